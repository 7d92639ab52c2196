"""GPU parity of Algorithm 2's initialisation (fjofc_init_cmds) against the float64
oracle (oracle.initial_configuration: numpy.linalg.eigh for classical MDS,
numpy.linalg.svd for the Procrustes fit), through the C ABI.

The device solves the eigenproblems by float32 subspace iteration, so X_(0) is compared
at relative Frobenius error 1e-4: each product S V carries float32 rounding of its n-term
sums (~1e-6 relative), which the eigenvectors amplify by the spectrum's gap ratio, about
10 on these generators.  Both sides use the same sign convention, so no alignment is
applied before the comparison.
"""
import numpy as np
import pytest

from oracle import fjofc_oracle as O
import synthetic

pytestmark = pytest.mark.gpu

X_TOL = 1e-4


@pytest.fixture(scope="module")
def fj():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import ensure_library
    return ensure_library()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - np.asarray(b, np.float64)) /
                 max(np.linalg.norm(np.asarray(b, np.float64)), 1e-300))


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("m,n,d,latent", [(2, 200, 2, 5), (3, 150, 3, 5), (2, 300, 5, 10), (2, 1000, 3, 10),
                                          (2, 9, 3, 5)])
def test_init_matches_oracle(fj, m, n, d, latent):
    prob = synthetic.make_insample(0, n=n, m=m, d=d, latent=latent, seed=300 + n + m)
    dev = [fj.to_device_delta(D) for D in prob.deltas]
    X, iters = fj.init_cmds(dev, d)
    ref = O.initial_configuration([_f32(D) for D in prob.deltas], d)
    assert len(iters) == m + 1 and all(1 <= k <= 200 for k in iters)
    assert _rel(X.cpu().numpy(), ref) <= X_TOL


def test_init_paper_generator_and_half_precision(fj):
    """The paper's Sec. 4.3 generator (m = 3, n = 400, d = 2), float32 and float16 Delta
    (the float16 result against the oracle on the float16-rounded Delta)."""
    import torch
    deltas = synthetic.paper_jitter_modalities(n=400, m=3, dim=2, seed=11)
    for dt in (torch.float32, torch.float16):
        dev = [fj.to_device_delta(D, dtype=dt) for D in deltas]
        X, _ = fj.init_cmds(dev, 2)
        rounded = [D.float().cpu().numpy().astype(np.float64) for D in dev]
        ref = O.initial_configuration(rounded, 2)
        assert _rel(X.cpu().numpy(), ref) <= X_TOL, dt


def test_identical_modalities_share_one_configuration(fj):
    """Delta_i = D(Y) for every i: every modality block is the same (commensurability 0)
    and the configuration reproduces Y's Gram matrix (Torgerson)."""
    rng = np.random.default_rng(21)
    n, m, d = 256, 3, 2
    Y = rng.standard_normal((n, d)) * np.array([3.0, 1.0])
    Y -= Y.mean(0)
    D = np.sqrt(((Y[:, None] - Y[None]) ** 2).sum(-1))
    dev = [fj.to_device_delta(D) for _ in range(m)]
    X, _ = fj.init_cmds(dev, d)
    X = X.cpu().numpy().astype(np.float64).reshape(m, n, d)
    for i in range(1, m):
        assert _rel(X[i], X[0]) <= 1e-5
    assert _rel(X[0] @ X[0].T, Y @ Y.T) <= 1e-4
    np.testing.assert_allclose(X.mean(1), 0, atol=1e-4 * np.abs(X).max())


def test_init_then_embed(fj):
    """Algorithm 2 end to end on the device: X_(0) from the initialisation, then 30
    transforms; against the oracle's Algorithm 1 loop from its own X_(0)."""
    import torch
    prob = synthetic.make_insample(0, n=300, m=2, d=2, seed=333)
    dev = [fj.to_device_delta(D) for D in prob.deltas]
    X, _ = fj.init_cmds(dev, 2)
    X0_gpu = X.cpu().numpy().astype(np.float64)
    res = fj.embed(dev, prob.W, X, max_iter=30)
    torch.cuda.synchronize()
    ref = O.jofc_embed([_f32(D) for D in prob.deltas], prob.W, X0_gpu, max_iter=30)
    assert _rel(X.cpu().numpy(), ref.X) <= 1e-5
    np.testing.assert_allclose(res.history, ref.stress, rtol=1e-6)
    assert res.stress < ref.stress[0]
