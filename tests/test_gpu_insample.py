"""GPU parity of the in-sample path (fjofc_embed / fjofc_stress) against the float64
oracle, through the C ABI.

Tolerances (float32 arithmetic on the device vs float64 in the oracle, same float32
inputs): X after T transforms within relative Frobenius error 1e-5, stress within 1e-6
relative.  Sizes span several RB x CW tiles with ragged tails; edge cases cover the
smallest n, duplicate points (d_ij = 0), a non-zero Delta diagonal, general weights,
float16/bfloat16 Delta, the stopping rule, determinism and non-finite input.
"""
import numpy as np
import pytest

from oracle import fjofc_oracle as O
import synthetic

pytestmark = pytest.mark.gpu

X_TOL = 1e-5
S_TOL = 1e-6


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


def _run(fj, deltas, W, X0, iters, tol=-1.0, tol_mode="relative", dtype=None, scales=None):
    import torch
    dev = [fj.to_device_delta(D, dtype=dtype, scale=(scales[i] if scales else 1.0)) for i, D in enumerate(deltas)]
    X = torch.as_tensor(np.asarray(X0, dtype=np.float32)).cuda().contiguous()
    res = fj.embed(dev, W, X, max_iter=iters, tol=tol, tol_mode=tol_mode, delta_scale=scales)
    torch.cuda.synchronize()
    return X.cpu().numpy().astype(np.float64), res


def _oracle(deltas, W, X0, iters, **kw):
    return O.jofc_embed([_f32(D) for D in deltas], W, _f32(X0), max_iter=iters, **kw)


CASES = [  # m, n, d
    (2, 200, 2), (1, 37, 2), (2, 2, 1), (2, 3, 2), (3, 65, 3), (2, 127, 3), (2, 128, 3), (2, 129, 3),
    (2, 130, 2), (3, 64, 5), (2, 100, 8), (2, 70, 10), (2, 50, 16), (4, 33, 2), (2, 300, 4),
]


@pytest.mark.parametrize("m,n,d", CASES)
def test_parity_fixed_iterations(fj, m, n, d):
    prob = synthetic.make_insample(0, n=n, m=m, d=d, seed=100 + 7 * n + m + d)
    T = 20
    X, res = _run(fj, prob.deltas, prob.W, prob.X0, T)
    assert res.status == 0 and res.iters == T
    ref = _oracle(prob.deltas, prob.W, prob.X0, T)
    assert _rel(X, ref.X) <= X_TOL, _rel(X, ref.X)
    np.testing.assert_allclose(res.history, ref.stress, rtol=S_TOL)
    # the returned stress is that of the returned X
    assert abs(res.stress - O.stress_blocks([_f32(D) for D in prob.deltas], prob.W, X)) <= S_TOL * res.stress
    # Guttman outputs are centred per modality
    for l in range(m):
        assert np.abs(X[l * n:(l + 1) * n].mean(0)).max() <= 1e-6 * np.abs(X).max()


def test_parity_against_float64_delta(fj):
    """Workload 0 (m=2, n=200, d=2, w=0.5) against the oracle on the unrounded float64
    Delta: the float32 input rounding stays inside the same tolerances."""
    prob = synthetic.make_insample(0)
    X, res = _run(fj, prob.deltas, prob.W, prob.X0, 20)
    ref = O.jofc_embed(prob.deltas, prob.W, prob.X0, max_iter=20)
    assert _rel(X, ref.X) <= X_TOL
    np.testing.assert_allclose(res.history, ref.stress, rtol=S_TOL)


def test_workload0_100_iterations(fj):
    """Workload 0 at its full 100 transforms: stress matches at every iterate."""
    prob = synthetic.make_insample(0)
    X, res = _run(fj, prob.deltas, prob.W, prob.X0, 100)
    ref = _oracle(prob.deltas, prob.W, prob.X0, 100)
    np.testing.assert_allclose(res.history, ref.stress, rtol=S_TOL)
    assert _rel(X, ref.X) <= 1e-4


def test_full_size_workload1_steps(fj):
    """Workload 1 at full size (m=2, n=5000, d=3) in the launch configuration the
    benchmark uses: three transforms against the oracle's Cor. 1 form and blockwise
    stress (both pinned to the dense definitions at small n)."""
    prob = synthetic.make_insample(1)
    T = 3
    X, res = _run(fj, prob.deltas, prob.W, prob.X0, T)
    d32 = [_f32(D) for D in prob.deltas]
    Xr = _f32(prob.X0)
    hist = [O.stress_blocks(d32, prob.W, Xr)]
    for _ in range(T):
        Xr = O.guttman_step_closed_form(d32, prob.W, Xr)
        hist.append(O.stress_blocks(d32, prob.W, Xr))
    assert _rel(X, Xr) <= X_TOL
    np.testing.assert_allclose(res.history, hist, rtol=S_TOL)


def test_duplicate_points_and_nonzero_diagonal(fj):
    """d_ij = 0 pairs contribute nothing to B(X) (Eq. B) and the Delta diagonal is
    ignored (its weight is 0 in Eq. W)."""
    prob = synthetic.make_insample(0, n=90, m=2, d=2, seed=5)
    X0 = prob.X0.copy()
    X0[3] = X0[7]
    X0[90 + 10] = X0[90 + 11]
    noisy = [D.copy() for D in prob.deltas]
    for D in noisy:
        np.fill_diagonal(D, 3.0)
    X, res = _run(fj, noisy, prob.W, X0, 15)
    ref = _oracle(prob.deltas, prob.W, X0, 15)
    assert _rel(X, ref.X) <= X_TOL
    np.testing.assert_allclose(res.history, ref.stress, rtol=S_TOL)


@pytest.mark.parametrize("kind", ["W2", "W3"])
def test_general_weights(fj, kind):
    """Per-modality fidelity and per-pair commensurability weights (Eq. W2), and the
    product weights of Eq. (W3)."""
    rng = np.random.default_rng(11)
    m, n, d = 3, 150, 3
    prob = synthetic.make_insample(0, n=n, m=m, d=d, seed=12)
    if kind == "W2":
        A = rng.uniform(0.2, 2.0, (m, m))
        W = np.triu(A) + np.triu(A, 1).T
    else:
        w = rng.uniform(0.3, 1.5, m)
        W = np.outer(w, w)
        np.fill_diagonal(W, w)
    X, res = _run(fj, prob.deltas, W, prob.X0, 20)
    ref = _oracle(prob.deltas, W, prob.X0, 20)
    assert _rel(X, ref.X) <= X_TOL
    np.testing.assert_allclose(res.history, ref.stress, rtol=S_TOL)


@pytest.mark.parametrize("dt", ["float16", "bfloat16"])
def test_half_precision_delta(fj, dt):
    """Delta stored as float16/bfloat16 divided by a per-modality scale: the device result
    matches the oracle run on the same rounded dissimilarities (scale * stored value)."""
    import torch
    dtype = getattr(torch, dt)
    prob = synthetic.make_insample(0, n=260, m=2, d=3, seed=21)
    scales = [float(np.max(D)) / 64.0 for D in prob.deltas]
    X, res = _run(fj, prob.deltas, prob.W, prob.X0, 20, dtype=dtype, scales=scales)
    rounded = [scales[i] * torch.as_tensor(prob.deltas[i] / scales[i]).to(dtype).double().numpy()
               for i in range(2)]
    ref = O.jofc_embed(rounded, prob.W, _f32(prob.X0), max_iter=20)
    assert _rel(X, ref.X) <= X_TOL
    np.testing.assert_allclose(res.history, ref.stress, rtol=S_TOL)


@pytest.mark.parametrize("mode,tol", [("relative", 1e-4), ("abs_normalized", 1e-5)])
def test_stopping_rule(fj, mode, tol):
    """The loop stops at the first transform whose decrease is within the tolerance
    (Algorithm 1 with the sign reading), and the returned X is that iterate."""
    prob = synthetic.make_insample(0, n=120, m=2, d=2, seed=31)
    X, res = _run(fj, prob.deltas, prob.W, prob.X0, 400, tol=tol, tol_mode=mode)
    h = res.history
    T = res.iters
    assert 1 <= T < 400 and len(h) == T + 1
    npairs = (240 * 239) // 2
    dec = lambda t: (h[t - 1] - h[t]) / (h[t - 1] if mode == "relative" else npairs)  # noqa: E731
    assert all(dec(t) > tol for t in range(1, T))
    assert dec(T) <= tol
    ref = _oracle(prob.deltas, prob.W, prob.X0, T)
    assert _rel(X, ref.X) <= 1e-4


def test_max_iter_zero_and_stress_entry(fj):
    import torch
    prob = synthetic.make_insample(0, n=333, m=3, d=4, seed=41)
    X0 = prob.X0 + 0.25          # uncentred input is used as given
    X, res = _run(fj, prob.deltas, prob.W, X0, 0)
    assert res.iters == 0
    np.testing.assert_array_equal(X, _f32(X0))
    ref = O.stress_blocks([_f32(D) for D in prob.deltas], prob.W, _f32(X0))
    assert abs(res.stress - ref) <= S_TOL * ref
    dev = [fj.to_device_delta(D) for D in prob.deltas]
    Xt = torch.as_tensor(np.asarray(X0, np.float32)).cuda()
    s = fj.stress(dev, prob.W, Xt)
    assert abs(s - ref) <= S_TOL * ref
    np.testing.assert_array_equal(Xt.cpu().numpy(), np.asarray(X0, np.float32))


def test_bitwise_deterministic(fj):
    prob = synthetic.make_insample(0, n=700, m=2, d=3, seed=51)
    X1, r1 = _run(fj, prob.deltas, prob.W, prob.X0, 10)
    X2, r2 = _run(fj, prob.deltas, prob.W, prob.X0, 10)
    np.testing.assert_array_equal(X1, X2)
    np.testing.assert_array_equal(r1.history, r2.history)


def test_nonfinite_input_reported(fj):
    prob = synthetic.make_insample(0, n=50, m=2, d=2, seed=61)
    X0 = prob.X0.copy()
    X0[5, 0] = np.nan
    X, res = _run_nocheck(fj, prob.deltas, prob.W, X0, 5)
    assert res.status == fj.FJOFC_ERR_NONFINITE


def _run_nocheck(fj, deltas, W, X0, iters):
    import torch
    dev = [fj.to_device_delta(D) for D in deltas]
    X = torch.as_tensor(np.asarray(X0, dtype=np.float32)).cuda()
    res = fj.embed(dev, W, X, max_iter=iters, check=False)
    return X.cpu().numpy(), res


def test_padded_row_stride_is_transparent(fj):
    """The same Delta with two different row strides gives bitwise equal results."""
    import torch
    prob = synthetic.make_insample(0, n=96, m=2, d=2, seed=71)
    outs = []
    for extra in (0, 36):
        dev = []
        for D in prob.deltas:
            buf = torch.zeros((96, 96 + extra), dtype=torch.float32, device="cuda")
            buf[:, :96] = torch.as_tensor(D, dtype=torch.float32)
            dev.append(buf[:, :96])
        X = torch.as_tensor(np.asarray(prob.X0, np.float32)).cuda()
        fj.embed(dev, prob.W, X, max_iter=8)
        outs.append(X.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])


@pytest.mark.parametrize("m,n,d", [(2, 300, 3), (3, 257, 2), (2, 90, 10), (2, 2200, 9)])
def test_persistent_and_per_pass_launches_agree(fj, m, n, d):
    """The default path (one persistent cooperative kernel for the whole loop) and the
    one-launch-per-pass path (profile=1) compute the same partials in the same order:
    bitwise equal X, iteration counts and stress histories."""
    import torch
    prob = synthetic.make_insample(0, n=n, m=m, d=d, seed=81 + n)
    dev = [fj.to_device_delta(D) for D in prob.deltas]
    outs = []
    for prof in (0, 1, 2):
        X = torch.as_tensor(np.asarray(prob.X0, np.float32)).cuda()
        r = fj.embed(dev, prob.W, X, max_iter=60, tol=1e-6, tol_mode="relative", profile=prof)
        outs.append((X.cpu().numpy(), r))
    for X, r in outs[1:]:
        np.testing.assert_array_equal(X, outs[0][0])
        assert r.iters == outs[0][1].iters
        np.testing.assert_array_equal(r.history, outs[0][1].history)
    assert outs[1][1].passes == outs[1][1].iters + 1 and outs[1][1].ms_pass > 0
    assert outs[2][1].passes == outs[2][1].iters + 1 and outs[2][1].ms_pass > 0


@pytest.mark.parametrize("m,n,d,relax", [(2, 150, 3, 1.5), (3, 129, 2, 2.0), (2, 300, 5, 1.8)])
def test_relaxed_updates_match_oracle(fj, m, n, d, relax):
    """Relaxed updates (opts.relax, the Conclusion's suggested acceleration) against the
    oracle's relaxed loop: X after 20 transforms within 1e-5, every stress within 1e-6;
    no centring of the iterates (the oracle's definition), and the persistent and
    per-pass launches agree bit for bit."""
    import torch
    prob = synthetic.make_insample(0, n=n, m=m, d=d, seed=91 + n)
    ref = _oracle(prob.deltas, prob.W, prob.X0, 20, relax=relax)
    dev = [fj.to_device_delta(D) for D in prob.deltas]
    outs = []
    for prof in (0, 1):
        X = torch.as_tensor(np.asarray(prob.X0, np.float32)).cuda()
        r = fj.embed(dev, prob.W, X, max_iter=20, profile=prof, relax=relax)
        outs.append((X.cpu().numpy(), r))
    X, r = outs[0]
    assert r.status == 0 and r.iters == 20
    assert _rel(X, ref.X) <= X_TOL
    np.testing.assert_allclose(r.history, ref.stress, rtol=S_TOL)
    np.testing.assert_array_equal(outs[1][0], X)
    np.testing.assert_array_equal(outs[1][1].history, r.history)


def test_relaxed_updates_reach_tolerance_in_fewer_transforms(fj):
    """Over-relaxation shortens the run to a relative stress change of 1e-6 on the m=2,
    n=400, d=2 generator, and the final stress is no worse than the plain run's (within
    1e-3 relative): what the relaxed updates are for."""
    import torch
    prob = synthetic.make_insample(0, n=400, seed=97)
    dev = [fj.to_device_delta(D) for D in prob.deltas]
    runs = {}
    for relax in (1.0, 1.9):
        X = torch.as_tensor(np.asarray(prob.X0, np.float32)).cuda()
        runs[relax] = fj.embed(dev, prob.W, X, max_iter=3000, tol=1e-6, tol_mode="relative", relax=relax)
    assert runs[1.9].iters < runs[1.0].iters
    assert runs[1.9].stress <= runs[1.0].stress * (1 + 1e-3)
    st = np.asarray(runs[1.9].history)
    assert np.all(np.diff(st) <= 1e-6 * st[:-1])       # float32 rounding aside, no increase
