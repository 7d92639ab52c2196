"""GPU parity of the in-sample path (fjofc_embed / fjofc_stress) against the float64
oracle, through the C ABI.

Tolerances (float32 arithmetic on the device vs float64 in the oracle, same float32
inputs; ``tests/parity_rule.py``): X after T transforms within relative Frobenius
error 1e-5; every stress within 1e-6 relative plus the fidelity error that float32
distances alone cause, 2 |Delta - d| eps_d d + (eps_d d)^2 per pair with eps_d =
2^-22.9 + (d + 3) 2^-25 (negligible except near zero stress).  Sizes span several
RB x CW tiles with ragged tails; edge cases cover the smallest n, duplicate points
(d_ij = 0), a non-zero Delta diagonal, exact configurations (zero stress), general
weights, float16/bfloat16 Delta, the stopping rule, determinism and non-finite input.
"""
import numpy as np
import pytest

from oracle import fjofc_oracle as O
import synthetic
from parity_rule import X_TOL, S_TOL, assert_history, assert_stress

pytestmark = pytest.mark.gpu


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
    return O.jofc_embed([_f32(D) for D in deltas], W, _f32(X0), max_iter=iters, keep_iterates=True, **kw)


def _hist(res, ref, deltas, W, where=""):
    """The device's stress history against the oracle's (the parity rule)."""
    assert_history(res.history, ref.stress, [_f32(D) for D in deltas], W, ref.iterates, where)


CASES = [  # m, n, d
    (2, 200, 2), (1, 37, 2), (2, 2, 1), (2, 3, 2), (3, 65, 3), (2, 127, 3), (2, 128, 3), (2, 129, 3),
    (2, 130, 2), (3, 64, 5), (2, 100, 8), (2, 70, 10), (2, 50, 16), (4, 33, 2), (2, 300, 4),
    (9, 40, 2), (12, 45, 3), (30, 20, 2), (32, 9, 5),      # beyond 8 modalities: the rolled mix
]


@pytest.mark.parametrize("m,n,d", CASES)
def test_parity_fixed_iterations(fj, m, n, d):
    prob = synthetic.make_insample(0, n=n, m=m, d=d, seed=100 + 7 * n + m + d)
    T = 20
    X, res = _run(fj, prob.deltas, prob.W, prob.X0, T)
    assert res.status == 0 and res.iters == T
    ref = _oracle(prob.deltas, prob.W, prob.X0, T)
    assert _rel(X, ref.X) <= X_TOL, _rel(X, ref.X)
    _hist(res, ref, prob.deltas, prob.W)
    # the returned stress is that of the returned X
    d32 = [_f32(D) for D in prob.deltas]
    assert_stress(res.stress, O.stress_blocks(d32, prob.W, X), d32, prob.W, X)
    # Guttman outputs are centred per modality
    for l in range(m):
        assert np.abs(X[l * n:(l + 1) * n].mean(0)).max() <= 1e-6 * np.abs(X).max()


def test_parity_against_float64_delta(fj):
    """Workload 0 (m=2, n=200, d=2, w=0.5) against the oracle on the unrounded float64
    Delta: the float32 input rounding stays inside the same tolerances."""
    prob = synthetic.make_insample(0)
    X, res = _run(fj, prob.deltas, prob.W, prob.X0, 20)
    ref = O.jofc_embed(prob.deltas, prob.W, prob.X0, max_iter=20, keep_iterates=True)
    assert _rel(X, ref.X) <= X_TOL
    assert_history(res.history, ref.stress, prob.deltas, prob.W, ref.iterates)


def test_workload0_100_iterations(fj):
    """Workload 0 at its full 100 transforms: stress matches at every iterate."""
    prob = synthetic.make_insample(0)
    X, res = _run(fj, prob.deltas, prob.W, prob.X0, 100)
    ref = _oracle(prob.deltas, prob.W, prob.X0, 100)
    _hist(res, ref, prob.deltas, prob.W)
    # past the 20-transform gate the float32 and float64 trajectories may part slowly
    # (near-flat directions of the stress); X is held to 1e-4 here, its stress to the rule
    assert _rel(X, ref.X) <= 1e-4


def test_full_size_workload1_steps(fj):
    """Workload 1 at full size (m=2, n=5000, d=3) in the launch configuration the
    benchmark uses: twenty transforms (the parity gate) against the oracle's Cor. 1 form,
    X within 1e-5 after the twentieth, and the stress of iterates 0, 1, 2, 3, 5, 10, 15
    and 20 against the oracle's blockwise stress (both oracle forms pinned to the dense
    definitions at small n) under the parity rule."""
    prob = synthetic.make_insample(1)
    T = 20
    X, res = _run(fj, prob.deltas, prob.W, prob.X0, T)
    assert res.status == 0 and res.iters == T
    d32 = [_f32(D) for D in prob.deltas]
    Xr = _f32(prob.X0)
    checked = (0, 1, 2, 3, 5, 10, 15, 20)
    for t in range(T + 1):
        if t > 0:
            Xr = O.guttman_step_closed_form(d32, prob.W, Xr)
        if t in checked:
            assert_stress(res.history[t], O.stress_blocks(d32, prob.W, Xr), d32, prob.W, Xr, t)
    assert _rel(X, Xr) <= X_TOL, _rel(X, Xr)


def _exact_problem(n, m, d, seed):
    """Every Delta_i holds the distances of one centred configuration Y (float32), so
    X = [Y; ...; Y] has zero stress (Eq. stress) and is a fixed point of the transform."""
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((n, d))
    Y -= Y.mean(0)
    Y = _f32(Y)
    Dy = np.sqrt(((Y[:, None, :] - Y[None, :, :]) ** 2).sum(-1))
    W = synthetic.weights_matrix(m, 1.0, 0.5)
    return Y, [Dy] * m, W, rng


@pytest.mark.parametrize("n,m,d", [(300, 2, 2), (257, 3, 3)])
def test_exact_configuration_fixed_point(fj, n, m, d):
    """X_0 = [Y; ...; Y] with Delta_i = D(Y): sigma(X_0) = 0 up to float32 distances (the
    rule's bound, with sigma = 0) and one transform returns X_0 within 1e-5."""
    Y, deltas, W, _ = _exact_problem(n, m, d, seed=1100 + n)
    X0 = np.vstack([Y] * m)
    X, res = _run(fj, deltas, W, X0, 1)
    d32 = [_f32(D) for D in deltas]
    assert res.status == 0 and res.iters == 1
    assert_stress(res.history[0], 0.0, d32, W, X0, "sigma(X_0)")
    assert_stress(res.history[1], O.stress_blocks(d32, W, X), d32, W, X, "sigma(X_1)")
    assert _rel(X, X0) <= X_TOL, _rel(X, X0)
    ref = _oracle(deltas, W, X0, 1)
    assert _rel(X, ref.X) <= X_TOL


def test_exact_configuration_recovery(fj):
    """From X_0 = [Y; Y] + 0.01 N(0, 1) the loop heads back to the zero-stress
    configuration along the oracle's trajectory: X after 20 transforms within 1e-5 of the
    oracle's, every stress of 200 transforms under the parity rule (whose float32
    distance term is what remains of the tolerance as sigma falls), and sigma(X_200)
    below 1e-6 sigma(X_0) (the float64 oracle reaches 2.8e-7 here; the slow part is the
    rotation of one modality against the other, held only by the commensurability
    weight)."""
    n, m, d = 400, 2, 2
    Y, deltas, W, rng = _exact_problem(n, m, d, seed=1200)
    X0 = _f32(np.vstack([Y] * m) + 0.01 * rng.standard_normal((m * n, d)))
    X, res = _run(fj, deltas, W, X0, 20)
    ref = _oracle(deltas, W, X0, 20)
    assert _rel(X, ref.X) <= X_TOL, _rel(X, ref.X)
    X, res = _run(fj, deltas, W, X0, 200)
    ref = _oracle(deltas, W, X0, 200)
    _hist(res, ref, deltas, W)
    assert res.history[-1] <= 1e-6 * res.history[0], (res.history[-1], res.history[0])


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
    _hist(res, ref, prob.deltas, prob.W)


@pytest.mark.parametrize("kind,m", [("W2", 3), ("W3", 3), ("W2", 12), ("W3", 20)])
def test_general_weights(fj, kind, m):
    """Per-modality fidelity and per-pair commensurability weights (Eq. W2), and the
    product weights of Eq. (W3), with few and with many modalities."""
    rng = np.random.default_rng(11 + m)
    n, d = (150, 3) if m <= 8 else (30, 3)
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
    _hist(res, ref, prob.deltas, W)


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
    ref = O.jofc_embed(rounded, prob.W, _f32(prob.X0), max_iter=20, keep_iterates=True)
    assert _rel(X, ref.X) <= X_TOL
    assert_history(res.history, ref.stress, rounded, prob.W, ref.iterates)


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
    d32 = [_f32(D) for D in prob.deltas]
    ref = O.stress_blocks(d32, prob.W, _f32(X0))
    assert_stress(res.stress, ref, d32, prob.W, _f32(X0))
    dev = [fj.to_device_delta(D) for D in prob.deltas]
    Xt = torch.as_tensor(np.asarray(X0, np.float32)).cuda()
    s = fj.stress(dev, prob.W, Xt)
    assert_stress(s, ref, d32, prob.W, _f32(X0))
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


@pytest.mark.parametrize("m,n,d", [(2, 300, 3), (3, 257, 2), (2, 90, 10), (2, 2200, 9), (14, 70, 3)])
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
    assert_history(r.history, ref.stress, [_f32(D) for D in prob.deltas], prob.W, ref.iterates)
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
