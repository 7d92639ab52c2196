"""GPU parity of the out-of-sample path (fjofc_oos) against the float64 oracle.

Each new object is an independent out-of-sample problem (Sec. 3).  The device result
after T transforms must match the oracle's dense Eq. (joosupdate) iteration (small n) or
its pinned O(nmd) form (large n) within relative error 1e-5 per object, stresses within
1e-6.  Cases: k not a multiple of the object group, n not a multiple of the point tile,
general weights, float16 delta, per-object stopping, exact-configuration fixed points.
Stresses follow the parity rule of ``tests/parity_rule.py`` (1e-6 relative plus the
fidelity error float32 distances alone cause, which decides only near zero stress).
Each case runs both kernel forms: the streaming one (one warp slot per object, the
dissimilarities streamed every iteration) and the resident one (one CTA per object with
-X^T and the object's dissimilarities in shared memory; d <= 8).
"""
import numpy as np
import pytest

from oracle import fjofc_oracle as O
import synthetic
from parity_rule import X_TOL, oos_stress_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fj():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import ensure_library
    return ensure_library()


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _device_inputs(fj, X, delta_new, Y0, dtype=None, scale=None):
    import torch
    k, m, n = delta_new.shape
    dn = fj.empty_oos_delta(k, m, n, dtype=dtype)
    src = delta_new if scale is None else delta_new / np.asarray(scale)[None, :, None]
    dn.copy_(torch.as_tensor(src).to(dn.dtype))
    Xd = torch.as_tensor(np.asarray(X, np.float32)).cuda().contiguous()
    Yd = torch.as_tensor(np.asarray(Y0, np.float32)).cuda().contiguous()
    it = torch.zeros(k, dtype=torch.int32, device="cuda")
    st = torch.zeros(k, dtype=torch.float64, device="cuda")
    return dn, Xd, Yd, it, st


def _setup(m, n, d, k, seed, w=0.5):
    prob = synthetic.make_insample(0, n=n, m=m, d=d, seed=seed, w_comm=w)
    # an in-sample configuration: a few oracle transforms from X0 (float32-representable)
    X = _f32(O.jofc_embed(prob.deltas, prob.W, prob.X0, max_iter=5).X) if m * n <= 900 else _f32(prob.X0)
    _, dnew, Y0 = synthetic.make_oos_objects(prob, k, stream=1)
    return prob, X, dnew, Y0


FORMS = ["streaming", "resident"]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("m,n,d,k", [(2, 10, 2, 1), (2, 63, 3, 7), (3, 64, 2, 33), (2, 65, 5, 9),
                                     (2, 200, 3, 17), (3, 130, 10, 5), (2, 40, 16, 3), (1, 50, 2, 4),
                                     (8, 301, 3, 3), (4, 257, 8, 2), (12, 70, 3, 5), (30, 40, 2, 4),
                                     (32, 33, 8, 3), (20, 50, 10, 2)])
def test_oos_parity_fixed_iterations(fj, m, n, d, k, form):
    if form == "resident" and d > 8:
        pytest.skip("the resident form is built for d <= 8")
    T = 15
    prob, X, dnew, Y0 = _setup(m, n, d, k, seed=300 + n + m + d)
    dn, Xd, Yd, it, st = _device_inputs(fj, X, dnew, Y0)
    res = fj.oos(Xd, dn, prob.W, Yd, max_iter=T, iters_out=it, stress_out=st, form=form)
    assert res.status == 0 and res.max_iters == T
    Y = Yd.cpu().numpy()
    sig = st.cpu().numpy()
    assert np.all(it.cpu().numpy() == T)
    # the dense Eq. (joosupdate) oracle; its pinned O(nmd) form above m n = 1000 (time)
    oracle = O.oos_embed if m * n <= 1000 else O.oos_embed_closed_form
    for o in range(k):
        ref = oracle(X, _f32(dnew[o]), _f32(Y0[o]), prob.W, max_iter=T)
        err = np.linalg.norm(Y[o] - ref.y) / np.linalg.norm(ref.y)
        assert err <= X_TOL, (o, err)
        assert abs(sig[o] - ref.stress[-1]) <= oos_stress_tol(ref.stress[-1], X, _f32(dnew[o]), ref.y, prob.W)
    assert abs(res.stress_sum - sig.sum()) <= 1e-12 * sig.sum()


def test_oos_full_size_workload(fj):
    """The learned-form in-sample size (m=2, n=10000, d=5) with 40 new objects, against the
    oracle's O(nmd) form (pinned to the dense update at small n)."""
    prob = synthetic.make_insample(4, with_deltas=False)
    X = _f32(prob.X0)
    _, dnew, Y0 = synthetic.make_oos_objects(prob, 40, stream=2)
    T = 10
    dn, Xd, Yd, it, st = _device_inputs(fj, X, dnew, Y0)
    fj.oos(Xd, dn, prob.W, Yd, max_iter=T, iters_out=it, stress_out=st)
    Y = Yd.cpu().numpy()
    sig = st.cpu().numpy()
    for o in range(0, 40, 3):
        ref = O.oos_embed_closed_form(X, _f32(dnew[o]), _f32(Y0[o]), prob.W, max_iter=T)
        assert np.linalg.norm(Y[o] - ref.y) / np.linalg.norm(ref.y) <= X_TOL
        assert abs(sig[o] - ref.stress[-1]) <= oos_stress_tol(ref.stress[-1], X, _f32(dnew[o]), ref.y, prob.W)


@pytest.mark.parametrize("form", FORMS)
def test_oos_general_weights_and_half_delta(fj, form):
    import torch
    rng = np.random.default_rng(3)
    m, n, d, k = 3, 77, 3, 6
    prob, X, dnew, Y0 = _setup(m, n, d, k, seed=401)
    A = rng.uniform(0.3, 2.0, (m, m))
    W = np.triu(A) + np.triu(A, 1).T
    scale = [float(dnew[:, j].max()) / 32 for j in range(m)]
    dn, Xd, Yd, it, st = _device_inputs(fj, X, dnew, Y0, dtype=torch.float16, scale=scale)
    fj.oos(Xd, dn, W, Yd, max_iter=12, delta_scale=scale, stress_out=st, form=form)
    Y = Yd.cpu().numpy()
    rounded = dn.double().cpu().numpy() * np.asarray(scale)[None, :, None]
    for o in range(k):
        ref = O.oos_embed(X, rounded[o], _f32(Y0[o]), W, max_iter=12)
        assert np.linalg.norm(Y[o] - ref.y) / np.linalg.norm(ref.y) <= 1e-5


@pytest.mark.parametrize("form", FORMS)
def test_oos_per_object_stopping(fj, form):
    m, n, d, k = 2, 90, 2, 12
    prob, X, dnew, Y0 = _setup(m, n, d, k, seed=501)
    tol = 1e-5
    dn, Xd, Yd, it, st = _device_inputs(fj, X, dnew, Y0)
    fj.oos(Xd, dn, prob.W, Yd, max_iter=300, tol=tol, tol_mode="relative", iters_out=it, stress_out=st,
           form=form)
    iters = it.cpu().numpy()
    Y = Yd.cpu().numpy()
    assert iters.min() >= 1 and iters.max() < 300
    assert len(set(iters.tolist())) > 1          # objects stop independently
    for o in range(k):
        ref = O.oos_embed(X, _f32(dnew[o]), _f32(Y0[o]), prob.W, max_iter=int(iters[o]))
        h = ref.stress
        assert np.linalg.norm(Y[o] - ref.y) / np.linalg.norm(ref.y) <= 1e-4
        # the oracle's own history would also have stopped there (allowing float32 noise
        # in the last decrease)
        assert (h[-2] - h[-1]) <= tol * h[-2] * 1.5 + 1e-9 * h[-2]


@pytest.mark.parametrize("form", FORMS)
def test_oos_exact_configuration_fixed_point(fj, form):
    """A new object that repeats in-sample object j of a zero-stress embedding stays at
    X_j (Sec. 3 fixed point)."""
    rng = np.random.default_rng(9)
    n, m, d = 70, 2, 2
    Yc = rng.standard_normal((n, d))
    Yc -= Yc.mean(0)
    Yc = _f32(Yc)
    Dy = np.sqrt(((Yc[:, None] - Yc[None]) ** 2).sum(-1))
    X = np.vstack([Yc, Yc])
    W = synthetic.weights_matrix(2, 1.0, 0.5)
    idx = [3, 40, 69]
    dnew = np.stack([np.stack([Dy[j], Dy[j]]) for j in idx])
    Y0 = np.stack([np.stack([Yc[j], Yc[j]]) for j in idx])
    dn, Xd, Yd, it, st = _device_inputs(fj, X, dnew, Y0)
    fj.oos(Xd, dn, W, Yd, max_iter=5, stress_out=st, form=form)
    np.testing.assert_allclose(Yd.cpu().numpy(), Y0, atol=2e-5)
    sig = st.cpu().numpy()
    for o in range(len(idx)):
        # the oracle's stress there is zero: the rule leaves the float32 distance term
        assert sig[o] <= oos_stress_tol(0.0, X, dnew[o], Y0[o], W), (o, sig[o])


def test_oos_forms_agree_and_auto_picks_resident_for_few_objects(fj):
    """Both forms on the same inputs (one object per CTA against a small in-sample set, 60
    transforms): results within float32 reduction-order noise; the automatic choice (few
    objects, small in-sample set) equals the resident result bit for bit."""
    import torch
    m, n, d, k = 3, 400, 3, 5
    prob, X, dnew, Y0 = _setup(m, n, d, k, seed=777)
    outs = {}
    for form in ("streaming", "resident", "auto"):
        dn, Xd, Yd, it, st = _device_inputs(fj, X, dnew, Y0)
        fj.oos(Xd, dn, prob.W, Yd, max_iter=60, iters_out=it, stress_out=st, form=form)
        torch.cuda.synchronize()
        outs[form] = (Yd.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy())
    Ys, its, ss = outs["streaming"]
    Yr, itr, sr = outs["resident"]
    assert np.all(its == 60) and np.all(itr == 60)
    for o in range(k):
        assert np.linalg.norm(Yr[o] - Ys[o]) / np.linalg.norm(Ys[o]) <= 1e-5, o
    np.testing.assert_allclose(sr, ss, rtol=1e-6)
    np.testing.assert_array_equal(outs["auto"][0], Yr)
    np.testing.assert_array_equal(outs["auto"][2], sr)
