"""Precision form: Delta stored as float16 / bfloat16 (divided by a per-modality scale
s_l = max(Delta_l) / 2^10, so that entries stay in float16's normal range), distances,
b_ij and the update in float32, at the m=3, n=20000, d=10 workload and on a 2000-object
subsample of its generator.

* Arithmetic parity: against the float64 oracle run on the same rounded dissimilarities
  (s_l times the stored value), X within relative Frobenius 1e-5 -- at full size on
  sampled objects after one transform (the oracle computes those rows one by one), on
  the subsample after 20 transforms (every stress under the parity rule of
  ``tests/parity_rule.py``: 1e-6 relative plus the float32 distance term).
* Input error, stated rather than gated at 1e-5: the same runs against the oracle on the
  exact float64 dissimilarities.
* Final stress: iterated to the relative tolerance, the 16-bit result re-scored with
  float32 Delta is within 1e-3 of the float32 path's final stress.
"""
import numpy as np
import pytest

from oracle import fjofc_oracle as O
import synthetic
from parity_rule import X_TOL, assert_stress

pytestmark = pytest.mark.gpu

DTYPES = ["float32", "float16", "bfloat16"]


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


def _device_deltas(fj, F, dtype_name):
    """Delta_l on the device in the requested storage type, with its scale."""
    import torch
    dtype = getattr(torch, dtype_name)
    out, scales = [], []
    for Fi in F:
        full = synthetic.torch_distances(Fi, "cuda", torch.float32)
        s = 1.0 if dtype == torch.float32 else float(full.max().item()) / 1024.0
        buf = fj.empty_delta(full.shape[0], dtype)
        buf.copy_((full / s).to(dtype) if s != 1.0 else full)
        del full
        out.append(buf)
        scales.append(s)
    return out, scales


def _rows(dev, scales, idx):
    """Rows idx of every stored Delta_l as the float64 values the device uses."""
    import torch
    ii = torch.as_tensor(idx, device="cuda")
    return [dev[l].index_select(0, ii).double().cpu().numpy() * scales[l] for l in range(len(dev))]


@pytest.fixture(scope="module")
def full_problem():
    return synthetic.make_insample(2, with_deltas=False)


@pytest.mark.parametrize("dt", DTYPES)
def test_full_size_one_transform_sampled_rows(fj, full_problem, dt):
    import torch
    prob = full_problem
    m, n, d = prob.spec.m, prob.spec.n, prob.spec.d
    dev, scales = _device_deltas(fj, prob.F, dt)
    X0 = np.asarray(prob.X0, dtype=np.float32)
    X = torch.as_tensor(X0).cuda()
    res = fj.embed(dev, prob.W, X, max_iter=1, delta_scale=None if dt == "float32" else scales)
    assert res.status == 0 and res.iters == 1
    X1 = X.cpu().numpy().astype(np.float64)
    idx = np.random.default_rng(20).choice(n, size=40, replace=False)
    rows = _rows(dev, scales, idx)
    want = O.guttman_rows(rows, prob.W, X0.astype(np.float64), idx)
    got = np.stack([X1[j * n + idx] for j in range(m)])
    assert _rel(got, want) <= X_TOL
    if dt != "float32":
        # input error of the 16-bit storage (the rounding of Delta; loose gate)
        exact = [synthetic.euclidean_distances(prob.F[l][idx], prob.F[l]) for l in range(m)]
        err = _rel(got, O.guttman_rows(exact, prob.W, X0.astype(np.float64), idx))
        print(f"{dt}: one transform vs exact-Delta oracle, sampled rows: {err:.3e}")
        assert err <= 5e-3
    del dev
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dt", DTYPES)
def test_subsample_twenty_transforms(fj, dt):
    import torch
    prob = synthetic.make_insample(2, n=2000)
    m, n = prob.spec.m, prob.spec.n
    dtype = getattr(torch, dt)
    scales = [1.0 if dt == "float32" else float(np.max(D)) / 1024.0 for D in prob.deltas]
    dev = [fj.to_device_delta(D, dtype=dtype, scale=scales[l]) for l, D in enumerate(prob.deltas)]
    X0 = np.asarray(prob.X0, dtype=np.float32)
    X = torch.as_tensor(X0).cuda()
    res = fj.embed(dev, prob.W, X, max_iter=20, delta_scale=None if dt == "float32" else scales, history=True)
    assert res.status == 0 and res.iters == 20
    got = X.cpu().numpy().astype(np.float64)
    rounded = [dev[l].double().cpu().numpy() * scales[l] for l in range(m)]
    Xo = X0.astype(np.float64)
    assert_stress(res.history[0], O.stress_blocks(rounded, prob.W, Xo), rounded, prob.W, Xo, 0)
    for t in range(1, 21):
        Xo = O.guttman_step_closed_form(rounded, prob.W, Xo)
        assert_stress(res.history[t], O.stress_blocks(rounded, prob.W, Xo), rounded, prob.W, Xo, t)
    assert _rel(got, Xo) <= X_TOL
    assert res.stress == res.history[20]
    if dt != "float32":
        Xe = X0.astype(np.float64)
        for _ in range(20):
            Xe = O.guttman_step_closed_form(prob.deltas, prob.W, Xe)
        err = _rel(got, Xe)
        print(f"{dt}: 20 transforms vs exact-Delta oracle (n=2000): {err:.3e}")
        assert err <= 5e-3


@pytest.mark.parametrize("dt", ["float16", "bfloat16"])
def test_full_size_final_stress_matches_float32(fj, full_problem, dt):
    import torch
    prob = full_problem
    X0 = torch.as_tensor(np.asarray(prob.X0, dtype=np.float32)).cuda()
    dev32, _ = _device_deltas(fj, prob.F, "float32")
    X32 = X0.clone()
    r32 = fj.embed(dev32, prob.W, X32, max_iter=300, tol=1e-7, tol_mode="relative")
    dev16, scales = _device_deltas(fj, prob.F, dt)
    X16 = X0.clone()
    r16 = fj.embed(dev16, prob.W, X16, max_iter=300, tol=1e-7, tol_mode="relative", delta_scale=scales)
    assert r32.status == 0 and r16.status == 0
    s16 = fj.stress(dev32, prob.W, X16)          # 16-bit result scored with float32 Delta
    rel = abs(s16 - r32.stress) / r32.stress
    print(f"{dt}: final stress {s16:.9e} vs float32 path {r32.stress:.9e} (rel {rel:.2e}), "
          f"iterations {r16.iters} vs {r32.iters}")
    assert rel <= 1e-3
    del dev32, dev16
    torch.cuda.empty_cache()
