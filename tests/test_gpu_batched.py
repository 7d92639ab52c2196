"""GPU tests of batched plans (fjofc_plan_*): many independent problems of uneven m, n, d
scheduled together (large ones on groups of SMs with their own barriers, small ones
sharing an SM one after another), captured in one CUDA graph.

* every problem's X after 20 transforms matches the float64 oracle (relative 1e-5), and
  its stress matches the oracle's stress of the same X (1e-6 relative plus the bound of
  the float32 distance error, which matters only for small, well-fitted problems),
  including a float16-Delta problem in its own class;
* with the relative tolerance each problem stops on its own: the same transform count
  and, within float32 reduction-order differences, the same X as a single fjofc_embed;
* re-running the plan from the same X_0 gives bitwise the same results;
* the plan runs as one CUDA graph and gives some problems groups of several SMs.
"""
import numpy as np
import pytest

from oracle import fjofc_oracle as O
import synthetic
from parity_rule import X_TOL, assert_stress

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


SHAPES = [  # m, n, d, delta type
    (2, 37, 2, "float32"), (3, 150, 3, "float32"), (1, 90, 5, "float32"), (2, 300, 3, "float32"),
    (2, 257, 2, "float32"), (3, 64, 5, "float32"), (2, 700, 3, "float32"), (2, 129, 3, "float16"),
    (2, 2, 2, "float32"), (3, 420, 2, "float32"), (12, 60, 3, "float32"),
]


def _check_stress(got, p, ref, where):
    """The device's stress of its own X_T against the oracle's stress of that X_T under
    the parity rule (1e-6 relative plus the float32 distance term, which carries the
    small, well-fitted problems of this batch), and the oracle's stresses of the device
    and oracle iterates against each other (1e-5 relative, as X)."""
    Xg = p["X"].cpu().numpy().astype(np.float64)
    s_dev_x = O.stress_blocks(p["rounded"], p["prob"].W, Xg)
    assert_stress(got, s_dev_x, p["rounded"], p["prob"].W, Xg, where)
    assert abs(s_dev_x - ref.stress[-1]) <= X_TOL * ref.stress[-1], where


def _problems(fj, shapes, seed0=500):
    import torch
    out = []
    for i, (m, n, d, dt) in enumerate(shapes):
        prob = synthetic.make_insample(0, n=n, m=m, d=d, seed=seed0 + i)
        dtype = getattr(torch, dt)
        scales = None if dt == "float32" else [float(np.max(D)) / 64.0 for D in prob.deltas]
        dev = [fj.to_device_delta(D, dtype=dtype, scale=(scales[l] if scales else 1.0))
               for l, D in enumerate(prob.deltas)]
        rounded = [dev[l].double().cpu().numpy() * (scales[l] if scales else 1.0) for l in range(m)]
        X0 = np.asarray(prob.X0, np.float32)
        out.append(dict(prob=prob, dev=dev, scales=scales, rounded=rounded, X0=X0,
                        X=torch.as_tensor(X0).cuda().contiguous()))
    return out


def test_mixed_batch_matches_oracle(fj):
    P = _problems(fj, SHAPES)
    plan = fj.Plan([(p["dev"], p["prob"].W, p["X"], p["scales"]) for p in P], max_iter=20)
    info = plan.info()
    assert info["graphed"]
    assert info["groups"].max() >= 2
    plan.run()
    res = plan.results()
    assert np.all(res.status == 0) and np.all(res.iters == 20)
    for i, p in enumerate(P):
        ref = O.jofc_embed(p["rounded"], p["prob"].W, p["X0"].astype(np.float64), max_iter=20)
        got = p["X"].cpu().numpy().astype(np.float64)
        assert _rel(got, ref.X) <= X_TOL, (i, SHAPES[i])
        _check_stress(res.stress[i], p, ref, (SHAPES[i], i))
    plan.close()


def test_rerun_is_bitwise_identical(fj):
    P = _problems(fj, SHAPES[:6], seed0=900)
    plan = fj.Plan([(p["dev"], p["prob"].W, p["X"], p["scales"]) for p in P], max_iter=15)
    plan.run()
    first = [p["X"].clone() for p in P]
    r1 = plan.results()
    for p in P:
        p["X"].copy_(__import__("torch").as_tensor(p["X0"]).cuda())
    plan.run()
    r2 = plan.results()
    for p, f in zip(P, first):
        assert bool((p["X"] == f).all())
    np.testing.assert_array_equal(r1.stress, r2.stress)


def test_per_problem_stopping_matches_single_calls(fj):
    import torch
    shapes = [(2, 180, 2, "float32"), (2, 333, 3, "float32"), (3, 120, 5, "float32"), (2, 600, 2, "float32")]
    P = _problems(fj, shapes, seed0=700)
    plan = fj.Plan([(p["dev"], p["prob"].W, p["X"], p["scales"]) for p in P], max_iter=400, tol=1e-6)
    plan.run()
    res = plan.results()
    for i, p in enumerate(P):
        Xs = torch.as_tensor(p["X0"]).cuda().contiguous()
        r = fj.embed(p["dev"], p["prob"].W, Xs, max_iter=400, tol=1e-6)
        assert abs(int(res.iters[i]) - r.iters) <= 1, (i, res.iters[i], r.iters)
        if int(res.iters[i]) == r.iters:
            assert _rel(p["X"].cpu().numpy(), Xs.cpu().numpy()) <= 1e-4
            assert abs(res.stress[i] - r.stress) <= 1e-5 * r.stress


@pytest.mark.parametrize("d", [2, 3, 5])
def test_more_problems_than_sms_share_them(fj, d):
    """400 small problems of one class: every problem on one SM, two or three one after
    another on each SM (the ring's barriers are retired and set up again in between)."""
    rng = np.random.default_rng(3 + d)
    shapes = [(int(rng.integers(1, 3)), int(rng.integers(20, 60)), d, "float32") for _ in range(400)]
    P = _problems(fj, shapes, seed0=1300)
    plan = fj.Plan([(p["dev"], p["prob"].W, p["X"], p["scales"]) for p in P], max_iter=12)
    info = plan.info()
    assert info["graphed"] and np.all(info["groups"] == 1)
    plan.run()
    res = plan.results()
    assert np.all(res.status == 0) and np.all(res.iters == 12)
    for i, p in enumerate(P):
        ref = O.jofc_embed(p["rounded"], p["prob"].W, p["X0"].astype(np.float64), max_iter=12)
        assert _rel(p["X"].cpu().numpy(), ref.X) <= X_TOL, (i, shapes[i])
        _check_stress(res.stress[i], p, ref, (shapes[i], i))


def test_autotuned_plan_matches_oracle_and_keeps_X0(fj):
    """The tuner's probe runs leave every X at X_0; the tuned plan (float16 storage
    allowed) gives oracle parity on the rounded Delta it chose."""
    import torch
    shapes = [(2, 300, 3, "float32"), (3, 180, 2, "float32"), (2, 640, 5, "float32"), (1, 90, 3, "float32")]
    P = _problems(fj, shapes, seed0=1700)
    plan = fj.Plan([(p["dev"], p["prob"].W, p["X"], p["scales"]) for p in P], max_iter=10, autotune=True,
                   probe_iters=3, allow_f16=True)
    assert plan.tuning["candidates"] == 8
    for p in P:
        assert bool((p["X"] == torch.as_tensor(p["X0"]).cuda()).all())
    plan.run()
    res = plan.results()
    for i, p in enumerate(P):
        deltas = p["rounded"]
        if plan.tuning["float16_delta"]:
            # the tuner's storage: Delta / s rounded to float16, s = max |Delta| / 2^10
            deltas = []
            for D in p["rounded"]:
                s = np.float32(np.float32(D.max()) / np.float32(1024.0))
                deltas.append((np.asarray(D, np.float32) * np.float32(1.0 / s)).astype(np.float16).astype(np.float64) * s)
        ref = O.jofc_embed(deltas, p["prob"].W, p["X0"].astype(np.float64), max_iter=10)
        assert _rel(p["X"].cpu().numpy(), ref.X) <= X_TOL, (i, shapes[i], plan.tuning)
