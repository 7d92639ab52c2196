"""Packed storage of the symmetric Delta (fjofc_pack_delta, delta_layout = PACKED): the
all-pairs pass reads the same values from the packed band layout (128-row bands from the
diagonal on, bands b and nB - 1 - b side by side), so the results must equal the full
layout's bit for bit, for every kernel shape (d = 3: column-strip layout, d = 5 and
d = 10: row-band layouts with 64- and 32-row blocks inside a band), ragged and exact band
counts, 16-bit Delta, and the batched plans; the packed matrices hold about half the
elements.  Also checked against the float64 oracle at one size."""
import numpy as np
import pytest

from oracle import fjofc_oracle as O
import synthetic
from parity_rule import X_TOL, assert_history, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fj():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import ensure_library
    return ensure_library()


@pytest.mark.parametrize("m,n,d,dt", [(2, 300, 3, "float32"), (2, 256, 3, "float32"), (3, 700, 5, "float32"),
                                      (2, 333, 10, "float32"), (2, 129, 2, "float16"), (1, 1000, 4, "bfloat16"),
                                      (2, 5, 3, "float32")])
def test_packed_equals_full_bitwise(fj, m, n, d, dt):
    import torch
    dtype = getattr(torch, dt)
    prob = synthetic.make_insample(0, n=n, m=m, d=d, seed=3400 + n + d)
    scales = None if dt == "float32" else [float(np.max(D)) / 256.0 for D in prob.deltas]
    full = [fj.to_device_delta(D, dtype=dtype, scale=(scales[i] if scales else 1.0)) for i, D in enumerate(prob.deltas)]
    packed = [fj.pack_delta(D) for D in full]
    assert packed[0].numel() <= n * (n + 256) // 2 + 128 * packed[0].shape[1]
    outs = []
    for deltas, layout in ((full, "full"), (packed, "packed")):
        X = torch.as_tensor(np.asarray(prob.X0, np.float32)).cuda()
        r = fj.embed(deltas, prob.W, X, max_iter=25, tol=1e-6, delta_scale=scales, layout=layout, n=n)
        outs.append((X.cpu().numpy(), r))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    assert outs[0][1].iters == outs[1][1].iters
    np.testing.assert_array_equal(outs[0][1].history, outs[1][1].history)


def test_packed_matches_oracle(fj):
    import torch
    prob = synthetic.make_insample(0, n=400, m=2, d=3, seed=3500)
    packed = [fj.pack_delta(fj.to_device_delta(D)) for D in prob.deltas]
    X = torch.as_tensor(np.asarray(prob.X0, np.float32)).cuda()
    r = fj.embed(packed, prob.W, X, max_iter=20, layout="packed", n=400)
    d32 = [np.asarray(D, np.float32).astype(np.float64) for D in prob.deltas]
    ref = O.jofc_embed(d32, prob.W, np.asarray(prob.X0, np.float32).astype(np.float64), max_iter=20,
                       keep_iterates=True)
    assert rel_fro(X.cpu().numpy(), ref.X) <= X_TOL
    assert_history(r.history, ref.stress, d32, prob.W, ref.iterates)


def test_packed_batched_plan(fj):
    """A batched plan over packed matrices equals the plan over the full ones."""
    import torch
    probs = [synthetic.make_insample(0, n=n, m=2, d=3, seed=3600 + n) for n in (150, 300)]
    res = []
    for layout in ("full", "packed"):
        Xs = []
        items = []
        for p in probs:
            dev = [fj.to_device_delta(D) for D in p.deltas]
            if layout == "packed":
                dev = [fj.pack_delta(D) for D in dev]
            X = torch.as_tensor(np.asarray(p.X0, np.float32)).cuda()
            Xs.append(X)
            items.append((dev, p.W, X))
        plan = fj.Plan(items, max_iter=15, layout=layout, n=[p.spec.n for p in probs])
        plan.run()
        torch.cuda.synchronize()
        res.append([X.cpu().numpy() for X in Xs])
    for a, b in zip(*res):
        np.testing.assert_array_equal(a, b)
