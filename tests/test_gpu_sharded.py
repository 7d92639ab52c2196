"""Row-block sharding on one GPU: fjofc_transform_rows over several object ranges must
add up to one whole Guttman transform (Eq. update), and the sharded loop
(paper_1502_03391_gb300/sharded.py, its ranges exchanged in one process) must follow
the float64 oracle under the parity rule (tests/parity_rule.py).  The exchange across
processes is tested on the CPU (test_sharded_host.py); several GPUs are not available
here."""
import numpy as np
import pytest

from oracle import fjofc_oracle as O
import synthetic
from parity_rule import X_TOL, assert_history, assert_stress, rel_fro

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


def _dev_rows(fj, deltas, r0, r1):
    import torch
    return [torch.as_tensor(np.ascontiguousarray(D[r0:r1]), dtype=torch.float32).cuda() for D in deltas]


@pytest.mark.parametrize("m,n,d,world", [(2, 300, 3, 3), (3, 129, 2, 4), (12, 40, 3, 2), (2, 70, 10, 3)])
def test_ranges_add_up_to_one_transform(fj, m, n, d, world):
    import torch
    from paper_1502_03391_gb300 import sharded
    prob = synthetic.make_insample(0, n=n, m=m, d=d, seed=3200 + n)
    X0 = torch.as_tensor(np.asarray(prob.X0, np.float32)).cuda()
    rows, parts = [], np.zeros(2 + m * d)
    for r0, r1 in sharded.partition(n, world):
        Xo, p = fj.transform_rows(_dev_rows(fj, prob.deltas, r0, r1), prob.W, X0, r0, r1)
        rows.append(Xo.cpu().numpy().astype(np.float64))
        parts += p
    X1 = np.concatenate(rows, axis=1).reshape(m * n, d)
    d32 = [_f32(D) for D in prob.deltas]
    ref = O.jofc_embed(d32, prob.W, _f32(prob.X0), max_iter=1)
    assert rel_fro(X1, ref.X) <= X_TOL, rel_fro(X1, ref.X)
    assert_stress(parts[0] + parts[1], ref.stress[0], d32, prob.W, _f32(prob.X0))
    np.testing.assert_allclose(parts[2:], X1.reshape(m, n, d).sum(axis=1).reshape(-1),
                               atol=1e-5 * np.abs(X1).sum() / n)
    # the same transform by the single-call path (its X_1 is centred)
    Xd = X0.clone()
    fj.embed([fj.to_device_delta(D) for D in prob.deltas], prob.W, Xd, max_iter=1)
    Xc = X1.reshape(m, n, d) - X1.reshape(m, n, d).mean(axis=1, keepdims=True)
    assert rel_fro(Xd.cpu().numpy(), Xc.reshape(m * n, d)) <= X_TOL


def test_sharded_loop_matches_oracle(fj):
    """Twenty transforms of the sharded loop with three ranges, exchanged in-process."""
    import torch
    from paper_1502_03391_gb300 import sharded
    m, n, d, world = 2, 260, 3, 3
    prob = synthetic.make_insample(0, n=n, m=m, d=d, seed=3300)
    ranges = sharded.partition(n, world)
    fns = [sharded.cuda_rows_fn(_dev_rows(fj, prob.deltas, r0, r1), prob.W, r0, r1) for r0, r1 in ranges]

    def rows_fn(X, mu):                      # every range's rows and parts, this process
        outs = [f(X, mu) for f in fns]
        return [o[0] for o in outs], [o[1] for o in outs]

    def exchange(rows, parts):
        full = torch.cat(rows, dim=1).reshape(m * n, d)
        return full, np.sum(parts, axis=0)

    X0 = torch.as_tensor(np.asarray(prob.X0, np.float32)).cuda()
    res = sharded.embed_sharded(rows_fn, exchange, X0, n, m, d, max_iter=20)
    d32 = [_f32(D) for D in prob.deltas]
    ref = O.jofc_embed(d32, prob.W, _f32(prob.X0), max_iter=20, keep_iterates=True)
    assert res.status == 0 and res.iters == 20
    assert rel_fro(res.X.cpu().numpy(), ref.X) <= X_TOL
    assert_history(res.history, ref.stress, d32, prob.W, ref.iterates)
