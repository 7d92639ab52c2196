"""Row-block sharding of the in-sample loop (paper_1502_03391_gb300/sharded.py) on the
CPU: two gloo ranks, each computing its object block's rows of every Guttman transform
with the float64 oracle (``guttman_rows``: rows of Eq. update from the Delta rows of
those objects, pinned to the dense step) and its parts of sigma and of the column sums;
the driver all-gathers the rows, all-reduces the parts and decides when to stop.  The
result must be Algorithm 1's (the oracle's dense loop) to 1e-10, under both stopping
rules.  This is the exchange and reassembly logic the multi-GPU path runs over NCCL."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def oracle_rows_fn(deltas, Wm, r0, r1):
    """rows_fn of one rank from the oracle: rows [r0, r1) of X_t (uncentred, as the
    device entry point returns them) and the parts of sigma(X_{t-1}) (fidelity over the
    block's full rows, halved; commensurability of the block's objects) and of X_t's
    column sums."""
    import torch
    from oracle import fjofc_oracle as O
    m = len(deltas)
    n = deltas[0].shape[0]
    Wm = np.asarray(Wm, dtype=np.float64)

    def fn(X, mu):
        Xc = X.numpy().astype(np.float64).reshape(m, n, -1)
        if mu is not None:
            Xc = Xc - mu[:, None, :]
        d = Xc.shape[2]
        idx = np.arange(r0, r1)
        rows = O.guttman_rows([D[r0:r1] for D in deltas], Wm, Xc.reshape(m * n, d), idx)   # (m, nr, d)
        fid = 0.0
        for l in range(m):
            diff = Xc[l][idx][:, None, :] - Xc[l][None, :, :]
            dist = np.sqrt((diff ** 2).sum(-1))
            e2 = (deltas[l][r0:r1] - dist) ** 2
            e2[np.arange(r1 - r0), idx] = 0.0
            fid += Wm[l, l] * e2.sum() / 2.0
        comm = sum(Wm[j, l] * float(((Xc[j][idx] - Xc[l][idx]) ** 2).sum())
                   for j in range(m) for l in range(j + 1, m))
        parts = np.concatenate([[fid, comm], rows.sum(axis=1).reshape(-1)])
        return torch.as_tensor(rows), parts
    return fn


CASES = [("relative", -1.0), ("relative", 1e-4), ("abs_normalized", 1e-6)]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import synthetic
    from paper_1502_03391_gb300 import sharded
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = synthetic.make_insample(0, n=45, m=3, d=2, seed=3100)
    ranges = sharded.partition(45, world)
    r0, r1 = ranges[rank]
    out = []
    for mode, tol in CASES:
        res = sharded.embed_sharded(oracle_rows_fn(prob.deltas, prob.W, r0, r1),
                                    sharded.dist_exchange(ranges, 3, 2), torch.as_tensor(prob.X0), 45, 3, 2,
                                    max_iter=60, tol=tol, tol_mode=mode)
        out.append((res.X.numpy(), res.iters, list(res.history), res.status))
    q.put((rank, out))
    dist.destroy_process_group()


def test_sharded_loop_gloo_world2_matches_oracle():
    """Fixed count (60 transforms) and both stopping rules, on two gloo ranks."""
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    pytest.importorskip("torch")
    # the package loads the CUDA library, which the CPU build provides
    from conftest import ensure_library
    ensure_library()
    import synthetic
    from oracle import fjofc_oracle as O
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    res = sorted((q.get(timeout=10) for _ in range(2)), key=lambda r: r[0])
    prob = synthetic.make_insample(0, n=45, m=3, d=2, seed=3100)
    for c, (mode, tol) in enumerate(CASES):
        ref = O.jofc_embed(prob.deltas, prob.W, prob.X0, max_iter=60, tol=tol, tol_mode=mode)
        for _, out in res:
            X, iters, hist, status = out[c]
            assert status == 0 and iters == ref.iters, (mode, tol)
            assert np.linalg.norm(X - ref.X) / np.linalg.norm(ref.X) <= 1e-10
            np.testing.assert_allclose(hist, ref.stress, rtol=1e-10)
        np.testing.assert_array_equal(res[0][1][c][0], res[1][1][c][0])   # every rank holds the same X


def test_partition_covers_the_objects():
    sys.path.insert(0, ROOT)
    from conftest import ensure_library
    ensure_library()
    from paper_1502_03391_gb300 import sharded
    for n, w in [(10, 3), (5000, 8), (7, 7)]:
        p = sharded.partition(n, w)
        assert p[0][0] == 0 and p[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(p, p[1:]))
        assert max(r1 - r0 for r0, r1 in p) - min(r1 - r0 for r0, r1 in p) <= 1
