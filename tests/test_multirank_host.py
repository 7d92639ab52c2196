"""The N > 1 path of bench.py on the CPU, with the gloo backend: the benchmark runs N
independent replicas (the method's problems do not share data; no collective on the
data path), and the whole-job figures are the slowest rank's time and the summed work;
the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, w = bench.aggregate_ranks(dist, torch.device("cpu"), elapsed_ms=10.0 + 5.0 * rank, work=100 * (rank + 1))
    q.put((rank, t, w))
    dist.destroy_process_group()


def test_aggregate_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, t, w in res:
        assert t == 15.0            # the slowest rank
        assert w == 300.0           # all ranks' work


def test_aggregate_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(None, None, 12.5, 7) == (12.5, 7.0)


def test_reference_arm_runs_on_rank0_only():
    """Under torchrun with two ranks only rank 0 prints the reference line; the other
    rank exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="4")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1 and '"impl": "reference"' in lines[0]
