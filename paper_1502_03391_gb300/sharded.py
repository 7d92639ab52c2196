"""Row-block sharding of the in-sample loop across GPUs (one process per GPU).

Eq. (update) mixes each object's rows (B_l X^(l))_i, and those rows need only row i of
every Delta_l and the whole previous iterate (Eq. B).  So with the objects split into
contiguous blocks [r0, r1), one per process, each process holds rows r0..r1-1 of every
Delta_l and, per Guttman transform:

1. computes its rows of X_t and its parts of sigma(X_{t-1}) and of the column sums of
   X_t (``fjofc_transform_rows`` on its GPU);
2. all-gathers the rows into the whole X_t and all-reduces the 2 + m d float64 parts
   (``torch.distributed``; NCCL between GPUs, gloo on the CPU);
3. applies the stopping rule of Algorithm 1 (decrease reading, Remark eps) to
   sigma(X_{t-1}), the same decision in every process, and centres X_t by its means
   (Guttman outputs are centred in exact arithmetic, Sec. 1.2.2) before the next
   transform.

The loop is written over two functions so that its logic runs anywhere: ``rows_fn(X,
mu)`` returns this process's rows of the next iterate and its parts, and
``exchange(rows, parts)`` returns the whole next iterate and the summed parts.
``cuda_rows_fn`` and ``dist_exchange`` are the GPU / torch.distributed versions.
The semantics are those of ``fjofc_embed``: X_0 is used as given, sigma(X_t) is the
stress of the centred X_t, the returned X_T is centred, T transforms were applied.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np


def partition(n: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous object blocks [r0, r1), one per process (sizes differ by at most one)."""
    return [(n * g // world, n * (g + 1) // world) for g in range(world)]


@dataclasses.dataclass
class ShardedResult:
    X: object                 # the returned iterate X_T (centred), (m n) x d
    iters: int                # T
    history: List[float]      # sigma(X_0) .. sigma(X_T)
    status: int               # 0, or -3 (FJOFC_ERR_NONFINITE): X holds the last finite iterate


def embed_sharded(rows_fn: Callable, exchange: Callable, X0, n: int, m: int, d: int, max_iter: int,
                  tol: float = -1.0, tol_mode: str = "relative") -> ShardedResult:
    """The in-sample loop over the row blocks (see the module docstring).  ``X0`` is the
    whole X_0 (the same in every process); ``rows_fn(X, mu)`` and ``exchange(rows,
    parts)`` as above; ``mu`` is an m x d float64 array or None."""
    npairs = (m * n) * (m * n - 1) / 2.0
    X, mu = X0, None
    hist: List[float] = []
    last_good = (X0, None, 0)
    for t in range(1, max_iter + 2):
        rows, parts = rows_fn(X, mu)             # rows of X_t, parts of sigma(X_{t-1}) and of X_t's sums
        Xn, tot = exchange(rows, parts)
        sigma = float(tot[0] + tot[1])           # sigma(X_{t-1})
        tp = t - 1
        if not math.isfinite(sigma):
            Xf, muf, T = last_good
            return ShardedResult(_centred(Xf, muf, m, n), T, hist, -3)
        hist.append(sigma)
        last_good = (X, mu, tp)
        stop = tp == max_iter
        if not stop and tp >= 1 and tol >= 0.0:
            dec = hist[-2] - hist[-1]
            cont = (dec > tol * hist[-2]) if tol_mode == "relative" else (dec / npairs > tol)
            stop = not cont
        if stop:
            return ShardedResult(_centred(X, mu, m, n), tp, hist, 0)
        X = Xn
        mu = np.asarray(tot[2:], dtype=np.float64).reshape(m, d) / n
    raise AssertionError("unreachable")


def _centred(X, mu, m, n):
    if mu is None:
        return X
    out = X.reshape(m, n, -1).clone() if hasattr(X, "clone") else X.reshape(m, n, -1).copy()
    for j in range(m):
        if hasattr(out, "clone"):
            import torch
            out[j] -= torch.as_tensor(mu[j], dtype=out.dtype, device=out.device)
        else:
            out[j] -= mu[j]
    return out.reshape(m * n, -1)


def cuda_rows_fn(delta_rows: Sequence, weights, r0: int, r1: int, delta_scale=None, stream=None):
    """rows_fn on this process's GPU: ``fjofc_transform_rows`` over rows [r0, r1)."""
    import paper_1502_03391_gb300 as fj

    def fn(X, mu):
        return fj.transform_rows(delta_rows, weights, X, r0, r1, mu=mu, delta_scale=delta_scale, stream=stream)
    return fn


def dist_exchange(ranges: Sequence[Tuple[int, int]], m: int, d: int, group=None):
    """exchange over torch.distributed: all-gather of the row blocks (padded to the
    largest block) into the whole (m n) x d iterate, all-reduce (sum) of the float64
    parts.  Works with NCCL (CUDA tensors) and gloo (CPU tensors)."""
    import torch
    import torch.distributed as dist

    world = len(ranges)
    n = ranges[-1][1]
    rmax = max(r1 - r0 for r0, r1 in ranges)

    def fn(rows, parts):
        dev = rows.device
        pad = torch.zeros((m, rmax, d), dtype=rows.dtype, device=dev)
        pad[:, :rows.shape[1]] = rows
        out = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(out, pad, group=group)
        full = torch.empty((m, n, d), dtype=rows.dtype, device=dev)
        for g, (r0, r1) in enumerate(ranges):
            full[:, r0:r1] = out[g][:, :r1 - r0]
        tot = torch.as_tensor(np.asarray(parts, dtype=np.float64), device=dev)
        dist.all_reduce(tot, group=group)
        return full.reshape(m * n, d), tot.cpu().numpy()
    return fn
