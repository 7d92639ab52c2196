"""Seeded synthetic inputs for the fJOFC workloads.

This module only *generates inputs*: latent features, per-modality
dissimilarity matrices Delta_i (Euclidean distances between the synthetic
feature vectors, i.e. the method's given data, Sec. 1.2), initial
configurations X0 and new out-of-sample objects.  It holds none of the
method's arithmetic (no weights, no Laplacian, no Guttman transform, no
stress) and is shared by the CPU oracle, the tests and the benchmark.

Recipe (all draws from ``numpy.random.default_rng``; the seed of workload
``k`` and repetition ``rep`` is ``1000*k + rep``):

* draw order: latent ``Z`` (n x latent), then ``A_1..A_m`` (latent x latent,
  standard Gaussian), then noise ``E_1..E_m`` (n x latent), then
  ``X0 ~ N(0, I)`` of shape (m*n) x d, rows modality-major;
* modality features ``F_i = Z A_i + noise * E_i``;
* ``Delta_i[a, b] = ||F_i[a] - F_i[b]||_2`` computed in float64.

New (out-of-sample) objects reuse the same ``A_i`` with fresh ``Z`` and noise
drawn from an independent, named sub-stream.  The paper's own Gaussian-plus-
uniform-jitter generator (Sec. 4.1 and Sec. 4.3) is provided as
``paper_jitter_modalities``.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "WORKLOADS",
    "Workload",
    "InSample",
    "make_insample",
    "make_oos_objects",
    "euclidean_distances",
    "cross_distances",
    "paper_jitter_modalities",
    "batched_problem_shapes",
    "weights_matrix",
]


@dataclasses.dataclass(frozen=True)
class Workload:
    """Shape of one synthetic workload (sizes follow the paper-shaped configs)."""

    name: str
    m: int
    n: int
    d: int
    latent: int
    noise: float
    w_fid: float = 1.0      # fidelity weight w_ii
    w_comm: float = 0.5     # commensurability weight w_ij (i != j)


# Workload k uses seed 1000*k + rep.
WORKLOADS = {
    0: Workload("insample-m2-n200-d2", m=2, n=200, d=2, latent=5, noise=0.1),
    1: Workload("insample-m2-n5000-d3", m=2, n=5000, d=3, latent=10, noise=0.2),
    2: Workload("insample-m3-n20000-d10", m=3, n=20000, d=10, latent=20, noise=0.3),
    3: Workload("batched-256", m=2, n=0, d=0, latent=5, noise=0.1),
    4: Workload("oos-m2-n10000-d5", m=2, n=10000, d=5, latent=10, noise=0.2),
}


def weights_matrix(m: int, w_fid: float = 1.0, w_comm: float = 0.5) -> np.ndarray:
    """m x m weight parameters: ``w_fid`` on the diagonal, ``w_comm`` elsewhere.

    This is only the *parameter* layout the library and the oracle take (Eq. W2
    weights ``w_ij``); it builds no omnibus matrix.
    """
    W = np.full((m, m), float(w_comm))
    np.fill_diagonal(W, float(w_fid))
    return W


def euclidean_distances(F: np.ndarray, G: Optional[np.ndarray] = None) -> np.ndarray:
    """float64 Euclidean distances between the rows of F (and G), by explicit
    coordinate differences (no Gram-matrix shortcut), blocked to bound memory."""
    F = np.asarray(F, dtype=np.float64)
    G = F if G is None else np.asarray(G, dtype=np.float64)
    out = np.empty((F.shape[0], G.shape[0]), dtype=np.float64)
    step = max(1, int(4_000_000 // max(1, G.shape[0] * F.shape[1])))
    for a in range(0, F.shape[0], step):
        diff = F[a:a + step, None, :] - G[None, :, :]
        out[a:a + step] = np.sqrt(np.einsum("abk,abk->ab", diff, diff))
    if G is F:
        np.fill_diagonal(out, 0.0)
    return out


def cross_distances(F_new: np.ndarray, F: np.ndarray) -> np.ndarray:
    """float64 distances from each new object's features to every in-sample object."""
    return euclidean_distances(F_new, F)


@dataclasses.dataclass
class InSample:
    """One in-sample problem: features, dissimilarities and the initial configuration."""

    spec: Workload
    seed: int
    Z: np.ndarray
    A: List[np.ndarray]
    F: List[np.ndarray]
    X0: np.ndarray                       # (m*n) x d float64, modality-major rows
    deltas: Optional[List[np.ndarray]]   # m arrays n x n float64 (None when not materialised)

    @property
    def W(self) -> np.ndarray:
        return weights_matrix(self.spec.m, self.spec.w_fid, self.spec.w_comm)


def make_insample(k: int, rep: int = 0, *, n: Optional[int] = None, m: Optional[int] = None,
                  d: Optional[int] = None, latent: Optional[int] = None,
                  noise: Optional[float] = None, seed: Optional[int] = None,
                  with_deltas: bool = True, w_fid: Optional[float] = None,
                  w_comm: Optional[float] = None) -> InSample:
    """Generate workload ``k`` (optionally with overridden sizes).

    ``with_deltas=False`` skips the float64 n x n distance matrices (large
    workloads build them on the device from ``F`` instead).
    """
    base = WORKLOADS[k]
    spec = dataclasses.replace(
        base,
        n=base.n if n is None else int(n),
        m=base.m if m is None else int(m),
        d=base.d if d is None else int(d),
        latent=base.latent if latent is None else int(latent),
        noise=base.noise if noise is None else float(noise),
        w_fid=base.w_fid if w_fid is None else float(w_fid),
        w_comm=base.w_comm if w_comm is None else float(w_comm),
    )
    seed = 1000 * k + rep if seed is None else int(seed)
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((spec.n, spec.latent))
    A = [rng.standard_normal((spec.latent, spec.latent)) for _ in range(spec.m)]
    E = [rng.standard_normal((spec.n, spec.latent)) for _ in range(spec.m)]
    X0 = rng.standard_normal((spec.m * spec.n, spec.d))
    F = [Z @ A[i] + spec.noise * E[i] for i in range(spec.m)]
    deltas = [euclidean_distances(Fi) for Fi in F] if with_deltas else None
    return InSample(spec=spec, seed=seed, Z=Z, A=A, F=F, X0=X0, deltas=deltas)


def make_oos_objects(prob: InSample, count: int, stream: int = 1, *, with_deltas: bool = True):
    """New objects drawn from the generator of ``prob`` (same ``A_i``).

    Returns ``(F_new, delta_new, Y0)``: ``F_new`` is a list of m arrays
    (count x latent); ``delta_new`` is (count, m, n) float64 (or None) with
    ``delta_new[o, j, k] = ||F_new[j][o] - F[j][k]||``; ``Y0 ~ N(0, I)`` of
    shape (count, m, d) is the standard out-of-sample initialisation.
    ``stream`` selects an independent sub-stream (e.g. 1 = training objects,
    2 = test objects).
    """
    spec = prob.spec
    rng = np.random.default_rng([prob.seed, 7919, int(stream)])
    Zn = rng.standard_normal((count, spec.latent))
    En = [rng.standard_normal((count, spec.latent)) for _ in range(spec.m)]
    Y0 = rng.standard_normal((count, spec.m, spec.d))
    F_new = [Zn @ prob.A[j] + spec.noise * En[j] for j in range(spec.m)]
    delta_new = None
    if with_deltas:
        delta_new = np.empty((count, spec.m, spec.n), dtype=np.float64)
        for j in range(spec.m):
            delta_new[:, j, :] = cross_distances(F_new[j], prob.F[j])
    return F_new, delta_new, Y0


def paper_jitter_modalities(n: int = 400, m: int = 3, dim: int = 2, seed: int = 0,
                            anomalies: int = 0):
    """The paper's Sec. 4.1 / 4.3 generator: Y ~ N((5,..,5), I), z = max(Y) - min(Y),
    Y_i = Y + E_i with E_i ~ U(-z/50, z/50) entrywise.  With ``anomalies > 0`` the
    last modality's first ``anomalies`` rows are redrawn from N((8,..,8), 2 I)
    (the anomaly setting).  Returns the list of m float64 distance matrices."""
    rng = np.random.default_rng(seed)
    Y = rng.normal(5.0, 1.0, size=(n, dim))
    z = Y.max() - Y.min()
    mods = []
    for i in range(m):
        base = Y
        if anomalies and i == m - 1:
            base = Y.copy()
            base[:anomalies] = rng.normal(8.0, np.sqrt(2.0), size=(anomalies, dim))
        E = rng.uniform(-z / 50.0, z / 50.0, size=(n, dim))
        mods.append(euclidean_distances(base + E))
    return mods


def batched_problem_shapes(count: int = 256, seed: int = 3000):
    """Shapes of the batched workload: n ~ U[100, 4000], m in {2, 3}, d in {2, 3, 5};
    problem p uses seed ``seed*10 + p`` with the small workload's generator."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(100, 4001, size=count)
    ms = rng.choice([2, 3], size=count)
    ds = rng.choice([2, 3, 5], size=count)
    return [dict(n=int(ns[p]), m=int(ms[p]), d=int(ds[p]), seed=int(seed * 10 + p))
            for p in range(count)]


def torch_distances(F: np.ndarray, device, out_dtype, G: Optional[np.ndarray] = None,
                    chunk: int = 4096):
    """Device-side float64 Euclidean distances (explicit differences, no Gram
    shortcut) cast to ``out_dtype``; used to build large inputs quickly."""
    import torch

    Ft = torch.as_tensor(np.asarray(F, dtype=np.float64), device=device)
    Gt = Ft if G is None else torch.as_tensor(np.asarray(G, dtype=np.float64), device=device)
    out = torch.empty((Ft.shape[0], Gt.shape[0]), dtype=out_dtype, device=device)
    for a in range(0, Ft.shape[0], chunk):
        blk = torch.cdist(Ft[a:a + chunk], Gt, compute_mode="donot_use_mm_for_euclid_dist")
        out[a:a + chunk] = blk.to(out_dtype)
    if G is None:
        out.fill_diagonal_(0)
    return out
