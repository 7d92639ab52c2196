"""FP64 CPU oracle for fJOFC (Lyzinski et al., "Fast Embedding for JOFC Using the
Raw Stress Criterion", arXiv 1502.03391).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The CUDA library never
calls it and shares no code with it.

What it computes is the plain definition of the JOFC method, written with dense
matrices and numpy float64 so that every step can be checked against the paper by
eye:

* the omnibus dissimilarity (Eq. jofcdelta) and weight matrix (Eq. W / Eq. W2),
* the combinatorial Laplacian ``L = D - W`` (Sec. 1.2.2, item 2),
* ``B(X)`` of Eq. (B) and the raw stress of Eq. (stress) as the double sum
  ``sum_{i<j} W_ij (Delta_ij - d_ij(X))^2``,
* Algorithm 1's loop ``X_t = L^+ B(X_{t-1}) X_{t-1}`` with ``L^+`` the
  Moore-Penrose pseudoinverse from ``numpy.linalg.pinv`` (SVD, rank-revealing cutoff),
* the out-of-sample Guttman transform of Eq. (joosupdate) with the dense blocks
  ``L_12, L_22, B_12, B_22`` of Sec. 3 and ``numpy.linalg.inv(L_22)``,
* Algorithm 2's initialisation: classical MDS (``numpy.linalg.eigh`` of the
  double-centred squared dissimilarities) and the orthogonal Procrustes fit
  (``numpy.linalg.svd``).

Readings of the paper taken here:

* stopping rule: Algorithm 1 prints ``sigma(X_t) - sigma(X_{t-1}) > eps``, which a
  descent method never satisfies; the loop continues while the *decrease*
  ``sigma(X_{t-1}) - sigma(X_t)`` exceeds the tolerance.  The tolerance is either
  the paper's normalised one (Remark eps: decrease of sigma/C(mn,2)) or relative
  (decrease / sigma(X_{t-1})).  A negative tolerance runs exactly ``max_iter``
  transforms.  The returned configuration is the last computed iterate.
* Eq. (B)'s diagonal sums over all off-diagonal entries of row i (the printed index
  range is a typo).
* General weights (Eq. W2) carry over to the out-of-sample problem: a new point in
  modality j has weight ``w_jj`` to the in-sample points of modality j and weight
  ``w_ij`` to the new point of modality i.  For Eq. (W) this is the paper's W^(o).
* Several new objects are independent problems (Sec. 3, last paragraph).
* Initialisation (Algorithm 2): the Procrustes fit of ``xi_i`` onto
  ``xi_0`` is ``xi_i V U'`` for ``xi_0' xi_i = U S V'`` (the printed ``xi_i U V'`` is
  the inverse rotation); cMDS eigenvectors get a sign convention (largest-magnitude
  entry positive).
* Relaxed updates (the Conclusion's suggested acceleration): ``X_t = X_{t-1} + r
  (L^+ B(X_{t-1}) X_{t-1} - X_{t-1})`` with ``0 <= r <= 2``, applied to the iterates as
  they are (no centring step: the plain transform's output is centred by itself, a
  relaxed one keeps ``(1 - r)`` times the previous iterate's column means).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "modified_weight_matrix",
    "omnibus_weights",
    "omnibus_dissimilarity",
    "laplacian",
    "pseudoinverse",
    "pairwise_distances",
    "guttman_B",
    "raw_stress",
    "EmbedResult",
    "jofc_embed",
    "guttman_step",
    "oos_blocks",
    "oos_stress",
    "OOSResult",
    "oos_embed",
    "continue_iterating",
    "modality_BX",
    "guttman_step_closed_form",
    "stress_blocks",
    "oos_step_closed_form",
    "oos_stress_direct",
    "oos_embed_closed_form",
]


# ---------------------------------------------------------------------------
# Weights and dissimilarities (Sec. 1.2.2 and Sec. 2.1)
# ---------------------------------------------------------------------------

def modified_weight_matrix(Wm: np.ndarray, n: int) -> np.ndarray:
    """The m x m matrix of Eq. (modW): diagonal ``n w_ii + sum_{j != i} w_ij``,
    off-diagonal ``-w_ij``."""
    Wm = np.asarray(Wm, dtype=np.float64)
    m = Wm.shape[0]
    M = -Wm.copy()
    for i in range(m):
        M[i, i] = n * Wm[i, i] + sum(Wm[i, j] for j in range(m) if j != i)
    return M


def omnibus_weights(Wm: np.ndarray, n: int) -> np.ndarray:
    """Dense mn x mn weight matrix of Eq. (W2): block (i,i) is ``w_ii (J_n - I_n)``,
    block (i,j) is ``w_ij I_n``.  With ``w_ii = 1`` and ``w_ij = w`` this is Eq. (W)."""
    Wm = np.asarray(Wm, dtype=np.float64)
    m = Wm.shape[0]
    W = np.zeros((m * n, m * n))
    J = np.ones((n, n))
    I = np.eye(n)
    for i in range(m):
        for j in range(m):
            blk = Wm[i, i] * (J - I) if i == j else Wm[i, j] * I
            W[i * n:(i + 1) * n, j * n:(j + 1) * n] = blk
    return W


def omnibus_dissimilarity(deltas: Sequence[np.ndarray]) -> np.ndarray:
    """Dense mn x mn omnibus dissimilarity of Eq. (jofcdelta): ``Delta_i`` on the
    diagonal blocks, the eta blocks elsewhere (0 on the matched diagonal; the NA
    entries carry weight 0, so any finite value works and 0 is stored)."""
    m = len(deltas)
    n = np.asarray(deltas[0]).shape[0]
    D = np.zeros((m * n, m * n))
    for i in range(m):
        D[i * n:(i + 1) * n, i * n:(i + 1) * n] = np.asarray(deltas[i], dtype=np.float64)
    return D


def laplacian(W: np.ndarray) -> np.ndarray:
    """Combinatorial Laplacian ``L = D - W`` with ``D_ii = sum_j W_ij``."""
    return np.diag(W.sum(axis=1)) - W


def pseudoinverse(L: np.ndarray) -> np.ndarray:
    """Moore-Penrose pseudoinverse of the symmetric Laplacian by SVD (``numpy.linalg.pinv``),
    with the rank-revealing cutoff N * eps * sigma_max.  The Laplacian of a connected
    JOFC weight graph has exactly one zero singular value (its null space is the constant
    vector, Prop. 1); numpy's default cutoff (1e-15 * sigma_max) can keep that singular
    value's rounding residue and return a wrong pseudoinverse."""
    N = L.shape[0]
    cut = N * np.finfo(np.float64).eps
    try:
        return np.linalg.pinv(L, rtol=cut, hermitian=True)
    except TypeError:                      # numpy < 2.0 names the cutoff rcond
        return np.linalg.pinv(L, rcond=cut, hermitian=True)


# ---------------------------------------------------------------------------
# Distances, B(X) and stress (Eq. B, Eq. stress)
# ---------------------------------------------------------------------------

def pairwise_distances(X: np.ndarray) -> np.ndarray:
    """``d_ij(X) = ||x_i - x_j||_2`` for all rows, by explicit differences."""
    X = np.asarray(X, dtype=np.float64)
    diff = X[:, None, :] - X[None, :, :]
    return np.sqrt(np.einsum("ijk,ijk->ij", diff, diff))


def guttman_B(X: np.ndarray, W: np.ndarray, Delta: np.ndarray) -> np.ndarray:
    """Eq. (B): off-diagonal ``-W_ij Delta_ij / d_ij(X)`` where ``d_ij != 0`` and 0
    where ``d_ij = 0``; diagonal = minus the sum of the row's off-diagonal entries."""
    D = pairwise_distances(X)
    N = D.shape[0]
    B = np.zeros((N, N))
    off = ~np.eye(N, dtype=bool)
    nz = off & (D != 0.0)
    B[nz] = -W[nz] * Delta[nz] / D[nz]
    B[np.diag_indices(N)] = -B.sum(axis=1)
    return B


def raw_stress(X: np.ndarray, W: np.ndarray, Delta: np.ndarray) -> float:
    """Raw stress ``sum_{i<j} W_ij (Delta_ij - d_ij(X))^2`` (Eq. stress written over
    the omnibus matrix, Sec. 1.2.2)."""
    D = pairwise_distances(X)
    iu = np.triu_indices(D.shape[0], k=1)
    return float(np.sum(W[iu] * (Delta[iu] - D[iu]) ** 2))


def continue_iterating(prev: float, cur: float, tol: float, tol_mode: str, n_pairs: int) -> bool:
    """Algorithm 1's loop test with the sign reading: keep going while the decrease
    exceeds the tolerance.  ``tol < 0`` never stops early."""
    if tol < 0:
        return True
    dec = prev - cur
    if tol_mode == "abs_normalized":          # Remark eps: sigma_N = sigma / C(nm, 2)
        return dec / n_pairs > tol
    if tol_mode == "relative":
        return dec > tol * prev
    raise ValueError(tol_mode)


# ---------------------------------------------------------------------------
# Algorithm 1 (JOFC with a dense pseudoinverse)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class EmbedResult:
    X: np.ndarray                 # final configuration, (m*n) x d
    iters: int                    # number of Guttman transforms applied
    stress: List[float]           # sigma(X_0), ..., sigma(X_iters)
    iterates: Optional[List[np.ndarray]] = None


def guttman_step(X: np.ndarray, Lp: np.ndarray, W: np.ndarray, Delta: np.ndarray) -> np.ndarray:
    """One Guttman transform ``L^+ B(X) X`` (Algorithm 1, loop body)."""
    return Lp @ (guttman_B(X, W, Delta) @ X)


def relaxed_step(X: np.ndarray, Lp: np.ndarray, W: np.ndarray, Delta: np.ndarray, relax: float) -> np.ndarray:
    """The relaxed update of iterative majorization that the paper names as the next
    acceleration of fJOFC (Conclusion, with de Leeuw and Heiser's relaxed updates):
    move from ``X`` towards the Guttman transform and ``relax`` times as far,
    ``X + relax (L^+ B(X) X - X)``.  ``relax = 1`` is the plain transform.  For
    ``0 <= relax <= 2`` the result stays inside the majorizing quadratic's level set of
    ``X`` (Eq. major: tau(., X) is a quadratic in the new configuration, minimised by
    the Guttman transform, and the relaxed point mirrors ``X`` about that minimiser at
    most), so the stress does not increase."""
    G = guttman_step(X, Lp, W, Delta)
    return X + relax * (G - X)


def jofc_embed(deltas: Sequence[np.ndarray], Wm: np.ndarray, X0: np.ndarray, max_iter: int,
               tol: float = -1.0, tol_mode: str = "relative", keep_iterates: bool = False,
               Lp: Optional[np.ndarray] = None, relax: float = 1.0) -> EmbedResult:
    """Algorithm 1 from a given ``X_0`` (its cMDS initialisation is not part of the
    loop): compute sigma(X_0); then repeat ``X_t = L^+ B(X_{t-1}) X_{t-1}`` (or, with
    ``relax != 1``, the relaxed update ``relaxed_step``) and sigma(X_t) until the
    stopping test fails or ``max_iter`` transforms are done."""
    m = len(deltas)
    n = np.asarray(deltas[0]).shape[0]
    W = omnibus_weights(Wm, n)
    Delta = omnibus_dissimilarity(deltas)
    if Lp is None:
        Lp = pseudoinverse(laplacian(W))
    X = np.array(X0, dtype=np.float64)
    n_pairs = (m * n) * (m * n - 1) // 2
    hist = [raw_stress(X, W, Delta)]
    its = [X.copy()] if keep_iterates else None
    t = 0
    while t < max_iter:
        X = guttman_step(X, Lp, W, Delta) if relax == 1.0 else relaxed_step(X, Lp, W, Delta, relax)
        t += 1
        hist.append(raw_stress(X, W, Delta))
        if keep_iterates:
            its.append(X.copy())
        if not continue_iterating(hist[-2], hist[-1], tol, tol_mode, n_pairs):
            break
    return EmbedResult(X=X, iters=t, stress=hist, iterates=its)


# ---------------------------------------------------------------------------
# Initialisation (Algorithm 2)
# ---------------------------------------------------------------------------

def cmds(D: np.ndarray, d: int) -> np.ndarray:
    """Classical MDS (Torgerson; the initialisation of Algorithm 1) of an n x n
    dissimilarity matrix: the double-centred matrix ``-1/2 J D^2 J`` (``J = I - 11'/n``, ``D^2`` elementwise)
    by ``numpy.linalg.eigh``, its d largest eigenpairs, coordinates ``v_k sqrt(max(l_k,
    0))``.  Sign convention (eigenvectors are defined up to sign): in every column the
    entry of largest magnitude is positive."""
    D = np.asarray(D, dtype=np.float64)
    n = D.shape[0]
    J = np.eye(n) - np.ones((n, n)) / n
    S = -0.5 * J @ (D * D) @ J
    lam, V = np.linalg.eigh(S)
    top = np.argsort(lam)[::-1][:d]
    xi = V[:, top] * np.sqrt(np.maximum(lam[top], 0.0))
    for k in range(xi.shape[1]):
        if xi[np.argmax(np.abs(xi[:, k])), k] < 0:
            xi[:, k] = -xi[:, k]
    return xi


def procrustes_fit(xi: np.ndarray, xi0: np.ndarray) -> np.ndarray:
    """The orthogonal Procrustes fit of ``xi`` onto ``xi0`` (Algorithm 2's Procrustes
    step): the rotation R (orthogonal d x d) minimising ||xi R - xi0||_F.  With ``T = xi0' xi =
    U S V'`` this is ``R = V U'``; the printed ``xi U V'`` is the inverse rotation (read
    as a transposition slip: the text asks for the fit of xi onto xi0)."""
    T = np.asarray(xi0, dtype=np.float64).T @ np.asarray(xi, dtype=np.float64)
    U, _, Vt = np.linalg.svd(T)
    return xi @ (Vt.T @ U.T)


def initial_configuration(deltas: Sequence[np.ndarray], d: int) -> np.ndarray:
    """Algorithm 2's initialisation: ``xi_0`` = cMDS of the average dissimilarity ``sum_i
    Delta_i / m``, centred; for every modality ``xi_i`` = cMDS of ``Delta_i``, centred,
    and ``X^(i)_(0)`` its Procrustes fit onto ``xi_0``; the rows stacked modality-major
    into the (m n) x d ``X_(0)``."""
    m = len(deltas)
    avg = sum(np.asarray(D, dtype=np.float64) for D in deltas) / m
    xi0 = cmds(avg, d)
    xi0 = xi0 - xi0.mean(0)
    blocks = []
    for D in deltas:
        xi = cmds(D, d)
        xi = xi - xi.mean(0)
        blocks.append(procrustes_fit(xi, xi0))
    return np.vstack(blocks)


# ---------------------------------------------------------------------------
# Out-of-sample embedding (Sec. 3)
# ---------------------------------------------------------------------------

def oos_blocks(X: np.ndarray, delta_new: np.ndarray, y: np.ndarray, Wm: np.ndarray):
    """Dense out-of-sample quantities for one new object.

    ``X`` is the (m*n) x d in-sample configuration, ``delta_new`` the m x n
    dissimilarities delta_j(k) of the new object to in-sample object k in modality j,
    ``y`` the m x d configuration of the new object.  Returns ``(Wo, Do, Xo)``: the
    (mn+m) x (mn+m) weight matrix W^(o) (in-sample points first, then y_1..y_m), the
    omnibus dissimilarity Delta^(o) in the same order and the stacked configuration.
    """
    Wm = np.asarray(Wm, dtype=np.float64)
    m = Wm.shape[0]
    n = X.shape[0] // m
    N = m * n + m
    Wo = np.zeros((N, N))
    Do = np.zeros((N, N))
    for j in range(m):
        rows = slice(j * n, (j + 1) * n)
        col = m * n + j
        Wo[rows, col] = Wm[j, j]
        Wo[col, rows] = Wm[j, j]
        Do[rows, col] = delta_new[j]
        Do[col, rows] = delta_new[j]
        for i in range(m):
            if i != j:
                Wo[m * n + i, col] = Wm[i, j]      # matched new points: Delta = 0
    Xo = np.vstack([X, y])
    return Wo, Do, Xo


def oos_stress(X: np.ndarray, delta_new: np.ndarray, y: np.ndarray, Wm: np.ndarray) -> float:
    """Eq. (joos) as the omnibus double sum ``sum_{i<j} W^(o)_ij (Delta^(o)_ij - d_ij)^2``."""
    Wo, Do, Xo = oos_blocks(X, delta_new, y, Wm)
    return raw_stress(Xo, Wo, Do)


@dataclasses.dataclass
class OOSResult:
    y: np.ndarray                 # m x d
    iters: int
    stress: List[float]


def oos_step(X: np.ndarray, delta_new: np.ndarray, y: np.ndarray, Wm: np.ndarray) -> np.ndarray:
    """Eq. (joosupdate): ``y_t = L22^+ (B12^T - L12^T) X + L22^+ B22 y_{t-1}`` with the
    blocks of the Laplacian of W^(o) and of B(X^(o)) (Eq. B), L22 inverted by
    ``numpy.linalg.inv`` (it is non-singular when every ``w_jj > 0``)."""
    m = np.asarray(Wm).shape[0]
    mn = X.shape[0]
    Wo, Do, Xo = oos_blocks(X, delta_new, y, Wm)
    Lo = laplacian(Wo)
    Bo = guttman_B(Xo, Wo, Do)
    L12, L22 = Lo[:mn, mn:], Lo[mn:, mn:]
    B12, B22 = Bo[:mn, mn:], Bo[mn:, mn:]
    L22inv = np.linalg.inv(L22)
    return L22inv @ ((B12.T - L12.T) @ X) + L22inv @ (B22 @ y)


def oos_embed(X: np.ndarray, delta_new: np.ndarray, y0: np.ndarray, Wm: np.ndarray,
              max_iter: int, tol: float = -1.0, tol_mode: str = "relative") -> OOSResult:
    """Out-of-sample procedure of Sec. 3 for one new object from ``y0``."""
    y = np.array(y0, dtype=np.float64)
    m = y.shape[0]
    hist = [oos_stress(X, delta_new, y, Wm)]
    # weighted terms of Eq. (joos): m*n fidelity distances + C(m,2) commensurability ones
    n_pairs = X.shape[0] + m * (m - 1) // 2
    t = 0
    while t < max_iter:
        y = oos_step(X, delta_new, y, Wm)
        t += 1
        hist.append(oos_stress(X, delta_new, y, Wm))
        if not continue_iterating(hist[-2], hist[-1], tol, tol_mode, n_pairs):
            break
    return OOSResult(y=y, iters=t, stress=hist)


# ---------------------------------------------------------------------------
# Large-n forms used to check full-size runs.  Both are pinned against the dense
# definitions above at small sizes (tests/test_oracle_pins.py).
# ---------------------------------------------------------------------------

def modality_BX(delta: np.ndarray, Xl: np.ndarray, w_ll: float = 1.0, row_block: int = 1024) -> np.ndarray:
    """The diagonal block B_l X^(l) of B(X) X (Eq. B restricted to modality l, whose only
    non-zero weights are w_ll on the off-diagonal pairs), in float64 by row blocks:
    (B_l X)_i = sum_{j != i, d_ij != 0} w_ll Delta_ij / d_ij (x_i - x_j)."""
    Xl = np.asarray(Xl, dtype=np.float64)
    n = Xl.shape[0]
    out = np.zeros_like(Xl)
    for a in range(0, n, row_block):
        blk = slice(a, min(n, a + row_block))
        diff = Xl[blk, None, :] - Xl[None, :, :]
        dist = np.sqrt(np.einsum("ijk,ijk->ij", diff, diff))
        coef = np.zeros_like(dist)
        nz = dist != 0.0
        idx = np.arange(blk.start, blk.stop)
        nz[np.arange(len(idx)), idx] = False
        coef[nz] = w_ll * np.asarray(delta, dtype=np.float64)[blk][nz] / dist[nz]
        out[blk] = np.einsum("ij,ijk->ik", coef, diff)
    return out


def guttman_step_closed_form(deltas: Sequence[np.ndarray], Wm: np.ndarray, X: np.ndarray) -> np.ndarray:
    """One Guttman transform L^+ B(X) X with L^+ written as in Cor. 1 (Appendix A):
    L^+ = Wmod^-1 (x) I_n + [Z - J_m/(mn)] (x) J_n,
    Z = -(Wmod + n(J_m/(mn) - diag w_ii))^-1 (J_m/(mn) - diag w_ii) Wmod^-1,
    applied to the block-diagonal B(X) X (the J_n term is kept, not assumed zero)."""
    Wm = np.asarray(Wm, dtype=np.float64)
    m = Wm.shape[0]
    n = X.shape[0] // m
    BX = [modality_BX(deltas[l], X[l * n:(l + 1) * n], Wm[l, l]) for l in range(m)]
    Wmod = modified_weight_matrix(Wm, n)
    Winv = np.linalg.inv(Wmod)
    Jm = np.ones((m, m))
    dw = np.diag(np.diag(Wm))
    Z = -np.linalg.inv(Wmod + n * (Jm / (m * n) - dw)) @ (Jm / (m * n) - dw) @ Winv - Jm / (m * n)
    colsum = [b.sum(axis=0) for b in BX]
    out = np.zeros_like(np.asarray(X, dtype=np.float64))
    for j in range(m):
        blk = sum(Winv[j, l] * BX[l] for l in range(m))
        blk = blk + sum(Z[j, l] * colsum[l] for l in range(m))[None, :]
        out[j * n:(j + 1) * n] = blk
    return out


def guttman_rows(delta_rows: Sequence[np.ndarray], Wm: np.ndarray, X: np.ndarray, idx) -> np.ndarray:
    """Rows ``idx`` of one Guttman transform L^+ B(X) X, for every modality, from the Delta
    rows of those objects only (for problems too large for the dense step).

    Eq. (update) / Cor. 1: row i of modality j is sum_l [Wmod^-1]_{jl} (B_l X^(l))_i with
    (B_l X^(l))_i = sum_{j' != i, d != 0} w_ll Delta_l[i, j'] / d_ij' (x_i - x_j') (Eq. B).
    The Z (x) J_n part of Cor. 1 adds sum_l Z_jl 1^T B_l X^(l), which is zero because every
    column of B_l sums to zero (Sec. 2.1), so it is left out here; the test of this
    function checks that claim against the full closed-form step.
    ``delta_rows[l]`` is len(idx) x n (row a holds Delta_l[idx[a], :]).  Returns an
    (m, len(idx), d) float64 array."""
    Wm = np.asarray(Wm, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    m = Wm.shape[0]
    n = X.shape[0] // m
    idx = np.asarray(idx)
    Winv = np.linalg.inv(modified_weight_matrix(Wm, n))
    BX = np.zeros((m, len(idx), X.shape[1]))
    for l in range(m):
        Xl = X[l * n:(l + 1) * n]
        for a, i in enumerate(idx):
            diff = Xl[i][None, :] - Xl
            dist = np.sqrt(np.einsum("jk,jk->j", diff, diff))
            coef = np.zeros(n)
            nz = dist != 0.0
            nz[i] = False
            coef[nz] = Wm[l, l] * np.asarray(delta_rows[l][a], dtype=np.float64)[nz] / dist[nz]
            BX[l, a] = coef @ diff
    return np.einsum("jl,lak->jak", Winv, BX)


def stress_blocks(deltas: Sequence[np.ndarray], Wm: np.ndarray, X: np.ndarray, row_block: int = 1024) -> float:
    """Eq. (stress) summed block by block: sum_l w_ll sum_{i<j} (Delta_l,ij - d_ij(X^(l)))^2
    + sum_{i<j} w_ij ||X^(i) - X^(j)||_F^2 (the omnibus double sum restricted to its
    non-zero weights), in float64 for large n."""
    Wm = np.asarray(Wm, dtype=np.float64)
    m = Wm.shape[0]
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0] // m
    tot = 0.0
    for l in range(m):
        Xl = X[l * n:(l + 1) * n]
        Dl = np.asarray(deltas[l], dtype=np.float64)
        for a in range(0, n, row_block):
            b = min(n, a + row_block)
            diff = Xl[a:b, None, :] - Xl[None, :, :]
            dist = np.sqrt(np.einsum("ijk,ijk->ij", diff, diff))
            mask = np.arange(n)[None, :] > np.arange(a, b)[:, None]
            tot += Wm[l, l] * float(np.sum(((Dl[a:b] - dist) ** 2)[mask]))
    for i in range(m):
        for j in range(i + 1, m):
            tot += Wm[i, j] * float(np.sum((X[i * n:(i + 1) * n] - X[j * n:(j + 1) * n]) ** 2))
    return tot


def oos_step_closed_form(X: np.ndarray, delta_new: np.ndarray, y: np.ndarray, Wm: np.ndarray) -> np.ndarray:
    """The O(nmd) out-of-sample update of Sec. 3 with general weights:
    xi_j = w_jj sum_k (1 - delta_j(k)/d_jk) X^(j)_k, psi_j = w_jj sum_k delta_j(k)/d_jk (terms
    with d_jk = 0 contribute X^(j)_k to xi_j and nothing to psi_j, Eq. B), and
    y_t = L22^-1 (xi + psi o y_{t-1}) with L22 the modified weight matrix of Eq. (modW)."""
    Wm = np.asarray(Wm, dtype=np.float64)
    m = Wm.shape[0]
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0] // m
    y = np.asarray(y, dtype=np.float64)
    xi = np.zeros_like(y)
    psi = np.zeros(m)
    for j in range(m):
        Xj = X[j * n:(j + 1) * n]
        dist = np.sqrt(np.sum((Xj - y[j]) ** 2, axis=1))
        ratio = np.zeros(n)
        nz = dist != 0.0
        ratio[nz] = np.asarray(delta_new[j], dtype=np.float64)[nz] / dist[nz]
        xi[j] = Wm[j, j] * ((1.0 - ratio)[:, None] * Xj).sum(axis=0)
        psi[j] = Wm[j, j] * ratio.sum()
    return np.linalg.inv(modified_weight_matrix(Wm, n)) @ (xi + psi[:, None] * y)


def oos_stress_direct(X: np.ndarray, delta_new: np.ndarray, y: np.ndarray, Wm: np.ndarray) -> float:
    """Eq. (joos) with general weights, summed directly."""
    Wm = np.asarray(Wm, dtype=np.float64)
    m = Wm.shape[0]
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0] // m
    y = np.asarray(y, dtype=np.float64)
    s = 0.0
    for j in range(m):
        dist = np.sqrt(np.sum((X[j * n:(j + 1) * n] - y[j]) ** 2, axis=1))
        s += Wm[j, j] * float(np.sum((np.asarray(delta_new[j], dtype=np.float64) - dist) ** 2))
    for i in range(m):
        for j in range(i + 1, m):
            s += Wm[i, j] * float(np.sum((y[i] - y[j]) ** 2))
    return s


def oos_embed_closed_form(X, delta_new, y0, Wm, max_iter: int, tol: float = -1.0,
                          tol_mode: str = "relative") -> OOSResult:
    """The out-of-sample loop with the O(nmd) update and direct stress (for large n)."""
    y = np.array(y0, dtype=np.float64)
    m = y.shape[0]
    n = np.asarray(X).shape[0] // m
    hist = [oos_stress_direct(X, delta_new, y, Wm)]
    n_pairs = m * n + m * (m - 1) // 2
    t = 0
    while t < max_iter:
        y = oos_step_closed_form(X, delta_new, y, Wm)
        t += 1
        hist.append(oos_stress_direct(X, delta_new, y, Wm))
        if not continue_iterating(hist[-2], hist[-1], tol, tol_mode, n_pairs):
            break
    return OOSResult(y=y, iters=t, stress=hist)
