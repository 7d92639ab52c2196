"""The parity rule every GPU parity test applies (one rule, one place).

The device computes in float32, the oracle in float64 on the same float32-rounded
inputs.  After T Guttman transforms (Algorithm 1's loop, Eq. update):

* X: relative Frobenius error ``X_TOL`` = 1e-5 (per object for the out-of-sample
  update, Eq. joosupdate).
* stress (Eq. stress, Eq. joos): ``S_TOL`` = 1e-6 relative, plus the error that float32
  distances put into the fidelity sum whatever the summation does.  The device's
  distance ``d' = d^2' rsqrt(d^2')`` carries a relative error ``|e| <= eps_d``: the
  hardware reciprocal square root (relative error at most 2^-22.9, the PTX ISA's bound
  for ``rsqrt.approx.f32``), the rounding of the squared distance (the coordinate
  differences, 2^-24 each, so 2^-23 on each square, and the d fused multiply-adds that
  sum the squares: at most (d + 2) 2^-24 on d^2, half of that on d) and the scaling of
  the coordinates into Delta's stored units (2^-25): ``eps_d = 2^-22.9 + (d + 3) 2^-25``
  (the residual d' - Delta is one fused multiply-add, whose rounding is relative to
  the residual itself and sits inside S_TOL).  A fidelity term then moves by
  ``|(Delta - d')^2 - (Delta - d)^2| <=
  2 |Delta - d| eps_d d + (eps_d d)^2``, so the stress tolerance is
  ``S_TOL sigma + sum_l w_ll sum_{i<j} (2 |Delta_ij - d_ij| eps_d d_ij + (eps_d d_ij)^2)``.
  For the workloads' residuals the added term is far below ``S_TOL sigma`` (the rule is
  the flat 1e-6 there); it matters where sigma is near zero (exact configurations).
"""
import numpy as np

X_TOL = 1e-5
S_TOL = 1e-6
RSQRT_REL = 2.0 ** -22.9


def distance_eps(d: int) -> float:
    """Bound of the relative error of one float32 distance in d dimensions."""
    return RSQRT_REL + (int(d) + 3) * 2.0 ** -25


def rel_fro(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _pair_bound(delta_block, dist, eps):
    return float(np.sum(2.0 * np.abs(delta_block - dist) * eps * dist + (eps * dist) ** 2))


def fidelity_bound(deltas, W, X, row_block: int = 1024) -> float:
    """sum_l w_ll sum_{i<j} (2 |Delta - d| eps_d d + (eps_d d)^2) at configuration X."""
    X = np.asarray(X, np.float64)
    W = np.asarray(W, np.float64)
    m = len(deltas)
    n = X.shape[0] // m
    eps = distance_eps(X.shape[1])
    tot = 0.0
    for l in range(m):
        Xl = X[l * n:(l + 1) * n]
        Dl = np.asarray(deltas[l], np.float64)
        for a in range(0, n, row_block):
            b = min(n, a + row_block)
            diff = Xl[a:b, None, :] - Xl[None, :, :]
            dist = np.sqrt(np.einsum("ijk,ijk->ij", diff, diff))
            mask = np.arange(n)[None, :] > np.arange(a, b)[:, None]
            tot += W[l, l] * _pair_bound(Dl[a:b][mask], dist[mask], eps)
    return tot


def stress_tol(sigma: float, deltas, W, X) -> float:
    return S_TOL * abs(sigma) + fidelity_bound(deltas, W, X)


def assert_stress(got: float, want: float, deltas, W, X, where=""):
    """|got - want| within the rule, the bound taken at configuration X."""
    tol = stress_tol(want, deltas, W, X)
    assert abs(got - want) <= tol, (where, got, want, tol)


def assert_history(got, want, deltas, W, iterates, where=""):
    """Every sigma(X_t) of a run against the oracle's, the bound taken at the oracle's
    iterate X_t."""
    got = np.asarray(got, np.float64)
    assert len(got) == len(want), (where, len(got), len(want))
    for t, (g, w, Xt) in enumerate(zip(got, want, iterates)):
        assert_stress(g, w, deltas, W, Xt, (where, t))


def oos_stress_tol(sigma: float, X, delta_o, y, W) -> float:
    """The rule for one new object's out-of-sample stress (Eq. joos): the fidelity terms
    are its m n distances to the in-sample points."""
    X = np.asarray(X, np.float64)
    W = np.asarray(W, np.float64)
    y = np.asarray(y, np.float64)
    m, d = y.shape
    n = X.shape[0] // m
    eps = distance_eps(d)
    tot = 0.0
    for j in range(m):
        dist = np.sqrt(((X[j * n:(j + 1) * n] - y[j][None, :]) ** 2).sum(-1))
        tot += W[j, j] * _pair_bound(np.asarray(delta_o[j], np.float64), dist, eps)
    return S_TOL * abs(sigma) + tot
