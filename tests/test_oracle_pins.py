"""Pins of the float64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the paper's
printed closed forms (hand-evaluated golden values and the general formulas of
Sec. 2.1 / Appendix A), the paper's fast update (Eq. update) and out-of-sample
simplification (Sec. 3), textbook SMACOF for m = 1, exact identities (Eq. stress,
Eq. comm, Remark faststress), the majorization guarantee, exact-configuration fixed
points and invariances.  All run on the CPU in a few seconds.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import fjofc_oracle as O
import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        rows.append(line.split())
    return rows


def _eqW(m, w):
    return synthetic.weights_matrix(m, 1.0, w)


def _lp(Wm, n):
    return O.pseudoinverse(O.laplacian(O.omnibus_weights(Wm, n)))


def _rand_sym_weights(rng, m, lo=0.2, hi=2.0):
    A = rng.uniform(lo, hi, size=(m, m))
    return np.triu(A) + np.triu(A, 1).T


# ---------------------------------------------------------------- closed forms

def test_golden_closed_forms_pin_pinv_and_L22():
    """The oracle's pinv(L) (built from Eq. W) splits as Winv (x) I_n + Z (x) J_n with the
    hand-evaluated Eq. (W1inv) and J-coefficient values; inv(L22) of the oracle's
    out-of-sample blocks equals the printed L22^+ (Sec. 3)."""
    for row in _golden():
        name = row[0]
        if name in ("Winv_eqW", "Z_eqW"):
            m, n, w = int(row[1]), int(row[2]), float(row[3])
            diag, off = float(Fraction(row[4])), float(Fraction(row[5]))
            Lp = _lp(_eqW(m, w), n)
            # Winv (x) I_n + Z (x) J_n: block (a,b) entry (0,0) = Winv_ab + Z_ab, entry (0,1) = Z_ab
            Zo = Lp[0:n * m:n, 1:n * m:n]                  # (a,b) -> entry (a*n, b*n+1)
            Wo = Lp[0:n * m:n, 0:n * m:n] - Zo
            got = Wo if name == "Winv_eqW" else Zo
            exp = np.full((m, m), off)
            np.fill_diagonal(exp, diag)
            np.testing.assert_allclose(got, exp, rtol=1e-10, atol=1e-13)
        elif name == "L22inv":
            m, n, w = int(row[1]), int(row[2]), float(row[3])
            diag, off = float(Fraction(row[4])), float(Fraction(row[5]))
            rng = np.random.default_rng(1)
            X = rng.standard_normal((m * n, 2))
            Wo, Do, Xo = O.oos_blocks(X, rng.uniform(1, 2, (m, n)), rng.standard_normal((m, 2)), _eqW(m, w))
            L22 = O.laplacian(Wo)[m * n:, m * n:]
            exp = np.full((m, m), off)
            np.fill_diagonal(exp, diag)
            np.testing.assert_allclose(np.linalg.inv(L22), exp, rtol=1e-12)
        elif name == "W3inv":
            n, w11, w22 = int(row[1]), float(row[2]), float(row[3])
            Wm = np.array([[w11, w11 * w22], [w11 * w22, w22]])
            exp = np.array([[Fraction(row[4]), Fraction(row[5])], [Fraction(row[5]), Fraction(row[6])]], dtype=float)
            np.testing.assert_allclose(np.linalg.inv(O.modified_weight_matrix(Wm, n)), exp, rtol=1e-13)
            # and W3 Laplacian: pinv(L) restricted to the I_n part carries the same Winv
            Lp = _lp(Wm, n)
            Zo = Lp[0:2 * n:n, 1:2 * n:n]
            np.testing.assert_allclose(Lp[0:2 * n:n, 0:2 * n:n] - Zo, exp, rtol=1e-10, atol=1e-13)
        else:
            raise AssertionError(name)


@pytest.mark.parametrize("m,n", [(2, 3), (3, 4), (4, 5), (2, 9)])
def test_corollary1_general_weights(m, n):
    """Cor. 1 / Thm 1 (Appendix A) for random Eq. (W2) weights: pinv(L) equals
    Winv (x) I_n + [Z - J_m/(mn)] (x) J_n; Prop. 1: pinv(L) = inv(L + J/mn) - J/mn;
    and L = Wmod (x) I_n - diag(w_ii) (x) J_n."""
    rng = np.random.default_rng(100 + m * 10 + n)
    Wm = _rand_sym_weights(rng, m)
    L = O.laplacian(O.omnibus_weights(Wm, n))
    Lp = O.pseudoinverse(L)
    Wmod = O.modified_weight_matrix(Wm, n)
    Jm = np.ones((m, m))
    dw = np.diag(np.diag(Wm))
    np.testing.assert_allclose(L, np.kron(Wmod, np.eye(n)) - np.kron(dw, np.ones((n, n))), atol=1e-13)
    Winv = np.linalg.inv(Wmod)
    Zm = -np.linalg.inv(Wmod + n * (Jm / (m * n) - dw)) @ (Jm / (m * n) - dw) @ Winv - Jm / (m * n)
    np.testing.assert_allclose(Lp, np.kron(Winv, np.eye(n)) + np.kron(Zm, np.ones((n, n))), atol=1e-12)
    N = m * n
    np.testing.assert_allclose(Lp, np.linalg.inv(L + np.ones((N, N)) / N) - np.ones((N, N)) / N, atol=1e-12)


def test_woodbury_kronecker_identity():
    """Remark after Eq. (W1inv): (A (x) I_n + B (x) J_n)^-1 = A^-1 (x) I_n - (A + nB)^-1 B A^-1 (x) J_n,
    checked on the oracle's L + J/mn for random weights."""
    rng = np.random.default_rng(5)
    m, n = 3, 6
    Wm = _rand_sym_weights(rng, m)
    L = O.laplacian(O.omnibus_weights(Wm, n))
    A = O.modified_weight_matrix(Wm, n)
    Bm = np.ones((m, m)) / (m * n) - np.diag(np.diag(Wm))
    lhs = np.linalg.inv(L + np.ones((m * n, m * n)) / (m * n))
    Ai = np.linalg.inv(A)
    rhs = np.kron(Ai, np.eye(n)) - np.kron(np.linalg.inv(A + n * Bm) @ Bm @ Ai, np.ones((n, n)))
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


# ---------------------------------------------------------------- the Guttman step

def _small_problem(m=2, n=12, d=2, seed=3, w=0.5):
    prob = synthetic.make_insample(0, n=n, m=m, d=d, seed=seed, w_comm=w)
    return prob.deltas, prob.W, prob.X0


@pytest.mark.parametrize("m,n,d,w", [(2, 12, 2, 0.5), (3, 9, 3, 2.0), (4, 7, 1, 0.1)])
def test_fast_update_equals_dense_step(m, n, d, w):
    """Eq. (update) with the reading of Algorithm 2's coefficient typo: the oracle's
    pinv(L) B(X) X equals (1/(n+mw)) B_j X^(j) + (w/(n(n+mw))) sum_l B_l X^(l), with the
    B_l the diagonal blocks of B(X) built from a plain per-modality loop."""
    deltas, Wm, X = _small_problem(m, n, d, seed=10 + m, w=w)
    W = O.omnibus_weights(Wm, n)
    D = O.omnibus_dissimilarity(deltas)
    Xn = O.guttman_step(X, _lp(Wm, n), W, D)
    # per-modality B_l X^(l) by loops over pairs (fidelity weight 1)
    BX = []
    for l in range(m):
        Xl = X[l * n:(l + 1) * n]
        out = np.zeros_like(Xl)
        for i in range(n):
            for j in range(n):
                if i == j:
                    continue
                dij = np.linalg.norm(Xl[i] - Xl[j])
                if dij > 0:
                    out[i] += deltas[l][i, j] / dij * (Xl[i] - Xl[j])
        BX.append(out)
    S = sum(BX)
    for j in range(m):
        exp = BX[j] / (n + m * w) + w / (n * (n + m * w)) * S
        np.testing.assert_allclose(Xn[j * n:(j + 1) * n], exp, rtol=1e-11, atol=1e-12)


def test_B_structure():
    """B(X) is block diagonal with zero row and column sums (Sec. 2.2)."""
    deltas, Wm, X = _small_problem(3, 8, 2)
    n, m = 8, 3
    B = O.guttman_B(X, O.omnibus_weights(Wm, n), O.omnibus_dissimilarity(deltas))
    np.testing.assert_allclose(B.sum(0), 0, atol=1e-12)
    np.testing.assert_allclose(B.sum(1), 0, atol=1e-12)
    for a in range(m):
        for b in range(m):
            if a != b:
                assert np.all(B[a * n:(a + 1) * n, b * n:(b + 1) * n] == 0)


def test_zero_distance_rule():
    """Eq. (B) sets b_ij = 0 when d_ij = 0: two coincident points do not pull each other."""
    deltas, Wm, X = _small_problem(2, 6, 2)
    X = X.copy()
    X[1] = X[0]
    W = O.omnibus_weights(Wm, 6)
    B = O.guttman_B(X, W, O.omnibus_dissimilarity(deltas))
    assert B[0, 1] == 0 and B[1, 0] == 0
    assert np.all(np.isfinite(B))


def test_m1_is_textbook_smacof():
    """m = 1: the Guttman transform is the unit-weight SMACOF update X <- n^-1 B(X) X
    (Borg & Groenen, Ch. 8), written here as an explicit loop."""
    deltas, Wm, X = _small_problem(1, 10, 2, seed=4)
    n = 10
    Wm = np.array([[1.0]])
    Xn = O.guttman_step(X, _lp(Wm, n), O.omnibus_weights(Wm, n), O.omnibus_dissimilarity(deltas))
    exp = np.zeros_like(X)
    for i in range(n):
        for j in range(n):
            if i != j:
                dij = np.sqrt(np.sum((X[i] - X[j]) ** 2))
                exp[i] += deltas[0][i, j] / dij * (X[i] - X[j])
    np.testing.assert_allclose(Xn, exp / n, rtol=1e-12, atol=1e-13)


def test_commensurability_weight_extremes():
    """Sec. 1.2.1 on the weight w of Eq. W: w = 0 embeds every Delta_i on its own (each
    block of one transform is the unit-weight SMACOF update of its modality, written as
    an explicit loop), and a large w forces the modalities' configurations together
    (after one transform the blocks differ by O(1/w))."""
    m, n, d = 2, 9, 2
    deltas, _, X = _small_problem(m, n, d, seed=12)
    D = O.omnibus_dissimilarity(deltas)
    W0 = _eqW(m, 0.0)
    Xn = O.guttman_step(X, _lp(W0, n), O.omnibus_weights(W0, n), D)
    for l in range(m):
        Xl = X[l * n:(l + 1) * n]
        exp = np.zeros_like(Xl)
        for i in range(n):
            for j in range(n):
                if i != j:
                    dij = np.sqrt(np.sum((Xl[i] - Xl[j]) ** 2))
                    exp[i] += deltas[l][i, j] / dij * (Xl[i] - Xl[j])
        # w = 0 leaves the blocks disconnected: L^+ acts per block, and each block of
        # B(X) X is centred, so the step is the per-modality update
        np.testing.assert_allclose(Xn[l * n:(l + 1) * n], exp / n, rtol=1e-10, atol=1e-12)
    gaps = []
    for w in (1e2, 1e4):
        Ww = _eqW(m, w)
        Xw = O.guttman_step(X, _lp(Ww, n), O.omnibus_weights(Ww, n), D)
        gaps.append(np.linalg.norm(Xw[:n] - Xw[n:]) / np.linalg.norm(Xw))
    assert gaps[1] < 1e-3 and 0.5e2 < gaps[0] / gaps[1] < 2e2, gaps


# ---------------------------------------------------------------- stress identities

def test_stress_identity_and_majorizer():
    """sigma(X) = sum W Delta^2 + tr X'LX - 2 tr X'B(X)X (Sec. 1.2.2) and the majorizer of
    Eq. (major) bounds sigma(Y) from above for a Y other than X."""
    deltas, Wm, X = _small_problem(2, 10, 2, seed=8)
    n = 10
    W = O.omnibus_weights(Wm, n)
    D = O.omnibus_dissimilarity(deltas)
    L = O.laplacian(W)
    iu = np.triu_indices(2 * n, 1)
    c = np.sum(W[iu] * D[iu] ** 2)
    s = O.raw_stress(X, W, D)
    np.testing.assert_allclose(s, c + np.trace(X.T @ L @ X) - 2 * np.trace(X.T @ O.guttman_B(X, W, D) @ X), rtol=1e-12)
    rng = np.random.default_rng(0)
    for _ in range(5):
        Y = X + 0.3 * rng.standard_normal(X.shape)
        major = c + np.trace(Y.T @ L @ Y) - 2 * np.trace(Y.T @ O.guttman_B(X, W, D) @ X)
        assert O.raw_stress(Y, W, D) <= major + 1e-10


@pytest.mark.parametrize("m,w", [(2, 0.5), (3, 1.5)])
def test_faststress_and_commensurability_identities(m, w):
    """Remark faststress: the omnibus stress equals half the Frobenius fidelity plus
    w times commensurability; Eq. (comm): commensurability = m sum_i ||X^(i) - Xbar||^2."""
    n = 9
    deltas, Wm, X = _small_problem(m, n, 3, seed=20 + m, w=w)
    W = O.omnibus_weights(Wm, n)
    D = O.omnibus_dissimilarity(deltas)
    fid = 0.0
    for i in range(m):
        Xi = X[i * n:(i + 1) * n]
        Di = np.sqrt(((Xi[:, None, :] - Xi[None, :, :]) ** 2).sum(-1))
        fid += 0.5 * np.sum((deltas[i] - Di) ** 2)
    comm = sum(np.sum((X[i * n:(i + 1) * n] - X[j * n:(j + 1) * n]) ** 2)
               for i in range(m) for j in range(i + 1, m))
    np.testing.assert_allclose(O.raw_stress(X, W, D), fid + w * comm, rtol=1e-12)
    Xbar = sum(X[i * n:(i + 1) * n] for i in range(m)) / m
    np.testing.assert_allclose(comm, m * sum(np.sum((X[i * n:(i + 1) * n] - Xbar) ** 2) for i in range(m)), rtol=1e-12)


# ---------------------------------------------------------------- the loop

def test_monotone_descent_and_centering():
    """Majorization guarantees non-increasing stress (Sec. 1.2.2, Sec. 5); every
    Guttman output is centred (Sec. 1.2.2)."""
    deltas, Wm, X0 = _small_problem(2, 20, 2, seed=30)
    res = O.jofc_embed(deltas, Wm, X0, max_iter=60, keep_iterates=True)
    s = np.array(res.stress)
    assert np.all(np.diff(s) <= 1e-12 * s[:-1])
    assert s[-1] < s[0]
    for Xt in res.iterates[1:]:
        np.testing.assert_allclose(Xt.mean(0), 0, atol=1e-12)


@pytest.mark.parametrize("m,w", [(2, 0.5), (3, 1.2)])
def test_relaxed_update_stays_in_the_majorizer_level_set(m, w):
    """Relaxed updates (the Conclusion's suggested acceleration): tau(., X) of Eq. (major)
    is a quadratic in the new configuration minimised by the Guttman transform G, so at
    X + r (G - X) it equals tau(G, X) + (1 - r)^2 (sigma(X) - tau(G, X)), and
    sigma(X_r) <= tau(X_r, X) <= sigma(X) exactly when 0 <= r <= 2."""
    n = 11
    deltas, Wm, X = _small_problem(m, n, 2, seed=40 + m, w=w)
    W = O.omnibus_weights(Wm, n)
    D = O.omnibus_dissimilarity(deltas)
    L = O.laplacian(W)
    Lp = _lp(Wm, n)
    BX = O.guttman_B(X, W, D) @ X
    iu = np.triu_indices(m * n, 1)
    c = np.sum(W[iu] * D[iu] ** 2)

    def tau(Y):
        return c + np.trace(Y.T @ L @ Y) - 2 * np.trace(Y.T @ BX)

    sX = O.raw_stress(X, W, D)
    np.testing.assert_allclose(tau(X), sX, rtol=1e-12)
    G = O.guttman_step(X, Lp, W, D)
    tG = tau(G)
    for r in (0.0, 0.5, 1.0, 1.5, 2.0, 2.5):
        Xr = O.relaxed_step(X, Lp, W, D, r)
        np.testing.assert_allclose(tau(Xr), tG + (1 - r) ** 2 * (sX - tG), rtol=1e-10, atol=1e-10 * sX)
        if r <= 2.0:
            assert O.raw_stress(Xr, W, D) <= tau(Xr) + 1e-10 * sX
            assert tau(Xr) <= sX + 1e-10 * sX
        else:
            assert tau(Xr) > sX


def test_relaxed_loop_descends_keeps_fixed_points_and_r0_stays():
    """With 0 < r <= 2 the relaxed loop's stress never increases; r = 0 leaves X_0 in
    place; a zero-stress configuration is a fixed point of the relaxed map too."""
    deltas, Wm, X0 = _small_problem(2, 20, 2, seed=31)
    for r in (1.5, 1.9, 2.0):
        res = O.jofc_embed(deltas, Wm, X0, max_iter=60, relax=r)
        st = np.array(res.stress)
        assert np.all(np.diff(st) <= 1e-12 * st[:-1]), r
        assert st[-1] < st[0]
    res0 = O.jofc_embed(deltas, Wm, X0, max_iter=5, relax=0.0)
    np.testing.assert_array_equal(res0.X, X0)
    rng = np.random.default_rng(12)
    n = 12
    Y = rng.standard_normal((n, 2))
    Y -= Y.mean(0)
    Dy = np.sqrt(((Y[:, None] - Y[None]) ** 2).sum(-1))
    Wm2 = _eqW(2, 0.5)
    X = np.vstack([Y, Y])
    W = O.omnibus_weights(Wm2, n)
    D = O.omnibus_dissimilarity([Dy, Dy])
    np.testing.assert_allclose(O.relaxed_step(X, _lp(Wm2, n), W, D, 1.7), X, atol=1e-12)


def test_cmds_recovers_a_euclidean_configuration():
    """Torgerson's theorem: cMDS of the distance matrix of a centred Y in R^d returns Y up
    to an orthogonal transform (equal Gram matrices), centred, with the eigenvalues the
    squared singular values of Y; cMDS to fewer dimensions keeps the d' leading ones."""
    rng = np.random.default_rng(5)
    n, d = 30, 3
    Y = rng.standard_normal((n, d)) @ np.diag([3.0, 2.0, 1.0])
    Y -= Y.mean(0)
    D = np.sqrt(((Y[:, None] - Y[None]) ** 2).sum(-1))
    xi = O.cmds(D, d)
    np.testing.assert_allclose(xi @ xi.T, Y @ Y.T, atol=1e-9)
    np.testing.assert_allclose(xi.mean(0), 0, atol=1e-12)
    np.testing.assert_allclose(np.sort((xi ** 2).sum(0))[::-1], np.linalg.svd(Y, compute_uv=False) ** 2, rtol=1e-9)
    U, sv, Vt = np.linalg.svd(Y, full_matrices=False)
    np.testing.assert_allclose(np.abs(O.cmds(D, 1)[:, 0]), np.abs(U[:, 0] * sv[0]), atol=1e-9)
    k = np.argmax(np.abs(xi), axis=0)
    assert np.all(xi[k, np.arange(d)] > 0)


def test_procrustes_fit_undoes_a_rotation():
    """The fit of xi = xi0 Q (Q orthogonal, a reflection included) onto xi0 is xi0 itself;
    the printed xi U V' (the inverse rotation) would give xi0 Q^2."""
    rng = np.random.default_rng(6)
    xi0 = rng.standard_normal((25, 3))
    for Q in (np.linalg.qr(rng.standard_normal((3, 3)))[0], np.diag([1.0, -1.0, 1.0])):
        xi = xi0 @ Q
        np.testing.assert_allclose(O.procrustes_fit(xi, xi0), xi0, atol=1e-10)
    th = 0.7
    Q = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    xi0 = rng.standard_normal((20, 2))
    U, _, Vt = np.linalg.svd(xi0.T @ (xi0 @ Q))
    assert np.linalg.norm((xi0 @ Q) @ (U @ Vt) - xi0) > 0.1      # the printed form does not fit


def test_initial_configuration_of_identical_modalities():
    """With Delta_i = D(Y) for every i the initialisation puts every modality on the same
    configuration (commensurability 0) that cMDS gives for D(Y), and it is centred."""
    rng = np.random.default_rng(7)
    n, m, d = 18, 3, 2
    Y = rng.standard_normal((n, d)) * np.array([2.0, 1.0])
    Y -= Y.mean(0)
    D = np.sqrt(((Y[:, None] - Y[None]) ** 2).sum(-1))
    X = O.initial_configuration([D] * m, d)
    for i in range(m):
        np.testing.assert_allclose(X[i * n:(i + 1) * n], X[:n], atol=1e-10)
    np.testing.assert_allclose(X[:n] @ X[:n].T, Y @ Y.T, atol=1e-9)
    np.testing.assert_allclose(X.reshape(m, n, d).mean(1), 0, atol=1e-12)


def test_exact_configuration_fixed_point_and_recovery():
    """When every Delta_i holds the distances of one configuration Y, X = [Y; Y] has
    zero stress and is a fixed point; from a perturbed start stress falls to ~0."""
    rng = np.random.default_rng(11)
    n, m, d = 15, 2, 2
    Y = rng.standard_normal((n, d))
    Y -= Y.mean(0)
    Dy = np.sqrt(((Y[:, None] - Y[None]) ** 2).sum(-1))
    deltas = [Dy, Dy]
    Wm = _eqW(m, 0.5)
    X = np.vstack([Y, Y])
    W = O.omnibus_weights(Wm, n)
    D = O.omnibus_dissimilarity(deltas)
    assert O.raw_stress(X, W, D) < 1e-25
    np.testing.assert_allclose(O.guttman_step(X, _lp(Wm, n), W, D), X, atol=1e-12)
    X0 = X + 0.01 * rng.standard_normal(X.shape)
    res = O.jofc_embed(deltas, Wm, X0, max_iter=200)
    assert res.stress[-1] < 1e-8 * res.stress[0]


def test_invariances():
    """Translation of X0 leaves X_1 unchanged; rotation rotates it; a consistent
    permutation of objects permutes it; scaling all weights by c leaves X_1 unchanged
    and scales the stress by c."""
    n, m = 10, 2
    deltas, Wm, X0 = _small_problem(m, n, 2, seed=40)
    W = O.omnibus_weights(Wm, n)
    D = O.omnibus_dissimilarity(deltas)
    Lp = _lp(Wm, n)
    X1 = O.guttman_step(X0, Lp, W, D)
    np.testing.assert_allclose(O.guttman_step(X0 + np.array([3.0, -2.0]), Lp, W, D), X1, atol=1e-11)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    np.testing.assert_allclose(O.guttman_step(X0 @ R, Lp, W, D), X1 @ R, atol=1e-11)
    perm = np.random.default_rng(1).permutation(n)
    dp = [dl[np.ix_(perm, perm)] for dl in deltas]
    idx = np.concatenate([perm + l * n for l in range(m)])
    Xp = O.guttman_step(X0[idx], Lp, W, O.omnibus_dissimilarity(dp))
    np.testing.assert_allclose(Xp, X1[idx], atol=1e-11)
    c = 3.5
    Wc = O.omnibus_weights(c * Wm, n)
    np.testing.assert_allclose(O.guttman_step(X0, _lp(c * Wm, n), Wc, D), X1, atol=1e-11)
    np.testing.assert_allclose(O.raw_stress(X0, Wc, D), c * O.raw_stress(X0, W, D), rtol=1e-12)


def test_stopping_rule_semantics():
    """The loop stops at the first transform whose stress decrease is within the
    tolerance and returns that iterate; a negative tolerance runs max_iter transforms."""
    deltas, Wm, X0 = _small_problem(2, 15, 2, seed=50)
    fixed = O.jofc_embed(deltas, Wm, X0, max_iter=25, tol=-1)
    assert fixed.iters == 25 and len(fixed.stress) == 26
    tol = 1e-4
    res = O.jofc_embed(deltas, Wm, X0, max_iter=500, tol=tol, tol_mode="relative")
    s = res.stress
    assert res.iters < 500
    for t in range(1, res.iters):
        assert s[t - 1] - s[t] > tol * s[t - 1]
    assert s[-2] - s[-1] <= tol * s[-2]
    n_pairs = 30 * 29 // 2
    res2 = O.jofc_embed(deltas, Wm, X0, max_iter=500, tol=1e-6, tol_mode="abs_normalized")
    assert (res2.stress[-2] - res2.stress[-1]) / n_pairs <= 1e-6


# ---------------------------------------------------------------- out of sample

def _oos_setup(m=2, n=10, d=2, w=0.5, seed=60):
    rng = np.random.default_rng(seed)
    deltas, Wm, X0 = _small_problem(m, n, d, seed=seed, w=w)
    X = O.jofc_embed(deltas, Wm, X0, max_iter=30).X
    delta_new = rng.uniform(0.5, 3.0, size=(m, n))
    y0 = rng.standard_normal((m, d))
    return X, delta_new, y0, Wm


@pytest.mark.parametrize("m,w", [(2, 0.5), (3, 2.0)])
def test_oos_closed_form_update(m, w):
    """Sec. 3: the dense update of Eq. (joosupdate) equals the O(nmd) form
    y_j = xi_j/(n+mw) + w/(n(n+mw)) sum_k xi_k + psi_j y_j/(n+mw) + w/(n(n+mw)) sum_k psi_k y_k
    with xi_j = sum_k (1 - delta_j(k)/d_jk) X^(j)_k and psi_j = sum_k delta_j(k)/d_jk."""
    n, d = 10, 2
    X, dn, y, Wm = _oos_setup(m, n, d, w)
    got = O.oos_step(X, dn, y, Wm)
    xi = np.zeros((m, d))
    psi = np.zeros(m)
    for j in range(m):
        for k in range(n):
            dist = np.linalg.norm(X[j * n + k] - y[j])
            xi[j] += (1 - dn[j, k] / dist) * X[j * n + k]
            psi[j] += dn[j, k] / dist
    c1, c2 = 1 / (n + m * w), w / (n * (n + m * w))
    exp = np.array([xi[j] * c1 + c2 * xi.sum(0) + psi[j] * y[j] * c1 + c2 * (psi[:, None] * y).sum(0)
                    for j in range(m)])
    np.testing.assert_allclose(got, exp, rtol=1e-12, atol=1e-13)


def test_oos_stress_equals_eq_joos_and_descends():
    """The omnibus out-of-sample stress equals Eq. (joos) written directly, and the
    out-of-sample Guttman iterations do not increase it."""
    m, n, d, w = 2, 10, 2, 0.5
    X, dn, y0, Wm = _oos_setup(m, n, d, w)
    direct = sum((dn[j, k] - np.linalg.norm(X[j * n + k] - y0[j])) ** 2 for j in range(m) for k in range(n))
    direct += w * sum(np.sum((y0[i] - y0[j]) ** 2) for i in range(m) for j in range(i + 1, m))
    np.testing.assert_allclose(O.oos_stress(X, dn, y0, Wm), direct, rtol=1e-12)
    res = O.oos_embed(X, dn, y0, Wm, max_iter=40)
    s = np.array(res.stress)
    assert np.all(np.diff(s) <= 1e-12 * s[:-1])


def test_oos_fixed_point_exact_configuration():
    """If the new object repeats in-sample object k of a zero-stress embedding with
    equal X^(i), then y_j = X^(j)_k is a fixed point with zero out-of-sample stress."""
    rng = np.random.default_rng(70)
    n, m, d = 12, 2, 2
    Y = rng.standard_normal((n, d))
    Y -= Y.mean(0)
    Dy = np.sqrt(((Y[:, None] - Y[None]) ** 2).sum(-1))
    X = np.vstack([Y, Y])
    Wm = _eqW(m, 0.5)
    k = 4
    dn = np.stack([Dy[k], Dy[k]])
    y = np.stack([Y[k], Y[k]])
    assert O.oos_stress(X, dn, y, Wm) < 1e-25
    np.testing.assert_allclose(O.oos_step(X, dn, y, Wm), y, atol=1e-12)


def test_oos_general_weights_and_uncentred_X():
    """General weights (reading of Sec. 3 for Eq. W2): the out-of-sample L22 equals the
    in-sample modified weight matrix of Eq. (modW), and the update is
    y = Wmod^-1 (xi + psi * y) with xi_j = w_jj sum_k (1 - delta_j(k)/d_jk) X^(j)_k and
    psi_j = w_jj sum_k delta_j(k)/d_jk.  An uncentred in-sample X keeps the -L12' X term
    visible.  The stress matches Eq. (joos) with w_jj on fidelity and w_ij on
    commensurability."""
    rng = np.random.default_rng(80)
    m, n, d = 3, 8, 2
    Wm = _rand_sym_weights(rng, m)
    X = rng.standard_normal((m * n, d)) + np.array([1.5, -0.7])
    dn = rng.uniform(0.5, 3.0, size=(m, n))
    y = rng.standard_normal((m, d))
    Wo, Do, Xo = O.oos_blocks(X, dn, y, Wm)
    L22 = O.laplacian(Wo)[m * n:, m * n:]
    np.testing.assert_allclose(L22, O.modified_weight_matrix(Wm, n), atol=1e-13)
    xi = np.zeros((m, d))
    psi = np.zeros(m)
    for j in range(m):
        for k in range(n):
            dist = np.linalg.norm(X[j * n + k] - y[j])
            xi[j] += Wm[j, j] * (1 - dn[j, k] / dist) * X[j * n + k]
            psi[j] += Wm[j, j] * dn[j, k] / dist
    exp = np.linalg.inv(O.modified_weight_matrix(Wm, n)) @ (xi + psi[:, None] * y)
    np.testing.assert_allclose(O.oos_step(X, dn, y, Wm), exp, rtol=1e-11, atol=1e-12)
    direct = sum(Wm[j, j] * (dn[j, k] - np.linalg.norm(X[j * n + k] - y[j])) ** 2
                 for j in range(m) for k in range(n))
    direct += sum(Wm[i, j] * np.sum((y[i] - y[j]) ** 2) for i in range(m) for j in range(i + 1, m))
    np.testing.assert_allclose(O.oos_stress(X, dn, y, Wm), direct, rtol=1e-12)


@pytest.mark.parametrize("m,n,d", [(2, 11, 2), (3, 7, 3), (1, 9, 2)])
def test_large_n_forms_match_dense_definition(m, n, d):
    """The block forms used for full-size checks (Cor. 1's L^+ applied to B(X) X, and the
    block-wise stress) agree with the dense pinv step and the omnibus double sum, for
    general Eq. (W2) weights and with a duplicated point (d_ij = 0)."""
    rng = np.random.default_rng(90 + m)
    deltas, _, X = _small_problem(m, n, d, seed=91 + m)
    Wm = _rand_sym_weights(rng, m)
    X = X.copy()
    X[1] = X[0]
    W = O.omnibus_weights(Wm, n)
    D = O.omnibus_dissimilarity(deltas)
    dense = O.guttman_step(X, _lp(Wm, n), W, D)
    np.testing.assert_allclose(O.guttman_step_closed_form(deltas, Wm, X), dense, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(O.stress_blocks(deltas, Wm, X, row_block=4), O.raw_stress(X, W, D), rtol=1e-12)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_oos_large_n_forms_match_dense(m):
    """The O(nmd) out-of-sample forms used at large n agree with the dense Eq. (joosupdate)
    step and the omnibus stress, for general weights, an uncentred X and a new point that
    coincides with an in-sample point (d_jk = 0)."""
    rng = np.random.default_rng(95 + m)
    n, d = 9, 3
    Wm = _rand_sym_weights(rng, m)
    X = rng.standard_normal((m * n, d)) + 0.4
    dn = rng.uniform(0.5, 3.0, size=(m, n))
    y = rng.standard_normal((m, d))
    y[0] = X[2]
    np.testing.assert_allclose(O.oos_step_closed_form(X, dn, y, Wm), O.oos_step(X, dn, y, Wm), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(O.oos_stress_direct(X, dn, y, Wm), O.oos_stress(X, dn, y, Wm), rtol=1e-12)
    a = O.oos_embed_closed_form(X, dn, y, Wm, max_iter=8)
    b = O.oos_embed(X, dn, y, Wm, max_iter=8)
    np.testing.assert_allclose(a.y, b.y, rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(a.stress, b.stress, rtol=1e-11)


@pytest.mark.parametrize("seed,m,n", [(11, 3, 150), (12, 2, 200), (13, 4, 60)])
def test_pseudoinverse_moore_penrose_conditions(seed, m, n):
    """The oracle's L^+ satisfies the four Moore-Penrose conditions and Prop. 1 for random
    Eq. (W2) weights at sizes where the cutoff between L's zero singular value and the rest
    matters (n up to 200)."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(0.2, 2.0, (m, m))
    Wm = np.triu(A) + np.triu(A, 1).T
    L = O.laplacian(O.omnibus_weights(Wm, n))
    P = O.pseudoinverse(L)
    N = m * n
    scale = np.abs(L).max()
    assert np.abs(L @ P @ L - L).max() <= 1e-10 * scale
    assert np.abs(P @ L @ P - P).max() <= 1e-10 * np.abs(P).max()
    assert np.abs(L @ P - (L @ P).T).max() <= 1e-10
    assert np.abs(P @ L - (P @ L).T).max() <= 1e-10
    J = np.ones((N, N)) / N
    np.testing.assert_allclose(P, np.linalg.inv(L + J) - J, atol=1e-10 * np.abs(P).max())


def test_guttman_rows_match_full_step():
    """Sampled rows of one transform (no J_n term) equal the dense pinv step and the full
    closed-form step (which keeps the J_n term) on a random problem with general W2
    weights: pins that the column sums of B_l X^(l) vanish and that the row formula has
    no dropped or transposed term."""
    rng = np.random.default_rng(77)
    m, n, d = 3, 23, 4
    F = [rng.normal(size=(n, 3)) for _ in range(m)]
    deltas = [np.sqrt(((f[:, None, :] - f[None, :, :]) ** 2).sum(-1)) for f in F]
    Wm = rng.uniform(0.3, 1.7, size=(m, m))
    Wm = (Wm + Wm.T) / 2
    X = rng.normal(size=(m * n, d))
    full = O.jofc_embed(deltas, Wm, X, max_iter=1).X
    closed = O.guttman_step_closed_form(deltas, Wm, X)
    idx = np.array([0, 5, 11, 22])
    rows = O.guttman_rows([D[idx] for D in deltas], Wm, X, idx)
    for j in range(m):
        np.testing.assert_allclose(rows[j], full[j * n + idx], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(rows[j], closed[j * n + idx], rtol=1e-10, atol=1e-12)
