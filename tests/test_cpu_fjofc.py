"""The C float64 Algorithm 2 (``oracle/fjofc_cpu.c``, the CPU baseline bench.py times)
against the numpy oracle's Algorithm 1 with its dense pseudoinverse (CPU only).

fJOFC reaches exactly the iterates of Algorithm 1 with an exact L^+ (Sec. 2.1, Cor. 1),
so the two float64 programs agree to rounding: X and every stress within 1e-10
relative, the same transform count under both stopping rules, for general weights
(Eq. W2), one modality (plain SMACOF) and duplicate points (d_ij = 0, Eq. B).
"""
import numpy as np
import pytest

from oracle import fjofc_oracle as O
from oracle import fjofc_cpu as C
import synthetic


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.mark.parametrize("m,n,d,kind", [(3, 15, 2, "W2"), (2, 40, 3, "W"), (1, 12, 2, "W"), (4, 9, 5, "W2")])
def test_cpu_fjofc_matches_oracle(m, n, d, kind):
    prob = synthetic.make_insample(0, n=n, m=m, d=d, seed=2000 + 7 * n + m)
    W = prob.W
    if kind == "W2":
        rng = np.random.default_rng(5 + m)
        A = rng.uniform(0.2, 2.0, (m, m))
        W = np.triu(A) + np.triu(A, 1).T
    X, it, hist = C.cpu_embed(prob.deltas, W, prob.X0, 12)
    ref = O.jofc_embed(prob.deltas, W, prob.X0, max_iter=12)
    assert it == 12
    assert _rel(X, ref.X) <= 1e-10
    np.testing.assert_allclose(hist, ref.stress, rtol=1e-10)


@pytest.mark.parametrize("mode,tol", [("relative", 1e-4), ("abs_normalized", 1e-5)])
def test_cpu_fjofc_stopping_rule(mode, tol):
    prob = synthetic.make_insample(0, n=60, m=2, d=2, seed=2101)
    X, it, hist = C.cpu_embed(prob.deltas, prob.W, prob.X0, 500, tol=tol, tol_mode=mode)
    ref = O.jofc_embed(prob.deltas, prob.W, prob.X0, max_iter=500, tol=tol, tol_mode=mode)
    assert it == ref.iters and 1 <= it < 500
    assert _rel(X, ref.X) <= 1e-10
    np.testing.assert_allclose(hist, ref.stress, rtol=1e-10)


def test_cpu_fjofc_duplicate_points():
    prob = synthetic.make_insample(0, n=20, m=2, d=2, seed=2202)
    X0 = prob.X0.copy()
    X0[3] = X0[5]
    X, it, hist = C.cpu_embed(prob.deltas, prob.W, X0, 6)
    ref = O.jofc_embed(prob.deltas, prob.W, X0, max_iter=6)
    assert _rel(X, ref.X) <= 1e-10
    np.testing.assert_allclose(hist, ref.stress, rtol=1e-10)
