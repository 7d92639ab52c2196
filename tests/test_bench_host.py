"""Host-side helpers of bench.py's paper-shaped out-of-sample workload (no GPU needed)."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_held_out_rows_drop_the_last_object_of_every_modality():
    m, n = 3, 5
    keep = bench.held_out_rows(m, n)
    assert keep.shape == (m * n,) and keep.sum() == m * (n - 1)
    assert np.flatnonzero(~keep).tolist() == [j * n + n - 1 for j in range(m)]
    X = np.arange(m * n * 2, dtype=float).reshape(m * n, 2)
    # the kept rows are the configuration of the first n - 1 objects, modality-major
    np.testing.assert_array_equal(X[keep].reshape(m, n - 1, 2), X.reshape(m, n, 2)[:, :n - 1])


def test_procrustes_rotation_recovers_rotations_and_reflections():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((40, 3))
    for det in (1.0, -1.0):
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        if np.sign(np.linalg.det(Q)) != det:
            Q[:, 0] = -Q[:, 0]
        R = bench.procrustes_rotation(A, A @ Q)
        np.testing.assert_allclose(R, Q, atol=1e-12)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-12)


def test_loglog_slope_of_power_laws():
    x = np.array([2.0, 4.0, 6.0, 8.0])
    assert abs(bench._loglog_slope(x, 3.0 * x ** 2) - 2.0) < 1e-12
    assert abs(bench._loglog_slope(x, 0.5 * x) - 1.0) < 1e-12
    assert abs(bench._loglog_slope(x, np.full(4, 7.0))) < 1e-12
