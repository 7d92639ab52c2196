"""The seeded input generators (``synthetic``) follow the recipe they state, on the CPU:
the seed rule, the draw order, the shapes, and dissimilarities that are Euclidean
distances of the features (symmetric, zero diagonal, triangle inequality).  Both the
oracle and the CUDA path read their inputs from here, so a silent change of recipe
would move every stored number at once."""
import numpy as np
import pytest

import synthetic


def test_insample_seed_rule_and_draw_order():
    prob = synthetic.make_insample(0, rep=3, n=40)
    assert prob.seed == 1000 * 0 + 3
    spec = prob.spec
    rng = np.random.default_rng(prob.seed)
    Z = rng.standard_normal((spec.n, spec.latent))
    A = [rng.standard_normal((spec.latent, spec.latent)) for _ in range(spec.m)]
    E = [rng.standard_normal((spec.n, spec.latent)) for _ in range(spec.m)]
    X0 = rng.standard_normal((spec.m * spec.n, spec.d))
    np.testing.assert_array_equal(prob.Z, Z)
    for i in range(spec.m):
        np.testing.assert_array_equal(prob.A[i], A[i])
        np.testing.assert_allclose(prob.F[i], Z @ A[i] + spec.noise * E[i], rtol=0, atol=0)
    np.testing.assert_array_equal(prob.X0, X0)
    again = synthetic.make_insample(0, rep=3, n=40)
    for a, b in zip(prob.deltas, again.deltas):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("k", [0, 1, 2, 4])
def test_workload_shapes(k):
    spec = synthetic.WORKLOADS[k]
    prob = synthetic.make_insample(k, n=30)          # the workload's m, d, latent at a small n
    assert prob.X0.shape == (spec.m * 30, spec.d)
    assert len(prob.F) == spec.m and all(F.shape == (30, spec.latent) for F in prob.F)
    np.testing.assert_array_equal(prob.W, synthetic.weights_matrix(spec.m, spec.w_fid, spec.w_comm))


def _is_distance_matrix(D, F):
    n = D.shape[0]
    assert D.shape == (n, n)
    np.testing.assert_array_equal(D, D.T)
    assert np.all(np.diag(D) == 0) and np.all(D >= 0)
    # triangle inequality through every intermediate point
    assert np.all(D[:, None, :] <= D[:, :, None] + D[None, :, :] + 1e-12)
    i, j = 3, 7
    assert abs(D[i, j] - np.sqrt(np.sum((F[i] - F[j]) ** 2))) <= 1e-12 * max(1.0, D[i, j])


def test_insample_dissimilarities_are_feature_distances():
    prob = synthetic.make_insample(0, n=25, m=3)
    for D, F in zip(prob.deltas, prob.F):
        _is_distance_matrix(D, F)


def test_oos_objects_share_the_modality_maps():
    prob = synthetic.make_insample(0, n=30)
    F_new, dnew, Y0 = synthetic.make_oos_objects(prob, 6, stream=2)
    spec = prob.spec
    assert dnew.shape == (6, spec.m, spec.n) and Y0.shape == (6, spec.m, spec.d)
    rng = np.random.default_rng([prob.seed, 7919, 2])
    Zn = rng.standard_normal((6, spec.latent))
    En = [rng.standard_normal((6, spec.latent)) for _ in range(spec.m)]
    for j in range(spec.m):
        np.testing.assert_allclose(F_new[j], Zn @ prob.A[j] + spec.noise * En[j], rtol=0, atol=0)
        o, k = 4, 11
        assert abs(dnew[o, j, k] - np.linalg.norm(F_new[j][o] - prob.F[j][k])) <= 1e-12 * dnew[o, j, k]
    other = synthetic.make_oos_objects(prob, 6, stream=1)[0]
    assert not np.allclose(other[0], F_new[0])      # streams are independent


def test_paper_generator_jitter_bound():
    """Sec. 4.1 / 4.3: Y ~ N((5,..,5), I), every modality Y + U(-z/50, z/50) with
    z = max(Y) - min(Y): each point moves by at most sqrt(dim) z / 50, so a distance by at
    most twice that; modalities differ (independent jitter)."""
    n, m, dim, seed = 60, 3, 2, 9
    deltas = synthetic.paper_jitter_modalities(n=n, m=m, dim=dim, seed=seed)
    Y = np.random.default_rng(seed).normal(5.0, 1.0, size=(n, dim))
    z = Y.max() - Y.min()
    DY = synthetic.euclidean_distances(Y)
    bound = 2 * np.sqrt(dim) * z / 50
    for D in deltas:
        np.testing.assert_array_equal(D, D.T)
        assert np.all(np.diag(D) == 0)
        assert np.max(np.abs(D - DY)) <= bound + 1e-12
    assert not np.allclose(deltas[0], deltas[1])


def test_device_distances_match_host_distances():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    F = rng.standard_normal((50, 5))
    G = rng.standard_normal((20, 5))
    got = synthetic.torch_distances(F, "cpu", torch.float64, G=G).numpy()
    np.testing.assert_allclose(got, synthetic.cross_distances(F, G), rtol=1e-13, atol=1e-13)
    sq = synthetic.torch_distances(F, "cpu", torch.float32).numpy()
    np.testing.assert_allclose(sq, synthetic.euclidean_distances(F).astype(np.float32), rtol=1e-6, atol=1e-6)
