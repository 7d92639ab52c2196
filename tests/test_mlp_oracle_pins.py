"""Pins of the float64 warm-start network oracle (oracle/mlp_oracle.py) against facts that
do not come from the oracle itself: textbook values of the normal CDF, central finite
differences of the loss, closed forms of the first Adam step and of a network whose
weights are zero, and a hand-built feature example."""
import math

import numpy as np

from oracle import mlp_oracle as M


def test_gelu_textbook_values():
    # Phi(1) = 0.8413447460685429, Phi(-1) = 0.15865525393145707, Phi(2) = 0.9772498680518208
    z = np.array([0.0, 1.0, -1.0, 2.0, -8.0, 8.0])
    want = np.array([0.0, 0.8413447460685429, -0.15865525393145707, 2 * 0.9772498680518208,
                     -8.0 * 6.22096057427178e-16, 8.0])
    np.testing.assert_allclose(M.gelu(z), want, rtol=1e-12, atol=1e-14)


def test_gelu_grad_is_the_derivative():
    z = np.linspace(-6, 6, 49)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(M.gelu_grad(z), fd, rtol=1e-7, atol=1e-9)


def _random_net(rng, n_in=7, hidden=6, n_out=3):
    theta = rng.normal(scale=0.6, size=M.param_count(n_in, hidden, n_out))
    return theta, (n_in, hidden, n_out)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    theta, dims = _random_net(rng)
    X = rng.normal(size=(5, dims[0]))
    Y = rng.normal(size=(5, dims[2]))
    L, g = M.gradient(theta, X, Y, *dims)
    assert abs(L - M.loss(theta, X, Y, *dims)) < 1e-14
    h = 1e-6
    fd = np.empty_like(theta)
    for p in range(theta.size):
        e = np.zeros_like(theta)
        e[p] = h
        fd[p] = (M.loss(theta + e, X, Y, *dims) - M.loss(theta - e, X, Y, *dims)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_zero_weights_give_the_bias():
    n_in, hidden, n_out = 4, 3, 2
    theta = np.zeros(M.param_count(n_in, hidden, n_out))
    theta[-n_out:] = [0.5, -2.0]
    X = np.arange(12.0).reshape(3, 4)
    Y = np.array([[1.0, 1.0], [0.0, 0.0], [0.5, -2.0]])
    yhat, _ = M.forward(theta, X, n_in, hidden, n_out)
    np.testing.assert_array_equal(yhat, np.tile([0.5, -2.0], (3, 1)))
    # L = 1/(2B) sum ||b3 - y||^2 = (0.25 + 9 + 0.25 + 4 + 0) / 6
    assert abs(M.loss(theta, X, Y, n_in, hidden, n_out) - 13.5 / 6) < 1e-15


def test_first_adam_step_closed_form():
    # with m = v = 0 and t = 1 the bias-corrected moments are g and g^2, so the step is
    # lr * g / (|g| + eps)
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    new, m, v = M.adam_step(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    np.testing.assert_allclose(new, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_features_by_hand():
    d = np.arange(2 * 2 * 6, dtype=np.float64).reshape(2, 2, 6)   # k=2, m=2, n=6
    f = M.features(d, np.array([4, 1]), np.array([0.5, 2.0]))
    # object 0: modality 0 -> d[0,0,4]*0.5, d[0,0,1]*0.5; modality 1 -> d[0,1,4]*2, d[0,1,1]*2
    np.testing.assert_array_equal(f[0], [2.0, 0.5, 20.0, 14.0])
    np.testing.assert_array_equal(f[1], [8.0, 6.5, 44.0, 38.0])


def test_param_count_of_the_warm_start_network():
    assert M.param_count(512, 512, 5) == 527877
    assert math.isclose(M.param_count(512, 512, 5), 512 * 512 * 2 + 512 * 2 + 512 * 5 + 5)
