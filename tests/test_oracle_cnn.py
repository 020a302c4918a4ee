"""Pins of the warm-start network oracle (oracle/cnn.py) to truths outside it:
a library cross-correlation, special cases, finite differences, Adam's closed
first step."""
import numpy as np
import scipy.ndimage as ndi

from oracle import cnn


def _params(rng, dims):
    return [(rng.standard_normal((dims[i + 1], dims[i], 3, 3)) * 0.5, rng.standard_normal(dims[i + 1]) * 0.1)
            for i in range(len(dims) - 1)]


def test_conv_is_circular_cross_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 7, 5))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = cnn.conv3x3(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(ndi.correlate(x[n, c], w[o, c], mode="wrap") for c in range(3))
            np.testing.assert_allclose(y[n, o], ref, rtol=1e-12, atol=1e-12)


def test_conv_special_cases():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 2, 4, 6))
    w = np.zeros((2, 2, 3, 3))
    w[0, 0, 1, 1] = 1.0    # identity on channel 0
    w[1, 1, 1, 2] = 1.0    # channel 1 read one column to the right (wrapping)
    y = cnn.conv3x3(x, w, np.zeros(2))
    np.testing.assert_array_equal(y[0, 0], x[0, 0])
    np.testing.assert_array_equal(y[0, 1], np.roll(x[0, 1], -1, axis=1))


def _loss(params, x, y, mean, tau, log_xi):
    out, acts, pres = cnn.forward(params, x)
    loss, g = cnn.warmstart_loss(out, y, mean, tau, log_xi, 7.0)
    return loss, g, acts, pres


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    dims = [3, 4, 4, 6]
    params = _params(rng, dims)
    x = rng.standard_normal((2, 3, 5, 6))
    y = x[:, 0]
    mean = y + 0.1 * rng.standard_normal(y.shape)
    var = np.exp(rng.standard_normal((2, 5, 5, 6)))
    log_xi = np.array([-1.0, 0.5])
    loss, g, acts, pres = _loss(params, x, y, mean, var, log_xi)
    grads = cnn.backward(params, acts, pres, g)
    h = 1e-6
    for li in range(len(params)):
        w, b = params[li]
        for idx in [(0, 0, 0, 0), (1, 2, 2, 1), (dims[li + 1] - 1, dims[li] - 1, 1, 2)]:
            old = w[idx]
            w[idx] = old + h
            lp = _loss(params, x, y, mean, var, log_xi)[0]
            w[idx] = old - h
            lm = _loss(params, x, y, mean, var, log_xi)[0]
            w[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[li][0][idx]) <= 1e-6 * max(1.0, abs(fd)), (li, idx)
        for o in range(b.size):
            old = b[o]
            b[o] = old + h
            lp = _loss(params, x, y, mean, var, log_xi)[0]
            b[o] = old - h
            lm = _loss(params, x, y, mean, var, log_xi)[0]
            b[o] = old
            assert abs((lp - lm) / (2 * h) - grads[li][1][o]) <= 1e-6 * max(1.0, abs(lp))


def test_input_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    w = rng.standard_normal((3, 2, 3, 3))
    x = rng.standard_normal((1, 2, 4, 5))
    dout = rng.standard_normal((1, 3, 4, 5))
    dx, _, _ = cnn.conv3x3_backward(x, w, dout)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (0, 1, 3, 4), (0, 0, 2, 1)]:
        xp = x.copy(); xp[idx] += h
        xm = x.copy(); xm[idx] -= h
        fd = (np.sum(cnn.conv3x3(xp, w, np.zeros(3)) * dout) - np.sum(cnn.conv3x3(xm, w, np.zeros(3)) * dout)) / (2 * h)
        assert abs(fd - dx[idx]) < 1e-6


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([0.3, -2.0, 1e-3])
    p = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    cnn.adam_step(p, g, m, v, 1, 0.01, eps=0.0)
    np.testing.assert_allclose(p, -0.01 * np.sign(g), rtol=1e-12)
