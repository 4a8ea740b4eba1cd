"""Pins of the float64 network reference: gradients against central finite
differences, parameter count, feature definition against a direct DFT sum."""
import math

import numpy as np
import pytest

from oracle import cnn


def small_case(seed=0, B=2):
    rng = np.random.default_rng(seed)
    p = cnn.init_params(rng)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1     # non-zero biases exercise every term
    x = rng.standard_normal((B, 8, 64, 64))
    uv = rng.uniform(-1, 1, (B, 2))
    t = rng.standard_normal((B, 12))
    return p, x, uv, t


def test_parameter_count_about_half_a_million():
    p, *_ = small_case()
    assert cnn.param_count(p) == 459244


@pytest.mark.parametrize("name", ["w0", "b0", "w1", "w2", "b2", "w3", "b3", "w4", "b4", "w5", "b5"])
def test_gradients_match_central_differences(name):
    p, x, uv, t = small_case(1)
    _, g = cnn.loss_and_grads(p, x, uv, t)
    rng = np.random.default_rng(hash(name) % 2**32)
    flat = p[name].reshape(-1)
    gflat = g[name].reshape(-1)
    idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
    h = 1e-6
    for i in idx:
        old = flat[i]
        flat[i] = old + h
        lp, _ = cnn.loss_and_grads(p, x, uv, t)
        flat[i] = old - h
        lm, _ = cnn.loss_and_grads(p, x, uv, t)
        flat[i] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, i, fd, gflat[i])


def test_features_are_log_normalised_spectrum_magnitudes():
    rng = np.random.default_rng(3)
    I = rng.random((2, 16, 16)) + 1.0
    f = cnn.features(I)
    assert f.shape == (2, 64, 64)
    # direct DFT sum at one lag, kx = 3, ky = -2 (stored at [ky + 32, kx + 32])
    y, x = np.mgrid[0:16, 0:16]
    F = np.sum(I[1] * np.exp(-2j * math.pi * (3 * x / 16 + (-2) * y / 16)))
    ref = math.log(abs(F) / I[1].sum() + cnn.FEATURE_FLOOR)
    assert abs(f[1, -2 + 32, 3 + 32] - ref) < 1e-12
    assert abs(f[0, 32, 32] - math.log(1 + cnn.FEATURE_FLOOR)) < 1e-12


def test_position_input_reaches_the_dense_layer():
    """Closed form: with every convolution zeroed the pooled features are 0, so a dense
    layer reading only (u, v) gives out = (relu(u), relu(v), 0, ...)."""
    p, x, _, _ = small_case(2, B=4)
    for k in p:
        p[k] = np.zeros_like(p[k])
    p["w4"][0, cnn.CHANNELS[4]] = 1.0
    p["w4"][1, cnn.CHANNELS[4] + 1] = 1.0
    p["w5"][0, 0] = 1.0
    p["w5"][1, 1] = 1.0
    uv = np.array([[0.5, -0.25], [-0.75, 0.125], [0.0, 1.0], [0.3, 0.2]])
    out, _ = cnn.forward(p, x, uv)
    assert np.array_equal(out[:, :2], np.maximum(uv, 0.0))
    assert np.all(out[:, 2:] == 0)


def test_max_pool_ties_go_to_the_first_position():
    """Ties of the 2 x 2 max-pool take the first maximum in (dy, dx) order, and the
    backward pass routes the gradient there alone."""
    x = np.zeros((1, 1, 2, 4))
    x[0, 0] = [[1.0, 3.0, 2.0, 2.0],
               [3.0, 0.5, 2.0, 2.0]]
    y, arg = cnn._pool(x)
    assert y.tolist() == [[[[3.0, 2.0]]]]
    assert arg.tolist() == [[[[1, 0]]]]                     # (0, 1) in the first block, (0, 0) in the second
    g = cnn._pool_backward(np.ones((1, 1, 1, 2)), arg, x.shape)
    assert g[0, 0].tolist() == [[0.0, 1.0, 1.0, 0.0], [0.0, 0.0, 0.0, 0.0]]
