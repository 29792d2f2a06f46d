"""Pins of the CNN oracle (oracle/cnn.py) by finite differences and closed forms."""
import math

import numpy as np

from oracle import cnn


def test_conv_identity_and_shift():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 5, 6, 3))
    w = np.zeros((9, 3, 3))
    w[4] = np.eye(3)                                   # centre tap: identity
    np.testing.assert_allclose(cnn.conv3x3(x, w), x, atol=0)
    w = np.zeros((9, 3, 3))
    w[5] = np.eye(3)                                   # tap (dy=0, dx=+1): out(y,x) = in(y, x+1)
    np.testing.assert_allclose(cnn.conv3x3(x, w), np.roll(x, -1, axis=2), atol=0)


def test_gelu_closed_form_and_derivative():
    z = np.linspace(-4, 4, 41)
    Phi = np.array([0.5 * (1 + math.erf(t / math.sqrt(2))) for t in z])
    np.testing.assert_allclose(cnn.gelu(z), z * Phi, atol=1e-15)
    h = 1e-6
    fd = (cnn.gelu(z + h) - cnn.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(cnn.gelu_grad(z), fd, atol=1e-8)


def _loss(x, w, dout):
    return float(np.sum(cnn.conv3x3(x, w) * dout))


def test_conv_gradients_by_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 4, 5, 3))
    w = rng.normal(size=(9, 3, 2))
    dout = rng.normal(size=(2, 4, 5, 2))
    gx = cnn.conv3x3_grad_input(dout, w)
    gw, gb = cnn.conv3x3_grad_weight(x, dout)
    h = 1e-6
    for idx in [(0, 1, 2, 0), (1, 3, 4, 2), (0, 0, 0, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        assert abs((_loss(xp, w, dout) - _loss(xm, w, dout)) / (2 * h) - gx[idx]) < 1e-6
    for idx in [(0, 0, 0), (4, 2, 1), (8, 1, 0)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        assert abs((_loss(x, wp, dout) - _loss(x, wm, dout)) / (2 * h) - gw[idx]) < 1e-6
    np.testing.assert_allclose(gb, dout.sum(axis=(0, 1, 2)))


def test_adam_first_step_is_signed_lr():
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -0.1, 2.0])
    p1, m, v = cnn.adam(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(p1, p - 0.01 * np.sign(g), atol=1e-15)
