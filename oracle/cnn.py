"""FP64 numpy oracle of the learned-guess network's kernels.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Definitions (the network has no counterpart in the paper; these are the plain
mathematical definitions the CUDA kernels implement):
  * periodic 3x3 convolution, NHWC: out[b, y, x, co] = bias[co]
      + sum_{dy, dx in {-1, 0, 1}} sum_ci in[b, (y+dy) mod H, (x+dx) mod W, ci] w[tap, ci, co],
    tap = (dy+1)*3 + (dx+1);
  * GELU(z) = z Phi(z) with the exact normal CDF Phi(z) = (1 + erf(z / sqrt 2)) / 2;
  * mean squared error and its gradient; Adam (Kingma & Ba, bias-corrected).
Pinned by finite differences in tests/test_oracle_cnn.py.
"""
from __future__ import annotations

import math

import numpy as np

_erf = np.vectorize(math.erf)


def shift(x, dy, dx):
    """x[b, (y+dy) mod H, (x+dx) mod W, c] as an array indexed [b, y, x, c]."""
    return np.roll(np.roll(x, -dy, axis=1), -dx, axis=2)


def conv3x3(x, w, bias=None):
    """x [B,H,W,ci], w [9,ci,co] -> [B,H,W,co] (periodic)."""
    B, H, W, ci = x.shape
    co = w.shape[2]
    out = np.zeros((B, H, W, co))
    for tap in range(9):
        dy, dx = tap // 3 - 1, tap % 3 - 1
        out += np.einsum("bhwc,cd->bhwd", shift(x, dy, dx), w[tap])
    if bias is not None:
        out += bias
    return out


def conv3x3_grad_input(dout, w):
    """d(loss)/d(in) for out = conv3x3(in, w): sum_tap shift(dout, -off) w[tap]^T."""
    B, H, W, co = dout.shape
    ci = w.shape[1]
    g = np.zeros((B, H, W, ci))
    for tap in range(9):
        dy, dx = tap // 3 - 1, tap % 3 - 1
        g += np.einsum("bhwd,cd->bhwc", shift(dout, -dy, -dx), w[tap])
    return g


def conv3x3_grad_weight(x, dout):
    """d(loss)/d(w)[tap, ci, co] = sum_p x[p + off(tap), ci] dout[p, co]; and d(bias)."""
    ci, co = x.shape[3], dout.shape[3]
    gw = np.zeros((9, ci, co))
    for tap in range(9):
        dy, dx = tap // 3 - 1, tap % 3 - 1
        gw[tap] = np.einsum("bhwc,bhwd->cd", shift(x, dy, dx), dout)
    return gw, dout.sum(axis=(0, 1, 2))


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def mse(yhat, y):
    d = yhat - y
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


LAYERS = [(3, 32), (32, 32), (32, 32), (32, 32), (32, 1)]


def unpack(blob):
    """Model blob -> (norms[4], [(w [9,ci,co], b [co]) x 5])."""
    blob = np.asarray(blob, dtype=np.float64)
    norms = blob[:4]
    off = 4
    layers = []
    for ci, co in LAYERS:
        w = blob[off:off + 9 * ci * co].reshape(9, ci, co)
        off += 9 * ci * co
        b = blob[off:off + co]
        off += co
        layers.append((w, b))
    assert off == blob.size
    return norms, layers


def features(phik, phikm1, phikm2, norms):
    """Network input [H, W, 3] (channels of the learned guess) for one sample."""
    mean = phik.mean()
    return np.stack([(phik - mean) / norms[0], (phik - phikm1) / norms[1],
                     (phik - 2 * phikm1 + phikm2) / norms[2]], axis=-1)


def forward(x, layers):
    """x [B,H,W,3] -> prediction [B,H,W,1]; GELU after the first four layers."""
    a = x
    for i, (w, b) in enumerate(layers):
        z = conv3x3(a, w, b)
        a = gelu(z) if i < 4 else z
    return a
