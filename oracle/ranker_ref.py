"""CPU ORACLE (test infrastructure only): the decimation ranker's loss and
gradient in FP64 with numpy.

The ranker has no counterpart in the paper; it replaces the argmin of
Alg. 1 (SELECT-VN) by the highest score W2 . relu(W1 x + b1) + b2 over eight
candidate features.  Parameters: one 641-vector W1[64][8], b1[64], W2[64],
b2.  Loss of a record with label y: w_y (log(1 + e^z) - y z), w_1 =
pos_weight, w_0 = 1 (binary cross entropy with logits).  With quantize, W1
and W2 are rounded to multiples of 2^-6 within [-2, 2] and b1 to multiples
of 2^-7 within [-512, 512] (half to even) before use, and the gradient is taken with respect to
the rounded values (straight through the rounding).

The gradient is the chain rule of these three steps written out by hand;
relu'(0) = 0.
"""
import numpy as np


def quantize(p):
    p = np.asarray(p, np.float64).copy()
    p[:512] = np.clip(np.rint(p[:512] * 64.0), -128, 128) / 64.0
    p[512:576] = np.clip(np.rint(p[512:576] * 128.0), -65536, 65536) / 128.0
    p[576:640] = np.clip(np.rint(p[576:640] * 64.0), -128, 128) / 64.0
    return p


def _unpack(p):
    return p[:512].reshape(64, 8), p[512:576], p[576:640], p[640]


def forward(p, x, quant=False):
    """Scores z [n] of feature rows x [n, 8]."""
    p = quantize(p) if quant else np.asarray(p, np.float64)
    W1, b1, W2, b2 = _unpack(p)
    a = np.asarray(x, np.float64) @ W1.T + b1
    return np.maximum(a, 0.0) @ W2 + b2


def loss(p, x, y, pos_weight=1.0, quant=False):
    z = forward(p, x, quant)
    y = np.asarray(y, np.float64)
    w = np.where(y > 0.5, pos_weight, 1.0)
    return w * (np.logaddexp(0.0, z) - y * z)


def grad(p, x, y, pos_weight=1.0, quant=False):
    """d(sum of losses)/dp [641] and the per-record losses."""
    q = quantize(p) if quant else np.asarray(p, np.float64)
    W1, b1, W2, b2 = _unpack(q)
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    a = x @ W1.T + b1
    h = np.maximum(a, 0.0)
    z = h @ W2 + b2
    w = np.where(y > 0.5, pos_weight, 1.0)
    dz = w * (1.0 / (1.0 + np.exp(-z)) - y)
    dh = np.where(a > 0.0, dz[:, None] * W2[None, :], 0.0)
    g = np.zeros(641)
    g[:512] = (dh.T @ x).reshape(-1)
    g[512:576] = dh.sum(0)
    g[576:640] = h.T @ dz
    g[640] = dz.sum()
    return g, w * (np.logaddexp(0.0, z) - y * z)
