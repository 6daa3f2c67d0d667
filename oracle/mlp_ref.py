"""FP64 reference of the Ca_cr proposal network (TEST INFRASTRUCTURE: only
the test-suite may import this module).

Plain NumPy, float64, written from the definitions: layers
6 -> 128 -> 128 -> 128 -> 128 -> 4, GELU(x) = x Phi(x) with
Phi(x) = (1 + erf(x / sqrt 2)) / 2 after each hidden layer; loss = mean over
the batch of mask * ((y0-t0)^2 + (y1-t1)^2 + (y3-t3)^2) + BCE(sigmoid(y2), t2);
AdamW with bias-corrected moments and decoupled weight decay.  The
parameter vector is the interface format of lbfe_mlp.h: per layer the
transposed weights Wt[in][out] then the bias b[out].
"""
from __future__ import annotations

import math

import numpy as np

DIMS = (6, 128, 128, 128, 128, 4)
_erf = np.vectorize(math.erf)


def param_count() -> int:
    return sum(DIMS[l] * DIMS[l + 1] + DIMS[l + 1] for l in range(len(DIMS) - 1))


def unpack(p: np.ndarray):
    """List of (Wt[in][out], b[out]) views of the flat parameter vector."""
    out, o = [], 0
    for l in range(len(DIMS) - 1):
        i, j = DIMS[l], DIMS[l + 1]
        Wt = p[o:o + i * j].reshape(i, j)
        o += i * j
        b = p[o:o + j]
        o += j
        out.append((Wt, b))
    return out


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(p: np.ndarray, x: np.ndarray, keep: bool = False):
    layers = unpack(np.asarray(p, dtype=np.float64))
    a = np.asarray(x, dtype=np.float64)
    zs, as_ = [], [a]
    for l, (Wt, b) in enumerate(layers):
        z = a @ Wt + b
        zs.append(z)
        a = gelu(z) if l < len(layers) - 1 else z
        as_.append(a)
    return (a, zs, as_) if keep else a


def loss_grad(p: np.ndarray, x: np.ndarray, t: np.ndarray, mask: np.ndarray | None = None):
    """(loss, gradient) of the batch, float64."""
    p = np.asarray(p, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    B = x.shape[0]
    mk = np.ones(B) if mask is None else np.asarray(mask, dtype=np.float64)
    y, zs, as_ = forward(p, x, keep=True)
    e = y - t
    z = y[:, 2]
    bce = np.maximum(z, 0) - z * t[:, 2] + np.log1p(np.exp(-np.abs(z)))
    loss = float(np.mean(mk * (e[:, 0] ** 2 + e[:, 1] ** 2 + e[:, 3] ** 2) + bce))
    dy = np.zeros_like(y)
    dy[:, 0] = 2 * mk * e[:, 0]
    dy[:, 1] = 2 * mk * e[:, 1]
    dy[:, 3] = 2 * mk * e[:, 3]
    dy[:, 2] = 1.0 / (1.0 + np.exp(-z)) - t[:, 2]
    dy /= B
    layers = unpack(p)
    grads = []
    dz = dy
    for l in range(len(layers) - 1, -1, -1):
        Wt, b = layers[l]
        a_in = as_[l]
        grads.append((a_in.T @ dz, dz.sum(0)))
        if l > 0:
            dz = (dz @ Wt.T) * gelu_grad(zs[l - 1])
    grads.reverse()
    g = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return loss, g


def adamw(p, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    """One AdamW step at step number t (1-based); returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    p = p - lr * (mh / (np.sqrt(vh) + eps) + wd * p)
    return p, m, v
