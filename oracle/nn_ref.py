"""Plain FP64 reference of the warm-start network's operations (TEST
INFRASTRUCTURE ONLY; not in the paper).

Tensors are channels-last numpy arrays x[n, z, y, x, c].  The convolution is
3x3x3 with zero padding 1 and stride 1, weights w[tap, ci, co] with
tap = 9 dz + 3 dy + dx (dz, dy, dx in 0..2 standing for offsets -1, 0, +1):

    y[p, co] = sum_tap sum_ci w[tap, ci, co] x[p + off(tap), ci] + b[co]

Written as an explicit sum over the 27 taps of shifted copies of the padded
input; the tests check it against scipy.ndimage.correlate, its adjoint
identities and finite differences.
"""
from __future__ import annotations

import numpy as np

OFFSETS = [(dz - 1, dy - 1, dx - 1) for dz in range(3) for dy in range(3) for dx in range(3)]


def _shifted(x, off):
    """x[p + off] with zero padding, for every p (x is [n, z, y, x, c])."""
    dz, dy, dx = off
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    n, d, h, w, c = x.shape
    return xp[:, 1 + dz:1 + dz + d, 1 + dy:1 + dy + h, 1 + dx:1 + dx + w, :]


def conv3d(x, w, b=None, relu=False):
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    y = np.zeros(x.shape[:4] + (w.shape[2],))
    for tap, off in enumerate(OFFSETS):
        y += _shifted(x, off) @ w[tap]
    if b is not None:
        y += np.asarray(b, np.float64)
    return np.maximum(y, 0.0) if relu else y


def conv3d_bwd_data(dy, w):
    """dL/dx for y = conv3d(x, w): sum_tap dy[p - off(tap)] w[tap]^T."""
    dy = np.asarray(dy, np.float64)
    w = np.asarray(w, np.float64)
    dx = np.zeros(dy.shape[:4] + (w.shape[1],))
    for tap, off in enumerate(OFFSETS):
        dx += _shifted(dy, tuple(-o for o in off)) @ w[tap].T
    return dx


def conv3d_bwd_weight(x, dy):
    """dL/dw[tap, ci, co] = sum_p x[p + off(tap), ci] dy[p, co]; dL/db = sum_p dy."""
    x = np.asarray(x, np.float64)
    dy = np.asarray(dy, np.float64)
    cin, cout = x.shape[4], dy.shape[4]
    dw = np.zeros((27, cin, cout))
    for tap, off in enumerate(OFFSETS):
        dw[tap] = _shifted(x, off).reshape(-1, cin).T @ dy.reshape(-1, cout)
    return dw, dy.reshape(-1, cout).sum(axis=0)


def pool2(x):
    n, d, h, w, c = x.shape
    return np.asarray(x, np.float64).reshape(n, d // 2, 2, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4, 6))


def pool2_bwd(dy):
    return np.repeat(np.repeat(np.repeat(np.asarray(dy, np.float64), 2, 1), 2, 2), 2, 3) / 8.0


def up2(x):
    return np.repeat(np.repeat(np.repeat(np.asarray(x, np.float64), 2, 1), 2, 2), 2, 3)


def up2_bwd(dy):
    n, d, h, w, c = dy.shape
    return np.asarray(dy, np.float64).reshape(n, d // 2, 2, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4, 6))


def bf16_round(a):
    """Round to bfloat16 (nearest, ties to even) and return as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
