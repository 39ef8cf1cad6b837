"""Plain FP64 reference of the warm-start network's operations (TEST
INFRASTRUCTURE ONLY; not in the paper).

Tensors are channels-last numpy arrays x[n, z, y, x, c].  The convolution is
3x3x3 with zero padding 1 and stride 1, weights w[tap, ci, co] with
tap = 9 dz + 3 dy + dx (dz, dy, dx in 0..2 standing for offsets -1, 0, +1):

    y[p, co] = sum_tap sum_ci w[tap, ci, co] x[p + off(tap), ci] + b[co]

Along the axes set in ``wrap`` (bit 0 = x, bit 1 = y, bit 2 = z) the input is
periodic instead of zero-padded.  Written as an explicit sum over the 27 taps
of shifted copies of the padded input; the tests check it against
scipy.ndimage.correlate, its adjoint identities and finite differences.
"""
from __future__ import annotations

import numpy as np

OFFSETS = [(dz - 1, dy - 1, dx - 1) for dz in range(3) for dy in range(3) for dx in range(3)]


def _shifted(x, off, wrap=0):
    """x[p + off] for every p (x is [n, z, y, x, c]): zero outside the box,
    periodic along the axes set in `wrap`."""
    dz, dy, dx = off
    xp = x
    for axis, bit in ((1, 4), (2, 2), (3, 1)):
        width = [(0, 0)] * 5
        width[axis] = (1, 1)
        xp = np.pad(xp, width, mode="wrap" if wrap & bit else "constant")
    n, d, h, w, c = x.shape
    return xp[:, 1 + dz:1 + dz + d, 1 + dy:1 + dy + h, 1 + dx:1 + dx + w, :]


def conv3d(x, w, b=None, relu=False, wrap=0):
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    y = np.zeros(x.shape[:4] + (w.shape[2],))
    for tap, off in enumerate(OFFSETS):
        y += _shifted(x, off, wrap) @ w[tap]
    if b is not None:
        y += np.asarray(b, np.float64)
    return np.maximum(y, 0.0) if relu else y


def conv3d_bwd_data(dy, w, wrap=0):
    """dL/dx for y = conv3d(x, w): sum_tap dy[p - off(tap)] w[tap]^T."""
    dy = np.asarray(dy, np.float64)
    w = np.asarray(w, np.float64)
    dx = np.zeros(dy.shape[:4] + (w.shape[1],))
    for tap, off in enumerate(OFFSETS):
        dx += _shifted(dy, tuple(-o for o in off), wrap) @ w[tap].T
    return dx


def conv3d_bwd_weight(x, dy, wrap=0):
    """dL/dw[tap, ci, co] = sum_p x[p + off(tap), ci] dy[p, co]; dL/db = sum_p dy."""
    x = np.asarray(x, np.float64)
    dy = np.asarray(dy, np.float64)
    cin, cout = x.shape[4], dy.shape[4]
    dw = np.zeros((27, cin, cout))
    for tap, off in enumerate(OFFSETS):
        dw[tap] = _shifted(x, off, wrap).reshape(-1, cin).T @ dy.reshape(-1, cout)
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


def _ident(a):
    return a


def unet_forward(params, x, chans, wrap=0, rnd=_ident):
    """FP64 U-Net: per level on the way down conv+ReLU twice then 2x2x2 average
    pooling; two conv+ReLU at the bottom; per level on the way up nearest
    upsampling, concatenation [upsampled | skip], conv+ReLU twice; a linear
    head.  params[name] = (w[27, cin, cout], b[cout]) with the names enc<l>a,
    enc<l>b, mid_a, mid_b, dec<l>a, dec<l>b, head.  `rnd` is applied to every
    stored activation (bf16_round mirrors BF16 storage); the head output is
    not rounded.  Returns (y, cache)."""
    def conv(name, a, relu=True):
        w, b = params[name]
        return rnd(conv3d(a, w, b, relu, wrap))

    c = {}
    a, skips = x, []
    for lv in range(len(chans) - 1):
        c[f"enc{lv}_in"] = a
        c[f"enc{lv}a"] = conv(f"enc{lv}a", a)
        c[f"enc{lv}b"] = conv(f"enc{lv}b", c[f"enc{lv}a"])
        skips.append(c[f"enc{lv}b"])
        a = rnd(pool2(c[f"enc{lv}b"]))
    c["mid_in"] = a
    c["mid_a"] = conv("mid_a", a)
    c["mid_b"] = conv("mid_b", c["mid_a"])
    a = c["mid_b"]
    for lv in reversed(range(len(chans) - 1)):
        cat = np.concatenate([up2(a), skips[lv]], axis=4)
        c[f"dec{lv}_in"] = cat
        c[f"dec{lv}a"] = conv(f"dec{lv}a", cat)
        c[f"dec{lv}b"] = conv(f"dec{lv}b", c[f"dec{lv}a"])
        a = c[f"dec{lv}b"]
    c["head_in"] = a
    w, b = params["head"]
    return conv3d(a, w, b, False, wrap), c


def unet_backward(params, cache, dy, chans, wrap=0, rnd=_ident):
    """Gradients {name: (dw, db)} of sum(y * dy) for the network of
    unet_forward, by the chain rule layer by layer in reverse; `rnd` is
    applied to every stored activation gradient."""
    grads = {}

    def bwd(name, g, x_in, y_out, need_dx=True):
        w, _ = params[name]
        if y_out is not None:
            g = g * (y_out > 0)
        grads[name] = conv3d_bwd_weight(x_in, g, wrap)
        return rnd(conv3d_bwd_data(g, w, wrap)) if need_dx else None

    nl = len(chans)
    g = bwd("head", np.asarray(dy, np.float64), cache["head_in"], None)
    dskip = {}
    for lv in range(nl - 1):
        g = bwd(f"dec{lv}b", g, cache[f"dec{lv}a"], cache[f"dec{lv}b"])
        g = bwd(f"dec{lv}a", g, cache[f"dec{lv}_in"], cache[f"dec{lv}a"])
        ca = chans[lv + 1]
        dskip[lv] = g[..., ca:]
        g = rnd(up2_bwd(g[..., :ca]))
    g = bwd("mid_b", g, cache["mid_a"], cache["mid_b"])
    g = bwd("mid_a", g, cache["mid_in"], cache["mid_a"])
    for lv in reversed(range(nl - 1)):
        g = rnd(rnd(pool2_bwd(g)) + dskip[lv])
        g = bwd(f"enc{lv}b", g, cache[f"enc{lv}a"], cache[f"enc{lv}b"])
        g = bwd(f"enc{lv}a", g, cache[f"enc{lv}_in"], cache[f"enc{lv}a"], need_dx=lv > 0)
    return grads
