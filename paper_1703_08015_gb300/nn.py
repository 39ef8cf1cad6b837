"""Learned warm start (not in the paper).

A 3D U-Net maps a geometry (a 64^3 solid mask plus the body-force scalar as a
second input channel) to an initial density and velocity field.  The solver
starts from the equilibrium of that field instead of rest and so needs fewer
steps to reach its steady state; the LBM residual alone decides convergence,
and the zero start stays the fallback.

Every layer of the network runs in the in-tree CUDA library
(``include/lbm_nn.h``): 3x3x3 convolutions as implicit GEMMs on the tensor
cores (BF16 operands, FP32 accumulation) for the forward pass and for both
backward passes, and the pooling, upsampling, concatenation, loss and Adam
kernels of training.  PyTorch only allocates the buffers, gathers training
batches and supplies the stream.  The training data are steady states that the
solver itself computes (FP32 storage of the shifted PDFs) on seeded sphere
packs.

Output scaling: in creeping flow the steady velocity is linear in the body
force F and inversely proportional to the viscosity nu, and the density
deviation is linear in F, so the network predicts
``t = ((rho - 1) / (a_rho F), u / (a_u F / nu))`` with a_rho and a_u fixed from
the training set so that both have unit mean square over the fluid nodes.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import time

import numpy as np

from . import geometry as geo
from . import lbm

P, I, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
F32, F64 = ctypes.c_float, ctypes.c_double
_DIMS = [P, I, I, I, I, I, P, P]
_SIGS = {
    "lbm_nn_conv3d": [P, I, I, I, I, I, P, P, I, I, I, P, P, P],
    "lbm_nn_weight_flip": [P, I, I, P, P],
    "lbm_nn_conv3d_wgrad": [P, P, I, I, I, I, I, I, I, P, P, P],
    "lbm_nn_relu_mask": [P, P, SZ, P],
    "lbm_nn_pool2": _DIMS,
    "lbm_nn_pool2_bwd": _DIMS,
    "lbm_nn_up2": _DIMS,
    "lbm_nn_up2_bwd": _DIMS,
    "lbm_nn_concat": [P, I, P, I, SZ, P, P],
    "lbm_nn_split": [P, I, I, SZ, P, P, P],
    "lbm_nn_mse": [P, P, P, SZ, I, SZ, P, P, P],
    "lbm_nn_adam": [P, P, P, P, P, SZ, F32, F32, F32, F32, I, P],
    "lbm_nn_add": [P, P, SZ, P, P],
    "lbm_nn_mask_input": [P, SZ, F32, P, P],
    "lbm_nn_fields_to_target": [P, P, SZ, F64, F64, F64, P, P],
    "lbm_nn_target_to_fields": [P, SZ, F64, F64, F64, P, P, P],
    "lbm_nn_f32_to_bf16": [P, SZ, P, P],
    "lbm_nn_bf16_to_f32": [P, SZ, P, P],
    "lbm_nn_gemm_bf16": [P, P, P, I, I, I, P],
    "lbm_nn_conv3d_tc": [P, I, I, I, I, I, P, P, I, I, I, P, P, P],
    "lbm_nn_tc_timeouts": [P],
    "lbm_nn_conv_tune": [I, I],
}
EXPORTED = tuple(_SIGS)
_ready = False

FORCE_REF = 1e-6  # the force channel holds F / FORCE_REF
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "unet_spheres64.npz")


def _lib():
    global _ready
    lib = lbm.library()
    if not _ready:
        for name, sig in _SIGS.items():
            f = getattr(lib, name)
            f.argtypes = sig
            f.restype = ctypes.c_int
        _ready = True
    return lib


def _p(t):
    """Device pointer of a torch tensor, an integer address, or NULL."""
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


def _call(name, *args):
    rc = getattr(_lib(), name)(*args)
    if rc != lbm.LBM_OK:
        raise lbm.LBMError(rc, lbm.lbm_last_error())


# ---- the C entry points, same names and argument order (tensors or addresses) ----

def lbm_nn_gemm_bf16(a, b, c, m, n, k, stream=None):
    _call("lbm_nn_gemm_bf16", _p(a), _p(b), _p(c), m, n, k, stream)


def lbm_nn_conv3d_tc(x, n, d, h, w, cin, wgt, bias, cout, relu, wrap, y, y32, stream=None):
    _call("lbm_nn_conv3d_tc", _p(x), n, d, h, w, cin, _p(wgt), _p(bias), cout, int(relu), int(wrap), _p(y),
          _p(y32), stream)


def lbm_nn_conv_tune(bricks_z=0, cout_tile=0):
    """Fix the halo-tile convolution's bricks per block along z and output
    channels per block (0 = chosen per shape)."""
    _call("lbm_nn_conv_tune", int(bricks_z), int(cout_tile))


def lbm_nn_tc_timeouts():
    """Blocks of the tensor-core kernels whose bounded waits ran out since the
    last call (read and cleared)."""
    v = ctypes.c_uint(0)
    _call("lbm_nn_tc_timeouts", ctypes.byref(v))
    return int(v.value)


def lbm_nn_conv3d(x, n, d, h, w, cin, wgt, bias, cout, relu, wrap, y, y32, stream=None):
    _call("lbm_nn_conv3d", _p(x), n, d, h, w, cin, _p(wgt), _p(bias), cout, int(relu), int(wrap), _p(y), _p(y32),
          stream)


def lbm_nn_weight_flip(wgt, cin, cout, wt, stream=None):
    _call("lbm_nn_weight_flip", _p(wgt), cin, cout, _p(wt), stream)


def lbm_nn_conv3d_wgrad(x, dy, n, d, h, w, cin, cout, wrap, dw, dbias, stream=None):
    _call("lbm_nn_conv3d_wgrad", _p(x), _p(dy), n, d, h, w, cin, cout, int(wrap), _p(dw), _p(dbias), stream)


def lbm_nn_relu_mask(g, act, count, stream=None):
    _call("lbm_nn_relu_mask", _p(g), _p(act), count, stream)


def lbm_nn_pool2(x, n, d, h, w, c, y, stream=None):
    _call("lbm_nn_pool2", _p(x), n, d, h, w, c, _p(y), stream)


def lbm_nn_pool2_bwd(dy, n, d, h, w, c, dx, stream=None):
    _call("lbm_nn_pool2_bwd", _p(dy), n, d, h, w, c, _p(dx), stream)


def lbm_nn_up2(x, n, d, h, w, c, y, stream=None):
    _call("lbm_nn_up2", _p(x), n, d, h, w, c, _p(y), stream)


def lbm_nn_up2_bwd(dy, n, d, h, w, c, dx, stream=None):
    _call("lbm_nn_up2_bwd", _p(dy), n, d, h, w, c, _p(dx), stream)


def lbm_nn_concat(a, ca, b, cb, voxels, y, stream=None):
    _call("lbm_nn_concat", _p(a), ca, _p(b), cb, voxels, _p(y), stream)


def lbm_nn_split(y, ca, cb, voxels, a, b, stream=None):
    _call("lbm_nn_split", _p(y), ca, cb, voxels, _p(a), _p(b), stream)


def lbm_nn_mse(pred, target, mask, voxels, c, count, loss, dpred, stream=None):
    _call("lbm_nn_mse", _p(pred), _p(target), _p(mask), voxels, c, count, _p(loss), _p(dpred), stream)


def lbm_nn_adam(p, g, m, v, pb, count, lr, beta1, beta2, eps, t, stream=None):
    _call("lbm_nn_adam", _p(p), _p(g), _p(m), _p(v), _p(pb), count, lr, beta1, beta2, eps, t, stream)


def lbm_nn_add(a, b, count, y, stream=None):
    _call("lbm_nn_add", _p(a), _p(b), count, _p(y), stream)


def lbm_nn_mask_input(mask, voxels, value, x, stream=None):
    _call("lbm_nn_mask_input", _p(mask), voxels, value, _p(x), stream)


def lbm_nn_fields_to_target(rho, u, voxels, rho0, s_rho, s_u, t, stream=None):
    _call("lbm_nn_fields_to_target", _p(rho), _p(u), voxels, rho0, s_rho, s_u, _p(t), stream)


def lbm_nn_target_to_fields(t, voxels, rho0, s_rho, s_u, rho, u, stream=None):
    _call("lbm_nn_target_to_fields", _p(t), voxels, rho0, s_rho, s_u, _p(rho), _p(u), stream)


def lbm_nn_f32_to_bf16(x, count, y, stream=None):
    _call("lbm_nn_f32_to_bf16", _p(x), count, _p(y), stream)


def lbm_nn_bf16_to_f32(x, count, y, stream=None):
    _call("lbm_nn_bf16_to_f32", _p(x), count, _p(y), stream)


# ---- the network ----

class Layer:
    def __init__(self, name, cin, cout, relu, w_off, b_off):
        self.name, self.cin, self.cout, self.relu = name, cin, cout, relu
        self.w_off, self.b_off = w_off, b_off
        self.nw = 27 * cin * cout


def unet_layers(chans, cin, cout):
    """(name, cin, cout, relu) of the U-Net: two convolutions per level on the
    way down (2x2x2 average pooling between levels), two at the bottom, and on
    the way up nearest upsampling, concatenation [upsampled | skip] and two
    convolutions per level; a linear 3x3x3 head."""
    out = []
    c = cin
    for lv, ch in enumerate(chans[:-1]):
        out += [(f"enc{lv}a", c, ch, True), (f"enc{lv}b", ch, ch, True)]
        c = ch
    out += [("mid_a", c, chans[-1], True), ("mid_b", chans[-1], chans[-1], True)]
    c = chans[-1]
    for lv in reversed(range(len(chans) - 1)):
        out += [(f"dec{lv}a", c + chans[lv], chans[lv], True), (f"dec{lv}b", chans[lv], chans[lv], True)]
        c = chans[lv]
    out.append(("head", c, cout, False))
    return out


class UNet:
    """3D U-Net on channels-last BF16 activations [n][z][y][x][c].

    Parameters live in one flat FP32 master vector (per layer the weights
    [27][cin][cout], then the bias) with its BF16 copy, gradient and Adam
    moments, so that one Adam launch updates everything.  ``wrap`` marks the
    periodic axes of the convolutions (bit 0 = x)."""

    def __init__(self, chans=(16, 32, 64, 128), cin=2, cout=4, wrap=1, seed=0, device="cuda", stream=None):
        import torch

        self.torch = torch
        self.chans, self.cin, self.cout, self.wrap = tuple(chans), cin, cout, wrap
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.layers, off = [], 0
        for name, ci, co, relu in unet_layers(self.chans, cin, cout):
            w_off = off
            off += 27 * ci * co
            b_off = off
            off += co
            off = (off + 7) // 8 * 8  # 16-byte aligned BF16 slices
            self.layers.append(Layer(name, ci, co, relu, w_off, b_off))
        self.by_name = {L.name: L for L in self.layers}
        self.n_params = off
        host = np.zeros(off, np.float32)
        rng = np.random.default_rng(seed)
        for L in self.layers:
            std = math.sqrt((2.0 if L.relu else 0.25) / (27 * L.cin))
            host[L.w_off:L.w_off + L.nw] = rng.normal(0.0, std, L.nw).astype(np.float32)
        self.p = torch.from_numpy(host).to(self.device)
        self.g = torch.zeros_like(self.p)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        self.pb = torch.empty(off, dtype=torch.bfloat16, device=self.device)
        self.wt = torch.empty(off, dtype=torch.bfloat16, device=self.device)
        self.t = 0
        self.acts = None
        self.meta = {}
        lbm_nn_f32_to_bf16(self.p, off, self.pb, self._s())

    def _s(self):
        return ctypes.c_void_p(self.stream.cuda_stream)

    def _w(self, L):
        return self.pb.data_ptr() + 2 * L.w_off

    def _wt(self, L):
        return self.wt.data_ptr() + 2 * L.w_off

    def _b(self, L):
        return self.p.data_ptr() + 4 * L.b_off

    def _empty(self, dims, c, dtype=None):
        return self.torch.empty(tuple(dims) + (c,), dtype=dtype or self.torch.bfloat16, device=self.device)

    def _conv(self, name, x, dims, y32=None, bf16_out=True):
        L = self.by_name[name]
        y = self._empty(dims, L.cout) if bf16_out else None
        lbm_nn_conv3d(x, *dims, L.cin, self._w(L), self._b(L), L.cout, L.relu, self.wrap, y, y32, self._s())
        return y

    def forward(self, x, dims, keep=False):
        """x: BF16 [n][d][h][w][cin] (d, h, w divisible by 2^(levels-1)).
        Returns FP32 [n][d][h][w][cout]; with keep, stores the activations
        that backward() needs."""
        n = dims[0]
        A = {}
        a, cur, skips = x, tuple(dims), []
        for lv, ch in enumerate(self.chans[:-1]):
            a1 = self._conv(f"enc{lv}a", a, cur)
            a2 = self._conv(f"enc{lv}b", a1, cur)
            A[f"enc{lv}a"], A[f"enc{lv}b"], A[f"enc{lv}_in"] = a1, a2, a
            skips.append((a2, cur))
            half = (n, cur[1] // 2, cur[2] // 2, cur[3] // 2)
            pooled = self._empty(half, ch)
            lbm_nn_pool2(a2, *cur, ch, pooled, self._s())
            a, cur = pooled, half
        m1 = self._conv("mid_a", a, cur)
        m2 = self._conv("mid_b", m1, cur)
        A["mid_a"], A["mid_b"], A["mid_in"] = m1, m2, a
        a, ca = m2, self.chans[-1]
        for lv in reversed(range(len(self.chans) - 1)):
            skip, sd = skips[lv]
            cs = self.chans[lv]
            up = self._empty(sd, ca)
            lbm_nn_up2(a, *cur, ca, up, self._s())
            cat = self._empty(sd, ca + cs)
            lbm_nn_concat(up, ca, skip, cs, int(np.prod(sd)), cat, self._s())
            cur = sd
            d1 = self._conv(f"dec{lv}a", cat, cur)
            d2 = self._conv(f"dec{lv}b", d1, cur)
            A[f"dec{lv}a"], A[f"dec{lv}b"], A[f"dec{lv}_in"] = d1, d2, cat
            a, ca = d2, cs
        y32 = self._empty(cur, self.cout, self.torch.float32)
        self._conv("head", a, cur, y32=y32, bf16_out=False)
        A["head_in"] = a
        A["dims"] = cur
        self.acts = A if keep else None
        return y32

    def _bwd(self, name, g, x_in, y_out, dims, need_dx=True):
        """ReLU mask, weight and bias gradient, and the gradient of the input."""
        L = self.by_name[name]
        vox = int(np.prod(dims))
        if L.relu:
            lbm_nn_relu_mask(g, y_out, vox * L.cout, self._s())
        lbm_nn_conv3d_wgrad(x_in, g, *dims, L.cin, L.cout, self.wrap, self.g.data_ptr() + 4 * L.w_off,
                            self.g.data_ptr() + 4 * L.b_off, self._s())
        if not need_dx:
            return None
        dx = self._empty(dims, L.cin)
        lbm_nn_conv3d(g, *dims, L.cout, self._wt(L), None, L.cin, 0, self.wrap, dx, None, self._s())
        return dx

    def backward(self, dout):
        """Accumulate the parameter gradients of the last forward(keep=True)
        for dL/dy = dout (BF16, the layout of the output)."""
        A = self.acts
        if A is None:
            raise RuntimeError("backward() needs forward(keep=True) first")
        for L in self.layers:
            lbm_nn_weight_flip(self._w(L), L.cin, L.cout, self._wt(L), self._s())
        dims = A["dims"]
        n = dims[0]
        nl = len(self.chans)
        level = [dims]
        for _ in range(nl - 1):
            c = level[-1]
            level.append((n, c[1] // 2, c[2] // 2, c[3] // 2))
        g = self._bwd("head", dout, A["head_in"], None, dims)
        dskip = {}
        for lv in range(nl - 1):
            cur = level[lv]
            g = self._bwd(f"dec{lv}b", g, A[f"dec{lv}a"], A[f"dec{lv}b"], cur)
            g = self._bwd(f"dec{lv}a", g, A[f"dec{lv}_in"], A[f"dec{lv}a"], cur)
            ca, cs = self.chans[lv + 1], self.chans[lv]
            du, ds = self._empty(cur, ca), self._empty(cur, cs)
            lbm_nn_split(g, ca, cs, int(np.prod(cur)), du, ds, self._s())
            dskip[lv] = ds
            g = self._empty(level[lv + 1], ca)
            lbm_nn_up2_bwd(du, *level[lv + 1], ca, g, self._s())
        cur = level[nl - 1]
        g = self._bwd("mid_b", g, A["mid_a"], A["mid_b"], cur)
        g = self._bwd("mid_a", g, A["mid_in"], A["mid_a"], cur)
        for lv in reversed(range(nl - 1)):
            cur, ch = level[lv], self.chans[lv]
            gp = self._empty(cur, ch)
            lbm_nn_pool2_bwd(g, *cur, ch, gp, self._s())
            lbm_nn_add(gp, dskip[lv], int(np.prod(cur)) * ch, gp, self._s())
            g = self._bwd(f"enc{lv}b", gp, A[f"enc{lv}a"], A[f"enc{lv}b"], cur)
            g = self._bwd(f"enc{lv}a", g, A[f"enc{lv}_in"], A[f"enc{lv}a"], cur, need_dx=lv > 0)
        self.acts = None

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.t += 1
        lbm_nn_adam(self.p, self.g, self.m, self.v, self.pb, self.n_params, lr, beta1, beta2, eps, self.t,
                    self._s())

    # ---- persistence: BF16 weights (what the kernels read) and FP32 biases ----
    def state(self):
        bits = self.pb.cpu().view(self.torch.int16).numpy().view(np.uint16)
        biases = self.p.cpu().numpy()
        return bits, biases

    def save(self, path, **meta):
        bits, biases = self.state()
        keep = np.zeros(self.n_params, bool)
        for L in self.layers:
            keep[L.b_off:L.b_off + L.cout] = True
        self.meta.update(meta)
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        np.savez_compressed(path, weights_bf16=bits, biases=biases[keep],
                            config=json.dumps({"chans": self.chans, "cin": self.cin, "cout": self.cout,
                                               "wrap": self.wrap, **self.meta}))

    @classmethod
    def load(cls, path, device="cuda", stream=None):
        import torch

        z = np.load(path)
        cfg = json.loads(str(z["config"]))
        net = cls(cfg["chans"], cfg["cin"], cfg["cout"], cfg["wrap"], device=device, stream=stream)
        bits = np.asarray(z["weights_bf16"], np.uint16)
        if bits.size != net.n_params:
            raise ValueError(f"{path}: {bits.size} parameters, the network has {net.n_params}")
        host = (bits.astype(np.uint32) << 16).view(np.float32).copy()
        b = np.asarray(z["biases"], np.float32)
        k = 0
        for L in net.layers:
            host[L.b_off:L.b_off + L.cout] = b[k:k + L.cout]
            k += L.cout
        net.p.copy_(torch.from_numpy(host))
        net.pb.copy_(torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16))
        net.meta = {k_: v for k_, v in cfg.items() if k_ not in ("chans", "cin", "cout", "wrap")}
        return net


# ---- data: steady states computed by the solver ----

def percolates_x(mask):
    """True if a fluid cluster winds around the periodic x axis (18-connected,
    the D3Q19 links).  Without one the steady flow is zero and a relative
    residual cannot fall, so such geometries are not used.  Clusters are
    labelled without the wrap; each link across the x boundary joins two
    labels with a winding step of +1, and a cluster winds when two paths
    between the same labels differ in winding."""
    from scipy import ndimage

    lab, n = ndimage.label(mask.astype(bool), ndimage.generate_binary_structure(3, 2))
    if n == 0:
        return False
    nz, ny, _ = mask.shape
    right, left = lab[:, :, -1], lab[:, :, 0]
    edges = set()
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            if abs(dz) + abs(dy) > 1:  # x step plus at most one more axis: D3Q19 links
                continue
            z0, z1 = max(0, -dz), nz - max(0, dz)
            y0, y1 = max(0, -dy), ny - max(0, dy)
            a = right[z0:z1, y0:y1]
            b = left[z0 + dz:z1 + dz, y0 + dy:y1 + dy]
            both = (a > 0) & (b > 0)
            edges.update(zip(a[both].tolist(), b[both].tolist()))
    adj = {}
    for a, b in edges:
        adj.setdefault(a, []).append((b, 1))
        adj.setdefault(b, []).append((a, -1))
    wind = {}
    for start in adj:
        if start in wind:
            continue
        wind[start] = 0
        stack = [start]
        while stack:
            v = stack.pop()
            for w, step in adj[v]:
                if w not in wind:
                    wind[w] = wind[v] + step
                    stack.append(w)
                elif wind[w] != wind[v] + step:
                    return True
    return False


def sample_geometries(n, seed, side=64, phi=(0.1, 0.6)):
    """n seeded sphere packs (radius 4-12, fluid fraction uniform in phi) that
    percolate along x; returns (masks, infos)."""
    rng = np.random.default_rng(seed)
    masks, infos, k = [], [], 0
    while len(masks) < n:
        target = float(rng.uniform(*phi))
        m, info = geo.sphere_pack_3d(side, seed=seed * 1_000_003 + k, target_fluid=target)
        k += 1
        if percolates_x(m):
            masks.append(m)
            infos.append({"target_fluid": target, **info})
    return masks, infos


def steady_states(masks, tau=0.6, force=1e-6, storage=lbm.LBM_STORE_F32S, target=1e-6, check_every=100,
                  max_steps=150000, batch=64, filter_period2=True, device="cuda", log=None):
    """Runs every geometry to residual < target and returns the steady fields
    as FP32 [n][z][y][x][4] = (rho - 1, u_x, u_y, u_z) on the device, plus the
    per-sample step counts (None where it did not converge).  Geometries are
    batched (one concatenated tile list per batch) in order of fluid fraction,
    so that each batch holds samples of similar convergence time; with
    filter_period2 the period-2 mode is removed after every residual check
    (lbm_filter_period2)."""
    import torch

    dev = torch.device(device)
    side = masks[0].shape
    vox = int(np.prod(side))
    out = torch.empty((len(masks),) + side + (4,), dtype=torch.float32, device=dev)
    steps_to = [None] * len(masks)
    rho = torch.empty(vox, dtype=torch.float64, device=dev)
    u = torch.empty(3 * vox, dtype=torch.float64, device=dev)
    order = np.argsort([float(m.mean()) for m in masks], kind="stable")
    for c0 in range(0, len(masks), batch):
        ids = order[c0:c0 + batch]
        t0 = time.perf_counter()
        b = lbm.BatchSolver([masks[i] for i in ids], lbm.LBM_D3Q19, 4, (1, 0, 0), tau, (force, 0, 0),
                            storage=storage, device=dev)
        b.stats(residual=True)
        n = 0
        while n < max_steps:
            b.step(check_every)
            n += check_every
            st, _ = b.stats(residual=True)
            for k, s in enumerate(st):
                if steps_to[ids[k]] is None and s.residual < target:
                    steps_to[ids[k]] = n
            if all(steps_to[i] is not None for i in ids):
                break
            if filter_period2:
                b.filter_period2()
        for k, i in enumerate(ids):
            lbm.lbm_moments_sample(b.ctx, k, rho, u, lbm.LBM_OUT_DEVICE, b._s())
            lbm_nn_fields_to_target(rho, u, vox, 1.0, 1.0, 1.0, out[i], b._s())
        torch.cuda.synchronize(dev)
        b.close()
        if log:
            phis = [float(masks[i].mean()) for i in ids]
            log(f"steady states {c0 + len(ids)}/{len(masks)} (fluid {min(phis):.2f}-{max(phis):.2f}): {n} steps, "
                f"{sum(steps_to[i] is None for i in ids)} not converged, {time.perf_counter() - t0:.1f} s")
    return out, steps_to


def inputs_from_masks(masks_dev, force, stream=None):
    """BF16 network input [n][z][y][x][2] from device uint8 masks [n][z][y][x]."""
    import torch

    x = torch.empty(tuple(masks_dev.shape) + (2,), dtype=torch.bfloat16, device=masks_dev.device)
    lbm_nn_mask_input(masks_dev, masks_dev.numel(), float(force / FORCE_REF), x, stream)
    return x


def augment(x, t, m, code):
    """One of the 16 symmetries of creeping flow driven along a periodic x
    axis, applied to a batch (input x [n,z,y,x,2], target t [n,z,y,x,4] =
    (rho - 1, u_x, u_y, u_z), mask m [n,z,y,x]).  code bit 0: mirror y
    (u_y -> -u_y); bit 1: mirror z (u_z -> -u_z); bit 2: swap y and z (u_y <->
    u_z); bit 3: mirror x, which by linearity in the force negates u_y, u_z
    and rho - 1 and keeps u_x."""
    sign = [1.0, 1.0, 1.0, 1.0]
    if code & 1:
        x, t, m = x.flip(2), t.flip(2), m.flip(2)
        sign[2] = -sign[2]
    if code & 2:
        x, t, m = x.flip(1), t.flip(1), m.flip(1)
        sign[3] = -sign[3]
    if code & 4 and x.shape[1] == x.shape[2]:
        x, t, m = x.transpose(1, 2), t.transpose(1, 2)[..., [0, 1, 3, 2]], m.transpose(1, 2)
        sign[2], sign[3] = sign[3], sign[2]
    if code & 8:
        x, t, m = x.flip(3), t.flip(3), m.flip(3)
        sign[0], sign[2], sign[3] = -sign[0], -sign[2], -sign[3]
    if sign != [1.0, 1.0, 1.0, 1.0]:
        t = t * t.new_tensor(sign)
    return x.contiguous(), t.contiguous(), m.contiguous()


def train(net, masks_dev, fields, force, nu, epochs=20, batch=8, lr=2e-3, lr_min=2e-5, seed=0, log=None,
          log_every=50, augment_data=True):
    """Adam on the masked mean-squared error of the scaled (rho - 1, u).
    fields: FP32 [n][z][y][x][4] raw steady fields (rho - 1, u) from
    steady_states().  Fixes the output scales a_rho, a_u from the data.  With
    augment_data every batch is mapped by a random flow symmetry (augment()).
    Returns the loss history [(iteration, loss)]."""
    torch = net.torch
    dev = net.device
    n = fields.shape[0]
    dims_one = tuple(fields.shape[1:4])
    vox = int(np.prod(dims_one))
    fl = masks_dev.bool()
    # output scales: unit mean square over fluid nodes (normalisation metadata)
    r2 = float((fields[..., 0][fl].double() ** 2).mean()) / force ** 2
    u2 = float((fields[..., 1:][fl].double() ** 2).mean()) * (nu / force) ** 2
    a_rho, a_u = math.sqrt(max(r2, 1e-300)), math.sqrt(max(u2, 1e-300))
    net.meta.update({"a_rho": a_rho, "a_u": a_u, "force_ref": FORCE_REF})
    s_rho, s_u = a_rho * force, a_u * force / nu
    tgt = fields.clone()
    tgt[..., 0] /= s_rho
    tgt[..., 1:] /= s_u
    tgt[~fl] = 0.0
    x_all = inputs_from_masks(masks_dev, force, net._s())
    counts = fl.reshape(n, -1).sum(dim=1).cpu().numpy()
    loss_dev = torch.zeros(1, dtype=torch.float64, device=dev)
    rng = np.random.default_rng(seed)
    iters = epochs * (n // batch)
    hist, it = [], 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        order = rng.permutation(n)
        for b0 in range(0, n - batch + 1, batch):
            idx = torch.as_tensor(order[b0:b0 + batch], device=dev)
            xb = x_all.index_select(0, idx)
            tb = tgt.index_select(0, idx)
            mb = masks_dev.index_select(0, idx)
            if augment_data:
                xb, tb, mb = augment(xb, tb, mb, int(rng.integers(16)))
            dims = (batch,) + dims_one
            y = net.forward(xb, dims, keep=True)
            dout = torch.empty(y.shape, dtype=torch.bfloat16, device=dev)
            lbm_nn_mse(y, tb, mb, batch * vox, net.cout, int(counts[order[b0:b0 + batch]].sum()), loss_dev, dout,
                       net._s())
            net.backward(dout)
            frac = it / max(iters - 1, 1)
            net.adam(lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * frac)))
            if it % log_every == 0 or it == iters - 1:
                loss = float(loss_dev.item())
                hist.append((it, loss))
                if log:
                    log(f"epoch {ep} iter {it}/{iters} loss {loss:.4e} ({time.perf_counter() - t0:.0f} s)")
            it += 1
    return hist


def predict_fields(net, mask, force, nu, on_device=False):
    """Warm-start (rho[nz][ny][nx], u[3][nz][ny][nx]) FP64 fields for one
    geometry, computed on the device by the network: host arrays, or with
    on_device the device tensors (lbm_init reads them in place)."""
    torch = net.torch
    m = torch.from_numpy(np.ascontiguousarray(mask, np.uint8)).to(net.device)[None]
    x = inputs_from_masks(m, force, net._s())
    dims = (1,) + tuple(mask.shape)
    y = net.forward(x, dims)
    vox = int(np.prod(mask.shape))
    rho = torch.empty(vox, dtype=torch.float64, device=net.device)
    u = torch.empty(3 * vox, dtype=torch.float64, device=net.device)
    lbm_nn_target_to_fields(y, vox, 1.0, net.meta["a_rho"] * force, net.meta["a_u"] * force / nu, rho, u,
                            net._s())
    if on_device:  # work queued on the current stream after this sees the fields
        torch.cuda.current_stream(net.device).wait_stream(net.stream)
        return rho.view(tuple(mask.shape)), u.view((3,) + tuple(mask.shape))
    return rho.cpu().numpy().reshape(mask.shape), u.cpu().numpy().reshape((3,) + tuple(mask.shape))


def time_to_steady(mask, net=None, tau=0.6, force=1e-6, storage=lbm.LBM_STORE_F64, target=1e-6, check_every=100,
                   max_steps=60000, filter_period2=True, finish=None, stall_checks=10, device="cuda"):
    """Wall time and steps until the LBM residual (relative change of u over
    check_every steps) falls below target, from rest or from the network's
    prediction; the timed region includes tiling, initialisation and network
    inference.  With filter_period2 the state is replaced by the mean of two
    consecutive states after every residual check that has not converged
    (lbm_filter_period2).  With `finish` (a storage form), a run whose residual
    stops falling (no 5 % gain over `stall_checks` checks: the rounding floor
    of a reduced storage form) continues from its state in that storage; the
    residual of the finishing form still decides convergence.  Returns a dict
    (converged, steps, seconds, permeability, velocity field on the fluid
    nodes, steps taken before the switch)."""
    import torch

    dev = torch.device(device)
    nu = (tau - 0.5) / 3.0
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    rho0 = u0 = None
    if net is not None:
        rho0, u0 = predict_fields(net, mask, force, nu, on_device=True)
    s = lbm.Solver(mask, lbm.LBM_D3Q19, 4, (1, 0, 0), tau, (force, 0, 0), storage=storage, rho_init=rho0,
                   u_init=u0, device=dev)
    s.stats(residual=True)
    n, st, rc, hist, switched_at, floor = 0, None, 0, [], None, None
    while n < max_steps:
        s.step(check_every)
        n += check_every
        st, rc = s.stats(residual=True)
        if rc != 0 or st.residual < target:
            break
        hist.append(st.residual)
        if (finish is not None and switched_at is None and len(hist) > stall_checks
                and hist[-1] > 0.95 * hist[-1 - stall_checks]):
            # the reduced form has reached its floor: carry the state over
            pdfs = torch.empty((19,) + mask.shape, dtype=torch.float64, device=dev)
            lbm.lbm_export_pdfs(s.ctx, pdfs, lbm.LBM_OUT_DEVICE, s._s())
            s2 = lbm.Solver(mask, lbm.LBM_D3Q19, 4, (1, 0, 0), tau, (force, 0, 0), storage=finish, device=dev)
            lbm.lbm_import_pdfs(s2.ctx, pdfs, n, lbm.LBM_OUT_DEVICE, s2._s())
            s.close()
            del pdfs
            s, switched_at, floor = s2, n, min(hist)
            s.stats(residual=True)
            continue
        if filter_period2:
            s.filter_period2()
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    rho, u, _, _ = s.moments()
    s.close()
    fl = mask.astype(bool)
    return {"converged": bool(rc == 0 and st.residual < target), "steps": n, "seconds": dt,
            "residual": float(st.residual), "permeability": nu * float(np.sum(u[0][fl])) / mask.size / force,
            "u": u[:, fl], "status": int(rc), "switched_at": switched_at, "residual_floor_before_switch": floor}


def solve_to_steady(mask, net=None, **kw):
    """Warm start with the network when given, falling back to the zero start
    if the warm-started run does not converge; the LBM residual decides."""
    r = time_to_steady(mask, net, **kw)
    if net is not None and not r["converged"]:
        z = time_to_steady(mask, None, **kw)
        z["seconds"] += r["seconds"]
        z["fallback"] = True
        return z
    return r
