"""Python binding of the C ABI in include/lbm.h (argument marshalling only).

The functions below carry the C names and forward to the in-tree CUDA library
``_build/libpaper_lbm.so``; every step of the method runs in its kernels.
PyTorch supplies device memory (the two PDF copies) and the CUDA stream.
There is no CPU fallback: if the library is missing the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

LBM_OK = 0
ERRORS = {-1: "LBM_ERR_ARG", -2: "LBM_ERR_SHAPE", -3: "LBM_ERR_CUDA", -4: "LBM_ERR_OOM",
          -5: "LBM_ERR_DIVERGED", -6: "LBM_ERR_TIMEOUT", -7: "LBM_ERR_BOUNDS", -8: "LBM_ERR_CAPACITY"}
LBM_D2Q9, LBM_D3Q19 = 9, 19
LBM_QUASI_COMPRESSIBLE, LBM_INCOMPRESSIBLE = 0, 1
LBM_STORE_F64, LBM_STORE_F32, LBM_STORE_F16S, LBM_STORE_F32S = 0, 1, 2, 3
LBM_ARITH_AUTO, LBM_ARITH_F64, LBM_ARITH_FIXED, LBM_ARITH_FF, LBM_ARITH_FF_TABLE = 0, 1, 2, 3, 4
LBM_OUT_DEVICE, LBM_STATS_RESIDUAL = 1, 2
LBM_LAYOUT_T2C, LBM_LAYOUT_TGB = 0, 1

EXPORTED = ("lbm_build_tilemap", "lbm_init", "lbm_step", "lbm_moments", "lbm_export_pdfs",
            "lbm_import_pdfs", "lbm_get_tiling", "lbm_free", "lbm_last_error", "lbm_stats_noalloc",
            "lbm_build_tilemap_batch", "lbm_init_batch", "lbm_moments_batch", "lbm_export_pdfs_sample",
            "lbm_num_samples", "lbm_moments_sample", "lbm_filter_period2", "lbm_layer_range",
            "lbm_current_copy", "lbm_moments_layers")
LBM_NOALLOC_MAX_BLOCKS = 8192


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class lbm_params(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("model", ctypes.c_int), ("nx", ctypes.c_int),
                ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("tile_a", ctypes.c_int),
                ("periodic", ctypes.c_int * 3), ("tau", ctypes.c_double),
                ("force", ctypes.c_double * 3), ("rho0", ctypes.c_double), ("storage", ctypes.c_int),
                ("arith", ctypes.c_int), ("f16_scale", ctypes.c_double),
                ("block_nodes", ctypes.c_int), ("persistent", ctypes.c_int), ("layout", ctypes.c_int),
                ("prefetch_blocks", ctypes.c_int)]


class lbm_tiling(ctypes.Structure):
    _fields_ = [("ntx", ctypes.c_int32), ("nty", ctypes.c_int32), ("ntz", ctypes.c_int32),
                ("n_tiles", ctypes.c_int32), ("n_ftiles", ctypes.c_int32),
                ("nbr_per_tile", ctypes.c_int32), ("n_fluid", ctypes.c_int64),
                ("pdf_bytes", ctypes.c_size_t), ("ghost_bytes", ctypes.c_size_t)]


class lbm_stats(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3), ("u2", ctypes.c_double),
                ("du2", ctypes.c_double), ("residual", ctypes.c_double), ("n_fluid", ctypes.c_int64),
                ("step", ctypes.c_int64)]


_lib = None
_lock = threading.Lock()


def library(build: bool = True):
    """Load the CUDA library (building it in-tree first when `build`)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            P, I = ctypes.c_void_p, ctypes.c_int
            lib.lbm_build_tilemap.argtypes = [ctypes.POINTER(lbm_params), P, P, P, ctypes.POINTER(lbm_tiling)]
            lib.lbm_init.argtypes = [ctypes.POINTER(P), ctypes.POINTER(lbm_params), P, P, P,
                                     ctypes.c_size_t, P, P, P]
            lib.lbm_step.argtypes = [P, I, P]
            lib.lbm_moments.argtypes = [P, P, P, ctypes.POINTER(lbm_stats), I, P]
            lib.lbm_export_pdfs.argtypes = [P, P, I, P]
            lib.lbm_import_pdfs.argtypes = [P, P, ctypes.c_int64, I, P]
            lib.lbm_get_tiling.argtypes = [P, ctypes.POINTER(lbm_tiling)]
            lib.lbm_free.argtypes = [P]
            lib.lbm_stats_noalloc.argtypes = [P, P, P]
            lib.lbm_build_tilemap_batch.argtypes = [ctypes.POINTER(lbm_params), I, P, P, ctypes.POINTER(lbm_tiling)]
            lib.lbm_init_batch.argtypes = [ctypes.POINTER(P), ctypes.POINTER(lbm_params), I, P, P, P, P,
                                           ctypes.c_size_t, P]
            lib.lbm_moments_batch.argtypes = [P, P, I, P]
            lib.lbm_export_pdfs_sample.argtypes = [P, I, P, I, P]
            lib.lbm_num_samples.argtypes = [P]
            lib.lbm_moments_sample.argtypes = [P, I, P, P, I, P]
            lib.lbm_filter_period2.argtypes = [P, P]
            lib.lbm_layer_range.argtypes = [P, I, I, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
            lib.lbm_current_copy.argtypes = [P]
            lib.lbm_moments_layers.argtypes = [P, I, I, ctypes.POINTER(lbm_stats), I, P]
            lib.lbm_last_error.restype = ctypes.c_char_p
            for name in EXPORTED:
                getattr(lib, name).restype = getattr(lib, name).restype or ctypes.c_int
            lib.lbm_last_error.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def _check(rc):
    if rc != LBM_OK:
        raise LBMError(rc, lbm_last_error())
    return rc


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def lbm_last_error() -> str:
    return library().lbm_last_error().decode()


def make_params(lattice, shape, tile_a, periodic=(0, 0, 0), tau=0.6, force=(0.0, 0.0, 0.0),
                rho0=1.0, model=LBM_QUASI_COMPRESSIBLE, storage=LBM_STORE_F64,
                arith=LBM_ARITH_AUTO, f16_scale=0.0, block_nodes=0, persistent=0,
                layout=LBM_LAYOUT_T2C, prefetch_blocks=0) -> lbm_params:
    """lbm_params from a mask shape (nz, ny, nx) or (ny, nx)."""
    if len(shape) == 2:
        shape = (1,) + tuple(shape)
    nz, ny, nx = shape
    p = lbm_params()
    p.lattice, p.model, p.nx, p.ny, p.nz, p.tile_a = lattice, model, nx, ny, nz, tile_a
    for k in range(3):
        p.periodic[k] = int(bool(periodic[k])) if k < len(periodic) else 0
        p.force[k] = float(force[k]) if k < len(force) else 0.0
    p.tau, p.rho0, p.storage, p.arith, p.f16_scale = float(tau), float(rho0), storage, arith, float(f16_scale)
    p.block_nodes, p.persistent, p.layout = int(block_nodes), int(persistent), int(layout)
    p.prefetch_blocks = int(prefetch_blocks)
    return p


def lbm_build_tilemap(params: lbm_params, mask, want_map=True, want_nbr=True):
    """Returns (lbm_tiling, tile_map[ntz,nty,ntx] or None, nbr[n_ftiles,3^d] or None)."""
    lib = library()
    m = np.ascontiguousarray(mask, np.uint8)
    info = lbm_tiling()
    _check(lib.lbm_build_tilemap(ctypes.byref(params), _ptr(m), None, None, ctypes.byref(info)))
    tm = np.empty((info.ntz, info.nty, info.ntx), np.int32) if want_map else None
    nb = np.empty((info.n_ftiles, info.nbr_per_tile), np.int32) if want_nbr else None
    if want_map or want_nbr:
        _check(lib.lbm_build_tilemap(ctypes.byref(params), _ptr(m), _ptr(tm), _ptr(nb), ctypes.byref(info)))
    return info, tm, nb


def lbm_init(params: lbm_params, mask, pdf_a, pdf_b, pdf_bytes, rho_init=None, u_init=None, stream=None):
    """Returns an opaque context handle (ctypes.c_void_p)."""
    lib = library()
    ctx = ctypes.c_void_p()
    m = np.ascontiguousarray(mask, np.uint8)
    r, u = _field(rho_init), _field(u_init)
    _check(lib.lbm_init(ctypes.byref(ctx), ctypes.byref(params), _ptr(m), _ptr(pdf_a), _ptr(pdf_b),
                        pdf_bytes, _ptr(r), _ptr(u), stream))
    return ctx


def _field(x):
    """An initial field as a contiguous FP64 array: device tensors stay on the
    device (lbm_init reads them in place), anything else goes through numpy."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        import torch

        return x.detach().to(torch.float64).contiguous()
    return np.ascontiguousarray(x, np.float64)


def lbm_step(ctx, nsteps, stream=None):
    return _check(library().lbm_step(ctx, int(nsteps), stream))


def lbm_moments(ctx, rho=None, u=None, stats=None, flags=0, stream=None):
    """Fills rho/u (numpy host arrays or device tensors with LBM_OUT_DEVICE) and
    stats (lbm_stats); returns the status (LBM_ERR_DIVERGED is not raised)."""
    rc = library().lbm_moments(ctx, _ptr(rho), _ptr(u), None if stats is None else ctypes.byref(stats),
                               int(flags), stream)
    if rc not in (LBM_OK, -5):
        _check(rc)
    return rc


def lbm_export_pdfs(ctx, out, flags=0, stream=None):
    return _check(library().lbm_export_pdfs(ctx, _ptr(out), int(flags), stream))


def lbm_import_pdfs(ctx, pdfs, step, flags=0, stream=None):
    return _check(library().lbm_import_pdfs(ctx, _ptr(pdfs), int(step), int(flags), stream))


def lbm_get_tiling(ctx) -> lbm_tiling:
    info = lbm_tiling()
    _check(library().lbm_get_tiling(ctx, ctypes.byref(info)))
    return info


def lbm_stats_noalloc(ctx, stats_dev, stream=None):
    """Mass/momentum sums into a caller-allocated device buffer of 8 doubles,
    without any device allocation (see include/lbm.h)."""
    return _check(library().lbm_stats_noalloc(ctx, _ptr(stats_dev), stream))


def _batch_args(masks):
    ms = [np.ascontiguousarray(m[None] if m.ndim == 2 else m, np.uint8) for m in masks]
    dims = np.array([[m.shape[2], m.shape[1], m.shape[0]] for m in ms], np.int32)
    ptrs = (ctypes.c_void_p * len(ms))(*[m.ctypes.data for m in ms])
    return ms, dims, ptrs


def lbm_build_tilemap_batch(params: lbm_params, masks) -> lbm_tiling:
    ms, dims, ptrs = _batch_args(masks)
    info = lbm_tiling()
    _check(library().lbm_build_tilemap_batch(ctypes.byref(params), len(ms), _ptr(dims), ptrs,
                                             ctypes.byref(info)))
    return info


def lbm_init_batch(params: lbm_params, masks, pdf_a, pdf_b, pdf_bytes, stream=None):
    ms, dims, ptrs = _batch_args(masks)
    ctx = ctypes.c_void_p()
    _check(library().lbm_init_batch(ctypes.byref(ctx), ctypes.byref(params), len(ms), _ptr(dims), ptrs,
                                    _ptr(pdf_a), _ptr(pdf_b), pdf_bytes, stream))
    return ctx


def lbm_moments_batch(ctx, n_samples, flags=0, stream=None):
    """Per-sample lbm_stats (list); LBM_ERR_DIVERGED is returned, not raised."""
    arr = (lbm_stats * n_samples)()
    rc = library().lbm_moments_batch(ctx, ctypes.cast(arr, ctypes.c_void_p), int(flags), stream)
    if rc not in (LBM_OK, -5):
        _check(rc)
    return list(arr), rc


def lbm_filter_period2(ctx, stream=None):
    return _check(library().lbm_filter_period2(ctx, stream))


def lbm_moments_sample(ctx, sample, rho=None, u=None, flags=0, stream=None):
    return _check(library().lbm_moments_sample(ctx, int(sample), _ptr(rho), _ptr(u), int(flags), stream))


def lbm_export_pdfs_sample(ctx, sample, out, flags=0, stream=None):
    return _check(library().lbm_export_pdfs_sample(ctx, int(sample), _ptr(out), int(flags), stream))


def lbm_free(ctx):
    return _check(library().lbm_free(ctx))


def _pdf_buffers(tiling, layout, device):
    """The two device buffers lbm_init takes: two PDF copies, or (ghost-buffer
    layout) the copy and the two ghost sets."""
    import torch

    a = max(int(tiling.pdf_bytes), 256)
    b = max(int(tiling.ghost_bytes), 256) if layout == LBM_LAYOUT_TGB else a
    return [torch.empty(a, dtype=torch.uint8, device=device), torch.empty(b, dtype=torch.uint8, device=device)]


class BatchSolver:
    """A batch context (many geometries, one concatenated tile list) plus its
    two PDF copies held as PyTorch device tensors."""

    def __init__(self, masks, lattice, tile_a, periodic=(0, 0, 0), tau=0.6, force=(0, 0, 0), rho0=1.0,
                 model=LBM_QUASI_COMPRESSIBLE, storage=LBM_STORE_F32S, arith=LBM_ARITH_AUTO,
                 f16_scale=0.0, block_nodes=0, persistent=0, layout=LBM_LAYOUT_T2C, device="cuda",
                 prefetch_blocks=0):
        import torch

        self.masks = [np.ascontiguousarray(m[None] if m.ndim == 2 else m, np.uint8) for m in masks]
        self.q = lattice
        self.params = make_params(lattice, self.masks[0].shape, tile_a, periodic, tau, force, rho0, model,
                                  storage, arith, f16_scale, block_nodes, persistent, layout, prefetch_blocks)
        self.tiling = lbm_build_tilemap_batch(self.params, self.masks)
        nbytes = max(int(self.tiling.pdf_bytes), 256)
        self.device = torch.device(device)
        self.pdf = _pdf_buffers(self.tiling, layout, self.device)
        self.stream = torch.cuda.current_stream(self.device)
        self.ctx = lbm_init_batch(self.params, self.masks, self.pdf[0], self.pdf[1], nbytes, self._s())

    def _s(self):
        return ctypes.c_void_p(self.stream.cuda_stream)

    def step(self, n=1):
        lbm_step(self.ctx, n, self._s())

    def stats(self, residual=False):
        return lbm_moments_batch(self.ctx, len(self.masks), LBM_STATS_RESIDUAL if residual else 0, self._s())

    def filter_period2(self):
        lbm_filter_period2(self.ctx, self._s())

    def export_pdfs(self, k):
        out = np.empty((self.q,) + self.masks[k].shape, np.float64)
        lbm_export_pdfs_sample(self.ctx, k, out, 0, self._s())
        return out

    def close(self):
        if getattr(self, "ctx", None) is not None:
            lbm_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """A context plus its two PDF copies held as PyTorch device tensors."""

    def __init__(self, mask, lattice, tile_a, periodic=(0, 0, 0), tau=0.6, force=(0, 0, 0), rho0=1.0,
                 model=LBM_QUASI_COMPRESSIBLE, storage=LBM_STORE_F64, arith=LBM_ARITH_AUTO,
                 f16_scale=0.0, rho_init=None, u_init=None, block_nodes=0, persistent=0,
                 layout=LBM_LAYOUT_T2C, device="cuda", prefetch_blocks=0):
        import torch

        self.torch = torch
        mask = np.asarray(mask, np.uint8)
        if mask.ndim == 2:
            mask = mask[None]
        self.mask = np.ascontiguousarray(mask)
        self.shape = self.mask.shape
        self.q = lattice
        self.params = make_params(lattice, self.shape, tile_a, periodic, tau, force, rho0, model, storage,
                                  arith, f16_scale, block_nodes, persistent, layout, prefetch_blocks)
        self.tiling, _, _ = lbm_build_tilemap(self.params, self.mask, want_map=False, want_nbr=False)
        nbytes = max(int(self.tiling.pdf_bytes), 256)
        self.device = torch.device(device)
        self.pdf = _pdf_buffers(self.tiling, layout, self.device)
        self.stream = torch.cuda.current_stream(self.device)
        self.ctx = lbm_init(self.params, self.mask, self.pdf[0], self.pdf[1], nbytes, rho_init, u_init,
                            self._s())

    def _s(self):
        return ctypes.c_void_p(self.stream.cuda_stream)

    def step(self, n=1):
        lbm_step(self.ctx, n, self._s())

    def moments(self, residual=False):
        """(rho[nz,ny,nx], u[d,nz,ny,nx], lbm_stats, status) on the host."""
        d = 3 if self.q == LBM_D3Q19 else 2
        rho = np.empty(self.shape, np.float64)
        u = np.empty((d,) + self.shape, np.float64)
        st = lbm_stats()
        rc = lbm_moments(self.ctx, rho, u, st, LBM_STATS_RESIDUAL if residual else 0, self._s())
        return rho, u, st, rc

    def filter_period2(self):
        lbm_filter_period2(self.ctx, self._s())

    def stats(self, residual=False):
        st = lbm_stats()
        rc = lbm_moments(self.ctx, None, None, st, LBM_STATS_RESIDUAL if residual else 0, self._s())
        return st, rc

    def export_pdfs(self):
        out = np.empty((self.q,) + self.shape, np.float64)
        lbm_export_pdfs(self.ctx, out, 0, self._s())
        return out

    def import_pdfs(self, pdfs, step):
        lbm_import_pdfs(self.ctx, np.ascontiguousarray(pdfs, np.float64), step, 0, self._s())

    def close(self):
        if getattr(self, "ctx", None) is not None:
            lbm_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
