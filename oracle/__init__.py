"""Plain FP64 CPU oracle for the sparse-geometry BGK lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it; the CUDA library never imports it, and
the two share no code.

It computes the plain dense, masked LBM of Tomczak & Szafran
(arXiv:1703.08015): Eq. 7 time step, Eq. 2 BGK collision, Eq. 3
(quasi-compressible) or Eq. 4 (incompressible) equilibrium, Eq. 5 / Eq. 6
velocity, pull streaming that only propagates between non-solid nodes
(Sec. 3.2) with halfway bounce-back for the value that cannot be gathered,
periodic or walled domain edges, and Guo forcing (not in the paper).  The
arithmetic lives in ``lbm_ref.c``; this module only marshals numpy arrays.

Array layout: ``mask[z, y, x]`` (uint8, 1 = fluid) and ``f[i, z, y, x]``
(float64); 2D lattices use nz = 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import tilemap_ref  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_ref.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_ref.so")
_lock = threading.Lock()
_lib = None

D2Q9 = 9
D3Q19 = 19
QUASI_COMPRESSIBLE = 0
INCOMPRESSIBLE = 1


def build(force: bool = False) -> str:
    """Compile ``lbm_ref.c`` into ``oracle/_build/liblbm_ref.so`` (gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            lib.ref_lattice.argtypes = [I, P, P, P, P, P]
            lib.ref_equilibrium.argtypes = [I, I, D, P, P]
            lib.ref_collide.argtypes = [I, I, D, P, P, P]
            lib.ref_init.argtypes = [I, I, I, I, I, P, D, P, P, P]
            lib.ref_step.argtypes = [I, I, I, I, I, P, P, D, P, P, P, I]
            lib.ref_step_nodes.argtypes = [I, I, I, I, I, P, P, D, P, P, P,
                                           ctypes.c_int64, P]
            lib.ref_moments.argtypes = [I, I, I, I, I, P, P, P, P, P, P, I]
            lib.ref_total_mass.argtypes = [I, I, I, I, P, P]
            lib.ref_total_mass.restype = D
            lib.ref_threads.argtypes = [I]
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Lattice:
    """Velocity set of a DdQq lattice as the oracle defines it."""

    def __init__(self, lattice: int):
        lib = _load()
        q = ctypes.c_int()
        d = ctypes.c_int()
        c = np.zeros((19, 3), np.int32)
        w = np.zeros(19, np.float64)
        opp = np.zeros(19, np.int32)
        if lib.ref_lattice(lattice, ctypes.byref(q), ctypes.byref(d), _p(c), _p(w), _p(opp)):
            raise ValueError(f"unknown lattice {lattice}")
        self.id = lattice
        self.q = q.value
        self.d = d.value
        self.c = c[: self.q].copy()
        self.w = w[: self.q].copy()
        self.opp = opp[: self.q].copy()


def _dims(mask):
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    if mask.ndim == 2:
        mask = mask[None]
    nz, ny, nx = mask.shape
    return mask, nx, ny, nz


def _periodic(periodic):
    p = np.zeros(3, np.int32)
    p[: len(periodic)] = [1 if v else 0 for v in periodic]
    return p


def equilibrium(lattice: int, rho: float, u, model: int = QUASI_COMPRESSIBLE) -> np.ndarray:
    """f^eq of Eq. 3 (model 0) or Eq. 4 (model 1) for one node."""
    lib = _load()
    uu = np.zeros(3, np.float64)
    uu[: len(u)] = u
    feq = np.zeros(19, np.float64)
    lib.ref_equilibrium(lattice, model, float(rho), _p(uu), _p(feq))
    return feq[: Lattice(lattice).q].copy()


def collide(lattice: int, f, tau: float, force=(0.0, 0.0, 0.0),
            model: int = QUASI_COMPRESSIBLE) -> np.ndarray:
    """Post-collision values of one node from its q gathered values."""
    lib = _load()
    f = np.ascontiguousarray(f, np.float64)
    F = np.zeros(3, np.float64)
    F[: len(force)] = force
    out = np.zeros_like(f)
    lib.ref_collide(lattice, model, float(tau), _p(F), _p(f), _p(out))
    return out


def init(lattice: int, mask, rho0: float = 1.0, rho=None, u=None,
         model: int = QUASI_COMPRESSIBLE) -> np.ndarray:
    """Equilibrium start field f[i, z, y, x] (solid nodes hold 0)."""
    lib = _load()
    mask, nx, ny, nz = _dims(mask)
    q = Lattice(lattice).q
    f = np.zeros((q, nz, ny, nx), np.float64)
    r = None if rho is None else np.ascontiguousarray(np.broadcast_to(rho, (nz, ny, nx)), np.float64)
    uu = None
    if u is not None:
        uu = np.zeros((3, nz, ny, nx), np.float64)
        u = np.asarray(u, np.float64)
        uu[: u.shape[0]] = u.reshape((u.shape[0], nz, ny, nx))
    rc = lib.ref_init(lattice, model, nx, ny, nz, _p(mask), float(rho0),
                      None if r is None else _p(r), None if uu is None else _p(uu), _p(f))
    if rc:
        raise ValueError("ref_init failed")
    return f


def step(lattice: int, mask, periodic, tau: float, force, f, out=None,
         model: int = QUASI_COMPRESSIBLE, nthreads: int = 0) -> np.ndarray:
    """One time step; returns the new post-collision field."""
    lib = _load()
    mask, nx, ny, nz = _dims(mask)
    F = np.zeros(3, np.float64)
    F[: len(force)] = force
    f = np.ascontiguousarray(f, np.float64)
    if out is None:
        out = np.empty_like(f)
    rc = lib.ref_step(lattice, model, nx, ny, nz, _p(_periodic(periodic)), _p(mask),
                      float(tau), _p(F), _p(f), _p(out), int(nthreads))
    if rc:
        raise ValueError("ref_step failed")
    return out


def run(lattice: int, mask, periodic, tau: float, force, f, nsteps: int,
        model: int = QUASI_COMPRESSIBLE, nthreads: int = 0) -> np.ndarray:
    """`nsteps` time steps from f (two buffers, swapped each step)."""
    a = np.array(f, np.float64, copy=True)
    b = np.empty_like(a)
    for _ in range(int(nsteps)):
        step(lattice, mask, periodic, tau, force, a, out=b, model=model, nthreads=nthreads)
        a, b = b, a
    return a


def step_nodes(lattice: int, mask, periodic, tau: float, force, f, nodes,
               model: int = QUASI_COMPRESSIBLE) -> np.ndarray:
    """One step evaluated only at flat node indices `nodes` -> [len, q]."""
    lib = _load()
    mask, nx, ny, nz = _dims(mask)
    F = np.zeros(3, np.float64)
    F[: len(force)] = force
    f = np.ascontiguousarray(f, np.float64)
    nodes = np.ascontiguousarray(nodes, np.int64)
    q = Lattice(lattice).q
    out = np.zeros((len(nodes), q), np.float64)
    rc = lib.ref_step_nodes(lattice, model, nx, ny, nz, _p(_periodic(periodic)), _p(mask),
                            float(tau), _p(F), _p(f), _p(nodes), len(nodes), _p(out))
    if rc:
        raise ValueError("ref_step_nodes failed (node out of range or solid)")
    return out


def moments(lattice: int, mask, periodic, force, f, model: int = QUASI_COMPRESSIBLE,
            nthreads: int = 0):
    """(rho[z,y,x], u[3,z,y,x]) that the next step will collide with."""
    lib = _load()
    mask, nx, ny, nz = _dims(mask)
    F = np.zeros(3, np.float64)
    F[: len(force)] = force
    f = np.ascontiguousarray(f, np.float64)
    rho = np.empty((nz, ny, nx), np.float64)
    u = np.empty((3, nz, ny, nx), np.float64)
    rc = lib.ref_moments(lattice, model, nx, ny, nz, _p(_periodic(periodic)), _p(mask),
                         _p(F), _p(f), _p(rho), _p(u), int(nthreads))
    if rc:
        raise ValueError("ref_moments failed")
    return rho, u


def total_mass(lattice: int, mask, f) -> float:
    """Sum of all post-collision PDFs over fluid nodes."""
    lib = _load()
    mask, nx, ny, nz = _dims(mask)
    f = np.ascontiguousarray(f, np.float64)
    return float(lib.ref_total_mass(lattice, nx, ny, nz, _p(mask), _p(f)))


def residual(u_now, u_prev, mask) -> float:
    """Steady-state residual ||u(t) - u(t-K)||_2 / ||u(t)||_2 over fluid nodes
    (not in the paper; plain FP64 sums)."""
    m = np.asarray(mask).reshape(-1) != 0
    a = np.asarray(u_now, np.float64).reshape(u_now.shape[0], -1)[:, m]
    b = np.asarray(u_prev, np.float64).reshape(u_prev.shape[0], -1)[:, m]
    den = float(np.sqrt(np.sum(a * a)))
    return float(np.sqrt(np.sum((a - b) ** 2))) / den if den > 0 else float("inf")


def threads(nthreads: int = 0) -> int:
    """OpenMP thread count the oracle uses for `nthreads` (0 = all)."""
    return int(_load().ref_threads(int(nthreads)))
