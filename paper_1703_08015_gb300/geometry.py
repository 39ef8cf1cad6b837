"""Seeded synthetic geometries (input generators only).

The paper's own geometries (a cerebral aneurysm, an aorta coarctation, the
ChipA/ChipB microvascular images and its random sphere arrays, Sec. 4.1 and
Table 1) are not available, so every workload here is drawn from a seeded
numpy generator.  This module holds no lattice Boltzmann arithmetic: it only
decides which nodes are fluid.  Both the CUDA path and the CPU oracle consume
its masks, laid out ``mask[z, y, x]`` (uint8, 1 = fluid, 0 = solid; 2D masks
use nz = 1).

Generators:
  * ``circles_2d``      - non-overlapping solid discs (random sequential addition)
  * ``sphere_pack_3d``  - overlapping solid spheres (a Swiss-cheese pore space)
  * ``tube_tree_3d``    - fluid tubes branching by Murray's law in solid rock
  * ``duct_3d`` / ``channel_2d`` / ``all_fluid`` - closed-form test geometries
  * ``random_mask``     - iid fluid/solid nodes for edge-case tests
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def all_fluid(nx: int, ny: int, nz: int = 1) -> np.ndarray:
    return np.ones((nz, ny, nx), np.uint8)


def random_mask(nx: int, ny: int, nz: int = 1, fluid: float = 0.7, seed: int = 0) -> np.ndarray:
    """Independent fluid (probability `fluid`) or solid nodes."""
    return (_rng(seed).random((nz, ny, nx)) < fluid).astype(np.uint8)


def channel_2d(nx: int, h: int) -> np.ndarray:
    """All-fluid 2D slab of height h (walls lie outside rows 0 and h-1)."""
    return np.ones((1, h, nx), np.uint8)


def duct_3d(nx: int, side: int) -> np.ndarray:
    """All-fluid square duct side x side along x (walls outside the box)."""
    return np.ones((side, side, nx), np.uint8)


def circles_2d(nx: int = 128, ny: int = 128, seed: int = 0, r_min: float = 3.0,
               r_max: float = 8.0, target_fluid: float = 0.5,
               max_attempts: int = 100_000, x_periodic: bool = True):
    """Random sequential addition of solid discs.

    Centres are uniform reals in the box, radii uniform in [r_min, r_max]; a
    candidate is rejected when it comes within 1 lattice unit of an accepted
    disc (centre distance < r1 + r2 + 1; minimum image along a periodic x).
    Stops once the fluid fraction is <= target_fluid or after max_attempts.
    A node is solid when its squared distance to a centre is <= r^2.
    Returns (mask[1, ny, nx], info dict).
    """
    rng = _rng(seed)
    solid = np.zeros((ny, nx), bool)
    xs = np.arange(nx, dtype=np.float64)
    ys = np.arange(ny, dtype=np.float64)
    discs = []
    attempts = 0
    while attempts < max_attempts:
        attempts += 1
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        r = rng.uniform(r_min, r_max)
        ok = True
        for (ox, oy, orr) in discs:
            dx = cx - ox
            if x_periodic:
                dx -= nx * round(dx / nx)
            if math.hypot(dx, cy - oy) < r + orr + 1.0:
                ok = False
                break
        if not ok:
            continue
        discs.append((cx, cy, r))
        dx = xs[None, :] - cx
        if x_periodic:
            dx -= nx * np.round(dx / nx)
        solid |= dx * dx + (ys[:, None] - cy) ** 2 <= r * r
        if 1.0 - solid.mean() <= target_fluid:
            break
    mask = (~solid).astype(np.uint8)[None]
    return mask, {"kind": "circles_2d", "seed": seed, "n_discs": len(discs),
                  "attempts": attempts, "fluid_fraction": float(mask.mean())}


def sphere_pack_3d(n: int = 256, seed: int = 0, r_min: float = 4.0, r_max: float = 12.0,
                   target_fluid: float = 0.30, x_periodic: bool = True, shape=None):
    """Overlapping solid spheres added until the fluid fraction is <= target.

    Centres uniform reals in the box, radii uniform in [r_min, r_max], minimum
    image along a periodic x.  `shape` = (nx, ny, nz) overrides the cube n^3.
    Returns (mask[nz, ny, nx], info dict).
    """
    nx, ny, nz = shape if shape is not None else (n, n, n)
    rng = _rng(seed)
    fluid = np.ones((nz, ny, nx), bool)
    n_fluid = fluid.size
    target = target_fluid * fluid.size
    count = 0
    while n_fluid > target:
        cx, cy, cz = rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(0, nz)
        r = rng.uniform(r_min, r_max)
        count += 1
        x0, x1 = int(math.floor(cx - r)), int(math.ceil(cx + r)) + 1
        y0, y1 = max(0, int(math.floor(cy - r))), min(ny, int(math.ceil(cy + r)) + 1)
        z0, z1 = max(0, int(math.floor(cz - r))), min(nz, int(math.ceil(cz + r)) + 1)
        if x_periodic:
            xi = np.arange(x0, x1)
            xw = xi % nx
        else:
            xi = np.arange(max(0, x0), min(nx, x1))
            xw = xi
        if len(xi) == 0 or y0 >= y1 or z0 >= z1:
            continue
        dz = (np.arange(z0, z1) - cz)[:, None, None]
        dy = (np.arange(y0, y1) - cy)[None, :, None]
        dx = (xi - cx)[None, None, :]
        ball = dz * dz + dy * dy + dx * dx <= r * r
        if x_periodic and len(np.unique(xw)) != len(xw):  # sphere wider than the box
            ball2 = np.zeros((z1 - z0, y1 - y0, nx), bool)
            np.logical_or.at(ball2, (slice(None), slice(None), xw), ball)
            sub = fluid[z0:z1, y0:y1, :]
            n_fluid -= int(np.count_nonzero(sub & ball2))
            sub &= ~ball2
            continue
        sub = fluid[z0:z1, y0:y1][:, :, xw]
        hit = sub & ball
        n_fluid -= int(np.count_nonzero(hit))
        fluid[z0:z1, y0:y1, xw] = sub & ~ball
    mask = fluid.astype(np.uint8)
    return mask, {"kind": "sphere_pack_3d", "seed": seed, "n_spheres": count,
                  "fluid_fraction": float(mask.mean())}


def _paint_capsule(fluid, p0, p1, r, x_periodic):
    nz, ny, nx = fluid.shape
    lo = np.floor(np.minimum(p0, p1) - r).astype(int)
    hi = np.ceil(np.maximum(p0, p1) + r).astype(int) + 1
    ylo, yhi = max(0, lo[1]), min(ny, hi[1])
    zlo, zhi = max(0, lo[2]), min(nz, hi[2])
    if x_periodic:
        xi = np.arange(lo[0], hi[0])
    else:
        xi = np.arange(max(0, lo[0]), min(nx, hi[0]))
    if len(xi) == 0 or ylo >= yhi or zlo >= zhi:
        return
    X = xi[None, None, :].astype(np.float64)
    Y = np.arange(ylo, yhi, dtype=np.float64)[None, :, None]
    Z = np.arange(zlo, zhi, dtype=np.float64)[:, None, None]
    d = p1 - p0
    L2 = float(d @ d)
    t = ((X - p0[0]) * d[0] + (Y - p0[1]) * d[1] + (Z - p0[2]) * d[2]) / (L2 if L2 > 0 else 1.0)
    t = np.clip(t, 0.0, 1.0)
    ex = X - (p0[0] + t * d[0])
    ey = Y - (p0[1] + t * d[1])
    ez = Z - (p0[2] + t * d[2])
    inside = ex * ex + ey * ey + ez * ez <= r * r
    xw = xi % nx
    if len(np.unique(xw)) != len(xw):
        acc = np.zeros((zhi - zlo, yhi - ylo, nx), bool)
        np.logical_or.at(acc, (slice(None), slice(None), xw), inside)
        fluid[zlo:zhi, ylo:yhi, :] |= acc
    else:
        fluid[zlo:zhi, ylo:yhi, xw] |= inside


def tube_tree_3d(n: int = 256, seed: int = 0, r_min: float = 3.0, r_max: float = 10.0,
                 target_fluid: float = 0.05, x_periodic: bool = True, shape=None):
    """Branching fluid tubes (capsules) in a solid background.

    Each tree starts with a straight trunk of radius r_max along x spanning
    the whole (periodic) length at a uniform (y, z).  Every segment of radius
    r spawns two children of radius r * 2^(-1/3) (Murray's law) from uniform
    points along it, in uniform random directions, each of length uniform in
    [6 r, 12 r]; branching stops below r_min.  Trees are added until the fluid
    fraction is >= target_fluid.  Returns (mask[nz, ny, nx], info dict).
    """
    nx, ny, nz = shape if shape is not None else (n, n, n)
    rng = _rng(seed)
    fluid = np.zeros((nz, ny, nx), bool)
    n_trees = 0
    n_segments = 0
    while fluid.mean() < target_fluid:
        n_trees += 1
        yc = rng.uniform(r_max + 1, ny - r_max - 1)
        zc = rng.uniform(r_max + 1, nz - r_max - 1)
        trunk = (np.array([0.0, yc, zc]), np.array([float(nx - 1), yc, zc]), r_max)
        stack = [trunk]
        while stack:
            p0, p1, r = stack.pop()
            _paint_capsule(fluid, p0, p1, r, x_periodic)
            n_segments += 1
            rc = r * 2.0 ** (-1.0 / 3.0)
            if rc < r_min:
                continue
            for _ in range(2):
                s = rng.uniform(0.0, 1.0)
                start = p0 + s * (p1 - p0)
                v = rng.normal(size=3)
                v /= np.linalg.norm(v)
                length = rng.uniform(6.0 * rc, 12.0 * rc)
                end = start + length * v
                end[1] = min(max(end[1], 0.0), ny - 1.0)
                end[2] = min(max(end[2], 0.0), nz - 1.0)
                if not x_periodic:
                    end[0] = min(max(end[0], 0.0), nx - 1.0)
                stack.append((start, end, rc))
    mask = fluid.astype(np.uint8)
    return mask, {"kind": "tube_tree_3d", "seed": seed, "n_trees": n_trees,
                  "n_segments": n_segments, "fluid_fraction": float(mask.mean())}


# The synthetic workloads used by the tests and the benchmark ---------------

def workload(name: str, seed: int = None):
    """Named synthetic workload -> (mask, params dict, info dict).

    params holds the lattice id, tile edge, periodic axes, tau, force and
    rho0 of that workload; the sizes follow the paper's problem statement
    (Sec. 4.1: 2D microvascular chips, 3D porous and vascular geometries).
    """
    if name == "d2q9_circles_128":
        mask, info = circles_2d(128, 128, seed=1 if seed is None else seed)
        params = dict(lattice=9, tile_a=16, periodic=(1, 0, 0), tau=0.8,
                      force=(1e-6, 0.0, 0.0), rho0=1.0, steps=1000)
    elif name == "d3q19_spheres_256":
        mask, info = sphere_pack_3d(256, seed=2 if seed is None else seed)
        params = dict(lattice=19, tile_a=4, periodic=(1, 0, 0), tau=0.6,
                      force=(1e-6, 0.0, 0.0), rho0=1.0, steps=2000)
    elif name == "d3q19_spheres_128":
        mask, info = sphere_pack_3d(128, seed=2 if seed is None else seed)
        params = dict(lattice=19, tile_a=4, periodic=(1, 0, 0), tau=0.6,
                      force=(1e-6, 0.0, 0.0), rho0=1.0, steps=2000)
    elif name == "d3q19_tubes_256":
        mask, info = tube_tree_3d(256, seed=3 if seed is None else seed)
        params = dict(lattice=19, tile_a=4, periodic=(1, 0, 0), tau=0.6,
                      force=(1e-6, 0.0, 0.0), rho0=1.0, steps=2000)
    elif name == "d3q19_dense_256":
        mask, info = all_fluid(256, 256, 256), {"kind": "all_fluid", "fluid_fraction": 1.0}
        params = dict(lattice=19, tile_a=4, periodic=(1, 1, 1), tau=0.6,
                      force=(1e-6, 0.0, 0.0), rho0=1.0, steps=2000)
    else:
        raise KeyError(name)
    return mask, params, info


def batch_workload(n: int = 64, seed: int = 5, side_min: int = 32, side_max: int = 160,
                   phi_min: float = 0.1, phi_max: float = 0.6):
    """Independent porous samples of uneven size and sparsity: cube sides
    drawn uniformly from the multiples of 8 in [side_min, side_max] (so that
    4^3 and 8^3 tiles divide the periodic x axis), fluid fractions uniform in
    [phi_min, phi_max], overlapping sphere packs (radius 4-12) with their own
    seeds.  Returns (masks, info list)."""
    rng = _rng(seed)
    sides = np.arange(side_min, side_max + 1, 8)
    masks, infos = [], []
    for k in range(n):
        side = int(rng.choice(sides))
        phi = float(rng.uniform(phi_min, phi_max))
        m, info = sphere_pack_3d(side, seed=seed * 1000 + k, target_fluid=phi)
        masks.append(m)
        infos.append({"side": side, "target_fluid": phi, **info})
    return masks, infos
