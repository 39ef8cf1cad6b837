"""Reference tiling of a masked lattice (TEST INFRASTRUCTURE ONLY).

Sec. 3 of Tomczak & Szafran (arXiv:1703.08015) covers the geometry with a
uniform mesh of tiles of a nodes per edge, anchored at node (0,0), pads the
geometry with solid nodes when its size is not a multiple of a, and drops
every tile that holds only solid nodes.  The tileMap array (Sec. 3, and the
s_ti = 4 B index of Sec. 3.1.1.1) stores, for every tile of the mesh, the
index of that tile's data, or -1 for a removed tile.

Readings taken here (the paper leaves them open):
  * a non-empty tile's index is its rank among non-empty tiles in row-major
    scan order, x fastest, then y, then z;
  * a periodic axis must be a multiple of a (padding would break the wrap);
  * the neighbour record of a tile lists the 3^d surrounding tiles in the
    order (dz, dy, dx) with each offset in -1, 0, 1 and dx fastest, holding
    the neighbour's index, or -1 for a removed tile or one beyond a
    non-periodic edge (Fig. 5 keeps such a 3^3 copy of the tile bitmap).

Two implementations: ``build_tilemap`` (numpy) and ``build_tilemap_loops``
(pure-Python loops for tiny masks, used to check the first).
"""
from __future__ import annotations

import numpy as np


class ShapeError(ValueError):
    """A periodic axis whose length is not a multiple of the tile edge."""


def _setup(mask, a, periodic, dim):
    mask = np.asarray(mask)
    if mask.ndim == 2:
        mask = mask[None]
    if dim == 2 and mask.shape[0] != 1:
        raise ValueError("2D tiling needs nz == 1")
    nz, ny, nx = mask.shape
    n = [nx, ny, nz]
    per = [bool(periodic[k]) if k < len(periodic) else False for k in range(3)]
    for ax in range(dim):
        if per[ax] and n[ax] % a != 0:
            raise ShapeError(f"periodic axis {ax} of length {n[ax]} is not a multiple of {a}")
    nt = [-(-n[ax] // a) for ax in range(dim)] + [1] * (3 - dim)
    return mask, n, per, nt


def build_tilemap(mask, a: int, periodic=(False, False, False), dim: int = 3):
    """Return (tile_map[ntz,nty,ntx] int32, nbr[N_ftiles, 3^dim] int32,
    tile_mask[N_ftiles, a^dim] uint8 (node order x fastest), coords[N_ftiles, 3])."""
    mask, n, per, nt = _setup(mask, a, periodic, dim)
    ntx, nty, ntz = nt
    az = a if dim == 3 else 1
    pad = np.zeros((ntz * az, nty * a, ntx * a), np.uint8)
    pad[: mask.shape[0], : mask.shape[1], : mask.shape[2]] = mask != 0
    tiles = pad.reshape(ntz, az, nty, a, ntx, a).transpose(0, 2, 4, 1, 3, 5)
    tiles = tiles.reshape(ntz, nty, ntx, az * a * a)
    nonempty = tiles.any(axis=3)
    tile_map = np.full((ntz, nty, ntx), -1, np.int32)
    count = int(nonempty.sum())
    tile_map[nonempty] = np.arange(count, dtype=np.int32)
    tz, ty, tx = np.nonzero(nonempty)  # row-major order == rank order
    coords = np.stack([tx, ty, tz], axis=1).astype(np.int32)
    tile_mask = tiles[nonempty].astype(np.uint8)

    offs = [(dx, dy, dz) for dz in ((-1, 0, 1) if dim == 3 else (0,))
            for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    nbr = np.empty((count, len(offs)), np.int32)
    for k, (dx, dy, dz) in enumerate(offs):
        cx, cy, cz = tx + dx, ty + dy, tz + dz
        ok = np.ones(count, bool)
        for c, m, p in ((cx, ntx, per[0]), (cy, nty, per[1]), (cz, ntz, per[2])):
            out = (c < 0) | (c >= m)
            if p:
                c %= m
            else:
                ok &= ~out
        val = np.full(count, -1, np.int32)
        idx = np.nonzero(ok)[0]
        val[idx] = tile_map[cz[idx] % ntz, cy[idx] % nty, cx[idx] % ntx]
        nbr[:, k] = val
    return tile_map, nbr, tile_mask, coords


def build_tilemap_loops(mask, a: int, periodic=(False, False, False), dim: int = 3):
    """The same tiling written as plain loops over tiles and nodes (tiny masks)."""
    mask, n, per, nt = _setup(mask, a, periodic, dim)
    ntx, nty, ntz = nt
    az = a if dim == 3 else 1

    def fluid(x, y, z):
        if x >= n[0] or y >= n[1] or z >= n[2]:
            return 0  # padding is solid
        return 1 if mask[z, y, x] else 0

    tile_map = np.full((ntz, nty, ntx), -1, np.int32)
    coords, tmask = [], []
    count = 0
    for tz in range(ntz):
        for ty in range(nty):
            for tx in range(ntx):
                bits = []
                for lz in range(az):
                    for ly in range(a):
                        for lx in range(a):
                            bits.append(fluid(tx * a + lx, ty * a + ly, tz * az + lz))
                if any(bits):
                    tile_map[tz, ty, tx] = count
                    count += 1
                    coords.append((tx, ty, tz))
                    tmask.append(bits)
    nbr = []
    for (tx, ty, tz) in coords:
        rec = []
        for dz in ((-1, 0, 1) if dim == 3 else (0,)):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    c = [tx + dx, ty + dy, tz + dz]
                    ok = True
                    for ax in range(3):
                        if c[ax] < 0 or c[ax] >= nt[ax]:
                            if per[ax]:
                                c[ax] %= nt[ax]
                            else:
                                ok = False
                    rec.append(int(tile_map[c[2], c[1], c[0]]) if ok else -1)
        nbr.append(rec)
    nn = 27 if dim == 3 else 9
    return (tile_map,
            np.array(nbr, np.int32).reshape(count, nn),
            np.array(tmask, np.uint8).reshape(count, az * a * a),
            np.array(coords, np.int32).reshape(count, 3))


def tile_stats(mask, a: int, dim: int = 3):
    """N_tiles, N_ftiles, N_fnodes and the average tile porosity phi_t (Eq. 17)."""
    tile_map, _, tile_mask, _ = build_tilemap(mask, a, (False,) * 3, dim)
    n_ftiles = tile_mask.shape[0]
    n_fnodes = int(tile_mask.sum())
    phi_t = n_fnodes / (n_ftiles * tile_mask.shape[1]) if n_ftiles else 0.0
    return {"N_tiles": int(tile_map.size), "N_ftiles": n_ftiles,
            "N_fnodes": n_fnodes, "phi_t": phi_t}


__all__ = ["ShapeError", "build_tilemap", "build_tilemap_loops", "tile_stats"]
