"""Autotuner of the tile-to-block mapping (not in the paper).

For a set of geometries (a batch or a single one) it times every candidate
mapping -- tile edge a, fluid nodes per step-kernel block, persistent or
one-block-per-work-block grid, and for the latter the L2 prefetch of the
work block four per SM ahead on or off -- for a few steps with CUDA events on
the launching stream, keeps the fastest, and caches the choice per GPU,
lattice, storage and workload signature in ``_build/autotune.json``.  Every candidate
computes the same update (the tests check bit equality across mappings), so
tuning only changes speed.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import _build
from . import lbm

CACHE = os.path.join(_build.BUILD, "autotune.json")


def candidates(lattice, storage, masks, periodic):
    """Mappings compiled for this lattice / storage that fit the geometries."""
    edges = [4, 8] if lattice == lbm.LBM_D3Q19 else [8, 16, 32]
    out = []
    for a in edges:
        ok = True
        for m in masks:
            n = [m.shape[2], m.shape[1], m.shape[0]]
            if any(periodic[k] and n[k] % a for k in range(3 if lattice == lbm.LBM_D3Q19 else 2)):
                ok = False
        if not ok:
            continue
        nt = a ** (3 if lattice == lbm.LBM_D3Q19 else 2)
        blocks = [0] + ([128] if nt <= 128 and storage != lbm.LBM_STORE_F64 else [])
        pers = [0, 1] if storage != lbm.LBM_STORE_F64 else [0]
        for bn in blocks:
            for pe in pers:
                # the persistent grid takes no prefetch; copies that fit the
                # L2 can run faster without it
                for pf in ([0, -1] if not pe else [0]):
                    out.append({"tile_a": a, "block_nodes": bn, "persistent": pe, "prefetch_blocks": pf})
    return out


def mapping_name(cfg):
    return f"a{cfg['tile_a']}_b{cfg['block_nodes']}_p{cfg['persistent']}_f{cfg.get('prefetch_blocks', 0)}"


def _signature(lattice, storage, masks):
    import torch

    fluid = int(sum(int(np.count_nonzero(m)) for m in masks))
    return (f"{torch.cuda.get_device_name()}|D{3 if lattice == 19 else 2}Q{lattice}|storage{storage}|"
            f"n{len(masks)}|fluid{fluid}")


def time_mapping(masks, lattice, cfg, storage, periodic, tau, force, steps=40, device="cuda"):
    """MLUPS of one mapping (after a short warm-up), CUDA events on the stream."""
    import torch

    b = lbm.BatchSolver(masks, lattice, cfg["tile_a"], periodic, tau, force, storage=storage,
                        block_nodes=cfg["block_nodes"], persistent=cfg["persistent"],
                        prefetch_blocks=cfg.get("prefetch_blocks", 0), device=device)
    try:
        b.step(16)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        b.step(steps)
        e1.record(b.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        return int(b.tiling.n_fluid) * steps / (ms * 1e-3) / 1e6
    finally:
        b.close()


def tune(masks, lattice, storage=lbm.LBM_STORE_F32S, periodic=(1, 0, 0), tau=0.6, force=(1e-6, 0, 0),
         steps=40, use_cache=True, device="cuda", cache_path=None):
    """Returns (best mapping dict, {mapping: MLUPS} of every candidate tried).
    The choice is cached in `cache_path` (default _build/autotune.json) under
    the GPU / lattice / storage / workload key and reused by later calls."""
    cache_path = cache_path or CACHE
    masks = [np.ascontiguousarray(m[None] if m.ndim == 2 else m, np.uint8) for m in masks]
    key = _signature(lattice, storage, masks)
    cache = {}
    if use_cache and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache and "prefetch_blocks" in cache[key]["best"]:
            return cache[key]["best"], cache[key]["trials"]
    trials, by_name = {}, {}
    for cfg in candidates(lattice, storage, masks, periodic):
        name = mapping_name(cfg)
        by_name[name] = cfg
        trials[name] = time_mapping(masks, lattice, cfg, storage, periodic, tau, force, steps, device)
    best = by_name[max(trials, key=trials.get)]
    cache[key] = {"best": best, "trials": trials, "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
    with open(cache_path, "w") as f:
        json.dump(cache, f, indent=1)
    return best, trials
