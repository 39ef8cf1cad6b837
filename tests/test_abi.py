"""C-ABI checks that need no GPU: the library loads, exports every entry
point include/lbm.h declares, and its host tiling (lbm_build_tilemap, Sec. 3)
matches the reference tiling bit for bit."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import tilemap_ref as tr
from paper_1703_08015_gb300 import geometry as geo
from paper_1703_08015_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported():
    lib = lbm.library()
    declared = _declared()
    assert {"lbm_build_tilemap", "lbm_init", "lbm_step", "lbm_moments", "lbm_free"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def _check_tiling(mask, lattice, a, periodic):
    p = lbm.make_params(lattice, mask.shape, a, periodic)
    info, tm, nb = lbm.lbm_build_tilemap(p, mask)
    dim = 2 if lattice == lbm.LBM_D2Q9 else 3
    rtm, rnb, rmask, _ = tr.build_tilemap(mask, a, periodic, dim)
    assert np.array_equal(tm, rtm)
    assert np.array_equal(nb, rnb)
    assert info.n_ftiles == rmask.shape[0]
    assert info.n_tiles == rtm.size
    assert info.n_fluid == int(np.count_nonzero(mask))
    # compact layout: each tile stores only its fluid nodes, q links each
    assert info.pdf_bytes == int(rmask.sum()) * lattice * 8


@pytest.mark.parametrize("seed", range(8))
def test_tilemap_matches_reference(seed):
    rng = np.random.default_rng(100 + seed)
    if seed % 2:
        a = int(rng.choice([8, 16, 32]))
        shape = (1, int(rng.integers(5, 70)), a * int(rng.integers(1, 4)))
        lattice = lbm.LBM_D2Q9
        per = (1, int(rng.integers(0, 2)) if shape[1] % a == 0 else 0, 0)
    else:
        a = int(rng.choice([4, 8]))
        shape = (int(rng.integers(3, 20)), int(rng.integers(3, 20)), a * int(rng.integers(1, 4)))
        lattice = lbm.LBM_D3Q19
        per = (1, 0, int(rng.integers(0, 2)) if shape[0] % a == 0 else 0)
    mask = (rng.random(shape) < rng.uniform(0.02, 0.7)).astype(np.uint8)
    _check_tiling(mask, lattice, a, per)


def test_tilemap_workload_sphere_pack():
    mask, _ = geo.sphere_pack_3d(shape=(64, 48, 40), seed=7)
    _check_tiling(mask, lbm.LBM_D3Q19, 4, (1, 0, 0))


def _tiling_of(mask, a=4, per=(1, 0, 0)):
    p = lbm.make_params(lbm.LBM_D3Q19, mask.shape, a, per)
    info, tm, nb = lbm.lbm_build_tilemap(p, mask)
    return int(info.n_ftiles), int(info.pdf_bytes), tm, nb


def test_tiling_from_several_threads_at_once():
    """The host tiling runs its passes on a pool of threads started once; calls
    from several threads at once (one gets the pool, the others run serially)
    give the same tables as one call at a time."""
    import threading

    masks = [geo.sphere_pack_3d(shape=(48, 40, 32), seed=s, r_min=2, r_max=6)[0] for s in range(6)]
    want = [_tiling_of(m) for m in masks]
    got = [None] * len(masks)

    def run(k):
        for _ in range(3):
            got[k] = _tiling_of(masks[k])

    th = [threading.Thread(target=run, args=(k,)) for k in range(len(masks))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for w, g in zip(want, got):
        assert w[:2] == g[:2] and np.array_equal(w[2], g[2]) and np.array_equal(w[3], g[3])


def _tile_in_child(q):
    m = geo.sphere_pack_3d(shape=(32, 32, 32), seed=4, r_min=2, r_max=5)[0]
    q.put(_tiling_of(m)[:2])


@pytest.mark.filterwarnings("ignore:This process .* is multi-threaded:DeprecationWarning")
def test_tiling_in_a_forked_child():
    """A child forked after the pool has started has none of its threads: it
    starts its own pool and tiles to the same result (no hang)."""
    import multiprocessing as mp

    m = geo.sphere_pack_3d(shape=(32, 32, 32), seed=4, r_min=2, r_max=5)[0]
    want = _tiling_of(m)[:2]  # the parent's pool is running
    ctx = mp.get_context("fork")
    q = ctx.Queue()
    pr = ctx.Process(target=_tile_in_child, args=(q,))
    pr.start()
    pr.join(60)
    if pr.is_alive():
        pr.kill()
        pr.join()
        pytest.fail("tiling in a forked child did not finish")
    assert pr.exitcode == 0
    assert q.get(timeout=5) == want


def test_tilemap_edge_cases():
    z = np.zeros((8, 8, 8), np.uint8)
    p = lbm.make_params(lbm.LBM_D3Q19, z.shape, 4)
    info, tm, nb = lbm.lbm_build_tilemap(p, z)
    assert info.n_ftiles == 0 and np.all(tm == -1) and nb.shape == (0, 27) and info.pdf_bytes == 0
    m = np.ones((4, 4, 10), np.uint8)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_build_tilemap(lbm.make_params(lbm.LBM_D3Q19, m.shape, 4, (1, 0, 0)), m)
    assert e.value.code == -2
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_build_tilemap(lbm.make_params(lbm.LBM_D3Q19, m.shape, 5), m)
    assert e.value.code == -1
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_build_tilemap(lbm.make_params(lbm.LBM_D2Q9, m.shape, 16), m)  # nz != 1
    assert e.value.code == -1
    one = np.zeros((1, 20, 20), np.uint8)
    one[0, 17, 3] = 1
    info, tm, nb = lbm.lbm_build_tilemap(lbm.make_params(lbm.LBM_D2Q9, one.shape, 16), one)
    assert info.n_ftiles == 1 and tm.tolist() == [[[-1, -1], [0, -1]]]


def test_null_arguments_are_rejected():
    lib = lbm.library()
    info = lbm.lbm_tiling()
    assert lib.lbm_build_tilemap(None, None, None, None, ctypes.byref(info)) == -1
    assert lib.lbm_step(None, 1, None) == -1
    assert lib.lbm_moments(None, None, None, None, 0, None) == -1
    assert lib.lbm_free(None) == 0
    assert "NULL" in lbm.lbm_last_error() or lbm.lbm_last_error() != ""


def test_batch_tiling_sums_the_samples():
    masks = [geo.random_mask(8 * (k + 1), 12, 6 + k, fluid=0.4, seed=k) for k in range(4)]
    p = lbm.make_params(lbm.LBM_D3Q19, (1, 1, 1), 4, (1, 0, 0))
    total = lbm.lbm_build_tilemap_batch(p, masks)
    n_ftiles = pdf = fluid = 0
    for m in masks:
        info, _, _ = lbm.lbm_build_tilemap(lbm.make_params(lbm.LBM_D3Q19, m.shape, 4, (1, 0, 0)), m, False, False)
        n_ftiles += info.n_ftiles
        pdf += info.pdf_bytes
        fluid += info.n_fluid
    assert (total.n_ftiles, total.pdf_bytes, total.n_fluid) == (n_ftiles, pdf, fluid)
    bad = [masks[0], geo.random_mask(10, 12, 6, seed=9)]  # nx = 10 not a multiple of 4 on periodic x
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_build_tilemap_batch(p, bad)
    assert e.value.code == -2


def test_conv_tune_validates_its_arguments():
    """lbm_nn_conv_tune takes 0 (chosen per shape) or a valid launch shape of
    the halo-tile convolution, and rejects the rest (no GPU involved)."""
    lib = lbm.library()
    f = lib.lbm_nn_conv_tune
    f.argtypes = [ctypes.c_int, ctypes.c_int]
    f.restype = ctypes.c_int
    try:
        for bz, nt in [(0, 0), (1, 16), (4, 128), (3, 48), (0, 112), (4, 0)]:
            assert f(bz, nt) == 0, (bz, nt)
        for bz, nt in [(-1, 0), (5, 0), (0, 8), (0, 144), (0, -16), (4, 144), (1, 24)]:
            assert f(bz, nt) == -1, (bz, nt)
    finally:
        assert f(0, 0) == 0


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes structures of the binding have the size and field offsets
    that a C compiler gives the structures of include/lbm.h (a field added to
    one side only would shift every later field the library reads)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    checks = {
        "lbm_params": (lbm.lbm_params, ["lattice", "nx", "tile_a", "periodic", "tau", "force", "rho0", "storage",
                                        "arith", "f16_scale", "block_nodes", "persistent", "layout",
                                        "prefetch_blocks"]),
        "lbm_tiling": (lbm.lbm_tiling, ["ntx", "n_ftiles", "n_fluid", "pdf_bytes", "ghost_bytes"]),
        "lbm_stats": (lbm.lbm_stats, ["mass", "momentum", "u2", "du2", "residual", "n_fluid", "step"]),
    }
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "lbm.h"', "int main(void) {"]
    for st, (_, fields) in checks.items():
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for f in fields:
            lines.append(f'  printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st, (cls, fields) in checks.items():
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for f in fields:
            assert got[(st, f)] == getattr(cls, f).offset, (st, f)
