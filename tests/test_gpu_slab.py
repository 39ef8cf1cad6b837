"""The domain split on the GPU: several ranks' boxes, each a context of its
own on one GPU, exchanging their ghost tile layers (contiguous byte ranges of
the PDF copies, lbm_layer_range) after every step.  Their interiors must
equal the undivided run bit for bit, and the interior statistics must add up
to the undivided run's."""
import numpy as np
import pytest

from paper_1703_08015_gb300 import geometry as geo
from paper_1703_08015_gb300 import lbm
from paper_1703_08015_gb300 import slab

pytestmark = pytest.mark.gpu


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _cases():
    m3, _ = geo.sphere_pack_3d(shape=(24, 20, 34), seed=81, r_min=2, r_max=5, target_fluid=0.45)
    m3p, _ = geo.sphere_pack_3d(shape=(20, 16, 32), seed=82, r_min=2, r_max=4, target_fluid=0.5)
    m2, _ = geo.circles_2d(48, 70, seed=83, r_min=2, r_max=5, max_attempts=800)
    return [
        ("d3q19_walls_z_2", m3, 19, 4, (1, 0, 0), 0.6, (1e-5, 0, 2e-6), 2, 60),
        ("d3q19_walls_z_3", m3, 19, 4, (1, 0, 0), 0.6, (1e-5, 0, 2e-6), 3, 60),
        ("d3q19_periodic_z_2", m3p, 19, 4, (1, 0, 1), 0.7, (1e-5, 0, 3e-6), 2, 50),
        ("d3q19_periodic_z_4", m3p, 19, 4, (1, 0, 1), 0.7, (1e-5, 0, 3e-6), 4, 50),
        ("d2q9_split_y_3", m2, 9, 16, (1, 0, 0), 0.8, (1e-5, 2e-6, 0), 3, 80),
    ]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_split_run_equals_the_undivided_run(case):
    _cuda()
    name, mask, lat, a, per, tau, F, world, steps = case
    whole = lbm.Solver(mask, lat, a, per, tau, F)
    comm = slab.LocalComm()
    ranks = [slab.SlabSolver(mask, lat, a, per, tau, F, r, world, comm) for r in range(world)]
    try:
        whole.step(steps)
        ref = whole.export_pdfs()
        st_ref, _ = whole.stats()
        comm.step_all(steps)
        got = np.concatenate([s.export_interior() for s in ranks], axis=1 if lat == 19 else 2)
        parts = [s.stats() for s in ranks]
    finally:
        whole.close()
        for s in ranks:
            s.close()
    fl = np.broadcast_to(np.asarray(mask).astype(bool).reshape(ref.shape[1:]), ref.shape)
    assert got.shape == ref.shape
    assert np.array_equal(got[fl].view(np.uint64), ref[fl].view(np.uint64))
    assert sum(p["n_fluid"] for p in parts) == st_ref.n_fluid
    assert sum(p["mass"] for p in parts) == pytest.approx(st_ref.mass, rel=1e-14)
    for k in range(3 if lat == 19 else 2):
        assert sum(p["momentum"][k] for p in parts) == pytest.approx(st_ref.momentum[k], rel=1e-11, abs=1e-16)


def test_layer_ranges_tile_the_copy():
    """The layer ranges of a context are contiguous, in order, and cover the
    PDF copy; empty layers have empty ranges; bad ranges are rejected."""
    _cuda()
    import ctypes

    mask = np.zeros((24, 12, 16), np.uint8)
    mask[2:9] = 1        # layers 0..2 hold fluid
    mask[17:21, 3:9] = 1  # layers 4, 5
    s = lbm.Solver(mask, 19, 4, (1, 0, 0), 0.6, (0, 0, 0))
    try:
        lib = lbm.library()
        off, nb = ctypes.c_size_t(), ctypes.c_size_t()
        end = 0
        sizes = []
        for layer in range(6):
            assert lib.lbm_layer_range(s.ctx, layer, layer + 1, ctypes.byref(off), ctypes.byref(nb)) == 0
            assert off.value == end
            end += nb.value
            sizes.append(nb.value)
        assert end == s.tiling.pdf_bytes
        assert sizes[3] == 0 and all(sizes[k] > 0 for k in (0, 1, 2, 4, 5))
        assert lib.lbm_layer_range(s.ctx, 0, 6, ctypes.byref(off), ctypes.byref(nb)) == 0
        assert (off.value, nb.value) == (0, s.tiling.pdf_bytes)
        assert lib.lbm_layer_range(s.ctx, 2, 7, ctypes.byref(off), ctypes.byref(nb)) == -1
        assert lib.lbm_layer_range(s.ctx, 3, 2, ctypes.byref(off), ctypes.byref(nb)) == -1
        assert lib.lbm_current_copy(s.ctx) == 0
        s.step(3)
        assert lib.lbm_current_copy(s.ctx) == 1
    finally:
        s.close()
