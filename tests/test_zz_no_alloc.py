"""lbm_stats_noalloc against lbm_moments (GPU).

Callers that cannot allocate device memory when they want the mass and
momentum sums (a fixed memory budget owned by another allocator, monitoring
hooks that must not change the footprint, loops that cannot take cudaMalloc's
device-wide synchronisation) use lbm_stats_noalloc, whose partial sums live in
a static device array.  Its output must match the allocating entry point's
statistics on consecutive calls, and tilings too large for the static array
must be rejected.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1703_08015_gb300 import geometry as geo
from paper_1703_08015_gb300 import lbm

pytestmark = pytest.mark.gpu


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _noalloc(torch, s):
    out = torch.full((8,), float("nan"), dtype=torch.float64, device=s.device)
    lbm.lbm_stats_noalloc(s.ctx, out, s._s())
    torch.cuda.synchronize(s.device)
    return out.cpu().numpy()


@pytest.mark.parametrize("lattice,a", [(19, 4), (9, 16)])
def test_noalloc_matches_lbm_moments_twice(lattice, a):
    torch = _cuda()
    if lattice == 19:
        mask, _ = geo.sphere_pack_3d(shape=(40, 36, 28), seed=31, r_min=2, r_max=5, target_fluid=0.4)
        F = (1e-5, 2e-6, -1e-6)
    else:
        mask, _ = geo.circles_2d(96, 70, seed=32, max_attempts=4000)
        F = (1e-5, 1e-6, 0.0)
    s = lbm.Solver(mask, lattice, a, (1, 0, 0), 0.7, F)
    try:
        for _ in range(2):  # two calls in a row, the state advancing between them
            s.step(37)
            st, rc = s.stats()
            assert rc == 0
            got = _noalloc(torch, s)
            ref = np.array([st.mass, *st.momentum, st.u2, 0.0, float(st.n_fluid), 0.0])
            assert got[6] == float(mask.sum())
            # the same kernels over the same partial blocks: the same bits
            assert np.array_equal(got[[0, 1, 2, 3, 4, 6]], ref[[0, 1, 2, 3, 4, 6]])
            again = _noalloc(torch, s)
            assert np.array_equal(again, got)
    finally:
        s.close()


def test_noalloc_batch_sums_every_sample():
    torch = _cuda()
    masks = [geo.sphere_pack_3d(shape=(24, 16, 20), seed=40 + k, r_min=2, r_max=4, target_fluid=0.5)[0]
             for k in range(3)]
    b = lbm.BatchSolver(masks, 19, 4, (1, 0, 0), 0.7, (1e-5, 0.0, 0.0), storage=lbm.LBM_STORE_F64)
    try:
        for _ in range(2):
            b.step(21)
            per, rc = b.stats()
            assert rc == 0
            got = _noalloc(torch, b)
            # one launch over all samples' tiles against per-sample launches
            # summed on the host: the same terms, summed in another grouping
            assert got[6] == float(sum(int(m.sum()) for m in masks))
            assert got[0] == pytest.approx(sum(st.mass for st in per), rel=1e-14)
            for k in (1, 2, 3):
                assert got[k] == pytest.approx(sum(st.momentum[k - 1] for st in per), rel=1e-12, abs=1e-18)
    finally:
        b.close()


def test_noalloc_rejects_too_many_blocks():
    torch = _cuda()
    # 257 x 256 tiles of 16^2, one fluid node in each: 65,792 tiles in groups
    # of 8 per partial block = 8,224 blocks > 8,192
    mask = np.zeros((1, 256 * 16, 257 * 16), np.uint8)
    mask[0, 5::16, 7::16] = 1
    s = lbm.Solver(mask, 9, 16, (0, 0, 0), 0.8, (0, 0, 0))
    try:
        assert s.tiling.n_ftiles == 257 * 256
        out = torch.zeros(8, dtype=torch.float64, device=s.device)
        rc = lbm.library().lbm_stats_noalloc(s.ctx, ctypes.c_void_p(out.data_ptr()), s._s())
        assert rc == -8
        assert "static scratch" in lbm.lbm_last_error()
        assert torch.count_nonzero(out).item() == 0  # nothing was launched
    finally:
        s.close()
