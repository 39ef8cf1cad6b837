"""The autotuner's candidate mappings (host logic, no GPU): tile edges that
divide every sample's periodic axes, 128-node blocks only where a tile fits,
the persistent grid and the 128-node blocks only for the FP32 storage forms,
the L2 prefetch on and off only for the one-block-per-work-block grid."""
import numpy as np

from paper_1703_08015_gb300 import autotune
from paper_1703_08015_gb300 import lbm


def _masks(*shapes):
    return [np.ones(s, np.uint8) for s in shapes]


def test_fp32_candidates_cover_the_mappings():
    c = autotune.candidates(19, lbm.LBM_STORE_F32S, _masks((16, 16, 32), (24, 8, 40)), (1, 0, 0))
    names = {autotune.mapping_name(x) for x in c}
    assert names == {"a4_b0_p0_f0", "a4_b0_p0_f-1", "a4_b0_p1_f0", "a4_b128_p0_f0", "a4_b128_p0_f-1",
                     "a4_b128_p1_f0", "a8_b0_p0_f0", "a8_b0_p0_f-1", "a8_b0_p1_f0"}
    assert all(x["prefetch_blocks"] == 0 for x in c if x["persistent"])


def test_periodic_axes_must_divide():
    # x = 36 is not a multiple of 8: only 4^3 tiles
    c = autotune.candidates(19, lbm.LBM_STORE_F32S, _masks((16, 16, 32), (8, 8, 36)), (1, 0, 0))
    assert {x["tile_a"] for x in c} == {4}
    # nothing fits a periodic axis of 6 nodes
    assert autotune.candidates(19, lbm.LBM_STORE_F32S, _masks((8, 8, 6)), (1, 0, 0)) == []
    # the same length on a wall-bounded axis is padded, so both edges stay
    assert {x["tile_a"] for x in autotune.candidates(19, lbm.LBM_STORE_F32S, _masks((8, 8, 6)), (0, 0, 0))} == {4, 8}


def test_fp64_and_d2q9_candidates():
    c = autotune.candidates(19, lbm.LBM_STORE_F64, _masks((16, 16, 32)), (1, 0, 0))
    assert all(x["block_nodes"] == 0 and x["persistent"] == 0 for x in c)
    assert {x["prefetch_blocks"] for x in c} == {0, -1}
    c2 = autotune.candidates(9, lbm.LBM_STORE_F32, _masks((1, 64, 96)), (1, 0, 0))
    assert {x["tile_a"] for x in c2} == {8, 16, 32}
    # 8^2 tiles (64 nodes) fit 128-node blocks, 16^2 and 32^2 do not
    assert {x["tile_a"] for x in c2 if x["block_nodes"] == 128} == {8}
