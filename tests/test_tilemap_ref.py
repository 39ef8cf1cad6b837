"""Pins of the reference tiling (Sec. 3): hand cases plus the numpy version
against the plain-loop version on random masks."""
import numpy as np
import pytest

from oracle import tilemap_ref as tr


def test_all_solid_has_no_tiles():
    tm, nbr, tmask, coords = tr.build_tilemap(np.zeros((8, 8, 8), np.uint8), 4)
    assert tm.shape == (2, 2, 2) and np.all(tm == -1)
    assert nbr.shape == (0, 27) and tmask.shape == (0, 64)


def test_single_fluid_node():
    m = np.zeros((9, 10, 11), np.uint8)  # nz, ny, nx -> tiles 3 x 3 x 3 (padded)
    m[5, 2, 9] = 1                       # z=5, y=2, x=9 -> tile (2, 0, 1)
    tm, nbr, tmask, coords = tr.build_tilemap(m, 4)
    assert tm.shape == (3, 3, 3)
    assert np.count_nonzero(tm >= 0) == 1 and tm[1, 0, 2] == 0
    assert list(coords[0]) == [2, 0, 1]
    node = (9 - 8) + 4 * (2 - 0) + 16 * (5 - 4)
    assert tmask[0].sum() == 1 and tmask[0][node] == 1
    assert nbr[0][13] == 0 and np.count_nonzero(nbr[0] >= 0) == 1


def test_padding_is_solid():
    m = np.ones((5, 7, 10), np.uint8)
    tm, nbr, tmask, coords = tr.build_tilemap(m, 4)
    assert tm.shape == (2, 2, 3) and np.all(tm >= 0)
    last = tm[1, 1, 2]
    # tile (2,1,1) covers x 8..11, y 4..7, z 4..7: only x<10, y<7, z<5 are real
    assert tmask[last].sum() == 2 * 3 * 1


def test_periodic_needs_multiple_of_a():
    m = np.ones((4, 4, 10), np.uint8)
    with pytest.raises(tr.ShapeError):
        tr.build_tilemap(m, 4, periodic=(1, 0, 0))
    tr.build_tilemap(m, 4, periodic=(0, 1, 1))  # y, z are multiples of 4


def test_row_major_rank_and_periodic_neighbours():
    m = np.zeros((1, 16, 48), np.uint8)
    m[0, 0, 0] = 1     # tile (0,0)
    m[0, 0, 40] = 1    # tile (2,0)
    m[0, 15, 20] = 1   # y=15 lies in tile row 0 (a=16), x=20 in tile column 1
    tm, nbr, _, coords = tr.build_tilemap(m, 16, periodic=(1, 0, 0), dim=2)
    assert tm.tolist() == [[[0, 1, 2]]]
    # neighbour order (dy, dx) with dx fastest; index 4 is the tile itself
    assert nbr[0].tolist() == [-1, -1, -1, 2, 0, 1, -1, -1, -1]  # x wraps to tile 2
    assert nbr[2].tolist() == [-1, -1, -1, 1, 2, 0, -1, -1, -1]
    tm, nbr, _, _ = tr.build_tilemap(m, 16, periodic=(0, 0, 0), dim=2)
    assert nbr[0].tolist() == [-1, -1, -1, -1, 0, 1, -1, -1, -1]


@pytest.mark.parametrize("seed", range(6))
def test_numpy_matches_loops(seed):
    rng = np.random.default_rng(seed)
    dim = 2 if seed % 2 else 3
    a = int(rng.choice([2, 4])) if dim == 3 else int(rng.choice([4, 8]))
    if dim == 3:
        shape = tuple(int(v) for v in rng.integers(3, 13, 3))
    else:
        shape = (1,) + tuple(int(v) for v in rng.integers(5, 30, 2))
    per = [bool(rng.integers(0, 2)) for _ in range(3)]
    n = [shape[2], shape[1], shape[0]]
    per = [p and n[k] % a == 0 for k, p in enumerate(per)]
    m = (rng.random(shape) < rng.uniform(0.05, 0.6)).astype(np.uint8)
    A = tr.build_tilemap(m, a, per, dim)
    B = tr.build_tilemap_loops(m, a, per, dim)
    for x, y in zip(A, B):
        assert x.dtype == y.dtype and np.array_equal(x, y)
