"""Pins for the oracle's tile policy (Sec. 3.5, Table 2)."""
import pytest

from conftest import read_golden
from oracle.tiles import min_tile_side, tile_dims


def _table2():
    for r in read_golden("table4_colours.txt"):
        p, k, tz, tx, ty, tt = map(int, r[:6])
        yield p, k, [tx, ty, tz, tt]
    for r in read_golden("table4_colours_k8_10.txt"):
        yield int(r[0]), int(r[1]), [32, 32, 32, 32]


@pytest.mark.parametrize("p,k,tile", list(_table2()))
def test_table2_tiles_for_32cube_x_64(p, k, tile):
    """Table 2: the tiles chosen for a 32^3 x 64 lattice, displacement along z."""
    assert tile_dims([32, 32, 32, 64], 2, [p], k) == tile


def test_table2_covers_all_90_entries():
    assert sorted((p, k) for p, k, _ in _table2()) == [(p, k) for p in range(9) for k in range(1, 11)]


def test_sec35_worked_examples():
    """Sec. 3.5: the stated minima are 2(p + k) + 1 along the displacement and
    2k + 1 elsewhere (33 and 17 for (8, 8); the example beside them prints
    34 x 18^3, one more on every side, and the formulas are taken).  Either
    way the power-of-two tile is 64 x 32^3, and on a 32 x 64^3 lattice
    (displacement along the 32 side) the displaced side is capped at 32,
    giving 32^4, as in the paper."""
    assert min_tile_side(0, 0, [8], 8) == 33
    assert min_tile_side(1, 0, [8], 8) == 17
    assert tile_dims([64, 64, 64, 64], 0, [8], 8) == [64, 32, 32, 32]
    assert tile_dims([32, 64, 64, 64], 0, [8], 8) == [32, 32, 32, 32]


def test_multiple_displacements_take_the_largest_p():
    """Sec. 3.4: the union of neighbourhoods needs the side of the largest p."""
    assert tile_dims([64, 64, 64, 64], 3, [1, 2, 5], 2) == tile_dims([64, 64, 64, 64], 3, [5], 2)


def test_non_power_of_two_sides_take_the_smallest_divisor():
    """A side of 24 (a factor of three): the smallest divisor >= 2k+1."""
    assert tile_dims([24, 24, 24, 48], 2, [0], 2) == [6, 6, 6, 6]
    assert tile_dims([24, 24, 24, 48], 2, [8], 2) == [6, 6, 24, 6]
    assert tile_dims([24, 24, 24, 48], 2, [4], 4) == [12, 12, 24, 12]
