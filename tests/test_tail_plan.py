"""The tail-split planner of the tensor-core path (host logic, no GPU): its
bounds, the cases it must split and the ones it must leave alone."""
import itertools

import pytest


@pytest.fixture(scope="module")
def mm():
    from paper_1306_6192_gb300 import build
    build.build()
    import paper_1306_6192_gb300 as m
    return m


def plan(mm, tiles, grid, kt, bn, m, products=3.0):
    st, split_from, split_s = mm.mm_tail_plan(tiles, grid, kt, bn, m, products)
    assert st == mm.MM_OK
    return split_from, split_s


def test_bounds_over_a_sweep(mm):
    for tiles, grid, kt, bn, prod in itertools.product(
            (1, 2, 31, 100, 151, 152, 153, 160, 304, 321, 512, 2048, 4097),
            (1, 2, 76, 152), (1, 4, 8, 16, 31, 32, 64, 128, 256), (64, 128, 256),
            (0.5, 3.0, 6.0)):
        m = kt * 64
        f, s = plan(mm, tiles, grid, kt, bn, m, prod)
        assert 1 <= s <= 4
        if s == 1:
            assert f == tiles
            continue
        r = tiles - f
        assert 0 <= f < tiles and r >= 1
        assert r * s <= 2 * grid            # at most two rounds of parts
        assert kt // s >= 2                 # every part keeps two pack rows
        assert r in (tiles % grid, tiles % grid + grid)  # the last (or last two) waves
        assert not (tiles < grid and kt < 16)


def test_full_waves_are_not_split(mm):
    for waves in (1, 2, 13):
        assert plan(mm, 152 * waves, 152, 128, 256, 8192) == (152 * waves, 1)


def test_square_8192_splits_its_last_wave(mm):
    # 8192^3 with 128 x 256 tiles: 2048 tiles = 13 full waves of 152 + 72
    f, s = plan(mm, 2048, 152, 128, 256, 8192)
    assert f == 2048 - 72 and s >= 2


def test_small_products_of_grouped_tables_are_not_split(mm):
    # the grouped workload's products below m = 961 (kt <= 15): never split
    for tiles in range(1, 65):
        for kt in (1, 2, 8, 15):
            assert plan(mm, tiles, 152, kt, 128, kt * 64, 6.0)[1] == 1


def test_underfilled_1024_cube_is_split(mm):
    # 1024^3 on the three-part kind: 64 tiles of 128 x 128, 16 pack rows of
    # K, on 152 CTAs: half the SMs idle unless the tiles are cut along K
    f, s = plan(mm, 64, 152, 16, 128, 1024, 6.0)
    assert f == 0 and s >= 2


def test_one_long_tile_is_split(mm):
    # 64 x 16384 . 16384 x 64: one tile with 256 pack rows of K
    f, s = plan(mm, 1, 152, 256, 64, 16384)
    assert f == 0 and s == 4


def test_deterministic_and_arguments(mm):
    assert plan(mm, 512, 152, 64, 256, 4096) == plan(mm, 512, 152, 64, 256, 4096)
    st, _, _ = mm.mm_tail_plan(-1, 152, 64, 256, 4096, 3.0)
    assert st == mm.MM_EINVAL
    st, _, _ = mm.mm_tail_plan(10, 152, 64, 0, 4096, 3.0)
    assert st == mm.MM_EINVAL
    st, _, _ = mm.mm_tail_plan(10, 152, 64, 256, 4096, 0.0)
    assert st == mm.MM_EINVAL
