"""The K-slice planner of the SIMT FP32 and FP64 DGEMM paths (host logic, no
GPU): which products are cut along K, and the bounds every plan keeps (one
wave of at most two CTAs per SM, slices of at least 128 values, slices that
cover K exactly, partials of at most 256 MiB, the same plan for a product and
its transpose)."""
import itertools

import pytest


@pytest.fixture(scope="module")
def mm():
    from paper_1306_6192_gb300 import build
    build.build()
    import paper_1306_6192_gb300 as m
    return m


def plan(mm, n, m, p, dt, sms=152):
    st, S, ks, tile = mm.mm_simt_plan(n, m, p, dt, sms)
    assert st == mm.MM_OK
    return S, ks, tile


def cdiv(a, b):
    return -(-a // b)


SIZES = (1, 33, 64, 100, 128, 129, 200, 512, 1000, 2048)
KS = (1, 100, 127, 128, 129, 1000, 4999, 16384, 100000)


@pytest.mark.parametrize("sms", [148, 152])
def test_bounds_over_a_sweep(mm, sms):
    for (n, p, m), dt in itertools.product(itertools.product(SIZES, SIZES, KS),
                                           (mm.MM_F32, mm.MM_F64)):
        S, ks, tile = plan(mm, n, m, p, dt, sms)
        f64 = dt == mm.MM_F64
        big = 64 if f64 else 128  # the one-pass kernel's tile
        assert plan(mm, p, m, n, dt, sms) == (S, ks, tile), (n, m, p, dt)
        if 2 * cdiv(n, big) * cdiv(p, big) >= sms:
            assert (S, ks, tile) == (0, 0, big), (n, m, p, dt)
            continue
        assert S >= 1
        assert tile == (128 if not f64 and n >= 128 and p >= 128 else 64)
        tiles = cdiv(n, tile) * cdiv(p, tile)
        assert S * tiles <= 2 * sms, (n, m, p, dt)  # one wave
        assert ks % (8 if f64 else 16) == 0
        assert (S - 1) * ks < m <= S * ks, (n, m, p, dt)  # the slices cover K, none empty
        if S > 1:
            assert ks >= 128
            assert S * n * p * (8 if f64 else 4) <= 256 << 20
        assert S <= 1024


def test_skinny_product_is_cut_into_128_slices(mm):
    """64 x 16384 . 16384 x 64: one output tile, so 128 slices of 128 values
    (the K bound, below two per SM)."""
    for dt in (mm.MM_F32, mm.MM_F64):
        assert plan(mm, 64, 16384, 64, dt) == (128, 128, 64)


def test_products_that_fill_the_sms_are_not_cut(mm):
    assert plan(mm, 2048, 512, 2048, mm.MM_F32) == (0, 0, 128)
    assert plan(mm, 2048, 512, 2048, mm.MM_F64) == (0, 0, 64)
    # 38 tiles of 128 x 128 fill half of 76 SMs but not of 152
    assert plan(mm, 128 * 38, 4096, 128, mm.MM_F32, sms=76)[0] == 0
    assert plan(mm, 128 * 38, 4096, 128, mm.MM_F32, sms=152)[0] > 0


def test_short_k_takes_one_slice(mm):
    """K below 128 is one slice (the partials would cost more than they save);
    its length is K rounded up to the kernel's K step."""
    assert plan(mm, 64, 100, 64, mm.MM_F32) == (1, 112, 64)
    assert plan(mm, 64, 100, 64, mm.MM_F64) == (1, 104, 64)
    assert plan(mm, 64, 1, 64, mm.MM_F32) == (1, 16, 64)


def test_wide_tiles_for_fp32_only(mm):
    """FP32 products at least 128 wide both ways keep 128 x 128 tiles; FP64
    and narrower FP32 products take 64 x 64."""
    assert plan(mm, 200, 2048, 150, mm.MM_F32)[2] == 128
    assert plan(mm, 200, 2048, 100, mm.MM_F32)[2] == 64
    assert plan(mm, 200, 2048, 150, mm.MM_F64)[2] == 64


def test_empty_and_arguments(mm):
    assert plan(mm, 0, 100, 10, mm.MM_F32) == (0, 0, 128)
    assert plan(mm, 10, 0, 10, mm.MM_F64) == (0, 0, 64)
    assert mm.mm_simt_plan(-1, 10, 10, mm.MM_F32)[0] == mm.MM_EINVAL
    assert mm.mm_simt_plan(10, -1, 10, mm.MM_F64)[0] == mm.MM_EINVAL
    assert mm.mm_simt_plan(10, 10, 10, 7)[0] == mm.MM_EINVAL
    # sms <= 0 takes the device's count (148 before the library is
    # initialised); this product has the same plan on 148 and 152 SMs
    assert mm.mm_simt_plan(64, 16384, 64, mm.MM_F32, 0) == (mm.MM_OK, 128, 128, 64)
