"""The FP64 emulation's plan as the library computes it on the host
(mm_ozaki_plan, no GPU): its K chunk rule must be the one the oracle restates
independently (oracle/ozaki.py), its chunk count ceil(m / columns), its
argument checks as documented, and its scratch bound must cover the digit
packs and level sums the method stores, with the accuracy gate's slice and
planes."""
import math

import pytest

from oracle import ozaki


@pytest.fixture(scope="module")
def mm():
    from paper_1306_6192_gb300 import build
    build.build()
    import paper_1306_6192_gb300 as m
    return m


def test_chunk_rule_matches_oracle(mm):
    for S in range(ozaki.MIN_SLICES, ozaki.MAX_SLICES + 1):
        st, mc, q, _ = mm.mm_ozaki_plan(64, 1000, 64, S)
        assert st == mm.MM_OK
        assert mc == ozaki.chunk_columns(S)
        assert q == 1


@pytest.mark.parametrize("m", [0, 1, 127, 5376, 5377, 10752, 100000])
def test_chunk_count(mm, m):
    st, mc, q, b = mm.mm_ozaki_plan(300, m, 200, 12)
    assert st == mm.MM_OK and mc == 5376
    assert q == math.ceil(m / mc)
    if m == 0:
        assert b == 0


@pytest.mark.parametrize("n,m,p,S", [(4096, 4096, 4096, 12), (8192, 8192, 8192, 12),
                                      (300, 517, 260, 2), (129, 6000, 70, 11), (1, 1, 1, 12)])
def test_scratch_bound_covers_digits_and_level_sums(mm, n, m, p, S):
    st, mc, q, b = mm.mm_ozaki_plan(n, m, p, S)
    assert st == mm.MM_OK
    # S digit slices per operand plus the accuracy gate's slice, S level sums
    # per K chunk plus the gate's plane
    digits = (S + 1) * (math.ceil(n / 128) * 128 + math.ceil(p / 128) * 128) * m
    levels = q * (S + 1) * n * p * 4
    assert b >= digits + levels
    assert b <= 2 * (digits + levels) + (4 << 20)


def test_arguments(mm):
    assert mm.mm_ozaki_plan(4, 4, 4, 1)[0] == mm.MM_EINVAL
    assert mm.mm_ozaki_plan(4, 4, 4, 13)[0] == mm.MM_EINVAL
    assert mm.mm_ozaki_plan(-1, 4, 4, 12)[0] == mm.MM_EINVAL
    assert mm.mm_ozaki_plan(4, -4, 4, 12)[0] == mm.MM_EINVAL
    mc = ozaki.chunk_columns(12)
    assert mm.mm_ozaki_plan(4, 1024 * mc, 4, 12)[0] == mm.MM_OK
    assert mm.mm_ozaki_plan(4, 1024 * mc + 1, 4, 12)[0] == mm.MM_EINVAL
