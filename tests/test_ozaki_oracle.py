"""Pins of the Ozaki-scheme oracle (oracle/ozaki.py), which the GPU path of
MM_MODE_OZAKI must match bit for bit: the digit expansion against exact
rationals, a hand-worked digit example, exact integer products, the chunk
rule, the method's error bound against exact rational products, agreement
with the plain FP64 oracle, and the edge cases.  Runs without a GPU."""
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import ozaki

U64 = 2.0 ** -53


def test_hand_worked_digits():
    # row maximum 0.375 = 0.75 * 2^-1: ilogb = -2, sigma = 0; S = 2 keeps 10 bits
    #   0.375: F = 384 = 12*32 + 0            -> 12, 0
    #   0.3:   F = floor(307.2) = 307 = 9*32 + 19; 19 >= 16 -> -13, carry -> 10, -13
    #   -0.2:  F = floor(204.8) = 204 = 6*32 + 12 -> -6, -12
    d = ozaki.digits(np.array([[0.375, 0.3, -0.2]]), np.array([[0]]), 2)
    assert d[:, 0, 0].tolist() == [12, 0]
    assert d[:, 0, 1].tolist() == [10, -13]
    assert d[:, 0, 2].tolist() == [-6, -12]
    # 3 in a row whose maximum is 5 = 0.625 * 2^3: sigma = 4, 3 / 16 = 6 / 32
    row = np.array([[3.0, 5.0]])
    sig = ozaki.scales(np.max(np.abs(row), axis=1))
    assert sig.tolist() == [4]
    d = ozaki.digits(row, sig[:, None], 2)
    assert d[:, 0, 0].tolist() == [6, 0] and d[:, 0, 1].tolist() == [10, 0]
    # a top digit of 16: F = 15*32 + 31 -> carry into 15 -> 16, -1
    x = (15 * 32 + 31) / 1024.0
    d = ozaki.digits(np.array([[x]]), np.array([[0]]), 2)
    assert d[:, 0, 0].tolist() == [16, -1]


def test_scales_are_ilogb_plus_two():
    x = np.array([0.0, 1.0, 0.999, 0.5, 3.0, 2.0 ** -1074, 2.0 ** -1030, 1e300])
    want = [0, 2, 1, 1, 3, -1072, -1028, int(np.floor(np.log2(1e300))) + 2]
    assert ozaki.scales(x).tolist() == want


@pytest.mark.parametrize("slices", [2, 5, 11, 12])
def test_digit_expansion_against_rationals(slices):
    vals = np.concatenate([
        synth.uniform_pm1_f64(3000, 40),
        synth.uniform_pm1_f64(3001, 40) * synth.pow2_int(3002, 40, -60, 60).astype(np.float64),
        np.array([0.0, -0.0, 2.0 ** -1074, -3 * 2.0 ** -1060, 1.0 - 2.0 ** -53]),
    ])
    sig = ozaki.scales(np.array([np.max(np.abs(vals))]))[0]
    d = ozaki.digits(vals[None, :], np.array([[sig]]), slices)[:, 0, :]
    assert np.all(np.abs(d) <= 16)
    for k, x in enumerate(vals):
        fx = abs(Fraction(float(x))) / Fraction(2) ** int(sig)
        assert fx < Fraction(1, 2)
        sgn = -1 if np.signbit(x) else 1
        mags = [sgn * int(d[t, k]) for t in range(slices)]  # digits of |x|
        assert 0 <= mags[0] <= 16 and all(-16 <= v <= 15 for v in mags[1:]), (x, mags)
        s = sum(Fraction(v, 32 ** (t + 1)) for t, v in enumerate(mags))
        rem = fx - s
        assert 0 <= rem < Fraction(1, 32 ** slices), (x, slices)


def test_chunk_rule():
    # (2^24 - 1) / (256 * 12) = 5461.3; 42 * 128 = 5376
    assert ozaki.chunk_columns(12) == 5376
    for S in range(ozaki.MIN_SLICES, ozaki.MAX_SLICES + 1):
        mc = ozaki.chunk_columns(S)
        assert mc % 128 == 0 and 256 * S * mc < 2 ** 24 <= 256 * S * (mc + 128)


@pytest.mark.parametrize("slices", list(range(ozaki.MIN_SLICES, ozaki.MAX_SLICES + 1)))
def test_chunk_rule_worst_case_level_sum(slices):
    """Every level sum the chunk rule admits is exact in FP32: balanced digits
    have magnitude at most 16 (a value whose digits reach it: 16, -16, ...,
    -16), so with every digit product at 256 (the digit arrays are written
    directly) over one full chunk, the top level L = S - 1 has S pairs of 256
    per column, 256 S mc < 2^24.  One more 128-column block per chunk would
    reach 2^24, and the oracle refuses such a level sum."""
    mc = ozaki.chunk_columns(slices)
    # F = 16 (32^(S-1) - (32^(S-1) - 1) / 31) has the digits 16, -16, ..., -16
    F = 16 * (32 ** (slices - 1) - (32 ** (slices - 1) - 1) // 31)
    assert F < 2 ** (5 * slices - 1)
    if F < 2 ** 53:  # exact as a double
        x = float(Fraction(F, 2 ** (5 * slices)))
        d = ozaki.digits(np.array([[x]]), np.array([[0]]), slices)[:, 0, 0]
        assert d.tolist() == [16] + [-16] * (slices - 1)
    Ad = np.full((slices, 1, mc), -16, np.int64)
    Bd = np.full((slices, mc, 1), -16, np.int64)
    D = ozaki.level_sums(Ad, Bd, slices)
    assert D.shape == (1, slices, 1, 1)
    for L in range(slices):
        assert D[0, L, 0, 0] == 256 * (L + 1) * mc
    assert abs(D).max() < 2 ** 24
    # a chunk rule one block too long lets the top level reach 2^24
    wide = mc + 128
    Aw = np.full((slices, 1, wide), 16, np.int64)
    Bw = np.full((slices, wide, 1), 16, np.int64)
    orig = ozaki.chunk_columns
    try:
        ozaki.chunk_columns = lambda s: wide
        with pytest.raises(ArithmeticError):
            ozaki.level_sums(Aw, Bw, slices)
    finally:
        ozaki.chunk_columns = orig


@pytest.mark.parametrize("shape,slices", [((7, 33, 5), 2), ((9, 5000, 6), 12), ((4, 1, 3), 11)])
def test_small_integers_exact(shape, slices):
    n, m, p = shape
    A = synth.small_ints(3100, (n, m)).astype(np.float64)
    B = synth.small_ints(3101, (m, p)).astype(np.float64)
    C = ozaki.gemm(A, B, slices)
    exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    assert np.array_equal(C, exact)


def _exact(A, B):
    n, m = A.shape
    p = B.shape[1]
    C = [[Fraction(0)] * p for _ in range(n)]
    S = [[0.0] * p for _ in range(n)]
    for i in range(n):
        for j in range(p):
            c = Fraction(0)
            s = 0.0
            for r in range(m):
                c += Fraction(float(A[i, r])) * Fraction(float(B[r, j]))
                s += abs(float(A[i, r]) * float(B[r, j]))
            C[i][j] = c
            S[i][j] = s
    return C, S


@pytest.mark.parametrize("slices", [2, 3, 6, 12])
@pytest.mark.parametrize("wide", [False, True])
def test_error_bound_against_rationals(slices, wide):
    n, m, p = 3, 29, 4
    A = synth.uniform_pm1_f64(3200, (n, m))
    B = synth.uniform_pm1_f64(3201, (m, p))
    if wide:
        A = A * synth.pow2_int(3202, (n, m), -30, 30).astype(np.float64)
        B = B * synth.pow2_int(3203, (m, p), -30, 30).astype(np.float64)
    A[1, 3] = 0.0
    C = ozaki.gemm(A, B, slices)
    bound = ozaki.error_bound(A, B, slices)
    Cx, Sabs = _exact(A, B)
    worst = 0.0
    for i in range(n):
        for j in range(p):
            err = abs(Fraction(float(C[i, j])) - Cx[i][j])
            # plus the final rounding to a double (half an ulp of the result)
            tol = bound[i, j] * (1 + U64) + U64 * (abs(float(Cx[i][j])) + bound[i, j])
            assert float(err) <= tol, (i, j, float(err), tol)
            worst = max(worst, float(err) / Sabs[i][j])
    if slices == 2 and not wide:
        assert worst > 1e-7       # two digits keep ~10 bits: the bound is not vacuous
    if slices == 12 and not wide:
        assert worst < 1e-15


def test_close_to_plain_fp64_oracle(orc):
    A = synth.uniform_pm1_f64(3300, (37, 300))
    B = synth.uniform_pm1_f64(3301, (300, 23))
    C = ozaki.gemm(A, B, 12)
    ref, absref = orc.gemm(A, B, with_abs=True)
    e = np.abs(C - ref) / absref
    assert e.max() < 1e-15


def test_edges():
    A = synth.uniform_pm1_f64(3400, (5, 9))
    B = synth.uniform_pm1_f64(3401, (9, 4))
    A[2, :] = 0.0
    C = ozaki.gemm(A, B, 8)
    assert np.all(C[2] == 0) and not np.any(np.signbit(C[2]))
    A[3, 4] = np.nan
    B[6, 1] = np.inf
    C = ozaki.gemm(A, B, 8)
    assert np.all(np.isnan(C[3])) and np.all(np.isnan(C[:, 1]))
    keep = [0, 1, 2, 4]
    assert np.all(np.isfinite(C[np.ix_(keep, [0, 2, 3])]))
    assert ozaki.gemm(np.zeros((3, 0)), np.zeros((0, 2)), 4).tolist() == [[0.0] * 2] * 3
    assert ozaki.gemm(np.zeros((0, 3)), np.zeros((3, 2)), 4).shape == (0, 2)


def _digits_shifted(X, sigma, slices):
    """Planted mistake: digit t taken one position too low."""
    d = _ORIG_DIGITS(X, sigma, slices)
    return np.concatenate([np.zeros_like(d[:1]), d[:-1]])


def _scales_no_offset(maxabs):
    """Planted mistake: sigma = ilogb(max) + 1 (the largest entries reach 1/2
    and beyond)."""
    return _ORIG_SCALES(maxabs) - np.where(maxabs > 0, 1, 0)


def _levels_dropped_term(Ad, Bd, slices):
    """Planted mistake: each level above 0 misses its t = 0 pair."""
    D = _ORIG_LEVELS(Ad, Bd, slices)
    m = Ad.shape[2]
    mc = ozaki.chunk_columns(slices)
    for c, k0 in enumerate(range(0, m, mc)):
        k1 = min(m, k0 + mc)
        for L in range(1, slices):
            D[c, L] -= Ad[0][:, k0:k1].astype(float) @ Bd[L][k0:k1, :].astype(float)
    return D


def _combine_wrong_weight(D, sigma, tau, slices):
    """Planted mistake: the levels weighted one digit too high."""
    return _ORIG_COMBINE(D, sigma, tau, slices) * 32.0


def _combine_reversed_levels(D, sigma, tau, slices):
    """Planted mistake: level L weighted as level S-1-L."""
    return _ORIG_COMBINE(D[:, ::-1], sigma, tau, slices)


_ORIG_DIGITS, _ORIG_SCALES = ozaki.digits, ozaki.scales
_ORIG_LEVELS, _ORIG_COMBINE = ozaki.level_sums, ozaki.combine


@pytest.mark.parametrize("name,fake", [("digits", _digits_shifted), ("scales", _scales_no_offset),
                                       ("level_sums", _levels_dropped_term),
                                       ("combine", _combine_wrong_weight),
                                       ("combine", _combine_reversed_levels)])
def test_planted_mistakes_are_caught(monkeypatch, name, fake):
    monkeypatch.setattr(ozaki, name, fake)
    pins = [test_hand_worked_digits,
            lambda: test_small_integers_exact((7, 33, 5), 2),
            lambda: test_error_bound_against_rationals(12, False),
            lambda: test_digit_expansion_against_rationals(5)]
    failed = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed >= 1, name


_ORIG_CHUNK = ozaki.chunk_columns


@pytest.mark.parametrize("fake", [lambda s: _ORIG_CHUNK(s) + 128,
                                  lambda s: ((2 ** 24 - 1) // (256 * s) + 127) // 128 * 128,
                                  lambda s: ((2 ** 24 - 1) // (225 * s)) // 128 * 128])
def test_planted_chunk_rule_is_caught(monkeypatch, fake):
    """Planted mistakes in the chunk rule (one block too long, rounded up, the
    digit products bounded by 15 * 15 instead of 16 * 16): the worst-case level
    sum catches each."""
    monkeypatch.setattr(ozaki, "chunk_columns", fake)
    with pytest.raises((AssertionError, ArithmeticError)):
        for S in range(ozaki.MIN_SLICES, ozaki.MAX_SLICES + 1):
            test_chunk_rule_worst_case_level_sum(S)
