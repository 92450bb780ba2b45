"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each ``pin_*`` takes an ``oracle.Oracle`` and raises AssertionError when the
oracle disagrees with something other than itself: exact rational arithmetic
of the definition (brute force with ``fractions.Fraction``), a hand-worked
example, closed forms (identity, diagonal), an exact integer library routine,
the invariants (AB)^T = B^T A^T and (AB)x = A(Bx), and rounding-error bounds.
The definition pinned is the Cauchy product of the paper's Section
"Implementacje algorytmow" (c_ij = sum_r a_ir b_rj), in the order of Listing 1.

The same pins run against builds of the oracle with one planted mistake each
(tests/test_oracle_mutants.py) to show that every such mistake is caught.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

import synth

U64 = 2.0 ** -53  # unit roundoff of binary64


def _exact_product(A, B):
    """Definition of the Cauchy product in exact rationals (tiny inputs)."""
    n, m = A.shape
    p = B.shape[1]
    C = [[Fraction(0)] * p for _ in range(n)]
    S = [[Fraction(0)] * p for _ in range(n)]
    for i in range(n):
        for j in range(p):
            c = Fraction(0)
            s = Fraction(0)
            for r in range(m):
                a = Fraction(float(A[i, r]))
                b = Fraction(float(B[r, j]))
                c += a * b
                s += abs(a) * abs(b)
            C[i][j] = c
            S[i][j] = s
    return C, S


TINY_SHAPES = [(1, 1, 1), (2, 3, 4), (3, 3, 3), (4, 1, 5), (5, 7, 2), (7, 5, 3),
               (17, 5, 3), (3, 17, 7), (4, 4, 17)]


def pin_bruteforce_definition(orc):
    """FP64 oracle vs exact rationals: |c - c_exact| <= (m-1) u (|A||B|)_ij,
    the textbook bound for recursive summation of exact products."""
    for t, (n, m, p) in enumerate(TINY_SHAPES):
        A = synth.uniform_pm1(100 + t, (n, m))
        B = synth.uniform_pm1(200 + t, (m, p))
        C, absC = orc.gemm(A, B, with_abs=True)
        Cx, Sx = _exact_product(A, B)
        for i in range(n):
            for j in range(p):
                bound = (m - 1) * U64 * float(Sx[i][j]) * (1 + 1e-12)
                err = abs(Fraction(float(C[i, j])) - Cx[i][j])
                assert float(err) <= bound, (n, m, p, i, j, float(err), bound)
                errs = abs(Fraction(float(absC[i, j])) - Sx[i][j])
                assert float(errs) <= bound + 1e-300, ("abs", n, m, p, i, j)


def pin_small_ints_exact(orc):
    """Integer entries in [-8, 8]: every partial sum is an integer below 2^53,
    so the oracle must equal the exact integer product (numpy int64 matmul)."""
    for t, (n, m, p) in enumerate([(1, 1, 1), (33, 64, 17), (8, 4096, 5), (64, 64, 64)]):
        A = synth.small_ints(300 + t, (n, m))
        B = synth.small_ints(400 + t, (m, p))
        C, absC = orc.gemm(A, B, with_abs=True)
        Ci = A.astype(np.int64) @ B.astype(np.int64)
        Si = np.abs(A).astype(np.int64) @ np.abs(B).astype(np.int64)
        assert np.array_equal(C, Ci.astype(np.float64)), (n, m, p)
        assert np.array_equal(absC, Si.astype(np.float64)), (n, m, p)


def pin_hand_example(orc):
    """Products worked by hand from the definition (tests/golden/hand_worked.txt):
    the 3x3 size of the paper's walk-through before Listing 2, where the
    thread with thread_x = 0, thread_y = 1 reads row thread_y of A and column
    thread_x of B and so computes the entry in row 1, column 0 (84 here), and
    a 2x3 by 3x2 product that catches a swapped operand or index.  The
    normaliser |A||B| is worked by hand too."""
    import golden
    cases = golden.hand_worked()
    assert [c["name"] for c in cases] == ["walkthrough_3x3", "nonsquare_2x3x2"]
    for c in cases:
        C, S = orc.gemm(c["A"], c["B"], with_abs=True)
        assert C.shape == (c["n"], c["p"]), c["name"]
        assert np.array_equal(C, c["C"]), c["name"]
        assert np.array_equal(S, c["ABS"]), c["name"]
    assert cases[0]["C"][1, 0] == 84.0


def pin_identity(orc):
    """A.I = A and I.B = B exactly (one non-zero product per entry)."""
    A = synth.uniform_pm1(500, (37, 23))
    C = orc.gemm(A, synth.identity(23))
    assert np.array_equal(C, A.astype(np.float64))
    B = synth.uniform_pm1(501, (19, 41))
    C = orc.gemm(synth.identity(19), B)
    assert np.array_equal(C, B.astype(np.float64))


def pin_diagonal(orc):
    """Paper's special case of diagonal matrices: A.diag(d) has c_ij = a_ij d_j
    and diag(d).B has c_ij = d_i b_ij, exactly (products of two float32 values
    are exact in binary64)."""
    A = synth.uniform_pm1(600, (29, 31))
    d = synth.uniform_pm1(601, 31)
    C = orc.gemm(A, synth.diag_matrix(601, 31))
    assert np.array_equal(C, A.astype(np.float64) * d.astype(np.float64)[None, :])
    B = synth.uniform_pm1(602, (31, 13))
    C = orc.gemm(synth.diag_matrix(601, 31), B)
    assert np.array_equal(C, d.astype(np.float64)[:, None] * B.astype(np.float64))


def pin_transpose(orc):
    """(AB)^T = B^T A^T: each entry sums the same products in the same order,
    so the oracle must agree bit for bit."""
    A = synth.uniform_pm1(700, (23, 45))
    B = synth.uniform_pm1(701, (45, 31))
    C = orc.gemm(A, B)
    Ct = orc.gemm(B.T.copy(), A.T.copy())
    assert np.array_equal(C.T, Ct)


def pin_freivalds(orc):
    """(AB)x = A(Bx) within the rounding of both sides."""
    n, m, p = 40, 300, 50
    A = synth.uniform_pm1(800, (n, m))
    B = synth.uniform_pm1(801, (m, p))
    x = synth.freivalds_vector(802, p)
    C, absC = orc.gemm(A, B, with_abs=True)
    y, ya = orc.gemv(C, x)
    z, za = orc.freivalds_rhs(A, B, x)
    bound = 4 * (m + p) * U64 * za
    assert np.all(np.abs(y - z) <= bound), float(np.max(np.abs(y - z) / za))
    # a result with one wrong row must be caught
    Cb = C.copy()
    Cb[7, :] += 1e-6 * absC[7, :]
    yb, _ = orc.gemv(Cb, x)
    assert np.abs(yb[7] - z[7]) > bound[7]


def pin_threads_invariant(orc):
    """Rows are split over threads; the result must not depend on the split."""
    A = synth.uniform_pm1(900, (53, 77))
    B = synth.uniform_pm1(901, (77, 29))
    ref = orc.gemm(A, B, threads=1)
    for t in (2, 3, 8, 64):
        assert np.array_equal(orc.gemm(A, B, threads=t), ref)


def pin_empty_dims(orc):
    """m = 0 gives the empty sum (C = 0); n = 0 or p = 0 gives an empty C."""
    C = orc.gemm(np.zeros((4, 0), np.float32), np.zeros((0, 5), np.float32))
    assert C.shape == (4, 5) and np.all(C == 0)
    assert orc.gemm(np.zeros((0, 3), np.float32), np.ones((3, 2), np.float32)).shape == (0, 2)
    assert orc.gemm(np.ones((2, 3), np.float32), np.ones((3, 0), np.float32)).shape == (2, 0)


def _exact_dot(x, y):
    return sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y)), Fraction(0))


def pin_dot2_and_long_double(orc):
    """Dot2 error <= u|s| + gamma_{n}^2 sum|ab| (Ogita-Rump-Oishi, Prop. 5.5
    style bound, taken loosely with factor 2); long double error <=
    (m-1) 2^-LDBL_MANT_DIG sum|ab| + u|s| after rounding to double.  The data
    are ill-conditioned on purpose: the second half of the products cancels
    the first half up to a small remainder."""
    m = 200
    a = synth.uniform_pm1_f64(1000, m)
    b = synth.uniform_pm1_f64(1001, m)
    # y2 chosen so that a2*b2 nearly cancels a1*b1 (condition number ~1e15)
    A = np.concatenate([a, a]).reshape(1, 2 * m)
    B = np.concatenate([b, -b * (1 + 2.0 ** -40)]).reshape(2 * m, 1)
    ex = _exact_dot(A[0], B[:, 0])
    s_abs = float(sum(abs(Fraction(float(x)) * Fraction(float(y))) for x, y in zip(A[0], B[:, 0])))
    hi, lo, ab = orc.entries(A, B, np.array([0]), np.array([0]), "dot2")
    n2 = 2 * m
    gam = n2 * U64 / (1 - n2 * U64)
    bound = U64 * abs(float(ex)) + 2 * gam * gam * s_abs
    assert abs(float(Fraction(float(hi[0])) - ex)) <= bound, (float(hi[0]), float(ex))
    assert abs(ab[0] - s_abs) <= n2 * U64 * s_abs
    hl, ll, _ = orc.entries(A, B, np.array([0]), np.array([0]), "ld")
    ul = 2.0 ** -orc.ldbl_mant_dig()
    bound_ld = U64 * abs(float(ex)) + (n2 - 1) * ul * s_abs * 1.01
    assert abs(float(Fraction(float(hl[0])) - ex)) <= bound_ld
    # plain FP64 cannot meet the Dot2 bound on this data (shows the test bites)
    plain = orc.gemm(A, B)[0, 0]
    assert abs(float(Fraction(float(plain)) - ex)) > bound


def pin_gemv(orc):
    """gemv via Dot2 against exact rationals."""
    X = synth.uniform_pm1_f64(1100, (6, 25))
    v = synth.uniform_pm1_f64(1101, 25)
    y, ya = orc.gemv(X, v)
    for i in range(6):
        ex = _exact_dot(X[i], v)
        assert abs(float(Fraction(float(y[i])) - ex)) <= 2 * U64 * abs(float(ex)) + 1e-300


def pin_pow2_exact(orc):
    """Exact fixed-point sum for +-2^k inputs against exact rationals."""
    A = synth.pow2_int(1200, (5, 37))
    B = synth.pow2_int(1201, (37, 4))
    hi, lo = orc.pow2_exact(A, B, shift=50)
    Cx, _ = _exact_product(A, B)
    for i in range(5):
        for j in range(4):
            got = Fraction(float(hi[i, j])) + Fraction(float(lo[i, j]))
            assert got == Cx[i][j], (i, j)


def pin_complex(orc):
    """Complex product: exact Gaussian rationals on tiny shapes, numpy's exact
    complex product on small integers, and c = A.B with real A, B reducing to
    the real oracle."""
    def cfrac(z):
        return (Fraction(float(z.real)), Fraction(float(z.imag)))
    for t, (n, m, p) in enumerate([(1, 1, 1), (2, 3, 4), (5, 7, 3)]):
        A = synth.uniform_pm1(1300 + t, (n, m)) + 1j * synth.uniform_pm1(1310 + t, (n, m))
        B = synth.uniform_pm1(1320 + t, (m, p)) + 1j * synth.uniform_pm1(1330 + t, (m, p))
        C, absC = orc.cgemm(A, B)
        for i in range(n):
            for j in range(p):
                er = Fraction(0); ei = Fraction(0)
                for r in range(m):
                    ar, ai = cfrac(A[i, r]); br, bi = cfrac(B[r, j])
                    er += ar * br - ai * bi
                    ei += ar * bi + ai * br
                bound = 4 * m * U64 * float(absC[i, j]) + 1e-300
                assert abs(float(Fraction(float(C[i, j].real)) - er)) <= bound
                assert abs(float(Fraction(float(C[i, j].imag)) - ei)) <= bound
    Ai = synth.small_ints(1340, (20, 33)) + 1j * synth.small_ints(1341, (20, 33))
    Bi = synth.small_ints(1342, (33, 17)) + 1j * synth.small_ints(1343, (33, 17))
    C, _ = orc.cgemm(Ai, Bi)
    assert np.array_equal(C, Ai.astype(np.complex128) @ Bi.astype(np.complex128))
    Ar = synth.uniform_pm1(1344, (9, 11)); Br = synth.uniform_pm1(1345, (11, 6))
    C, absC = orc.cgemm(Ar, Br)
    Cr, Sr = orc.gemm(Ar, Br, with_abs=True)
    assert np.array_equal(C.real, Cr) and np.all(C.imag == 0) and np.array_equal(absC, Sr)


def pin_axpby(orc):
    """alpha (A.B) + beta D against exact rationals on tiny inputs (within the
    FP64 rounding of the product and of the two scalings), exact on small
    integers, and its special cases: alpha = 1, beta = 0 is the product
    itself; alpha = 0 is beta D without the product; D = C gives the same
    as a separate copy of D."""
    A = synth.uniform_pm1(3100, (3, 5)).astype(np.float64)
    B = synth.uniform_pm1(3101, (5, 4)).astype(np.float64)
    D = synth.uniform_pm1(3102, (3, 4)).astype(np.float64)
    alpha, beta = -0.3, 1.7
    got, norm = orc.axpby(alpha, A, B, beta, D)
    C, S = _exact_product(A, B)
    for i in range(3):
        for j in range(4):
            a, b, d = Fraction(alpha), Fraction(beta), Fraction(float(D[i, j]))
            exact = a * C[i][j] + b * d
            nrm = abs(a) * S[i][j] + abs(b) * abs(d)
            assert abs(Fraction(float(got[i, j])) - exact) <= 8 * Fraction(U64) * nrm
            assert abs(Fraction(float(norm[i, j])) - nrm) <= 8 * Fraction(U64) * nrm
    Ai = synth.small_ints(3103, (4, 6)).astype(np.float64)
    Bi = synth.small_ints(3104, (6, 5)).astype(np.float64)
    Di = synth.small_ints(3105, (4, 5)).astype(np.float64)
    got, _ = orc.axpby(3, Ai, Bi, -2, Di)
    want = [[3 * sum(int(Ai[i, r]) * int(Bi[r, j]) for r in range(6)) - 2 * int(Di[i, j])
             for j in range(5)] for i in range(4)]
    assert np.array_equal(got, np.array(want, np.float64))
    ref, ab = orc.gemm(A, B, with_abs=True)
    got, norm = orc.axpby(1.0, A, B, 0.0, None)
    assert np.array_equal(got, ref) and np.array_equal(norm, ab)
    got, norm = orc.axpby(0.0, None, None, -2.0, D)
    assert np.array_equal(got, -2.0 * D) and np.array_equal(norm, 2.0 * np.abs(D))


ALL_PINS = [
    pin_bruteforce_definition, pin_small_ints_exact, pin_hand_example,
    pin_identity, pin_diagonal, pin_transpose, pin_freivalds,
    pin_threads_invariant, pin_empty_dims, pin_dot2_and_long_double,
    pin_gemv, pin_pow2_exact, pin_complex, pin_axpby,
]
