"""Oracle of the FP64 product emulated by the Ozaki scheme.

TEST INFRASTRUCTURE ONLY, like the rest of this package: only tests/,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it.
It shares no code with the CUDA path.

Method: K. Ozaki, T. Ogita, S. Oishi, S. M. Rump, "Error-free transformations
of matrix multiplication by using fast routines of matrix multiplication and
its applicability", Numer. Algorithms 59 (2012): cut each operand into slices
whose pairwise products are computed without rounding by a fast low-precision
matrix product, then add the slice products in the working precision.  This is
not in the paper (whose "double" column multiplies in double directly); the
variant restated here, step by step, is the one the library's e4m3 tensor-core
path implements:

  1. Scales.  sigma_i = ilogb(max_r |a_ir|) + 2 for each row of A (so that
     |a_ir| 2^-sigma_i < 1/2), tau_j the same for each column of B; 0 for an
     all-zero row or column.
  2. Digits.  F = floor(|x| 2^(5S - sigma)), an integer below 2^(5S - 1)
     (S <= 12, so F fits 59 bits).  Its base-32 digits f_t (t = 0 most
     significant) are made balanced from the least significant one up: with a
     carry c = 0, for t = S-1 down to 1, v = f_t + c gives d_t = v - 32 and
     c = 1 when v >= 16, else d_t = v and c = 0; then d_0 = f_0 + c.  So
     d_t lies in [-16, 15] for t >= 1, d_0 in [0, 16], every digit is an
     integer e4m3 holds exactly, sum_t d_t 32^(S-1-t) = F, and with the sign
     of x on every digit x 2^-sigma = sum_t d_t 32^-(t+1) + (a remainder of
     magnitude below 2^-5S).
  3. K chunks.  The inner dimension is cut into chunks of
     mc = floor(floor((2^24 - 1) / (256 S)) / 128) * 128 columns (the last one
     shorter); with |d| <= 16 a level of S pairs over mc columns stays below
     2^24, so each level sum is an integer that FP32 holds exactly (the
     condition under which the tensor cores' FP32 accumulation of the digit
     products is error-free).  The chunking leaves the exact result unchanged;
     the oracle checks that condition on every level sum it forms and raises
     if a chunk rule ever lets one reach 2^24.
  4. Levels.  For each chunk c and L = 0..S-1,
         D[c][L] = sum_{t+u=L} A_t[:, chunk c] . B_u[chunk c, :]
     exactly (integers; float64 matrix products of integers whose partial
     sums stay below 2^53 are exact).  Pairs with t + u >= S are dropped.
  5. Sum.  v = sum over chunks and levels of D[c][L] 32^(S-1-L), an exact
     integer; c_ij = RN(v) 2^(sigma_i + tau_j - 5(S+1)), RN = the nearest
     double (ties to even), the power-of-two scaling rounding again only in
     the subnormal range.  Rows of A or columns of B that hold a NaN or an
     infinity give NaN.
"""
from __future__ import annotations

import numpy as np

MIN_SLICES, MAX_SLICES, DEFAULT_SLICES = 2, 12, 12


def chunk_columns(slices: int) -> int:
    """Step 3: inner-dimension columns per chunk."""
    return ((2 ** 24 - 1) // (256 * slices)) // 128 * 128


def scales(maxabs: np.ndarray) -> np.ndarray:
    """Step 1: ilogb(max) + 2 (0 for a zero maximum).  frexp writes a
    positive finite max as f 2^e with f in [0.5, 1), so ilogb(max) = e - 1."""
    _, e = np.frexp(np.where(np.isfinite(maxabs), maxabs, 0.0))
    return np.where(maxabs > 0, e + 1, 0).astype(np.int64)


def fixed_point(X: np.ndarray, sigma: np.ndarray, slices: int) -> np.ndarray:
    """F = floor(|x| 2^(5S - sigma)) (uint64) for a matrix whose element
    (i, k) is scaled by 2^-sigma[i] (sigma broadcast against X), from the
    float64 bit fields in integer arithmetic."""
    X = np.asarray(X, np.float64)
    ax = np.abs(np.where(np.isfinite(X), X, 0.0))
    f, e = np.frexp(ax)                       # ax = f 2^e, f in [0.5, 1) or 0
    mant = (f * 2.0 ** 53).astype(np.uint64)  # exact: f has at most 53 bits
    shift = e.astype(np.int64) - 53 + 5 * slices - np.broadcast_to(sigma, X.shape)
    F = np.zeros(X.shape, np.uint64)
    left = shift >= 0
    F[left] = mant[left] << shift[left].astype(np.uint64)
    right = (shift < 0) & (shift > -64)
    F[right] = mant[right] >> (-shift[right]).astype(np.uint64)
    return F


def digits(X: np.ndarray, sigma: np.ndarray, slices: int) -> np.ndarray:
    """Step 2: int64 array [slices, *X.shape] of signed balanced digits."""
    if not MIN_SLICES <= slices <= MAX_SLICES:
        raise ValueError("slices must lie in [%d, %d]" % (MIN_SLICES, MAX_SLICES))
    F = fixed_point(X, sigma, slices)
    f = [((F >> np.uint64(5 * (slices - 1 - t))) & np.uint64(31)).astype(np.int64)
         for t in range(slices)]
    out = np.empty((slices,) + F.shape, np.int64)
    carry = np.zeros(F.shape, np.int64)
    for t in range(slices - 1, 0, -1):
        v = f[t] + carry
        wrap = v >= 16
        out[t] = np.where(wrap, v - 32, v)
        carry = wrap.astype(np.int64)
    out[0] = f[0] + carry
    sign = np.where(np.signbit(np.asarray(X, np.float64)), -1, 1).astype(np.int64)
    return out * sign


def level_sums(Ad: np.ndarray, Bd: np.ndarray, slices: int) -> np.ndarray:
    """Steps 3-4: D[c][L] = sum_{t+u=L} A_t[:, chunk c] . B_u[chunk c, :] from
    the digit arrays Ad [S, n, m] and Bd [S, m, p]; float64 products of
    integers whose partial sums stay below 2^53, so exact."""
    m = Ad.shape[2]
    mc = chunk_columns(slices)
    chunks = [(k0, min(m, k0 + mc)) for k0 in range(0, m, mc)]
    Af = Ad.astype(np.float64)
    Bf = Bd.astype(np.float64)
    D = np.zeros((len(chunks), slices, Ad.shape[1], Bd.shape[2]))
    for c, (k0, k1) in enumerate(chunks):
        for L in range(slices):
            for t in range(L + 1):
                D[c, L] += Af[t][:, k0:k1] @ Bf[L - t][k0:k1, :]
    if D.size and float(np.max(np.abs(D))) >= 2.0 ** 24:
        raise ArithmeticError("a level sum reached 2^24: not exact in FP32 (K chunk too long)")
    return D


def combine(D: np.ndarray, sigma: np.ndarray, tau: np.ndarray, slices: int) -> np.ndarray:
    """Step 5: the exact integer v = sum_c sum_L D[c][L] 32^(S-1-L) (Python
    integers), rounded to the nearest double, times 2^(sigma_i + tau_j - 5(S+1))."""
    n, p = D.shape[2:]
    v = np.zeros((n, p), dtype=object)
    for c in range(D.shape[0]):
        for L in range(slices):
            Di = D[c, L].astype(np.int64).astype(object)
            v = v + Di * (1 << (5 * (slices - 1 - L)))
    rounded = np.array([[float(x) for x in row] for row in v], dtype=np.float64).reshape(n, p)
    k = (sigma[:, None] + tau[None, :] - 5 * (slices + 1)).astype(np.int32)
    return np.ldexp(rounded, k)


def gemm(A: np.ndarray, B: np.ndarray, slices: int = DEFAULT_SLICES) -> np.ndarray:
    """Steps 1-5: the emulated FP64 product of A (n x m) and B (m x p)."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    n, m = A.shape
    p = B.shape[1]
    if n == 0 or p == 0 or m == 0:
        return np.zeros((n, p))
    with np.errstate(invalid="ignore"):
        amax = np.max(np.abs(A), axis=1)
        bmax = np.max(np.abs(B), axis=0)
    fin_a = np.isfinite(amax)
    fin_b = np.isfinite(bmax)
    sigma = scales(np.where(fin_a, amax, 0.0))
    tau = scales(np.where(fin_b, bmax, 0.0))
    Ad = digits(np.where(fin_a[:, None], A, 0.0), sigma[:, None], slices)   # [S, n, m]
    Bd = digits(np.where(fin_b[None, :], B, 0.0), tau[None, :], slices)     # [S, m, p]
    C = combine(level_sums(Ad, Bd, slices), sigma, tau, slices)
    C[~fin_a, :] = np.nan
    C[:, ~fin_b] = np.nan
    return C


def error_bound(A: np.ndarray, B: np.ndarray, slices: int) -> np.ndarray:
    """Per-entry bound of |c_emulated - c| from the method (before the final
    rounding to a double): every term a_ir b_rj with both factors non-zero loses
    at most (S + 2) 2^(sigma_i + tau_j - 5S - 1), zero terms nothing.  With
    a' = a 2^-sigma, b' = b 2^-tau (both below 1/2) and a^, b^ their S-digit
    expansions (|a' - a^| < 2^-5S, |b^| <= |b'|), |a'b' - a^b^| < 2^-5S; the
    dropped pairs t + u >= S (at most S - 1 per level, each digit product at
    most 256) add at most 256 (S - 1) 32^-(S+2) 32/31 < (S - 1) 2^-5S / 3.8;
    both together stay below (S + 2) 2^(-5S - 1) for S >= 2."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    sigma = scales(np.max(np.abs(A), axis=1)) if A.size else np.zeros(A.shape[0], np.int64)
    tau = scales(np.max(np.abs(B), axis=0)) if B.size else np.zeros(B.shape[1], np.int64)
    nz = (A != 0).astype(np.float64) @ (B != 0).astype(np.float64)
    return (slices + 2) * np.ldexp(nz, (sigma[:, None] + tau[None, :] - 5 * slices - 1).astype(np.int32))
