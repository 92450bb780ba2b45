"""Seeded synthetic inputs for the dense matrix product C = A.B.

This module is shared by the CUDA path's tests/bench and by the CPU oracle.
It holds no arithmetic of the matrix product itself: it only turns a seed into
operand values, index samples and problem shapes.

The paper measures on square 4096x4096 matrices with unspecified values
(Section "Implementacje algorytmow", the 4096x4096 remark before Listing 3;
Table 2).  No dataset is involved, so seeded synthetic matrices stand in for
its inputs.

Generator: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style: draw number
``i`` of stream ``seed`` is the SplitMix64 output mixing function applied to
``seed + (i + 1) * 0x9E3779B97F4A7C15`` (mod 2**64), i.e. the (i+1)-th output
of a SplitMix64 generator started at state ``seed``.  Every value is therefore
addressable by index and identical on any machine.

Value recipes (all exact in the stated type):
  uniform_pm1    x = ((u >> 40) - 2**23) * 2**-23, a 24-bit grid on [-1, 1):
                 every value is exactly representable in float32.
  small_ints     integers in [lo, hi] (u mod (hi - lo + 1) + lo).
  pow2_real      s * 2**e, s = +-1 (bit 63 of a second draw), e uniform real
                 in [emin, emax), rounded once to float32.
  pow2_int       s * 2**k, k integer uniform in [emin, emax]: exact.
  diag_matrix    diag(d) with d = uniform_pm1.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "GAMMA", "splitmix64", "uniform_pm1", "uniform01_f64", "uniform_pm1_f64",
    "small_ints", "pow2_real", "pow2_int", "diag_matrix", "identity",
    "row_scale_exponents", "sample_indices", "freivalds_vector",
    "grouped_dims", "serving_stream",
]

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream separation: a single user seed feeds several independent streams
# (values, signs, exponents ...) by xoring a fixed tag into it.
_TAG_SIGN = 0x5157A9E5C0DE0001
_TAG_EXP = 0x5157A9E5C0DE0002
_TAG_COL = 0x5157A9E5C0DE0003


def _u64(x) -> np.uint64:
    return np.uint64(int(x) & 0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+count-1`` of SplitMix64 stream ``seed`` (uint64)."""
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _u64(seed) + idx * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _count(shape) -> int:
    if isinstance(shape, int):
        return shape
    return int(np.prod(shape, dtype=np.int64))


def uniform_pm1(seed: int, shape) -> np.ndarray:
    """float32 values on the 24-bit grid of [-1, 1) (exact in float32)."""
    u = splitmix64(seed, _count(shape))
    v = (u >> np.uint64(40)).astype(np.int64) - (1 << 23)
    return (v.astype(np.float64) * 2.0 ** -23).astype(np.float32).reshape(shape)


def uniform01_f64(seed: int, count: int) -> np.ndarray:
    """float64 values on the 53-bit grid of [0, 1)."""
    u = splitmix64(seed, count)
    return (u >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def uniform_pm1_f64(seed: int, shape) -> np.ndarray:
    """float64 values on the 53-bit grid of [-1, 1)."""
    u = splitmix64(seed, _count(shape))
    v = (u >> np.uint64(11)).astype(np.int64) - (1 << 52)
    return (v.astype(np.float64) * 2.0 ** -52).reshape(shape)


def small_ints(seed: int, shape, lo: int = -8, hi: int = 8) -> np.ndarray:
    """float32 integers uniform in [lo, hi] (small enough to be exact)."""
    u = splitmix64(seed, _count(shape))
    v = (u % np.uint64(hi - lo + 1)).astype(np.int64) + lo
    return v.astype(np.float32).reshape(shape)


def _signs(seed: int, n: int) -> np.ndarray:
    u = splitmix64(seed ^ _TAG_SIGN, n)
    return np.where((u >> np.uint64(63)) == 1, -1.0, 1.0)


def pow2_real(seed: int, shape, emin: float = -20.0, emax: float = 20.0) -> np.ndarray:
    """s * 2**e, e uniform real in [emin, emax), rounded once to float32."""
    n = _count(shape)
    e = emin + (emax - emin) * uniform01_f64(seed ^ _TAG_EXP, n)
    x = _signs(seed, n) * np.exp2(e)
    return x.astype(np.float32).reshape(shape)


def pow2_int(seed: int, shape, emin: int = -20, emax: int = 20) -> np.ndarray:
    """s * 2**k, k integer uniform in [emin, emax] (exact in float32)."""
    n = _count(shape)
    u = splitmix64(seed ^ _TAG_EXP, n)
    k = (u % np.uint64(emax - emin + 1)).astype(np.int64) + emin
    x = _signs(seed, n) * np.ldexp(1.0, k)
    return x.astype(np.float32).reshape(shape)


def diag_matrix(seed: int, n: int, dtype=np.float32) -> np.ndarray:
    """diag(d) with d drawn by uniform_pm1 (the diagonal case of the paper)."""
    d = uniform_pm1(seed, n)
    out = np.zeros((n, n), dtype=dtype)
    out[np.arange(n), np.arange(n)] = d
    return out


def identity(n: int, dtype=np.float32) -> np.ndarray:
    return np.eye(n, dtype=dtype)


def row_scale_exponents(seed: int, n: int, choices=(-120, 100)) -> np.ndarray:
    """Per-row power-of-two exponents drawn from ``choices`` (wide-range stress)."""
    u = splitmix64(seed ^ _TAG_COL, n)
    pick = (u % np.uint64(len(choices))).astype(np.int64)
    return np.asarray(choices, dtype=np.int64)[pick]


def sample_indices(seed: int, n: int, p: int, count: int):
    """``count`` seeded (i, j) output positions, each uniform over n x p."""
    u = splitmix64(seed, 2 * count)
    i = (u[0::2] % np.uint64(max(n, 1))).astype(np.int64)
    j = (u[1::2] % np.uint64(max(p, 1))).astype(np.int64)
    return i, j


def freivalds_vector(seed: int, p: int) -> np.ndarray:
    """float64 random vector x (53-bit grid on [-1, 1)) for (AB)x = A(Bx)."""
    return uniform_pm1_f64(seed, p)


def grouped_dims(seed: int, count: int, lo: int = 32, hi: int = 1024, step: int = 32):
    """``count`` (n, m, p) triples, each uniform over {lo, lo+step, ..., hi}."""
    k = (hi - lo) // step + 1
    u = splitmix64(seed, 3 * count)
    v = (u % np.uint64(k)).astype(np.int64) * step + lo
    return v.reshape(count, 3)


def serving_stream(seed: int, count: int, rate: float, lo: int = 64, hi: int = 4096,
                   f64_share: float = 0.2):
    """Poisson request stream: arrival times (s), dims log-uniform in [lo, hi]
    (rounded to int) and a per-request FP64 flag with probability f64_share."""
    u = uniform01_f64(seed, 5 * count).reshape(count, 5)
    gaps = -np.log1p(-u[:, 0]) / rate
    t = np.cumsum(gaps)
    llo, lhi = math.log(lo), math.log(hi)
    dims = np.rint(np.exp(llo + (lhi - llo) * u[:, 1:4])).astype(np.int64)
    dims = np.clip(dims, lo, hi)
    f64 = u[:, 4] < f64_share
    return t, dims, f64
