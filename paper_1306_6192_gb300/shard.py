"""Row-block sharding of one product C = A.B over the ranks of a job.

Every entry c_ij of the Cauchy product depends only on row i of A and column j
of B (the paper's definition, Section "Implementacje algorytmow"), so a
product splits across GPUs without any exchange during the computation: rank
r takes the rows [r0, r1) of A and of C, every rank holds all of B, and each
computes its block C[r0:r1] = A[r0:r1] . B with the library on its own GPU.
Only placing B on every rank (a broadcast, or each rank generating or loading
it) and an optional gather of the C blocks cross ranks.  Rows of a row-major
matrix are contiguous, so a rank's blocks of A and C are plain pointer
offsets into the full matrices.

This module is host logic only (the partition and the call on the local
block); the computation itself runs through the C ABI.
"""
from __future__ import annotations

TILE_ROWS = 128  # rows of A per output tile of the tensor-core kernels


def row_blocks(n: int, world: int, align: int = TILE_ROWS) -> list[tuple[int, int]]:
    """Rows [r0, r1) of each of `world` ranks for an n-row product.

    The blocks are disjoint, in rank order and cover [0, n) exactly.  They are
    cut at multiples of `align` (whole output tiles per rank) and balanced to
    within one tile; when n has fewer tiles than there are ranks the last ranks
    get empty blocks.  Every rank gets the same plan from (n, world, align)."""
    if n < 0 or world < 1 or align < 1:
        raise ValueError("row_blocks: n >= 0, world >= 1, align >= 1")
    tiles = (n + align - 1) // align
    base, extra = divmod(tiles, world)
    out, t0 = [], 0
    for r in range(world):
        t1 = t0 + base + (1 if r < extra else 0)
        out.append((min(n, t0 * align), min(n, t1 * align)))
        t0 = t1
    return out


def local_block(n: int, rank: int, world: int, align: int = TILE_ROWS) -> tuple[int, int]:
    """This rank's rows [r0, r1)."""
    return row_blocks(n, world, align)[rank]


def gemm_rows(mm, n, m, p, A, B, C, rank, world, dt=None, mode=None, stream=None):
    """Queues this rank's block C[r0:r1] = A[r0:r1] . B (torch tensors on the
    rank's GPU, row-major and dense; A n x m, B m x p, C n x p) with
    mm_gemm_async and returns (status, r0, r1).  An empty block queues
    nothing."""
    r0, r1 = local_block(n, rank, world)
    dt = mm.MM_F32 if dt is None else dt
    mode = mm.MM_MODE_SPLIT_BF16X3 if mode is None else mode
    if r1 <= r0:
        return mm.MM_OK, r0, r1
    st = mm.mm_gemm_async(r1 - r0, m, p, A[r0:r1], B, C[r0:r1], dt, mode, stream)
    return st, r0, r1
