"""Row-block sharding of one product over ranks, on CPU with gloo: the
partition (disjoint, in order, covering every row, cut at whole output tiles,
balanced, also when n is not a multiple of the ranks or of the tile), and a
sharded product whose blocks, computed by each rank with the CPU oracle
standing in for its GPU and gathered with gloo, equal the oracle's full
product bit for bit (each entry depends on its own row of A only)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1306_6192_gb300 import shard


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("n", [0, 1, 127, 128, 129, 300, 1000, 8192, 8193])
def test_row_blocks_partition(n, world):
    blocks = shard.row_blocks(n, world)
    assert len(blocks) == world
    assert blocks[0][0] == 0 and blocks[-1][1] == n
    for (a0, a1), (b0, b1) in zip(blocks, blocks[1:]):
        assert a1 == b0  # contiguous, disjoint, in rank order
    tiles = []
    for r0, r1 in blocks:
        assert 0 <= r0 <= r1 <= n
        assert r0 % shard.TILE_ROWS == 0 or r0 == n  # whole tiles per rank
        tiles.append((r1 - r0 + shard.TILE_ROWS - 1) // shard.TILE_ROWS)
    assert max(tiles) - min(tiles) <= 1
    assert sum(tiles) == (n + shard.TILE_ROWS - 1) // shard.TILE_ROWS
    for r in range(world):
        assert shard.local_block(n, r, world) == blocks[r]


def test_row_blocks_arguments():
    with pytest.raises(ValueError):
        shard.row_blocks(-1, 2)
    with pytest.raises(ValueError):
        shard.row_blocks(10, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, shape, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    n, m, p = shape
    A = synth.uniform_pm1(71, (n, m))   # every rank can form any row block of A
    B = synth.uniform_pm1(72, (m, p))   # B is replicated
    r0, r1 = shard.local_block(n, rank, world)
    block = oracle.Oracle().gemm(A[r0:r1], B) if r1 > r0 else np.zeros((0, p))
    # gather the blocks (padded to the largest) on every rank
    rows = max(b1 - b0 for b0, b1 in shard.row_blocks(n, world))
    buf = torch.zeros((rows, p), dtype=torch.float64)
    buf[: r1 - r0] = torch.from_numpy(block)
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    if rank == 0:
        C = np.concatenate([parts[r][: b1 - b0].numpy()
                            for r, (b0, b1) in enumerate(shard.row_blocks(n, world))])
        out["C"] = C
        out["ref"] = oracle.Oracle().gemm(A, B)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_product_equals_full(world):
    shape = (300, 70, 50)  # 3 output tiles of rows: uneven over 2 ranks, one each over 3
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, shape, out), nprocs=world, join=True)
    assert out["C"].shape == out["ref"].shape
    assert np.array_equal(out["C"], out["ref"])
