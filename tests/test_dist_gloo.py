"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): every
rank does its own work, the job time is the max over ranks and the job rate
counts the units of all ranks (weak scaling, no data collective)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 * (rank + 1)              # rank 1 is the slow one
    mx = bench.max_over_ranks(ms, dist, "cpu")
    rate = bench.whole_job_rate(2.0e12, world, mx)
    out[rank] = (mx, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1]
    mx, rate = out[0]
    assert mx == 20.0
    assert rate == pytest.approx(2 * 2.0e12 / 0.020)


def test_single_rank_identity():
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.whole_job_rate(1.0e12, 1, 1000.0) == pytest.approx(1.0e12)
