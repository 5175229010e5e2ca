"""The benchmark's multi-GPU mode runs independent replicas (one lattice per
GPU, no collective on the data path); its only cross-rank steps are the
barrier and the max-over-ranks timing.  Those are exercised here with two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    slowest = bench.max_over_ranks(1.0 + rank, world)          # rank 1 is the slow one
    rate = bench.whole_job_rate(100.0, 1.0 + rank, world)      # 2 ranks x 100 units / 2 s
    out[rank] = (slowest, rate)
    dist.destroy_process_group()


def test_two_rank_max_and_whole_job_rate():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        assert out[0] == out[1] == (2.0, 100.0)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10.0, 2.0, 1) == pytest.approx(5.0)
