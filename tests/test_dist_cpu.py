"""The multi-rank host logic of the benchmark on CPU: two gloo ranks, each
timing its own independent tile (weak scaling, no data exchange); the job's
time is the slowest rank's and its work the sum over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank          # rank 1 is the slower one
    units = 1000.0 * (rank + 1)     # different work per rank
    out[rank] = (bench._max_over_ranks(ms, dist, "cpu"), bench._sum_over_ranks(units, dist, "cpu"))
    dist.barrier()
    dist.destroy_process_group()


def test_max_and_sum_over_two_gloo_ranks():
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
        assert out[0] == out[1] == (15.0, 3000.0)


def test_single_rank_is_identity():
    import bench
    assert bench._max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench._sum_over_ranks(7.0, None, "cpu") == 7.0
