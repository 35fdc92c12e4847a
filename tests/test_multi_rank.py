"""Multi-process path of the benchmark (replicas, no data-path collective) with the gloo
backend on CPU, world_size 2: the whole-job rate uses the slowest rank's time."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [800.0, 1000.0][rank]            # rank 1 is the slow replica
    m = bench.max_over_ranks(local_ms)
    out[rank] = (m, bench.whole_job_rate(world, 8, 10, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_max_and_rate():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        m, rate = res[rank]
        assert m == 1000.0
        assert rate == pytest.approx(2 * 8 * 10 / 1.0)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(123.0) == 123.0
    assert bench.whole_job_rate(1, 8, 10, 500.0) == pytest.approx(160.0)
