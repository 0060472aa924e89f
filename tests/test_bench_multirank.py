"""CPU: the benchmark's N>1 host logic (replicas only, one process per GPU) with two gloo
ranks: the job's time is the slowest rank's, the rate aggregates every rank's bytes, and a
branch every rank must take together (the end-to-end run, which needs host memory for all
replicas) is taken only when every rank agrees."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(1.5 + rank, dist, device="cpu")     # rank 1 is the slow one
    rate = bench.whole_job_rate(3.0e9, world, ms)
    agree_one = bench.all_ranks_agree(rank == 0, dist)      # only rank 0 says yes
    agree_all = bench.all_ranks_agree(True, dist)
    out[rank] = (ms, rate, agree_one, agree_all)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_time_is_max_and_rate_aggregates():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, rate, agree_one, agree_all = out[r]
        assert ms == 2.5
        assert agree_one is False and agree_all is True
        assert abs(rate - 3.0e9 * 2 / 2.5e-3 / 1e9) < 1e-6


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(1.25) == 1.25
    assert abs(bench.whole_job_rate(1e9, 1, 1.0) - 1000.0) < 1e-9
    assert bench.all_ranks_agree(True) and not bench.all_ranks_agree(False)
    assert bench.host_mem_available() >= 0
