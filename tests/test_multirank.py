"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own batch
of points (weak scaling, no collective on the data path), timings reduced to
the slowest rank, throughput counting every rank's points."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.env_dist()
        ms = 3.0 + r  # the ranks' step times differ
        slowest = bench.max_over_ranks(ms, dist)
        seed = bench.rank_points_seed(r)
        seeds = [None] * w
        dist.all_gather_object(seeds, seed)
        out[rank] = (r, w, local, slowest, bench.job_throughput(w, 1024, slowest), tuple(seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        r, w, local, slowest, value, seeds = out[rank]
        assert (r, w, local) == (rank, world, rank)
        assert slowest == 4.0                       # max over ranks
        assert value == pytest.approx(2 * 1024 / 4e-3)  # all ranks' points / slowest time
        assert len(set(seeds)) == world             # every rank has its own points


def test_single_rank_defaults():
    import bench

    assert bench.max_over_ranks(5.0, None) == 5.0
    assert bench.job_throughput(1, 1024, 2.0) == pytest.approx(512000.0)
