"""bench.py on CPU.  The N > 1 path: two gloo ranks, each with its own batch
of points (weak scaling, no collective on the data path), timings reduced to
the slowest rank, throughput counting every rank's points.  The reference arm
(the oracle on the host cores) and its JSON line."""
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
        seed = bench.rank_points_seed(bench.CONFIG_INDEX, r)
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


def test_reference_arm_prints_one_json_line():
    """`bench.py --impl reference` (the oracle on the host cores, no GPU)
    prints one JSON line with the bench contract's keys."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                          "--reference-points", "2"],
                         cwd=root, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "evals/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["points_per_step"] == 2 and "n=128" in d["config"]["workload"]
