"""The multi-rank path of bench.py (replicas, one process per GPU) on CPU:
two gloo ranks agree on the slowest rank's time and on the whole-job
throughput, and a rank other than 0 prints nothing in the reference arm."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = 10.0 + 5.0 * rank  # rank 1 is slower
    ms = bench.max_over_ranks(mine, dist, "cpu")
    value = bench.job_throughput(1_000_000, world, ms)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"ms": ms, "value": value}, f)


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    assert res[0] == res[1]
    assert res[0]["ms"] == 15.0
    # two replicas of 1M triangles in 15 ms
    assert abs(res[0]["value"] - 2 * 1e6 / 15e-3 / 1e6) < 1e-9


def test_single_rank_helpers_are_identities():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(2e6, 1, 2.0) == pytest.approx(1000.0)


def test_reference_arm_prints_only_on_rank_0():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "3", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
