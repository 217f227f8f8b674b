"""The N > 1 path of bench.py on CPU: two gloo ranks (world_size 2).  Every
rank runs its own replica (the path shards with no data-path collective); the
only collectives are the barrier and the max over ranks of the timed region,
and the whole-job rate counts every rank's units over the slowest rank's time.
"""

import os
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [1.5, 2.0][rank]  # the second rank is the slower one
    dist.barrier()
    m = bench.max_over_ranks(elapsed, dist, "cpu")
    rate = bench.whole_job_rate(500_000, 3, world, m)
    out[rank] = (m, rate)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_count_all_units():
    port = 29500 + os.getpid() % 1000
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == (2.0, 500_000 * 3 * 2 / 2.0)


def test_reference_arm_non_zero_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
