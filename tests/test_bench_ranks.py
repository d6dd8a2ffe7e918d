"""The multi-rank logic of bench.py, on CPU with two gloo ranks.

Under torchrun every rank runs an independent replica of the workload (the
path has no data exchange: particles are independent once the metric is
known, Sec. 2.1).  What the ranks share is the timing: the slowest rank's time,
an element-wise MAX over ranks, and the whole-job value = units of all ranks /
that time.  Rank 0 alone prints; the CPU reference arm runs on rank 0 only.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as td

    import bench

    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        times = bench.max_over_ranks(td, [10.0 + rank, 5.0 - rank, 7.0], "cpu")
        p = bench.rank_params("c3_3x256", rank)
        q.put((rank, times, p["seed"], p["n_part"], p["n_grid"]))
    finally:
        td.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_distinct_seeds():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        rank, times, seed, n_part, n_grid = q.get(timeout=120)
        got[rank] = (times, seed, n_part, n_grid)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the maximum of every entry
    assert got[0][0] == got[1][0] == [11.0, 5.0, 7.0]
    # replicas: same shapes, different seeds
    assert got[0][1] != got[1][1]
    assert got[0][2:] == got[1][2:]


def test_whole_job_value_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench

    one = bench.whole_job_value(1, 1e9, 2.0)
    assert one == 5e8
    assert bench.whole_job_value(4, 1e9, 2.0) == 4 * one
    assert bench.max_over_ranks(None, [3, 1], "cpu") == [3.0, 1.0]


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
