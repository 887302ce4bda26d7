"""The N > 1 host path of bench.py with two gloo ranks on the CPU: the job
time is the slowest rank's, the throughput counts every replica's units,
and the reference arm does its work on rank 0 only.  (The evaluation does
not shard: each rank runs an independent replica, so there is no data-path
collective to test.)"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, results):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = [0.25, 0.4][rank]
        t_max = bench.max_over_ranks(mine, True, "cpu")
        dist.barrier()
        results[rank] = (t_max, bench.job_throughput(world, 1000, t_max))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    port = free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_rank, args=(2, port, results), nprocs=2, join=True)
        res = dict(results)
    assert res[0] == res[1] == (0.4, 2 * 1000 / 0.4)


def test_single_rank_is_its_own_max():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.125, False, "cpu") == 0.125
    assert bench.job_throughput(1, 48, 0.5) == 96.0


@pytest.mark.parametrize("rank,expect_line", [("0", True), ("1", False)])
def test_reference_arm_runs_on_rank_zero_only(rank, expect_line):
    env = dict(os.environ, RANK=rank, WORLD_SIZE="2", LOCAL_RANK=rank)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--cpu-seconds", "0.5"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    if expect_line:
        assert len(lines) == 1
        rec = json.loads(lines[0])
        assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
        assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["cpu_baseline"]["kind"] == "oracle"
    else:
        assert lines == []


def test_oracle_pool_runs_one_process_per_core():
    """The batched CPU baseline spreads the oracle over one spawned process per host core,
    each on its own share of the instances, and counts every process's instances."""
    sys.path.insert(0, ROOT)
    import bench
    for kind, n in (("contingency", 2304), ("mixed", 4096)):
        rate, m, el, cores = bench.oracle_pool(kind, n, 0.3)
        assert cores == len(os.sched_getaffinity(0))
        assert m >= cores and el >= 0.3 and rate == pytest.approx(m / el)
