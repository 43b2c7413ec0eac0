"""The multi-rank host logic of bench.py on CPU: two gloo ranks.

`bench.py --gpus N` runs N independent replicas, one per rank (the path
shards by independent problems, so there is no data-path collective): each
rank takes its own Philox seed, the timed region is the slowest rank's, the
whole-job throughput is every rank's particles over that time, and the
reference arm runs on rank 0 only.
"""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg = bench.replica_config({"seed": 7, "nx": 10}, rank)
        t_rank = [0.50, 0.75][rank]          # this rank's timed region (s)
        particles = [1000.0, 1200.0][rank]   # this rank's particle count
        t_max = bench.over_ranks(t_rank, world, "max")
        total = bench.over_ranks(particles, world, "sum")
        value = bench.job_throughput(particles, 10, t_max, world)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"seed": cfg["seed"], "nx": cfg["nx"], "t_max": t_max, "total": total, "value": value}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas_time_and_throughput(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(world)]
    # independent seeded replicas, the rest of the workload unchanged
    assert [x["seed"] for x in r] == [7, 1007] and all(x["nx"] == 10 for x in r)
    # every rank sees the slowest rank's time and the job's particle total
    assert all(x["t_max"] == 0.75 and x["total"] == 2200.0 for x in r)
    assert all(abs(x["value"] - 2200.0 * 10 / 0.75) < 1e-9 for x in r)


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        workload, steps, warmup = "cylinder2d_20m", 1, 0
    bench.run_reference(A())
    assert capsys.readouterr().out == ""


def test_single_rank_helpers_are_identities():
    import bench
    assert bench.over_ranks(3.5, 1, "max") == 3.5
    assert bench.job_throughput(100.0, 4, 2.0, 1) == 200.0
    assert bench.replica_config({"seed": 3}, 0)["seed"] == 3
