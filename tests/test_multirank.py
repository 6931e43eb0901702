"""The multi-rank path of bench.py on CPU (gloo, world size 2).

With N GPUs every rank solves its own problem (replicas: the solve has no
exchange step), times it between barriers, and the job's time is the slowest
rank's; rank 0 alone prints.  Here the ranks are CPU processes on gloo with
made-up per-rank times, and the reference arm is run as rank 1 (no output,
exit 0) and rank 0 (one JSON line) on the small 64 x 128 workload."""

import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    r, w, local = bench.init_ranks("gloo")
    ms = bench.max_over_ranks(10.0 + 5.0 * r, w, "cpu")       # rank 1 is the slow one
    value = bench.whole_job_value(1000, w, ms)
    dist.barrier()
    dist.destroy_process_group()
    out[r] = (r, w, local, ms, value)


def test_max_over_ranks_and_whole_job_value_on_gloo():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        r, w, local, ms, value = out[rank]
        assert (r, w, local) == (rank, world, rank)
        assert ms == 15.0                                         # the slowest rank's time
        assert value == pytest.approx(1000 * world / 15e-3)


def test_reference_arm_prints_on_rank_zero_only():
    base = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "sh20_64x128",
            "--steps", "2", "--warmup", "3"]
    env = dict(os.environ, WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    r1 = subprocess.run(base, env=dict(env, RANK="1", LOCAL_RANK="1"), capture_output=True, text=True, timeout=600)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = subprocess.run(base, env=dict(env, RANK="0", LOCAL_RANK="0"), capture_output=True, text=True, timeout=600)
    assert r0.returncode == 0
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "DOF/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
