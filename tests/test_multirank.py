"""The multi-rank path of bench.py on CPU (gloo, world size 2).

With N GPUs every rank solves its own problem (replicas: the solve has no
exchange step), times it between barriers, and the job's time is the slowest
rank's; rank 0 alone prints.  Here the ranks are CPU processes on gloo with
made-up per-rank times, and the reference arm is run as rank 1 (no output,
exit 0) and rank 0 (one JSON line) on the small 64 x 128 workload.  The batched
form is sharded, not replicated: each rank computes the same longest-processing-
time split of the 4096 uneven problems by itself and solves its own part."""

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


def _shard_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from synth import sh

    r, w, _ = bench.init_ranks("gloo")
    sizes, _ = sh.batched_sizes(4096)
    mine = bench.shard_lpt(sizes, w)[r]             # computed locally, no exchange
    gathered = [None] * w
    dist.all_gather_object(gathered, mine)          # only the test compares the ranks' parts
    dist.barrier()
    dist.destroy_process_group()
    out[r] = (mine, gathered, sizes)


@pytest.mark.parametrize("world", [2])
def test_batched_problems_are_sharded_by_lpt(world):
    out = mp.Manager().dict()
    mp.spawn(_shard_main, args=(world, _free_port(), out), nprocs=world, join=True)
    mine0, gathered, sizes = out[0]
    # every rank derived the same split on its own
    for r in range(world):
        assert out[r][1] == gathered and out[r][0] == gathered[r]
    # every problem exactly once
    flat = sorted(b for part in gathered for b in part)
    assert flat == list(range(len(sizes)))
    # balanced to within the largest problem, as the LPT rule guarantees
    loads = [sum(sizes[b][0] * sizes[b][1] for b in part) for part in gathered]
    largest = max(a * b for a, b in sizes)
    assert max(loads) - min(loads) <= largest
    assert len(gathered[0]) > 1000 and len(gathered[1]) > 1000
