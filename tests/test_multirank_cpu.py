"""The N > 1 path of the benchmark on CPU (no GPU): two gloo ranks on 127.0.0.1 run the
benchmark's own rank setup, barrier and max-over-ranks reduction, and the whole-job rate is the
units all ranks processed over the slowest rank's time ("replicas only": no data-path
collective)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import bench
world, rank, local = bench.dist_setup()
bench.barrier(world)
ms = [12.0, 20.0][rank]  # rank 1 is the slowest
ms_max = bench.max_over_ranks(world, ms)
rate = bench.job_rate(1000, 5, world, ms_max)
bench.barrier(world)
import torch.distributed as dist
dist.destroy_process_group()
print(json.dumps({{"rank": rank, "world": world, "ms_max": ms_max, "rate": rate}}))
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_agree_on_the_slowest_time():
    port = free_port()
    code = WORKER.format(root=ROOT)
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["world"] == 2 and o["ms_max"] == 20.0
        # 2 replicas x 1000 points x 3 stages x 5 steps over 20 ms
        assert o["rate"] == pytest.approx(2 * 1000 * 3 * 5 / 0.020)


def test_single_rank_defaults():
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    code = ("import sys; sys.path.insert(0, %r); import bench; "
            "print(bench.dist_setup(), bench.max_over_ranks(1, 3.5))" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "(1, 0, 0) 3.5"
