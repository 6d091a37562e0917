"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas, no collective on the data path)
agree on the slowest rank's time, aggregate the whole-job rate from it, and only rank 0 prints
the reference arm's line."""

import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
rank, _, world = bench.dist_info()
dist.init_process_group("gloo")
# rank r took (10 + r) ms for the P-ERK steps and (20 - r) ms for the full method
mx = bench.max_over_ranks([10.0 + rank, 20.0 - rank], world, "cpu")
rate = bench.replica_rate(1000.0, mx[0], world)
print(json.dumps({{"rank": rank, "max": mx, "rate": rate}}), flush=True)
dist.destroy_process_group()
"""


def run_ranks(code, world=2, extra_env=None, args=()):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code, *args], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(out)
    return outs


def test_two_gloo_ranks_take_the_slowest_time():
    outs = run_ranks(WORKER.format(root=ROOT))
    lines = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for ln in lines:
        assert ln["max"] == [11.0, 20.0]                 # max over ranks, element-wise
        assert ln["rate"] == pytest.approx(2 * 1000.0 / 11e-3)


def test_reference_arm_prints_on_rank_zero_only():
    code = ("import sys; sys.path.insert(0, %r); import bench; "
            "sys.argv = ['bench.py', '--impl', 'reference', '--workload', 'vortex', '--steps', '2', '--warmup', '3']; "
            "bench.main()" % ROOT)
    outs = run_ranks(code)
    line = json.loads(outs[0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert outs[1].strip() == ""
