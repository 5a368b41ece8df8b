"""The N > 1 path of bench.py (replicas only: every rank sorts the same sweep
on its own GPU, no data-path collective) on CPU with two gloo ranks: the
whole-job time is the slowest rank's, the value counts every rank's keys, and
the reference arm runs on rank 0 only."""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import importlib.util
import torch.distributed as dist
spec = importlib.util.spec_from_file_location("bench", os.path.join(os.environ["ROOT"], "bench.py"))
bench = importlib.util.module_from_spec(spec)
spec.loader.exec_module(bench)
dist.init_process_group("gloo")
rank = dist.get_rank()
ms, value = bench.replica_throughput(10.0 + 5.0 * rank, 1_000_000, dist, "cpu")
print(json.dumps({"rank": rank, "ms": ms, "value": value}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    env = dict(os.environ, ROOT=ROOT, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    return env


def test_max_over_ranks_and_whole_job_value():
    pytest.importorskip("torch")
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", WORKER], env=_env(r, 2, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    res = [json.loads(o.strip().splitlines()[-1]) for o, _ in outs]
    for r in res:
        assert r["ms"] == 15.0                               # the slowest rank's time
        assert abs(r["value"] - 2 * 1e6 / 15e-3 / 1e9) < 1e-9  # both ranks' keys over it


def test_single_rank_throughput_without_a_group():
    sys.path.insert(0, ROOT)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    ms, value = bench.replica_throughput(20.0, 3_000_000)
    assert ms == 20.0 and abs(value - 3e6 / 20e-3 / 1e9) < 1e-12


def test_reference_arm_runs_on_rank_zero_only():
    # the other ranks exit 0 without work; rank 0 prints the JSON line
    port = _free_port()
    args = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
            "--steps", "1", "--warmup", "3", "--n", "4096"]
    procs = [subprocess.Popen(args, env=_env(r, 2, port), stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                              text=True, cwd=ROOT) for r in range(2)]
    outs = [p.communicate(timeout=300) for p in procs]
    assert all(p.returncode == 0 for p in procs), [e for _, e in outs]
    assert outs[1][0].strip() == ""
    line = json.loads(outs[0][0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
