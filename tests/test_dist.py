"""Replica path of bench.py on CPU: two gloo ranks on 127.0.0.1 run the
same host logic the GPU job runs over NCCL (set-up, barrier, max over
ranks, whole-job aggregate), and the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys, time
sys.path.insert(0, os.environ["ROOT"])
import bench
world, rank, local = bench.dist_setup(None, backend="gloo")
bench.dist_barrier(world)
ms = 100.0 + 50.0 * rank            # rank 1 is the slow replica
m = bench.dist_max(ms, world)
v = bench.aggregate_value(57344, 10, m, world)
bench.dist_barrier(world)
print(json.dumps({"rank": rank, "world": world, "max": m, "value": v}), flush=True)
import torch.distributed as dist
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def launch(code, world=2):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, ROOT=ROOT, WORLD_SIZE=str(world), RANK=str(r), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=240)
        except subprocess.TimeoutExpired:
            p.kill()
            o, e = p.communicate()
        outs.append((p.returncode, o, e))
    return outs


def test_two_gloo_ranks_agree_on_the_slowest_time():
    outs = launch(CHILD)
    lines = []
    for rc, o, e in outs:
        assert rc == 0, e[-2000:]
        lines.append(json.loads([l for l in o.splitlines() if l.startswith("{")][-1]))
    for d in lines:
        assert d["world"] == 2 and d["max"] == 150.0
        # whole job: 2 replicas x 57,344 cells x 10 cycles in the slowest replica's 150 ms
        assert abs(d["value"] - 2 * 57344 * 10 / 0.150) < 1e-6 * d["value"]
    assert sorted(d["rank"] for d in lines) == [0, 1]


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_setup(None) == (1, 0, 0)
    assert bench.dist_max(3.5, 1) == 3.5
    assert bench.aggregate_value(1000, 4, 2.0, 1) == 1000 * 4 / 0.002


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm prints one line from rank 0; the
    other ranks exit 0 at once without work."""
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=240)
    assert r.returncode == 0 and not [l for l in r.stdout.splitlines() if l.startswith("{")], r.stdout


def test_bench_lines_are_strict_json_with_a_diverged_run():
    """A diverged sub-run (NaN residuals, an empty history) still prints a
    line that strict JSON parsers read: non-finite floats become null."""
    sys.path.insert(0, ROOT)
    import bench
    line = {"value": 1.5e9, "supersonic": {"res_first": float("nan"), "history": [float("nan")],
                                            "drop": float("inf"), "n": np.int64(3), "x": np.float64(-np.inf)}}
    text = json.dumps(bench.finite(line), allow_nan=False)

    def refuse(tok):
        raise ValueError(tok)
    d = json.loads(text, parse_constant=refuse)
    assert d["value"] == 1.5e9 and d["supersonic"]["res_first"] is None
    assert d["supersonic"]["history"] == [None] and d["supersonic"]["drop"] is None
    assert d["supersonic"]["n"] == 3 and d["supersonic"]["x"] is None


def test_host_cpu_names_model_and_cores():
    sys.path.insert(0, ROOT)
    import bench
    h = bench.host_cpu()
    assert isinstance(h["cpu_model"], str) and h["cpu_model"]
    assert h["nproc"] == os.cpu_count()
