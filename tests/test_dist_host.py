"""Host logic of the benchmark's multi-rank path on the CPU: two gloo ranks
(127.0.0.1) started the way torchrun starts them (RANK, WORLD_SIZE,
MASTER_ADDR, MASTER_PORT).  Each rank advances its own replica (weak scaling,
no collective on the data path); the only collective is the max of the timed
region, which every rank must receive; the reference arm runs on rank 0 only
and the other ranks exit 0 without work or output."""

import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO"])
import bench
ws, rank, local, dist = bench.dist_setup()
t = bench.max_over_ranks(dist, 1.5 + rank, "cpu")
v = bench.job_throughput(ws, 1000, 10, t)
print(json.dumps({"rank": rank, "ws": ws, "backend": dist.get_backend(), "max": t, "value": v}))
dist.barrier()
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def launch(code_or_args, ws=2, timeout=120):
    port = free_port()
    procs = []
    for r in range(ws):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(ws), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), REPO=ROOT, CUDA_VISIBLE_DEVICES="")
        cmd = [sys.executable, "-c", code_or_args] if isinstance(code_or_args, str) else code_or_args
        procs.append(subprocess.Popen(cmd, cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    out = []
    for p in procs:
        o, e = p.communicate(timeout=timeout)
        out.append((p.returncode, o, e))
    return out


def test_two_ranks_share_the_slowest_time():
    res = launch(WORKER)
    lines = []
    for rc, o, e in res:
        assert rc == 0, e[-2000:]
        lines.append(json.loads(o.strip().splitlines()[-1]))
    assert {d["rank"] for d in lines} == {0, 1}
    for d in lines:
        assert d["ws"] == 2 and d["backend"] == "gloo"
        assert d["max"] == 2.5  # the slower rank's time on both
        assert abs(d["value"] - 2 * 1000 * 10 / 2.5 / 1e6) < 1e-15


def test_reference_arm_runs_on_rank_zero_only():
    """Rank 1 of the reference arm returns before any work: exit 0, no line."""
    res = launch([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
                  "--ref-sample-steps", "1"], ws=2)
    rc1, o1, e1 = res[1]
    assert rc1 == 0 and o1.strip() == "", e1[-2000:]
    rc0, o0, e0 = res[0]
    assert rc0 == 0, e0[-2000:]
    line = json.loads(o0.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["cpu_baseline"]["kind"] == "oracle"
