"""The multi-process side of bench.py on CPU (gloo, world size 2, 127.0.0.1): every run here
has one GPU, so N > 1 means independent replicas; what needs checking is the host logic --
the process group, the barrier around the timed region, the max over ranks that the
whole-job throughput divides by, and that the reference arm runs on rank 0 alone."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench
ws, rank, local = bench.dist_env()
dist = bench.init_dist(ws)
bench.barrier(dist)
# each rank reports its own time; the job's time is the slowest rank's
t = bench.max_over_ranks(dist, 10.0 + rank)
bench.barrier(dist)
print(json.dumps({{"rank": rank, "ws": ws, "max": t}}), flush=True)
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def run_ranks(code, ws=2, extra_env=None, timeout=120):
    port = free_port()
    procs = []
    for r in range(ws):
        env = dict(os.environ, WORLD_SIZE=str(ws), RANK=str(r), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), **(extra_env or {}))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    try:
        for p in procs:
            out, err = p.communicate(timeout=timeout)
            outs.append((p.returncode, out, err))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    return outs


def test_replicas_barrier_and_max_over_ranks():
    pytest.importorskip("torch")
    outs = run_ranks(WORKER.format(root=ROOT))
    import json
    for rc, out, err in outs:
        assert rc == 0, err[-2000:]
    res = sorted((json.loads(o.strip().splitlines()[-1]) for _, o, _ in outs), key=lambda d: d["rank"])
    assert [d["rank"] for d in res] == [0, 1]
    assert all(d["ws"] == 2 and d["max"] == 11.0 for d in res)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm (the oracle on the host cores) runs on rank 0; other
    ranks exit 0 at once without printing a line."""
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "3", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
