"""The multi-process path of bench.py on CPU (gloo, world size 2): N GPUs run N
replicas of the workload, the job's time is the slowest rank's, and the rate
counts the units of all ranks."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import os, sys
sys.path.insert(0, %r)
import torch
import bench
torch.distributed.init_process_group("gloo")
ws, rank, local = bench.dist_env()
m = bench.max_over_ranks(1.5 + rank, ws)
v = bench.whole_job_rate(1000.0, ws, m)
print("RESULT", rank, ws, m, v, flush=True)
torch.distributed.destroy_process_group()
""" % ROOT


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_replica_timing_takes_the_slowest_rank():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                   LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", SCRIPT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    results = {}
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-2000:]
        for line in out.splitlines():
            if line.startswith("RESULT"):
                _, rank, ws, m, v = line.split()
                results[int(rank)] = (int(ws), float(m), float(v))
    assert sorted(results) == [0, 1]
    for ws, m, v in results.values():
        assert ws == 2
        assert m == 2.5                      # the slower rank's time
        assert v == pytest.approx(1000.0 * 2 / 2.5)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_on_a_non_zero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
