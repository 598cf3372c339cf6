"""bench.py's multi-rank arithmetic on the CPU: two gloo ranks, each with its own
replica; the whole-job value is the units of all ranks over the slowest rank's
time, and only rank 0 prints."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


CHILD = r"""
import os, sys, json
sys.path.insert(0, %r)
import torch.distributed as dist
import bench
rank, local, world = bench.dist_setup()
assert dist.get_backend() == "gloo" and world == 2
units = 1000.0 * (rank + 1)            # rank 0: 1000 updates, rank 1: 2000
secs = 2.0 if rank == 0 else 4.0       # rank 1 is the slowest
value, tmax, total = bench.aggregate(units, secs, world)
bench.barrier(world)
if rank == 0:
    print(json.dumps({"value": value, "tmax": tmax, "total": total}))
dist.destroy_process_group()
"""


def test_two_rank_aggregate_uses_max_time_and_total_units():
    port = _free_port()
    env_base = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2",
                    CUDA_VISIBLE_DEVICES="")
    procs = []
    for r in range(2):
        env = dict(env_base, RANK=str(r), LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD % ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            p.kill()
            pytest.fail("gloo rank timed out")
        assert p.returncode == 0, err
        outs.append(out.strip())
    import json
    rec = json.loads(outs[0])
    assert outs[1] == ""
    assert rec["tmax"] == 4.0 and rec["total"] == 3000.0
    assert rec["value"] == pytest.approx(750.0)


def test_single_rank_aggregate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(100, 4.0, 1) == (25.0, 4.0, 100)
