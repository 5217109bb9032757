"""bench.py's multi-process path on the CPU: two gloo ranks, the barrier and
the max / sum over ranks that frame the timing (replicas only: no data-path
collective), and the reference arm's rule that only rank 0 works."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RANK_SCRIPT = r"""
import json, os, sys, time
sys.path.insert(0, sys.argv[1])
import bench
rank, world, local = bench.dist_env()
dist = bench.init_dist(world, "gloo")
# ranks report different per-rank times and unit counts
t = 1.0 + rank
bench.barrier(dist)
tmax = bench.max_over_ranks(dist, t)
units = bench.sum_over_ranks(dist, 10.0 * (rank + 1))
bench.barrier(dist)
print(json.dumps({"rank": rank, "world": world, "local": local, "tmax": tmax, "units": units}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_max_and_sum():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", _RANK_SCRIPT, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["world"] == 2 and o["local"] == o["rank"]
        assert o["tmax"] == 2.0  # the slowest rank sets the job time
        assert o["units"] == 30.0  # value = units of all ranks / that time
    assert sorted(o["rank"] for o in outs) == [0, 1]


def test_single_process_helpers_are_identity():
    import bench

    assert bench.init_dist(1, "gloo") is None
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.sum_over_ranks(None, 7.0) == 7.0
    bench.barrier(None)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
