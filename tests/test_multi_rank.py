"""The N > 1 benchmark path on CPU: two gloo ranks, one independent map replica
each (no data-path collective); only the timing reduction crosses ranks.
Checks that throughput is total units over the slowest rank's time, and that
the reference arm runs on rank 0 alone."""
import json
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
d = bench.Dist("gloo")
# rank r processed (r + 1) * 1000 units in (r + 1) * 0.5 s
units = d.sum(float((d.rank + 1) * 1000))
slowest = d.max((d.rank + 1) * 0.5)
d.barrier()
print(json.dumps({{"rank": d.rank, "world": d.world, "units": units, "slowest": slowest}}))
d.close()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _spawn(code, world, port, extra_env=None):
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_two_gloo_ranks_reduce_timing_like_the_benchmark():
    outs = _spawn(WORKER.format(root=ROOT), 2, _free_port())
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for r in res:
        assert r["world"] == 2
        assert r["units"] == 3000.0      # weak scaling: all ranks' units
        assert r["slowest"] == 1.0       # the slowest rank's time
    assert sorted(r["rank"] for r in res) == [0, 1]


def test_reference_arm_runs_on_rank_zero_only():
    """Under a multi-rank launch every rank but 0 exits 0 without work."""
    code = ("import sys; sys.path.insert(0, %r); import bench, types; "
            "a = types.SimpleNamespace(gpus=2, steps=1, warmup=0); "
            "sys.exit(bench.run_reference(a) if __import__('os').environ['RANK'] != '0' else 0)"
            % ROOT)
    outs = _spawn(code, 2, _free_port())
    assert outs[1].strip() == ""
