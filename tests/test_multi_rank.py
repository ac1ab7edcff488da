"""Multi-rank paths on CPU, as two gloo ranks.

The benchmark runs one independent map replica per rank (no data-path
collective); only the timing reduction crosses ranks.  Checks that throughput
is total units over the slowest rank's time, and that the reference arm runs on
rank 0 alone.  The method's one exchange step, Algorithm 3 fusion, is checked
as a sum all-reduce of two agents' memories."""
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


FUSION_WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import numpy as np, torch, torch.distributed as dist
import oracle
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
g = oracle.Grid(W=32, H=24, res=0.125, x_min=-2.0, y_min=-1.5, tiles_x=2, tiles_y=2)
nx, ny = oracle.draw_nu(3, 128, 0.2)
rng = np.random.default_rng(0)                      # every rank draws the same scans
xy = rng.uniform([-2.2, -1.7], [2.2, 1.7], (90, 2)).astype(np.float32)
lab = rng.integers(0, 2, 90).astype(np.uint8)
part = slice(rank * 90 // world, (rank + 1) * 90 // world)   # each agent sees its share
mine = oracle.memories(g, nx, ny, xy[part], lab[part], "tile")
t = torch.from_numpy(np.ascontiguousarray(np.stack([mine.real, mine.imag], -1)))
dist.all_reduce(t, op=dist.ReduceOp.SUM)            # Algorithm 3: fusion is a sum
fused = t[..., 0].numpy() + 1j * t[..., 1].numpy()
union = oracle.memories(g, nx, ny, xy, lab, "tile")
err = float(np.abs(fused - union).max())
P_f = oracle.decode_map(g, nx, ny, fused, "tile")
P_u = oracle.decode_map(g, nx, ny, union, "tile")
print(json.dumps({{"rank": rank, "err": err, "perr": float(np.abs(P_f - P_u).max()),
                   "local_differs": bool(np.abs(mine - union).max() > 1e-6)}}))
dist.destroy_process_group()
"""


def test_fusion_across_two_gloo_ranks_is_a_sum_all_reduce():
    """Algorithm 3 across ranks: two agents bundle their own shares of the points;
    a sum all-reduce of the memories (the path's one exchange step) gives every
    rank the memories, and hence the map, of the union."""
    outs = _spawn(FUSION_WORKER.format(root=ROOT), 2, _free_port())
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert sorted(r["rank"] for r in res) == [0, 1]
    for r in res:
        assert r["err"] < 1e-10 and r["perr"] < 1e-10
        assert r["local_differs"]
