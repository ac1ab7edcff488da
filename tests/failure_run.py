"""Runs the bounded-wait failure test in its own process.  With the
environment variable VSAOGM_DEBUG_WAIT_NS set when a map is created, the
tensor-core decode's pipeline waits give up after that many nanoseconds and
its loader warp first stalls on a barrier that nothing arrives at for four
times as long, so the waits run out: the call must report E_TIMEOUT through
vsaogm_status, drain its MMAs and free its tensor memory.  A fresh map created
with the variable unset must then decode normally and match the oracle (the
context stays usable).  Prints one JSON line.  Used by test_gpu_failures.py."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from helpers import config_for, normwise, oracle_grid  # noqa: E402
from paper_2408_09066_gb300 import build, synth  # noqa: E402
from paper_2408_09066_gb300 import vsaogm as V  # noqa: E402


def status(m):
    try:
        m.status()
        return "ok"
    except V.VsaogmError as e:
        return {V.E_TIMEOUT: "E_TIMEOUT"}.get(e.code, str(e))


def query(m, wl, dev):
    m.encode_bundle(torch.from_numpy(wl.xy).to(dev), torch.from_numpy(wl.labels).to(dev))
    heat = torch.empty((2, wl.H, wl.W), dtype=torch.float32, device=dev)
    occ = torch.empty((wl.H, wl.W), dtype=torch.float32, device=dev)
    m.query(heat, occ)
    torch.cuda.synchronize()
    return heat, occ


def main():
    build.build()
    dev = torch.device("cuda")
    wl = synth.small_scan(D=8192)
    cfg = config_for(wl, decode_prec=V.DECODE_BF16X3)
    out = {}
    os.environ["VSAOGM_DEBUG_WAIT_NS"] = "200000"  # 200 us
    with V.Map(cfg) as m:
        query(m, wl, dev)
        out["single_map"] = status(m)
        # the batched decode kernel takes the same limit from each map
        with V.Batch([m]) as b:
            xy = torch.from_numpy(wl.xy).to(dev)
            lab = torch.from_numpy(wl.labels).to(dev)
            heat = torch.empty((2, wl.H, wl.W), dtype=torch.float32, device=dev)
            occ = torch.empty((wl.H, wl.W), dtype=torch.float32, device=dev)
            b.step([xy], [lab], [heat], [occ])
            torch.cuda.synchronize()
            out["batch"] = status(m)
    del os.environ["VSAOGM_DEBUG_WAIT_NS"]
    with V.Map(cfg) as m:
        heat, occ = query(m, wl, dev)
        out["fresh_map"] = status(m)
        g = oracle_grid(cfg)
        nx, ny = oracle.draw_nu(cfg.seed, cfg.D, float(np.float32(cfg.length_scale)))
        ref = oracle.pipeline(g, nx, ny, wl.xy, wl.labels, cfg.r_occ, cfg.r_emp, cfg.rho, "tile")
        out["fresh_P"] = normwise(heat.cpu().numpy(), ref["P"])
        out["fresh_pr1"] = float(np.abs(occ.cpu().numpy() - ref["pr1"]).max())
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
