"""Runs the hot path on the bounds-checked build (-DVSAOGM_CHECK) in its own
process: single maps of several shapes and precisions, a window query, a
captured and replayed batch, wide tiles with bundling patches and points far
outside the map.  Prints one JSON line with every status and the parity of
the small scan against the oracle.  Used by test_gpu_checked_build.py."""
import json
import os
import sys

os.environ["VSAOGM_CHECKED"] = "1"
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
        return str(e)


def main():
    build.build(checked=True)
    assert V.LIB_PATH.endswith("libvsaogm_checked.so")
    dev = torch.device("cuda")
    out = {"statuses": {}}
    wl = synth.small_scan()
    far = np.array([[-100.0, 50.0], [30.0, -2.0]], np.float32)
    xy = np.concatenate([wl.xy, far])
    lab = np.concatenate([wl.labels, np.array([0, 1], np.uint8)])
    for name, prec in (("fp32", V.DECODE_FP32), ("bf16", V.DECODE_BF16X3),
                       ("fp8", V.DECODE_FP8X3)):
        cfg = config_for(wl, decode_prec=prec)
        with V.Map(cfg) as m:
            m.encode_bundle(torch.from_numpy(xy).to(dev), torch.from_numpy(lab).to(dev))
            heat = torch.empty((2, wl.H, wl.W), device=dev)
            occ = torch.empty((wl.H, wl.W), device=dev)
            m.query(heat, occ)
            torch.cuda.synchronize()
            out["statuses"][name] = status(m)
            if name == "fp32":
                g = oracle_grid(cfg)
                nx, ny = oracle.draw_nu(cfg.seed, cfg.D, float(np.float32(cfg.length_scale)))
                ref = oracle.pipeline(g, nx, ny, xy, lab, cfg.r_occ, cfg.r_emp, cfg.rho, "tile")
                out["small_P"] = normwise(heat.cpu().numpy(), ref["P"])
                out["small_pr1"] = float(np.abs(occ.cpu().numpy() - ref["pr1"]).max())
    # a paper-shaped map with one wide tile (bundling patches), a window query
    tr = synth.paper_trajectory(n_scans=4, D=2048)
    cfg = V.default_config(D=2048, grid_w=400, grid_h=400, resolution=0.1, x_min=-20.0,
                           y_min=-20.0, tiles_x=1, tiles_y=1, decode_prec=V.DECODE_BF16X3)
    with V.Map(cfg) as m:
        m.encode_bundle(torch.from_numpy(tr.xy).to(dev), torch.from_numpy(tr.labels).to(dev))
        n = m.window_scratch(100, 120, 150, 130)
        heat = torch.empty(n, device=dev)
        occ = torch.empty((130, 150), device=dev)
        m.query_window(100, 120, 150, 130, heat, occ)
        torch.cuda.synchronize()
        out["statuses"]["wide_tile_window"] = status(m)
    # a batch of uneven maps, stepped, captured and replayed
    wls = synth.batch_maps(n_maps=5, seed=41, min_cells=40, max_cells=300, min_points=2000,
                           max_points=40000, dims=(1000, 2048, 4096))
    maps = [V.Map(config_for(w, decode_prec=V.DECODE_BF16X3)) for w in wls]
    xs = [torch.from_numpy(w.xy).to(dev) for w in wls]
    ls = [torch.from_numpy(w.labels).to(dev) for w in wls]
    hs = [torch.empty((2, w.H, w.W), device=dev) for w in wls]
    os_ = [torch.empty((w.H, w.W), device=dev) for w in wls]
    s = torch.cuda.Stream()
    with V.Batch(maps) as b:
        b.step(xs, ls, hs, os_, stream=s)
        b.capture(xs, ls, hs, os_, stream=s)
        b.replay(stream=s)
        s.synchronize()
        out["statuses"]["batch"] = [status(m) for m in maps]
    for m in maps:
        m.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
