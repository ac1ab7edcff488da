"""Shared helpers for the GPU tests: run the CUDA path through the C ABI and
build the oracle's grid from exactly the float32 values the library sees."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2408_09066_gb300 import vsaogm as V


def f32(x) -> float:
    return float(np.float32(x))


def oracle_grid(cfg: V.Config) -> oracle.Grid:
    return oracle.Grid(W=cfg.grid_w, H=cfg.grid_h, res=f32(cfg.resolution), x_min=f32(cfg.x_min),
                       y_min=f32(cfg.y_min), tiles_x=cfg.tiles_x, tiles_y=cfg.tiles_y)


def config_for(wl, **kw) -> V.Config:
    args = dict(D=wl.D, grid_w=wl.W, grid_h=wl.H, resolution=wl.res, x_min=wl.x_min,
                y_min=wl.y_min, tiles_x=wl.tiles_x, tiles_y=wl.tiles_y,
                length_scale=wl.length_scale, seed=wl.seed)
    args.update(kw)
    return V.default_config(**args)


def normwise(got, want) -> float:
    """max |got - want| / max |want| (0 when both vanish)."""
    got = np.asarray(got, np.float64) if not np.iscomplexobj(got) else np.asarray(got)
    want = np.asarray(want)
    den = np.abs(want).max() if want.size else 0.0
    num = np.abs(got - want).max() if want.size else 0.0
    return float(num / den) if den > 0 else float(num)


def run_gpu(cfg: V.Config, xy: np.ndarray, labels: np.ndarray, calls: int = 1):
    """Encode (optionally split into `calls` consecutive calls), then decode,
    query and entropy through the C ABI; returns host copies of everything."""
    import torch
    dev = torch.device("cuda")
    m = V.Map(cfg)
    try:
        n = len(labels)
        bounds = np.linspace(0, n, calls + 1).astype(int)
        txy = torch.from_numpy(np.ascontiguousarray(xy, np.float32)).to(dev)
        tlab = torch.from_numpy(np.ascontiguousarray(labels, np.uint8)).to(dev)
        for a, b in zip(bounds[:-1], bounds[1:]):
            m.encode_bundle(txy[a:b], tlab[a:b])
        H, W = cfg.grid_h, cfg.grid_w
        heat_raw = torch.empty((2, H, W), dtype=torch.float32, device=dev)
        occ_q = torch.empty((H, W), dtype=torch.float32, device=dev)
        m.query(heat_raw, occ_q)
        heat = torch.empty((2, H, W), dtype=torch.float32, device=dev)
        m.decode(heat)
        occ = torch.empty((H, W), dtype=torch.float32, device=dev)
        ogm = torch.empty((H, W), dtype=torch.float32, device=dev)
        cls = torch.empty((H, W), dtype=torch.uint8, device=dev)
        m.entropy(heat, occ, ogm, cls)
        omega = m.get_memory()
        torch.cuda.synchronize()
        m.status()
        nu = m.axis_frequencies()
        out = dict(omega=omega.cpu().numpy(), P=heat_raw.cpu().numpy(), Phat=heat.cpu().numpy(),
                   occ=occ.cpu().numpy(), occ_query=occ_q.cpu().numpy(), ogm=ogm.cpu().numpy(),
                   cls=cls.cpu().numpy(), nu=nu, rejected=m.rejected())
        # NaN / Inf scan of every floating output
        for k in ("omega", "P", "Phat", "occ", "occ_query", "ogm"):
            assert np.all(np.isfinite(out[k])), f"non-finite values in {k}"
    finally:
        m.close()
    return out
