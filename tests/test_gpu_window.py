"""Local map queries (vsaogm_query_window) against the oracle's window query,
for the FP32 and the tensor-core decodes: corner, edge, interior and whole-map
windows, several radii."""
import numpy as np
import pytest

import oracle
from helpers import config_for, oracle_grid
from paper_2408_09066_gb300 import synth
from paper_2408_09066_gb300 import vsaogm as V

pytestmark = pytest.mark.gpu

TOL_PR = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2408_09066_gb300 import build
    build.build()


WINDOWS = [(0, 0, 20, 17), (40, 3, 24, 30), (10, 12, 33, 40), (0, 0, 64, 64), (63, 63, 1, 1)]


@pytest.mark.parametrize("prec", [V.DECODE_FP32, V.DECODE_BF16X3])
@pytest.mark.parametrize("radii", [(3, 3), (1, 5)])
def test_window_queries_match_oracle(prec, radii):
    import torch
    wl = synth.small_scan(seed=77)
    cfg = config_for(wl, tiles_x=2, tiles_y=2, r_occ=radii[0], r_emp=radii[1], decode_prec=prec)
    dev = torch.device("cuda")
    g = oracle_grid(cfg)
    nx, ny = oracle.draw_nu(cfg.seed, cfg.D, float(np.float32(cfg.length_scale)))
    om = oracle.memories(g, nx, ny, wl.xy, wl.labels, "tile")
    with V.Map(cfg) as m:
        m.encode_bundle(torch.from_numpy(wl.xy).to(dev), torch.from_numpy(wl.labels).to(dev))
        for (x0, y0, w, h) in WINDOWS:
            heat = torch.empty(m.window_scratch(x0, y0, w, h), dtype=torch.float32, device=dev)
            occ = torch.empty((h, w), dtype=torch.float32, device=dev)
            ogm = torch.empty((h, w), dtype=torch.float32, device=dev)
            cls = torch.empty((h, w), dtype=torch.uint8, device=dev)
            m.query_window(x0, y0, w, h, heat, occ, ogm, cls)
            torch.cuda.synchronize()
            m.status()
            want = oracle.query_window(g, nx, ny, om, x0, y0, w, h, cfg.r_occ, cfg.r_emp)
            P = heat[:want["P"].size].cpu().numpy().reshape(want["P"].shape)
            perr = np.abs(P - want["P"]).max() / np.abs(want["P"]).max()
            assert perr <= 1e-4, (x0, y0, w, h, perr, P.reshape(2, -1).max(1), want["maxima"])
            assert np.abs(occ.cpu().numpy() - want["pr1"]).max() <= TOL_PR, (x0, y0, w, h)
            assert np.abs(ogm.cpu().numpy() - want["ogm"]).max() <= 2 * TOL_PR
            assert np.array_equal(cls.cpu().numpy(),
                                  oracle.classify_f32(ogm.cpu().numpy(), cfg.rho))


def test_whole_map_window_equals_map_query():
    import torch
    wl = synth.small_scan(seed=78)
    cfg = config_for(wl, tiles_x=2, tiles_y=2)
    dev = torch.device("cuda")
    with V.Map(cfg) as m:
        m.encode_bundle(torch.from_numpy(wl.xy).to(dev), torch.from_numpy(wl.labels).to(dev))
        heat = torch.empty((2, wl.H, wl.W), dtype=torch.float32, device=dev)
        occ = torch.empty((wl.H, wl.W), dtype=torch.float32, device=dev)
        m.query(heat, occ)
        heat2 = torch.empty(m.window_scratch(0, 0, wl.W, wl.H), dtype=torch.float32, device=dev)
        occ2 = torch.empty((wl.H, wl.W), dtype=torch.float32, device=dev)
        m.query_window(0, 0, wl.W, wl.H, heat2, occ2)
        torch.cuda.synchronize()
        assert torch.equal(occ, occ2)


def test_window_outside_the_map_is_rejected():
    wl = synth.small_scan(seed=79)
    with V.Map(config_for(wl)) as m:
        for bad in [(-1, 0, 4, 4), (0, 0, 65, 4), (60, 60, 5, 1), (0, 0, 0, 3)]:
            with pytest.raises(V.VsaogmError) as ei:
                m.window_scratch(*bad)
            assert ei.value.code == V.E_INVAL


@pytest.mark.parametrize("prec", [V.DECODE_FP32, V.DECODE_BF16X3])
def test_map_max_windows_equal_the_map_query(prec):
    """With VSAOGM_FLAG_WINDOW_MAP_MAX a window query normalises by the whole
    map's maxima (Eq. non-linearities, Fig. 2E): its outputs are those of the
    same cells of the map query and match the oracle's whole-map pipeline
    there; after more points are bundled the next window query decodes the map
    again.  The window's P is the map query's P bit for bit; its entropy sums
    the same disks, but as differences of running sums that start at the
    window's own blocks, so Pr differs from the map query's only by float
    rounding (held to 1e-5)."""
    import torch
    wl = synth.small_scan(seed=80)
    more = synth.small_scan(seed=81)
    cfg = config_for(wl, tiles_x=2, tiles_y=2, decode_prec=prec, flags=V.FLAG_WINDOW_MAP_MAX)
    dev = torch.device("cuda")
    g = oracle_grid(cfg)
    nx, ny = oracle.draw_nu(cfg.seed, cfg.D, float(np.float32(cfg.length_scale)))
    with V.Map(cfg) as m, V.Map(config_for(wl, tiles_x=2, tiles_y=2, decode_prec=prec)) as full:
        pts = []
        for w in (wl, more):
            xy, lab = torch.from_numpy(w.xy).to(dev), torch.from_numpy(w.labels).to(dev)
            m.encode_bundle(xy, lab)
            full.encode_bundle(xy, lab)
            pts.append(w)
            heat = torch.empty((2, wl.H, wl.W), dtype=torch.float32, device=dev)
            occ = torch.empty((wl.H, wl.W), dtype=torch.float32, device=dev)
            ogm = torch.empty((wl.H, wl.W), dtype=torch.float32, device=dev)
            full.query(heat, occ, ogm)
            ref = oracle.pipeline(g, nx, ny, np.concatenate([p.xy for p in pts]),
                                  np.concatenate([p.labels for p in pts]), cfg.r_occ,
                                  cfg.r_emp, cfg.rho)
            for (x0, y0, ww, hh) in WINDOWS:
                wheat = torch.empty(m.window_scratch(x0, y0, ww, hh), dtype=torch.float32,
                                    device=dev)
                wocc = torch.empty((hh, ww), dtype=torch.float32, device=dev)
                wogm = torch.empty((hh, ww), dtype=torch.float32, device=dev)
                m.query_window(x0, y0, ww, hh, wheat, wocc, wogm)
                torch.cuda.synchronize()
                m.status()
                sl = (slice(y0, y0 + hh), slice(x0, x0 + ww))
                assert (wocc - occ[sl]).abs().max().item() <= 1e-5, (x0, y0, ww, hh)
                assert (wogm - ogm[sl]).abs().max().item() <= 2e-5
                assert np.abs(wocc.cpu().numpy() - ref["pr1"][sl]).max() <= TOL_PR
                # heat receives P of the window's region, as in the local mode
                R = max(cfg.r_occ, cfg.r_emp)
                rx0, ry0 = max(0, x0 - R), max(0, y0 - R)
                rx1, ry1 = min(wl.W, x0 + ww + R), min(wl.H, y0 + hh + R)
                P = wheat[:2 * (rx1 - rx0) * (ry1 - ry0)].view(2, ry1 - ry0, rx1 - rx0)
                assert torch.equal(P, heat[:, ry0:ry1, rx0:rx1])


@pytest.mark.parametrize("prec", [V.DECODE_FP32, V.DECODE_BF16X3])
def test_decode_windows_match_oracle(prec):
    """vsaogm_decode_window: P_hat of a window (Eqs. vector-normalization,
    loc-query, non-linearities) normalised by the window's own per-class
    maxima, against the oracle's decode of the same cells put through its
    non-linearity; the whole map's window equals vsaogm_decode."""
    import torch
    wl = synth.small_scan(seed=82)
    cfg = config_for(wl, tiles_x=2, tiles_y=2, decode_prec=prec)
    dev = torch.device("cuda")
    g = oracle_grid(cfg)
    nx, ny = oracle.draw_nu(cfg.seed, cfg.D, float(np.float32(cfg.length_scale)))
    om = oracle.memories(g, nx, ny, wl.xy, wl.labels, "tile")
    with V.Map(cfg) as m:
        m.encode_bundle(torch.from_numpy(wl.xy).to(dev), torch.from_numpy(wl.labels).to(dev))
        for (x0, y0, w, h) in WINDOWS:
            heat = torch.empty((2, h, w), dtype=torch.float32, device=dev)
            m.decode_window(x0, y0, w, h, heat)
            torch.cuda.synchronize()
            m.status()
            jj, ii = np.meshgrid(np.arange(y0, y0 + h), np.arange(x0, x0 + w), indexing="ij")
            cells = np.stack([ii.ravel(), jj.ravel()], 1)
            P = oracle.decode_cells(g, nx, ny, om, cells, "tile").T.reshape(2, h, w)
            want, _ = oracle.nonlinear(P)
            err = np.abs(heat.cpu().numpy() - want).max()
            assert err <= 2e-4, (x0, y0, w, h, err)
        full = torch.empty((2, wl.H, wl.W), dtype=torch.float32, device=dev)
        m.decode(full)
        whole = torch.empty((2, wl.H, wl.W), dtype=torch.float32, device=dev)
        m.decode_window(0, 0, wl.W, wl.H, whole)
        torch.cuda.synchronize()
        assert torch.equal(full, whole)


@pytest.mark.parametrize("prec", [V.DECODE_FP32, V.DECODE_BF16X3])
def test_map_max_decode_windows_equal_the_map_decode(prec):
    """With VSAOGM_FLAG_WINDOW_MAP_MAX a decoded window is normalised by the
    whole map's maxima: bit for bit the same cells of vsaogm_decode, and after
    more points are bundled the next window decodes the map again."""
    import torch
    wl = synth.small_scan(seed=83)
    more = synth.small_scan(seed=84)
    cfg = config_for(wl, tiles_x=2, tiles_y=2, decode_prec=prec, flags=V.FLAG_WINDOW_MAP_MAX)
    dev = torch.device("cuda")
    with V.Map(cfg) as m:
        for w in (wl, more):
            m.encode_bundle(torch.from_numpy(w.xy).to(dev), torch.from_numpy(w.labels).to(dev))
            full = torch.empty((2, wl.H, wl.W), dtype=torch.float32, device=dev)
            m.decode(full)
            for (x0, y0, ww, hh) in WINDOWS:
                heat = torch.empty((2, hh, ww), dtype=torch.float32, device=dev)
                m.decode_window(x0, y0, ww, hh, heat)
                torch.cuda.synchronize()
                m.status()
                assert torch.equal(heat, full[:, y0:y0 + hh, x0:x0 + ww]), (x0, y0, ww, hh)


def test_decode_window_outside_the_map_is_rejected():
    import torch
    wl = synth.small_scan(seed=85)
    dev = torch.device("cuda")
    with V.Map(config_for(wl)) as m:
        heat = torch.empty((2, 4, 4), dtype=torch.float32, device=dev)
        for bad in [(-1, 0, 4, 4), (62, 0, 4, 4), (0, 61, 4, 4)]:
            with pytest.raises(V.VsaogmError) as ei:
                m.decode_window(*bad, heat)
            assert ei.value.code == V.E_INVAL
