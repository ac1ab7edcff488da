"""Element-by-element parity with the FP64 oracle at full size: the 400 x 400
cell, 4 x 4 tile, D = 8192 map of 2.268M points (in the launch configuration
the benchmark times: one map, encode + bundle, then the fused query), every
map of the 64-map batch (autotuned, captured and replayed as the benchmark
steps it), multi-map fusion (Algorithm 3) and the paper-shaped workloads
(ToySim-, Intel- and EviLOG-like rows of the dataset table).

Every memory at every frequency, every cell of P, P_hat, Pr(psi = 1) and OGM
is compared, and the classes bit-exactly (decided on the GPU's own float32
OGM).  Tolerances (normwise = max|gpu - oracle| / max|oracle|):
  * memories: 3e-5 normwise (the FP32 encode's phase error, see the parity
    tests of the small cases);
  * P and P_hat: 1e-4 for the FP32 path and the 16-bit split products (about
    16 significant bits per product), 1e-2 for FP8x3 (hi + lo e4m3, about
    8 significant bits per operand value);
  * Pr(psi = 1): 1e-3 absolute for every path; OGM = 2 Pr - 1: 2e-3.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from helpers import config_for, normwise, oracle_grid, run_gpu
from paper_2408_09066_gb300 import synth
from paper_2408_09066_gb300 import vsaogm as V

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL_OMEGA, TOL_PR = 3e-5, 1e-3
TOL_P = {V.DECODE_FP32: 1e-4, V.DECODE_BF16X3: 1e-4, V.DECODE_FP16X3: 1e-4,
         V.DECODE_FP8X3: 1e-2}
ALL_PRECS = [V.DECODE_FP32, V.DECODE_BF16X3, V.DECODE_FP16X3, V.DECODE_FP8X3]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2408_09066_gb300 import build
    build.build()


def _oracle(cfg, xy, lab):
    g = oracle_grid(cfg)
    nx, ny = oracle.draw_nu(cfg.seed, cfg.D, float(np.float32(cfg.length_scale)))
    out = oracle.pipeline(g, nx, ny, xy, lab, cfg.r_occ, cfg.r_emp, cfg.rho, "tile")
    out["nu"] = (nx, ny)
    return out


def _omega_c(got):
    if np.iscomplexobj(got):
        return got
    o = got.reshape(got.shape[0], -1, 2)
    return o[..., 0] + 1j * o[..., 1]


def _check_every_element(got, want, prec, what=""):
    """Every output of one map against the oracle; returns the errors."""
    err = dict(omega=normwise(_omega_c(got["omega"]), want["omega"]),
               P=normwise(got["P"], want["P"]),
               pr1=float(np.abs(got["occ"] - want["pr1"]).max()),
               ogm=float(np.abs(got["ogm"] - want["ogm"]).max()))
    if "Phat" in got:
        err["Phat"] = normwise(got["Phat"], want["Phat"])
    assert err["omega"] <= TOL_OMEGA, (what, err)
    assert err["P"] <= TOL_P[prec], (what, err)
    assert err.get("Phat", 0.0) <= TOL_P[prec], (what, err)
    assert err["pr1"] <= TOL_PR, (what, err)
    assert err["ogm"] <= 2 * TOL_PR, (what, err)
    return err


@pytest.fixture(scope="module")
def paper():
    wl = synth.paper_trajectory()
    cfg = config_for(wl)
    return wl, _oracle(cfg, wl.xy, wl.labels)


@pytest.mark.parametrize("prec", ALL_PRECS)
def test_paper_map_every_element(paper, prec):
    """400 x 400 cells, 4 x 4 tiles, D = 8192, 2,268,000 points: all 32 memories
    at all 8192 frequencies, and all 160,000 cells of both class maps."""
    wl, want = paper
    cfg = config_for(wl, decode_prec=prec)
    got = run_gpu(cfg, wl.xy, wl.labels)
    assert np.array_equal(got["nu"][0], want["nu"][0])
    assert np.array_equal(got["nu"][1], want["nu"][1])
    assert got["rejected"] == 0
    _check_every_element(got, want, prec, "paper map")
    assert np.array_equal(got["cls"], oracle.classify_f32(got["ogm"], cfg.rho))
    assert np.array_equal(got["occ_query"], got["occ"])


def test_batch64_every_map_every_element():
    """The 64-map batch (64^2 to 1024^2 cells, 1..8 x 8 tiles, D in {2048, 4096,
    8192}, 10k-500k points each) through the autotuned, captured and replayed
    step: every memory, cell and class of every map against the oracle."""
    import torch
    wls = synth.batch_maps()
    cfgs = [config_for(w, decode_prec=V.DECODE_BF16X3) for w in wls]
    dev = torch.device("cuda")
    maps = [V.Map(c) for c in cfgs]
    try:
        xy = [torch.from_numpy(np.ascontiguousarray(w.xy, np.float32)).to(dev) for w in wls]
        lab = [torch.from_numpy(np.ascontiguousarray(w.labels, np.uint8)).to(dev) for w in wls]
        heat = [torch.empty((2, w.H, w.W), dtype=torch.float32, device=dev) for w in wls]
        occ = [torch.empty((w.H, w.W), dtype=torch.float32, device=dev) for w in wls]
        ogm = [torch.empty((w.H, w.W), dtype=torch.float32, device=dev) for w in wls]
        s = torch.cuda.Stream()
        with V.Batch(maps) as b:
            with torch.cuda.stream(s):
                b.autotune(xy, lab, heat, occ, stream=s)
                b.capture(xy, lab, heat, occ, ogm, reset=True, stream=s)
                b.replay(stream=s)
            s.synchronize()
            b.status()
            got = [dict(omega=m.get_memory().cpu().numpy(), P=h.cpu().numpy(),
                        occ=o.cpu().numpy(), ogm=g.cpu().numpy())
                   for m, h, o, g in zip(maps, heat, occ, ogm)]
        worst = {}
        for w, cfg, g in zip(wls, cfgs, got):
            for k, v in g.items():
                assert np.all(np.isfinite(v)), (w.name, k)
            err = _check_every_element(g, _oracle(cfg, w.xy, w.labels), V.DECODE_BF16X3, w.name)
            for k, v in err.items():
                worst[k] = max(worst.get(k, 0.0), v)
        print("batch64 worst errors against the oracle:", worst)
    finally:
        for m in maps:
            m.close()


@pytest.mark.parametrize("prec", [V.DECODE_FP32, V.DECODE_BF16X3])
def test_fusion_matches_the_oracle_on_the_union(prec):
    """Algorithm 3 with two agents on a 4 x 4 tile map: agent A bundles the
    first half of a 20-scan trajectory, agent B the second half, A fuses B.
    The fused memories are the oracle's memories of the union (a sum of the
    agents' memories, Eq. bundling), and the fused map decodes to the oracle's
    P, Pr(psi = 1) and OGM of the union."""
    import torch
    wl = synth.paper_trajectory(n_scans=20, D=4096)
    cfg = config_for(wl, decode_prec=prec)
    want = _oracle(cfg, wl.xy, wl.labels)
    dev = torch.device("cuda")
    n = wl.n // 2
    xy = torch.from_numpy(wl.xy).to(dev)
    lab = torch.from_numpy(wl.labels).to(dev)
    H, W = wl.H, wl.W
    with V.Map(cfg) as a, V.Map(cfg) as b:
        a.encode_bundle(xy[:n], lab[:n])
        b.encode_bundle(xy[n:], lab[n:])
        a.fuse(b)
        heat = torch.empty((2, H, W), dtype=torch.float32, device=dev)
        occ = torch.empty((H, W), dtype=torch.float32, device=dev)
        ogm = torch.empty((H, W), dtype=torch.float32, device=dev)
        a.query(heat, occ, ogm)
        torch.cuda.synchronize()
        a.status()
        got = dict(omega=a.get_memory().cpu().numpy(), P=heat.cpu().numpy(),
                   occ=occ.cpu().numpy(), ogm=ogm.cpu().numpy())
    _check_every_element(got, want, prec, "fused map")


def _paper_shaped():
    return [synth.toysim_like(), synth.intel_like(n_scans=300), synth.evilog_like()]


@pytest.mark.parametrize("prec", [V.DECODE_FP32, V.DECODE_BF16X3])
@pytest.mark.parametrize("which", [0, 1, 2], ids=["toysim", "intel", "evilog"])
def test_paper_shaped_rows_every_element(prec, which):
    """ToySim-like (100 m world at 0.25 m, 2 x 2 tiles, D = 16000, l = 1 m),
    Intel-like (300 of its 910 scans of 421 beams, 380^2 cells, 8 x 8 tiles,
    D = 16000, l = 0.2 m) and EviLOG-like (one 48,000-point frame, 352 x 512
    cells of 0.16 m, one tile, D = 16000, l = 0.2 m): every output element."""
    wl = _paper_shaped()[which]
    cfg = config_for(wl, decode_prec=prec)
    got = run_gpu(cfg, wl.xy, wl.labels)
    want = _oracle(cfg, wl.xy, wl.labels)
    _check_every_element(got, want, prec, wl.name)
    assert np.array_equal(got["cls"], oracle.classify_f32(got["ogm"], cfg.rho))
