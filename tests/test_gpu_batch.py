"""Batched stepping of many maps (one launch per stage across all maps) against
the FP64 oracle map by map, against the same maps stepped one at a time, and
through CUDA-graph capture and replay.

Tolerances are those of the tensor-core decode: raw maps P <= 1e-4 normwise,
occupancy Pr(psi = 1) <= 1e-3 absolute, memories <= 3e-5 normwise (the FP32
encode's bound).
"""
import numpy as np
import pytest

import oracle
from helpers import config_for, normwise, oracle_grid
from paper_2408_09066_gb300 import synth
from paper_2408_09066_gb300 import vsaogm as V

pytestmark = pytest.mark.gpu

TOL_OMEGA, TOL_P, TOL_PR = 3e-5, 1e-4, 1e-3
# batch vs the same map stepped alone: the frequency slicing of the decode
# differs (the batch slices for all maps at once), so the FP32 accumulators sum
# other runs of split products.  Each path sits 0.3e-5 to 1.6e-5 off the
# oracle (the omitted lo*lo term of the BF16 split is 2^-16 relative per
# product), so they can differ by a few 1e-5 (6.3e-5 seen on a 423^2-cell
# D = 8192 map); both stay inside TOL_P of the oracle
TOL_SELF_P, TOL_SELF_PR = TOL_P, TOL_PR
PRECS = [V.DECODE_BF16X3, V.DECODE_FP16X3, V.DECODE_FP8X3]
# raw maps P of the FP8 split (about 8 significant bits per operand value: held
# to the P_hat bound, see the tensor-core decode tests for the derivation)
TOL_P_PREC = {V.DECODE_BF16X3: 1e-4, V.DECODE_FP16X3: 1e-4, V.DECODE_FP8X3: 1e-2}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2408_09066_gb300 import build
    build.build()


def _maps(n_maps=6, seed=7, **kw):
    args = dict(min_cells=40, max_cells=200, min_points=2000, max_points=30000,
                dims=(1000, 2048, 4096))
    args.update(kw)
    return synth.batch_maps(n_maps=n_maps, seed=seed, **args)


class _Run:
    """Device inputs and outputs of one batch of workloads."""

    def __init__(self, wls, prec):
        import torch
        dev = torch.device("cuda")
        self.wls = wls
        self.cfgs = [config_for(w, decode_prec=prec) for w in wls]
        self.maps = [V.Map(c) for c in self.cfgs]
        self.xy = [torch.from_numpy(np.ascontiguousarray(w.xy, np.float32)).to(dev) for w in wls]
        self.lab = [torch.from_numpy(np.ascontiguousarray(w.labels, np.uint8)).to(dev)
                    for w in wls]
        self.heat = [torch.empty((2, w.H, w.W), dtype=torch.float32, device=dev) for w in wls]
        self.occ = [torch.empty((w.H, w.W), dtype=torch.float32, device=dev) for w in wls]
        self.ogm = [torch.empty((w.H, w.W), dtype=torch.float32, device=dev) for w in wls]
        self.batch = V.Batch(self.maps)

    def host(self):
        import torch
        torch.cuda.synchronize()
        self.batch.status()
        out = [dict(omega=m.get_memory().cpu().numpy(), P=h.cpu().numpy(), occ=o.cpu().numpy(),
                    ogm=g.cpu().numpy())
               for m, h, o, g in zip(self.maps, self.heat, self.occ, self.ogm)]
        for d in out:  # NaN / Inf scan
            for k, v in d.items():
                assert np.all(np.isfinite(v)), f"non-finite values in {k}"
        return out

    def close(self):
        self.batch.close()
        for m in self.maps:
            m.close()


def _oracle(cfg, xy, lab):
    g = oracle_grid(cfg)
    nx, ny = oracle.draw_nu(cfg.seed, cfg.D, float(np.float32(cfg.length_scale)))
    return oracle.pipeline(g, nx, ny, xy, lab, cfg.r_occ, cfg.r_emp, cfg.rho, "tile")


def _omega_c(got):
    if np.iscomplexobj(got):
        return got
    o = got.reshape(got.shape[0], -1, 2)
    return o[..., 0] + 1j * o[..., 1]


def _check(got, want, what="", tol_p=TOL_P):
    assert normwise(_omega_c(got["omega"]), want["omega"]) <= TOL_OMEGA, what
    assert normwise(got["P"], want["P"]) <= tol_p, what
    assert np.abs(got["occ"] - want["pr1"]).max() <= TOL_PR, what
    assert np.abs(got["ogm"] - want["ogm"]).max() <= 2 * TOL_PR, what


@pytest.mark.parametrize("prec", PRECS)
def test_batch_matches_oracle(prec):
    """Six maps of uneven size, tiling and D (one D not a multiple of 32)."""
    r = _Run(_maps(), prec)
    try:
        r.batch.step(r.xy, r.lab, r.heat, r.occ, r.ogm)
        for w, cfg, got in zip(r.wls, r.cfgs, r.host()):
            _check(got, _oracle(cfg, w.xy, w.labels), w.name, TOL_P_PREC[prec])
    finally:
        r.close()


def test_batch_mixes_fused_and_separate_chunk_sums():
    """A batch holding a one-tile map with many points (its memories hold many
    chunks: their sums run in the separate reduction launch) beside many-tile
    maps with few points (their sums run inside the encode launch), checked
    against the oracle; a second step on reset maps gives bit-identical
    memories (both fixed-order paths are deterministic)."""
    import dataclasses
    wls = _maps(n_maps=3, seed=41, min_cells=64, max_cells=96, min_points=2000,
                max_points=4000, max_tiles=4, dims=(1000, 2048))
    dense = synth.batch_maps(n_maps=1, seed=43, min_cells=64, max_cells=64, min_points=60000,
                             max_points=60000, max_tiles=1, dims=(1000,))[0]
    wls = ([dataclasses.replace(dense, tiles_x=1, tiles_y=1)] +
           [dataclasses.replace(w, tiles_x=4, tiles_y=4) for w in wls])
    r = _Run(wls, V.DECODE_BF16X3)
    try:
        r.batch.set_timing(True)
        r.batch.step(r.xy, r.lab, r.heat, r.occ, r.ogm)
        got = r.host()
        st = r.batch.stage_times(reset=True)
        assert st["reduce"][1] == 1  # the dense map's sums
        for w, cfg, g in zip(r.wls, r.cfgs, got):
            _check(g, _oracle(cfg, w.xy, w.labels), w.name)
        r.batch.step(r.xy, r.lab, r.heat, r.occ, r.ogm, reset=True)
        again = r.host()
        for a, b in zip(got, again):
            assert np.array_equal(a["omega"], b["omega"])
    finally:
        r.close()


def test_batch_equals_single_maps():
    """The batch gives each map what vsaogm_encode_bundle + vsaogm_query give
    it alone, up to the summation order inside the memories."""
    import torch
    r = _Run(_maps(seed=11), V.DECODE_BF16X3)
    try:
        r.batch.step(r.xy, r.lab, r.heat, r.occ, r.ogm)
        got = r.host()
        for i, (w, cfg) in enumerate(zip(r.wls, r.cfgs)):
            with V.Map(cfg) as m:
                m.encode_bundle(r.xy[i], r.lab[i])
                heat = torch.empty_like(r.heat[i])
                occ = torch.empty_like(r.occ[i])
                m.query(heat, occ)
                torch.cuda.synchronize()
                assert normwise(got[i]["omega"], m.get_memory().cpu().numpy()) <= 1e-5, w.name
                assert normwise(got[i]["P"], heat.cpu().numpy()) <= TOL_SELF_P, w.name
                assert np.abs(got[i]["occ"] - occ.cpu().numpy()).max() <= TOL_SELF_PR, w.name
    finally:
        r.close()


def test_accumulate_empty_map_and_determinism():
    """reset = 0 bundles into the memories already there; a map with no new
    points is still queried; two runs are bit-identical."""
    import torch
    wls = _maps(n_maps=4, seed=13)
    r = _Run(wls, V.DECODE_BF16X3)
    try:
        half = [len(w.labels) // 2 for w in wls]
        first_xy = [x[:h] for x, h in zip(r.xy, half)]
        first_lab = [x[:h] for x, h in zip(r.lab, half)]
        r.batch.step(first_xy, first_lab, r.heat, r.occ, r.ogm, reset=True)
        rest_xy = [x[h:] for x, h in zip(r.xy, half)]
        rest_lab = [x[h:] for x, h in zip(r.lab, half)]
        rest_xy[1] = rest_xy[1][:0]   # map 1 gets its second half below, alone
        rest_lab[1] = rest_lab[1][:0]
        r.maps[1].encode_bundle(r.xy[1][half[1]:], r.lab[1][half[1]:])
        r.batch.step(rest_xy, rest_lab, r.heat, r.occ, r.ogm, reset=False)
        got = r.host()
        for w, cfg, g in zip(wls, r.cfgs, got):
            _check(g, _oracle(cfg, w.xy, w.labels), w.name)
        # the same two steps again on fresh maps: identical bits
        r2 = _Run(wls, V.DECODE_BF16X3)
        try:
            r2.batch.step(first_xy, first_lab, r2.heat, r2.occ, r2.ogm, reset=True)
            r2.maps[1].encode_bundle(r.xy[1][half[1]:], r.lab[1][half[1]:])
            r2.batch.step(rest_xy, rest_lab, r2.heat, r2.occ, r2.ogm, reset=False)
            for a, b in zip(got, r2.host()):
                for k in a:
                    assert np.array_equal(a[k], b[k]), k
        finally:
            r2.close()
        torch.cuda.synchronize()
    finally:
        r.close()


def test_capture_and_replay():
    """A captured step replays to the bits of an uncaptured step, also after
    the inputs are refilled in place."""
    import torch
    wls = _maps(n_maps=5, seed=17)
    r = _Run(wls, V.DECODE_BF16X3)
    s = torch.cuda.Stream()
    try:
        with torch.cuda.stream(s):
            r.batch.capture(r.xy, r.lab, r.heat, r.occ, r.ogm, reset=True, stream=s)
        s.synchronize()
        first = r.host()
        for w, cfg, g in zip(wls, r.cfgs, first):
            _check(g, _oracle(cfg, w.xy, w.labels), w.name)
        # new points, same counts: refill in place and replay
        rng = np.random.default_rng(3)
        new = []
        for w, x, lab in zip(wls, r.xy, r.lab):
            xy2 = np.ascontiguousarray(w.xy[rng.permutation(len(w.xy))] * np.float32(0.9))
            lab2 = np.ascontiguousarray(1 - w.labels).astype(np.uint8)
            x.copy_(torch.from_numpy(xy2))
            lab.copy_(torch.from_numpy(lab2))
            new.append((xy2, lab2))
        torch.cuda.synchronize()
        r.batch.replay(stream=s)
        s.synchronize()
        replayed = r.host()
        for (xy2, lab2), cfg, g, w in zip(new, r.cfgs, replayed, wls):
            _check(g, _oracle(cfg, xy2, lab2), w.name)
        r.batch.step(r.xy, r.lab, r.heat, r.occ, r.ogm, reset=True, stream=s)
        s.synchronize()
        for a, b in zip(replayed, r.host()):
            for k in a:
                assert np.array_equal(a[k], b[k]), k
        for _ in range(3):
            r.batch.replay(stream=s)
        s.synchronize()
        for a, b in zip(replayed, r.host()):
            for k in a:
                assert np.array_equal(a[k], b[k]), k
    finally:
        r.close()


def test_autotune_keeps_parity():
    wls = _maps(n_maps=4, seed=19)
    r = _Run(wls, V.DECODE_BF16X3)
    try:
        t = r.batch.autotune(r.xy, r.lab, r.heat, r.occ)
        assert t["poly_warps"] in (7, 8, 9, 10)
        assert t["items_per_cta"] in (8, 16, 32)
        assert t["decode_waves"] in (1, 2, 4)
        r.batch.step(r.xy, r.lab, r.heat, r.occ, r.ogm)
        for w, cfg, g in zip(wls, r.cfgs, r.host()):
            _check(g, _oracle(cfg, w.xy, w.labels), w.name)
    finally:
        r.close()


def test_full_batch_of_64_small_maps():
    """The largest batch: 64 maps, each checked against the oracle."""
    wls = _maps(n_maps=64, seed=23, min_cells=16, max_cells=96, min_points=300,
                max_points=4000, dims=(256, 512, 1000))
    r = _Run(wls, V.DECODE_FP16X3)
    try:
        r.batch.step(r.xy, r.lab, r.heat, r.occ, r.ogm)
        for w, cfg, g in zip(wls, r.cfgs, r.host()):
            _check(g, _oracle(cfg, w.xy, w.labels), w.name)
    finally:
        r.close()


def test_paper_shaped_batch_sampled():
    """The 64-map workload at full size (64^2 to 1024^2 cells, 1..8 x 8 tiles,
    D in {2048, 4096, 8192}, 10k-500k points), stepped as the benchmark steps
    it (autotuned, captured, replayed): every map's memories at 64 sampled
    frequencies against the oracle; P and occupancy of the whole map against
    the oracle for the three maps of least work; every map against its own
    single-map run on the GPU."""
    import torch
    wls = synth.batch_maps()
    r = _Run(wls, V.DECODE_BF16X3)
    s = torch.cuda.Stream()
    try:
        with torch.cuda.stream(s):
            r.batch.autotune(r.xy, r.lab, r.heat, r.occ, stream=s)
            r.batch.capture(r.xy, r.lab, r.heat, r.occ, r.ogm, reset=True, stream=s)
            r.batch.replay(stream=s)
        s.synchronize()
        got = r.host()
        rng = np.random.default_rng(29)
        for w, cfg, g in zip(wls, r.cfgs, got):
            ks = np.sort(rng.choice(cfg.D, 64, replace=False)).astype(np.int32)
            nx, ny = oracle.draw_nu(cfg.seed, cfg.D, float(np.float32(cfg.length_scale)))
            want = oracle.memories(oracle_grid(cfg), nx, ny, w.xy, w.labels, "tile", ks)
            om = _omega_c(g["omega"])[:, ks]
            # normwise over the sampled columns, against the whole memory's scale
            scale = np.abs(_omega_c(g["omega"])).max()
            assert np.abs(om - want).max() / scale <= TOL_OMEGA, w.name
            assert np.all((g["occ"] >= 0) & (g["occ"] <= 1)), w.name
        cheap = sorted(range(len(wls)), key=lambda i: len(wls[i].labels) * wls[i].D
                       + wls[i].W * wls[i].H * wls[i].D)[:3]
        for i in cheap:
            _check(got[i], _oracle(r.cfgs[i], wls[i].xy, wls[i].labels), wls[i].name)
        for i, (w, cfg) in enumerate(zip(wls, r.cfgs)):
            with V.Map(cfg) as m:
                m.encode_bundle(r.xy[i], r.lab[i])
                heat = torch.empty_like(r.heat[i])
                occ = torch.empty_like(r.occ[i])
                m.query(heat, occ)
                torch.cuda.synchronize()
                assert normwise(got[i]["P"], heat.cpu().numpy()) <= TOL_SELF_P, w.name
                assert np.abs(got[i]["occ"] - occ.cpu().numpy()).max() <= TOL_SELF_PR, w.name
    finally:
        r.close()


def test_rejected_configurations():
    import torch
    a = V.Map(V.default_config(D=256, grid_w=32, grid_h=32, decode_prec=V.DECODE_BF16X3))
    b = V.Map(V.default_config(D=256, grid_w=32, grid_h=32, decode_prec=V.DECODE_FP16X3))
    c = V.Map(V.default_config(D=256, grid_w=32, grid_h=32, decode_prec=V.DECODE_FP32))
    d = V.Map(V.default_config(D=256, grid_w=32, grid_h=32, decode_prec=V.DECODE_BF16X3,
                               flags=V.FLAG_ATOMIC))
    try:
        for maps in ([a, b], [c], [a, a], [d]):
            with pytest.raises(V.VsaogmError) as e:
                V.Batch(maps)
            assert e.value.code == V.E_INVAL
        bt = V.Batch([a])
        with pytest.raises(V.VsaogmError):
            bt.replay()   # nothing captured
        heat = torch.empty((2, 32, 32), dtype=torch.float32, device="cuda")
        occ = torch.empty((32, 32), dtype=torch.float32, device="cuda")
        xy = torch.zeros((4, 2), dtype=torch.float32, device="cuda")
        lab = torch.zeros((4,), dtype=torch.uint8, device="cuda")
        with pytest.raises(V.VsaogmError):
            bt.capture([xy], [lab], [heat], [occ], stream=0)   # default stream
        bt.close()
    finally:
        for m in (a, b, c, d):
            m.close()


def test_stage_timing_and_launch_counts():
    import torch
    wls = _maps(n_maps=3, seed=31)
    r = _Run(wls, V.DECODE_BF16X3)
    s = torch.cuda.Stream()
    try:
        r.batch.set_timing(True)
        r.batch.step(r.xy, r.lab, r.heat, r.occ, r.ogm, stream=s)
        st = r.batch.stage_times(reset=True)
        # maps with few chunks per memory sum them inside the encode launch;
        # the reduce launch runs only for the others
        # small maps sort in one CTA each (one launch), the others in four
        launched = {k: v[1] for k, v in st.items()}
        assert launched["reduce"] in (0, 1)
        assert launched["sort"] in (1, 4, 5)
        per_step = {"sort": launched["sort"], "encode": 1, "reduce": launched["reduce"],
                    "norms": 1, "decode": 3, "nonlinear": 0, "entropy": 1}
        assert launched == per_step
        assert all(st[k][0] > 0 for k in ("sort", "encode", "norms", "decode",
                                          "entropy"))
        r.batch.capture(r.xy, r.lab, r.heat, r.occ, r.ogm, stream=s)
        r.batch.stage_times(reset=True)
        r.batch.replay(stream=s)
        r.batch.replay(stream=s)
        st = r.batch.stage_times(reset=True)
        assert sum(v[1] for v in st.values()) == 2 * sum(per_step.values())
        s.synchronize()
    finally:
        r.close()
