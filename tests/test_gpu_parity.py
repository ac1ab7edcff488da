"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (normwise error = max|gpu - oracle| / max|oracle|):
  * memories omega: 3e-5.  Each phasor carries at most 2.5e-5 rad of phase
    error from the kernel's fast phase reduction (|nu . offset| < 32 turns;
    far points take an exact reduction, about 4e-7 rad) plus about 4e-7 from
    MUFU sin/cos; below 4 turns (every point inside the map, in its bundling
    patch) the phase goes unreduced to MUFU, whose own argument reduction
    costs about 1e-7 x |2 pi t| <= 5e-6 rad (measured on GB300), about 1e-5
    rad in all.  A memory of one point is a single phasor, so the bound is
    reached there, while sums of many phasors average it down;
  * quasi-probabilities P and P_hat of the FP32 decode: 1e-4;
  * occupancy Pr(psi = 1) and OGM: 1e-3 absolute (the entropy sums up to
    |disk| terms -P_hat ln P_hat whose slope grows like |ln P_hat|, so the
    heat-map bound is amplified before the softmax);
  * integer outputs (tile assignment, axis frequencies, classes decided on the
    GPU's own float32 OGM): bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
from helpers import config_for, normwise, oracle_grid, run_gpu
from paper_2408_09066_gb300 import synth
from paper_2408_09066_gb300 import vsaogm as V

pytestmark = pytest.mark.gpu

TOL_OMEGA = 3e-5
TOL_HEAT = 1e-4
TOL_PR = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2408_09066_gb300 import build
    build.build()


def _oracle_all(cfg, xy, lab):
    g = oracle_grid(cfg)
    nx, ny = oracle.draw_nu(cfg.seed, cfg.D, float(np.float32(cfg.length_scale)))
    valid = (lab <= 1) & np.all(np.isfinite(xy), axis=1)
    out = oracle.pipeline(g, nx, ny, xy[valid], lab[valid], cfg.r_occ, cfg.r_emp, cfg.rho, "tile")
    out["nu"] = (nx, ny)
    return out


def _check_all(cfg, got, want, tol_heat=TOL_HEAT, tol_pr=TOL_PR):
    assert np.array_equal(got["nu"][0], want["nu"][0]) and np.array_equal(got["nu"][1], want["nu"][1])
    assert normwise(got["omega"], want["omega"]) <= TOL_OMEGA
    assert normwise(got["P"], want["P"]) <= tol_heat
    assert normwise(got["Phat"], want["Phat"]) <= tol_heat
    assert np.abs(got["occ"] - want["pr1"]).max() <= tol_pr
    assert np.abs(got["ogm"] - want["ogm"]).max() <= 2 * tol_pr
    assert np.array_equal(got["occ_query"], got["occ"])
    assert np.array_equal(got["cls"], oracle.classify_f32(got["ogm"], cfg.rho))


def test_small_scan_full_parity():
    """One 360-beam scan on a 64 x 64 map, D = 1024: every output, every cell."""
    wl = synth.small_scan()
    cfg = config_for(wl)
    got = run_gpu(cfg, wl.xy, wl.labels)
    want = _oracle_all(cfg, wl.xy, wl.labels)
    _check_all(cfg, got, want)
    assert got["rejected"] == 0


@pytest.mark.parametrize("D", [1, 7, 1000, 2304, 4100])
def test_ragged_sizes_tiles_not_dividing_grid(D):
    """Tiles that do not divide the grid, points outside the map, D that is not
    a multiple of the kernels' k slices, n not a multiple of any block size."""
    rng = np.random.default_rng(D)
    n = 3 * 2048 + 17
    xy = rng.uniform(-3.0, 3.4, (n, 2)).astype(np.float32)
    lab = rng.integers(0, 2, n).astype(np.uint8)
    cfg = V.default_config(D=D, grid_w=50, grid_h=37, resolution=0.13, x_min=-2.9, y_min=-2.3,
                           tiles_x=3, tiles_y=2, length_scale=0.2, seed=77, r_occ=2, r_emp=4)
    _check_all(cfg, run_gpu(cfg, xy, lab), _oracle_all(cfg, xy, lab))


def test_points_on_tile_boundaries_go_to_the_lower_tile():
    """Exactly representable boundaries at x in {-2, 0, 2}, y in {-1, 1}."""
    cfg = V.default_config(D=256, grid_w=64, grid_h=48, resolution=0.125, x_min=-4.0, y_min=-3.0,
                           tiles_x=4, tiles_y=3, seed=5)
    pts = np.array([[-2, 0.3], [0, 0.3], [2, 0.3], [0.1, -1], [0.1, 1], [0, 1], [2, -1],
                    [-4, -3], [4, 3], [-100, 50], [100, -50], [-2, -1]], np.float32)
    lab = np.array([0, 1] * 6, np.uint8)
    got = run_gpu(cfg, pts, lab)
    want = _oracle_all(cfg, pts, lab)
    nz_got = sorted(np.nonzero(np.abs(got["omega"]).sum(1))[0].tolist())
    nz_want = sorted(np.nonzero(np.abs(want["omega"]).sum(1))[0].tolist())
    assert nz_got == nz_want
    err = np.abs(got["omega"] - want["omega"])
    mem, k = np.unravel_index(np.argmax(err), err.shape)
    assert normwise(got["omega"], want["omega"]) <= TOL_OMEGA, (
        f"memory {mem} k {k}: got {got['omega'][mem, k]} want {want['omega'][mem, k]}; "
        f"worst error per memory {err.max(1).tolist()}")


@pytest.mark.parametrize("x,y", [(-100.0, 50.0), (100.0, -50.0), (0.3, 0.2), (-3.9, 2.9),
                                 (1000.0, 1000.0)])
def test_single_point_phasors_anywhere(x, y):
    """One point: every element of its memory is a unit phasor whose phase the
    oracle knows exactly; near and far from the tile centre."""
    cfg = V.default_config(D=4096, grid_w=64, grid_h=48, resolution=0.125, x_min=-4.0,
                           y_min=-3.0, tiles_x=4, tiles_y=3, seed=5)
    pts = np.array([[x, y]], np.float32)
    got = run_gpu(cfg, pts, np.array([1], np.uint8))
    want = _oracle_all(cfg, pts, np.array([1], np.uint8))
    err = np.abs(got["omega"] - want["omega"]).max(0)
    k = int(np.argmax(err))
    nx, ny = want["nu"]
    far = max(abs(x), abs(y)) > 10.0  # exact reduction; near points take the fast one
    tol = 2e-6 if far else TOL_OMEGA
    assert err[k] <= tol, (f"k {k}: nu ({nx[k]}, {ny[k]}) got {got['omega'][:, k]} "
                           f"want {want['omega'][:, k]}")


@pytest.mark.parametrize("packed,poly,poly_warps",
                         [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 2, 0), (1, 3, 0), (1, 0, 3),
                          (1, 0, 8), (1, 0, 12), (1, 0, -1)])
@pytest.mark.parametrize("D", [1000, 8192])
def test_encode_kernel_variants(monkeypatch, packed, poly, poly_warps, D):
    """The scalar encode kernel and the f32x2 one with 0..3 frequency pairs per
    thread on the FMA-pipe polynomial (or one pair in some warps only, two in
    some with 12 of 32 pairs; -1 is the automatic share) match the oracle,
    near and far points."""
    monkeypatch.setenv("VSAOGM_ENCODE_PACKED", str(packed))
    monkeypatch.setenv("VSAOGM_ENCODE_POLY", str(poly))
    monkeypatch.setenv("VSAOGM_ENCODE_POLY_WARPS", str(poly_warps))
    wl = synth.small_scan(seed=31, D=D)
    far = np.array([[-100.0, 50.0], [40.0, -3.0]], np.float32)
    xy = np.concatenate([wl.xy, far])
    lab = np.concatenate([wl.labels, np.array([0, 1], np.uint8)])
    cfg = config_for(wl)
    _check_all(cfg, run_gpu(cfg, xy, lab), _oracle_all(cfg, xy, lab))


def test_empty_input_and_single_class():
    cfg = V.default_config(D=128, grid_w=20, grid_h=16, resolution=0.1, x_min=-1.0, y_min=-0.8,
                           tiles_x=2, tiles_y=2, rho=0.0)
    got = run_gpu(cfg, np.zeros((0, 2), np.float32), np.zeros(0, np.uint8))
    assert np.all(got["omega"] == 0) and np.all(got["P"] == 0) and np.all(got["Phat"] == 0)
    assert np.all(got["occ"] == 0.5) and np.all(got["ogm"] == 0) and np.all(got["cls"] == 1)
    # only occupied points: the empty class decodes to zero everywhere
    rng = np.random.default_rng(0)
    xy = rng.uniform(-1, 1, (300, 2)).astype(np.float32)
    lab = np.ones(300, np.uint8)
    got = run_gpu(cfg, xy, lab)
    want = _oracle_all(cfg, xy, lab)
    assert np.all(got["Phat"][0] == 0)
    _check_all(cfg, got, want)


def test_single_point_at_cell_centre():
    cfg = V.default_config(D=1024, grid_w=16, grid_h=12, resolution=0.125, x_min=-1.0,
                           y_min=-0.75, tiles_x=2, tiles_y=2, seed=3)
    i0, j0 = 11, 2
    xy = np.array([[-1.0 + (i0 + 0.5) * 0.125, -0.75 + (j0 + 0.5) * 0.125]], np.float32)
    got = run_gpu(cfg, xy, np.array([1], np.uint8))
    assert abs(got["P"][1, j0, i0] - math.sqrt(1024)) < 1e-4 * math.sqrt(1024)
    assert np.unravel_index(np.argmax(got["P"][1]), got["P"][1].shape) == (j0, i0)
    assert got["Phat"][1, j0, i0] == pytest.approx(1.0, abs=1e-6)


def test_rejected_points_are_skipped_and_counted():
    rng = np.random.default_rng(4)
    n = 5000
    xy = rng.uniform(-1, 1, (n, 2)).astype(np.float32)
    lab = rng.integers(0, 2, n).astype(np.uint8)
    lab[::97] = 2
    xy[5::101, 0] = np.nan
    xy[7::103, 1] = np.inf
    bad = (lab > 1) | ~np.all(np.isfinite(xy), 1)
    cfg = V.default_config(D=512, grid_w=20, grid_h=20, resolution=0.1, x_min=-1.0, y_min=-1.0,
                           tiles_x=2, tiles_y=2)
    got = run_gpu(cfg, xy, lab)
    assert got["rejected"] == int(bad.sum())
    _check_all(cfg, got, _oracle_all(cfg, xy, lab))
    # checked mode reports them as an error
    import torch
    cfg.flags = V.FLAG_CHECKED
    with V.Map(cfg) as m:
        with pytest.raises(V.VsaogmError) as ei:
            m.encode_bundle(torch.from_numpy(xy).cuda(), torch.from_numpy(lab).cuda())
        assert ei.value.code == V.E_DATA


def test_consecutive_calls_accumulate_like_one():
    """Eq. bundling across calls: three calls equal one call on the union."""
    wl = synth.small_scan(seed=1234)
    cfg = config_for(wl)
    got = run_gpu(cfg, wl.xy, wl.labels, calls=3)
    _check_all(cfg, got, _oracle_all(cfg, wl.xy, wl.labels))


def test_default_mode_is_bitwise_reproducible_and_atomic_mode_agrees():
    wl = synth.small_scan(seed=99)
    cfg = config_for(wl)
    a = run_gpu(cfg, wl.xy, wl.labels)
    b = run_gpu(cfg, wl.xy, wl.labels)
    for k in ("omega", "P", "Phat", "occ", "ogm", "cls"):
        assert np.array_equal(a[k], b[k]), k
    cfg.flags = V.FLAG_ATOMIC
    c = run_gpu(cfg, wl.xy, wl.labels)
    assert normwise(c["omega"], a["omega"]) <= TOL_OMEGA
    assert normwise(c["P"], a["P"]) <= TOL_HEAT


@pytest.mark.parametrize("r_occ,r_emp,rho", [(0, 0, 0.0), (1, 5, -0.3), (16, 2, 0.2), (3, 3, 0.9)])
def test_disk_radii_and_threshold(r_occ, r_emp, rho):
    wl = synth.small_scan(seed=7)
    cfg = config_for(wl, r_occ=r_occ, r_emp=r_emp, rho=rho)
    _check_all(cfg, run_gpu(cfg, wl.xy, wl.labels), _oracle_all(cfg, wl.xy, wl.labels))


def test_fusion_equals_bundling_the_union_and_memory_roundtrip():
    """Algorithm 3: fusing two maps with the same axis vectors and tiling equals
    one map of all points; get/set of memories is an exact copy."""
    import torch
    wl = synth.small_scan(seed=21)
    cfg = config_for(wl)
    n = wl.n // 2
    dev = torch.device("cuda")
    xy = torch.from_numpy(wl.xy).to(dev)
    lab = torch.from_numpy(wl.labels).to(dev)
    with V.Map(cfg) as a, V.Map(cfg) as b, V.Map(cfg) as u:
        a.encode_bundle(xy[:n], lab[:n])
        b.encode_bundle(xy[n:], lab[n:])
        u.encode_bundle(xy, lab)
        a.fuse(b)
        fa, fu = a.get_memory(), u.get_memory()
        torch.cuda.synchronize()
        assert normwise(fa.cpu().numpy(), fu.cpu().numpy()) <= TOL_OMEGA
        u.set_memory(fa)
        assert torch.equal(u.get_memory(), fa)
        other = config_for(wl, seed=cfg.seed + 1)
        with V.Map(other) as c:
            with pytest.raises(V.VsaogmError) as ei:
                a.fuse(c)
            assert ei.value.code == V.E_INVAL


def test_host_entry_point_matches_device_path():
    import torch
    wl = synth.small_scan(seed=3)
    cfg = config_for(wl)
    ref = run_gpu(cfg, wl.xy, wl.labels)
    with V.Map(cfg) as m:
        occ = np.empty((wl.H, wl.W), np.float32)
        m.update_query_host(wl.xy, wl.labels, occ)
    assert np.array_equal(occ, ref["occ"])


def test_large_dimension():
    wl = synth.small_scan(seed=5, D=16384)
    cfg = config_for(wl)
    _check_all(cfg, run_gpu(cfg, wl.xy, wl.labels), _oracle_all(cfg, wl.xy, wl.labels))


def test_paper_scale_trajectory_sampled():
    """The full 400 x 400, 4 x 4 tile, D = 8192 workload with its 2.27M points,
    in the launch configuration the benchmark uses: memories at sampled k for
    all 32 memories, P at sampled cells of two tiles (the oracle decodes those
    tiles from its own full memories), and properties of the occupancy."""
    wl = synth.paper_trajectory()
    cfg = config_for(wl)
    got = run_gpu(cfg, wl.xy, wl.labels)
    g = oracle_grid(cfg)
    nx, ny = oracle.draw_nu(cfg.seed, cfg.D, float(np.float32(cfg.length_scale)))
    assert np.array_equal(got["nu"][0], nx)
    rng = np.random.default_rng(0)
    ks = np.sort(rng.choice(cfg.D, 24, replace=False)).astype(np.int32)
    om_k = oracle.memories(g, nx, ny, wl.xy, wl.labels, "tile", ks=ks)
    assert normwise(got["omega"][:, ks], om_k) <= TOL_OMEGA
    # two tiles decoded in full precision by the oracle from their own points
    beta = oracle.assign(g, wl.xy)
    for tile in (5, 15):
        sel = beta == tile
        om_t = oracle.memories(g, nx, ny, wl.xy[sel], wl.labels[sel], "tile")
        bx, by = tile % 4, tile // 4
        ci = rng.integers(bx * 100, bx * 100 + 100, 40)
        cj = rng.integers(by * 100, by * 100 + 100, 40)
        cells = np.stack([ci, cj], 1).astype(np.int32)
        Pw = oracle.decode_cells(g, nx, ny, om_t, cells, "tile")
        Pg = got["P"][:, cj, ci].T
        scale = np.abs(got["P"]).max()
        assert np.abs(Pg - Pw).max() <= TOL_HEAT * scale
    occ, ogm = got["occ"], got["ogm"]
    assert np.all(np.isfinite(occ)) and occ.min() >= 0 and occ.max() <= 1
    assert np.abs(ogm - (2 * occ - 1)).max() <= 1e-6
    assert np.array_equal(got["cls"], oracle.classify_f32(ogm, cfg.rho))
    assert got["Phat"].max() == pytest.approx(1.0, abs=1e-6)


@pytest.mark.parametrize("patches", ["auto", "0"])
def test_bundling_patches_in_wide_tiles(monkeypatch, patches):
    """One 40 m tile (its points up to 28 m from the centre): by default each
    chunk is summed relative to the centre of its 40/6 m patch and turned into
    the tile frame afterwards; with patches switched off the far points take
    the exact phase reduction.  Both match the oracle, as do points far
    outside the map."""
    if patches == "0":
        monkeypatch.setenv("VSAOGM_ENCODE_PATCHES", "0")
    else:
        monkeypatch.delenv("VSAOGM_ENCODE_PATCHES", raising=False)
    wl = synth.paper_trajectory(n_scans=6, D=2048)
    far = np.array([[-100.0, 50.0], [40.0, -3.0], [19.99, 19.99]], np.float32)
    xy = np.concatenate([wl.xy, far])
    lab = np.concatenate([wl.labels, np.array([0, 1, 1], np.uint8)])
    cfg = V.default_config(D=2048, grid_w=400, grid_h=400, resolution=0.1, x_min=-20.0,
                           y_min=-20.0, tiles_x=1, tiles_y=1, length_scale=0.1, seed=77)
    _check_all(cfg, run_gpu(cfg, xy, lab), _oracle_all(cfg, xy, lab))


def test_single_point_far_from_a_wide_tile_centre():
    """A single point 19 m from the centre of a 40 m tile: a fast-reduced phasor
    relative to its patch, times the exactly reduced patch rotation."""
    cfg = V.default_config(D=4096, grid_w=400, grid_h=400, resolution=0.1, x_min=-20.0,
                           y_min=-20.0, tiles_x=1, tiles_y=1, seed=78)
    pts = np.array([[19.3, -18.7]], np.float32)
    got = run_gpu(cfg, pts, np.array([1], np.uint8))
    want = _oracle_all(cfg, pts, np.array([1], np.uint8))
    assert np.abs(got["omega"] - want["omega"]).max() <= TOL_OMEGA


@pytest.mark.parametrize("n", [8192, 8193])
def test_sort_paths_either_side_of_the_one_cta_bound(n):
    """Up to 8192 points the four sort steps run in one CTA, above it as four
    kernels; both give the oracle's memories and maps and are bitwise
    reproducible (a stable counting sort either way)."""
    import dataclasses
    wl = synth.batch_maps(n_maps=1, seed=51, min_cells=80, max_cells=80, min_points=9000,
                          max_points=9000, max_tiles=1, dims=(1024,))[0]
    wl = dataclasses.replace(wl, xy=wl.xy[:n].copy(), labels=wl.labels[:n].copy(), tiles_x=4,
                             tiles_y=4)
    cfg = config_for(wl)
    a = run_gpu(cfg, wl.xy, wl.labels)
    _check_all(cfg, a, _oracle_all(cfg, wl.xy, wl.labels))
    b = run_gpu(cfg, wl.xy, wl.labels)
    for k in ("omega", "P", "occ"):
        assert np.array_equal(a[k], b[k]), k
