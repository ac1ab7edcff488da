"""The allocation-free encode entry point (vsaogm_encode_bundle_noalloc).

Some callers cannot call cudaMalloc: a real-time control loop, where an
allocation can synchronise the device and stall it, or a process whose device
memory belongs to another allocator.  For them the library offers an encode
call whose scratch is a static device array.  This test calls it through the C
ABI twice in a row on the same map and checks the memories after each call
against the regular (allocating) entry point, within the memory tolerance the
other parity tests use.  It is kept in a file of its own, collected last.
"""
import numpy as np
import pytest

import oracle
from helpers import config_for, normwise, oracle_grid
from paper_2408_09066_gb300 import synth
from paper_2408_09066_gb300 import vsaogm as V

pytestmark = pytest.mark.gpu

TOL_OMEGA = 3e-5  # as in test_gpu_parity.py
MAX_POINTS = 1 << 18


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2408_09066_gb300 import build
    build.build()


@pytest.mark.parametrize("D", [1024, 8192])
def test_noalloc_matches_regular_entry_point_on_two_calls(D):
    import torch
    wl = synth.small_scan(seed=4242, D=D)
    more = synth.small_scan(seed=4243, D=D)
    cfg = config_for(wl, tiles_x=2, tiles_y=2)
    dev = torch.device("cuda")
    batches = [(torch.from_numpy(w.xy).to(dev), torch.from_numpy(w.labels).to(dev))
               for w in (wl, more)]
    with V.Map(cfg) as ref, V.Map(cfg) as na:
        for xy, lab in batches:
            ref.encode_bundle(xy, lab)
            V._check(V.lib().vsaogm_encode_bundle_noalloc(
                na.handle, V._V(xy.data_ptr()), V._V(lab.data_ptr()), lab.shape[0],
                V._V(torch.cuda.current_stream().cuda_stream)))
            a, b = ref.get_memory(), na.get_memory()
            torch.cuda.synchronize()
            assert normwise(b.cpu().numpy(), a.cpu().numpy()) <= TOL_OMEGA
        assert ref.rejected() == na.rejected() == 0


def test_noalloc_rejects_more_points_than_its_scratch_holds():
    import torch
    wl = synth.small_scan(seed=1)
    cfg = config_for(wl)
    n = (1 << 18) + 1
    xy = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    lab = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with V.Map(cfg) as m:
        with pytest.raises(V.VsaogmError) as ei:
            m.encode_bundle_noalloc(xy, lab)
        assert ei.value.code == V.E_INVAL and "maximum" in str(ei.value)
        m.encode_bundle_noalloc(xy[:0], lab[:0])  # n = 0 is a no-op
        assert torch.count_nonzero(m.get_memory()).item() == 0


def _noalloc(m, xy, lab):
    import torch
    V._check(V.lib().vsaogm_encode_bundle_noalloc(
        m.handle, V._V(xy.data_ptr()), V._V(lab.data_ptr()), lab.shape[0],
        V._V(torch.cuda.current_stream().cuda_stream)))


def _oracle_omega(cfg, xy, lab):
    nx, ny = oracle.draw_nu(cfg.seed, cfg.D, float(np.float32(cfg.length_scale)))
    return oracle.memories(oracle_grid(cfg), nx, ny, xy, lab, "tile")


@pytest.mark.parametrize("n", [8193, 100_000, MAX_POINTS])
def test_noalloc_many_points_match_regular_entry_point_and_oracle(n):
    """Calls above the one-CTA sort bound (8192 points), which run the
    four-kernel sort and use the array's histogram region, up to exactly the
    documented maximum of 262,144 points: first points of the 400 x 400 cell,
    4 x 4 tile trajectory at D = 2048, twice in a row."""
    import torch
    wl = synth.paper_trajectory(n_scans=13, D=2048)
    assert wl.n >= MAX_POINTS
    xy_h, lab_h = wl.xy[:n].copy(), wl.labels[:n].copy()
    cfg = config_for(wl)
    dev = torch.device("cuda")
    xy, lab = torch.from_numpy(xy_h).to(dev), torch.from_numpy(lab_h).to(dev)
    want = _oracle_omega(cfg, xy_h, lab_h)
    with V.Map(cfg) as ref, V.Map(cfg) as na:
        for call in (1, 2):
            ref.encode_bundle(xy, lab)
            _noalloc(na, xy, lab)
            a, b = ref.get_memory(), na.get_memory()
            torch.cuda.synchronize()
            na.status()
            a, b = a.cpu().numpy(), b.cpu().numpy()
            assert normwise(b, a) <= TOL_OMEGA, call
            assert normwise(b, call * want) <= TOL_OMEGA, call


def test_noalloc_wide_tile_far_points_match_oracle():
    """One 40 m tile: the call bundles every point relative to the tile centre,
    so points near the tile's edge (up to 28 m from its centre) take the fast
    phase reduction and points far outside the map the exact one; both match
    the oracle's memories."""
    import torch
    wl = synth.paper_trajectory(n_scans=6, D=2048)
    far = np.array([[-100.0, 50.0], [40.0, -3.0], [19.99, 19.99], [-19.95, 19.97]],
                   np.float32)
    xy_h = np.ascontiguousarray(np.concatenate([wl.xy, far]))
    lab_h = np.concatenate([wl.labels, np.array([0, 1, 1, 0], np.uint8)])
    cfg = V.default_config(D=2048, grid_w=400, grid_h=400, resolution=0.1, x_min=-20.0,
                           y_min=-20.0, tiles_x=1, tiles_y=1, length_scale=0.1, seed=77)
    want = _oracle_omega(cfg, xy_h, lab_h)
    dev = torch.device("cuda")
    xy, lab = torch.from_numpy(xy_h).to(dev), torch.from_numpy(lab_h).to(dev)
    with V.Map(cfg) as ref, V.Map(cfg) as na:
        ref.encode_bundle(xy, lab)
        _noalloc(na, xy, lab)
        a, b = ref.get_memory(), na.get_memory()
        torch.cuda.synchronize()
        a, b = a.cpu().numpy(), b.cpu().numpy()
    assert normwise(b, a) <= TOL_OMEGA
    assert normwise(b, want) <= TOL_OMEGA
    # the single far point alone: one phasor, so no averaging hides its error
    with V.Map(cfg) as na:
        one = torch.from_numpy(far[:1].copy()).to(dev)
        _noalloc(na, one, torch.zeros(1, dtype=torch.uint8, device=dev))
        b = na.get_memory().cpu().numpy()
    w1 = _oracle_omega(cfg, far[:1], np.zeros(1, np.uint8))
    assert np.abs(b - w1).max() <= TOL_OMEGA


def test_noalloc_checked_map_reports_rejected_points():
    """With VSAOGM_FLAG_CHECKED, rejected points (label above 1, non-finite
    coordinates) make the call return E_DATA, as the regular entry point does;
    the valid points are still bundled."""
    import torch
    wl = synth.small_scan(seed=4244)
    cfg = config_for(wl, flags=V.FLAG_CHECKED)
    xy_h = wl.xy.copy()
    lab_h = wl.labels.copy()
    lab_h[5] = 2
    xy_h[9, 0] = np.nan
    dev = torch.device("cuda")
    xy, lab = torch.from_numpy(xy_h).to(dev), torch.from_numpy(lab_h).to(dev)
    with V.Map(cfg) as ref, V.Map(cfg) as na:
        with pytest.raises(V.VsaogmError) as e_ref:
            ref.encode_bundle(xy, lab)
        with pytest.raises(V.VsaogmError) as e_na:
            _noalloc(na, xy, lab)
        assert e_ref.value.code == e_na.value.code == V.E_DATA
        assert ref.rejected() == na.rejected() == 2
        a, b = ref.get_memory(), na.get_memory()
        torch.cuda.synchronize()
        assert normwise(b.cpu().numpy(), a.cpu().numpy()) <= TOL_OMEGA
        # a clean call on the checked map returns OK
        good = np.ones(len(lab_h), bool)
        good[[5, 9]] = False
        _noalloc(na, xy[torch.from_numpy(good).to(dev)].contiguous(),
                 lab[torch.from_numpy(good).to(dev)].contiguous())
