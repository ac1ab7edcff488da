"""Failure detection without a GPU fault.

* Bounded waits: the tensor-core decode gives every mbarrier wait a limit; a
  test knob (VSAOGM_DEBUG_WAIT_NS at map creation) shortens it and makes the
  loader warp stall on a barrier nothing arrives at, so the waits run out.  The
  call must report E_TIMEOUT, free its tensor memory and leave the context
  usable: a fresh map then matches the oracle.  Runs in its own process.
* Allocation failures: with VSAOGM_FAIL_ALLOC=n the n-th device allocation of
  one call fails as if the device were out of memory.  Map creation, scratch
  reservation, growing scratch in encode and query, and batch creation and
  stepping must each return E_NOMEM and keep nothing allocated
  (vsaogm_device_bytes), and the map must stay usable.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from helpers import config_for
from paper_2408_09066_gb300 import synth
from paper_2408_09066_gb300 import vsaogm as V

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2408_09066_gb300 import build
    build.build()


def test_bounded_waits_time_out_and_the_context_stays_usable():
    r = subprocess.run([sys.executable, os.path.join(HERE, "failure_run.py")],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["single_map"] == "E_TIMEOUT", res
    assert res["batch"] == "E_TIMEOUT", res
    assert res["fresh_map"] == "ok", res
    assert res["fresh_P"] <= 1e-4 and res["fresh_pr1"] <= 1e-3, res


def _fails_then_succeeds(monkeypatch, call, exact=True, max_n=64):
    """Runs call() with the n-th allocation failing for n = 1, 2, ... until it
    succeeds; each failing run must raise E_NOMEM and, for calls that create
    an object (exact), leave the library's device bytes where they were (a
    call that grows an existing map's scratch keeps what it grew before the
    failure; the map frees it when it is destroyed).  Returns the number of
    allocations seen and the call's result."""
    for n in range(1, max_n + 1):
        before = V.device_bytes()
        monkeypatch.setenv("VSAOGM_FAIL_ALLOC", str(n))
        try:
            result = call()
        except V.VsaogmError as e:
            assert e.code == V.E_NOMEM, (n, e)
            if exact:
                assert V.device_bytes() == before, n
            continue
        finally:
            monkeypatch.delenv("VSAOGM_FAIL_ALLOC", raising=False)
        return n - 1, result
    raise AssertionError("the call never succeeded")


@pytest.mark.parametrize("prec", [V.DECODE_FP32, V.DECODE_BF16X3])
def test_map_creation_frees_everything_on_allocation_failure(monkeypatch, prec):
    wl = synth.small_scan()
    cfg = config_for(wl, tiles_x=2, tiles_y=2, decode_prec=prec)
    base = V.device_bytes()
    n, m = _fails_then_succeeds(monkeypatch, lambda: V.Map(cfg))
    assert n >= 10  # tables, memories, counters (and the decode tables)
    assert V.device_bytes() > base
    m.close()
    assert V.device_bytes() == base


def test_scratch_growth_failures_leave_the_map_usable(monkeypatch):
    import torch
    dev = torch.device("cuda")
    wl = synth.small_scan(seed=17)
    cfg = config_for(wl, decode_prec=V.DECODE_BF16X3)
    xy = torch.from_numpy(wl.xy).to(dev)
    lab = torch.from_numpy(wl.labels).to(dev)
    heat = torch.empty((2, wl.H, wl.W), dtype=torch.float32, device=dev)
    occ = torch.empty((wl.H, wl.W), dtype=torch.float32, device=dev)
    with V.Map(cfg) as ref:
        ref.encode_bundle(xy, lab)
        ref.query(heat, occ)
        want = occ.cpu().numpy()
    base = V.device_bytes()
    with V.Map(cfg) as m:
        # reserve: every scratch buffer it grows can fail
        n, _ = _fails_then_succeeds(monkeypatch, lambda: m.reserve(1 << 20), exact=False)
        assert n >= 1
    assert V.device_bytes() == base
    with V.Map(cfg) as m:
        # the first encode and the first query grow their scratch (before any
        # launch, so a failed call bundles nothing)
        _fails_then_succeeds(monkeypatch, lambda: m.encode_bundle(xy, lab), exact=False)
        _fails_then_succeeds(monkeypatch, lambda: m.query(heat, occ), exact=False)
        torch.cuda.synchronize()
        m.status()
        assert np.array_equal(occ.cpu().numpy(), want)
    assert V.device_bytes() == base


def test_batch_allocation_failures(monkeypatch):
    import torch
    dev = torch.device("cuda")
    wls = synth.batch_maps(n_maps=3, seed=61, min_cells=40, max_cells=90, min_points=2000,
                           max_points=6000, dims=(1000, 2048))
    maps = [V.Map(config_for(w, decode_prec=V.DECODE_BF16X3)) for w in wls]
    try:
        xy = [torch.from_numpy(w.xy).to(dev) for w in wls]
        lab = [torch.from_numpy(w.labels).to(dev) for w in wls]
        heat = [torch.empty((2, w.H, w.W), dtype=torch.float32, device=dev) for w in wls]
        occ = [torch.empty((w.H, w.W), dtype=torch.float32, device=dev) for w in wls]
        base = V.device_bytes()
        _, b = _fails_then_succeeds(monkeypatch, lambda: V.Batch(maps))
        try:
            n, _ = _fails_then_succeeds(monkeypatch, lambda: b.step(xy, lab, heat, occ),
                                        exact=False)
            assert n >= 1  # the first step grows the batch's scratch
            torch.cuda.synchronize()
            b.status()
            assert all(np.all((o.cpu().numpy() >= 0) & (o.cpu().numpy() <= 1)) for o in occ)
        finally:
            b.close()
        assert V.device_bytes() == base
    finally:
        for m in maps:
            m.close()
