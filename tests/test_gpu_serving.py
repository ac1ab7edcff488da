"""Continuous-batching serving: every query returns the same occupancy whether
its requests run alone (one slot, one request at a time) or mixed with other
robots' requests on concurrent streams; and the window results match the
oracle for one robot."""
import numpy as np
import pytest

import oracle
from helpers import oracle_grid
from paper_2408_09066_gb300 import serving, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2408_09066_gb300 import build
    build.build()


def _fresh(reqs):
    return [serving.Request(r.kind, r.robot, r.arrival, xy=r.xy, labels=r.labels,
                            window=r.window) for r in reqs]


def test_results_alone_equal_results_in_the_mix():
    fleet = synth.robot_fleet(4, seed=77, min_cells=256, max_cells=384, scans_per_robot=2,
                              beams=360, n_empty=10)
    cfgs = serving.fleet_configs(fleet, D=2048)
    reqs = serving.poisson_requests(fleet, rate=500.0, duration=0.08, query_frac=0.5, seed=3,
                                    win_lo=32, win_hi=96)
    assert sum(r.kind == "query" for r in reqs) >= 5 and sum(r.kind == "update" for r in reqs) >= 5
    reqs_m, reqs_a = _fresh(reqs), _fresh(reqs)
    mixed = serving.Server(cfgs, max_points=360 * 11, max_window=96, n_slots=4)
    try:
        got_mixed = mixed.run(reqs_m, realtime=False)
    finally:
        mixed.close()
    alone = serving.Server(cfgs, max_points=360 * 11, max_window=96, n_slots=1)
    try:
        got_alone = alone.run(reqs_a, realtime=False)
    finally:
        alone.close()
    assert len(got_mixed) == len(got_alone) == len(reqs)
    for ra, rm in zip(reqs_a, reqs_m):
        if ra.kind == "query":
            assert ra.result.shape == rm.result.shape
            assert np.abs(ra.result - rm.result).max() <= 1e-6


def test_served_window_matches_oracle():
    fleet = synth.robot_fleet(1, seed=78, min_cells=256, max_cells=256, scans_per_robot=1,
                              beams=360, n_empty=10)
    cfg = serving.fleet_configs(fleet, D=1024)[0]
    xy, lab = fleet[0].scans[0]
    reqs = [serving.Request("update", 0, 0.0, xy=xy, labels=lab),
            serving.Request("query", 0, 0.0, window=(100, 90, 60, 70))]
    srv = serving.Server([cfg], max_points=len(lab), max_window=70, n_slots=2)
    try:
        srv.run(reqs, realtime=False)
    finally:
        srv.close()
    g = oracle_grid(cfg)
    nx, ny = oracle.draw_nu(cfg.seed, cfg.D, float(np.float32(cfg.length_scale)))
    om = oracle.memories(g, nx, ny, xy, lab, "tile")
    want = oracle.query_window(g, nx, ny, om, 100, 90, 60, 70, cfg.r_occ, cfg.r_emp)
    assert np.abs(reqs[1].result - want["pr1"]).max() <= 1e-3
