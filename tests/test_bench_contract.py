"""The benchmark's JSON line keeps its contract (CPU: the oracle arm).

``bench.py --impl reference`` times the FP64 oracle on the host cores and prints
one JSON line with the same metric, unit and config as the GPU arm, plus
``impl``, a ``cpu_baseline`` describing the run and an ``e2e`` object with no
host-device traffic.  Run here on the small workload, which takes a second.
"""
import contextlib
import io
import json
import types

import bench


def _reference_line(workload, steps=2, warmup=1):
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.run_reference(types.SimpleNamespace(gpus=1, steps=steps, warmup=warmup,
                                                       workload=workload))
    assert rc == 0
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1, "one JSON line"
    return json.loads(lines[0])


def test_reference_line_has_the_contract_keys():
    d = _reference_line("small")
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "points/s"
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 1)
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["vs_baseline"] is None and d["dtype"] == "f64"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["p50_ms"] <= d["p99_ms"]
    assert d["data"].startswith("synthetic") and "small" in d["data"]
    assert d["config"]["workload"].startswith("small_64x64_1tile")
    assert d["config"]["points_per_step"] == 3960
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert isinstance(cb["cores"], int) and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}
    assert d["gpu_launches"] == 0
    # throughput is the points the timed steps processed over their measured
    # time: the whole workload per step when it fits the step budget
    assert d["points_per_sampled_step"] == 3960
    assert abs(d["value"] * d["ms_per_step"] / 1e3 - 3960) < 1e-6 * 3960
    # one whole, unsampled step is timed too
    assert d["full_step"]["s"] > 0
    assert abs(d["full_step"]["points_per_s"] * d["full_step"]["s"] - 3960) < 1e-6 * 3960


def test_reference_steps_are_measured_samples_of_the_paper_workload(monkeypatch):
    """On a workload too large for one step within the budget, each step is a
    random sample with the workload's mix of points and cells, and `value` is
    what the samples processed over their measured time (no extrapolation)."""
    from paper_2408_09066_gb300 import synth
    wl = synth.paper_trajectory(n_scans=4, D=2048)
    monkeypatch.setattr(bench, "make_workload", lambda name, rank=0: wl)
    monkeypatch.setattr(bench, "sample_fraction", lambda w, budget, rng: 0.125)
    d = _reference_line("paper", steps=2, warmup=0)
    n, c = d["points_per_sampled_step"], d["cells_per_sampled_step"]
    assert n == round(0.125 * wl.n) and c == round(0.125 * wl.W * wl.H)
    assert abs(d["value"] * d["ms_per_step"] / 1e3 - n) < 1e-6 * n
    assert "fraction 0.125" in d["cpu_baseline"]["sample"]


def test_data_field_names_the_workload():
    from paper_2408_09066_gb300 import synth
    assert bench.data_of("paper", None) == bench.DATA
    w = synth.small_scan()
    assert bench.data_of("small", w).endswith("(small_64x64_1tile, 3960 points)")
