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
    # throughput is the workload's points over the mean step time
    assert abs(d["value"] * d["ms_per_step"] / 1e3 - 3960) < 1e-6 * 3960


def test_data_field_names_the_workload():
    from paper_2408_09066_gb300 import synth
    assert bench.data_of("paper", None) == bench.DATA
    w = synth.small_scan()
    assert bench.data_of("small", w).endswith("(small_64x64_1tile, 3960 points)")
