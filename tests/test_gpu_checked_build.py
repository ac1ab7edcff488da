"""The bounds-checked build (-DVSAOGM_CHECK, the library's sanitizer stand-in):
every guarded index of the hot path stays in range on single maps of three
decode precisions, a window query on a wide tile with bundling patches, and a
captured and replayed batch; the small scan still matches the oracle."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_reports_no_out_of_range_access():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_run.py")],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    st = res["statuses"]
    assert st["fp32"] == st["bf16"] == st["fp8"] == st["wide_tile_window"] == "ok", st
    assert all(x == "ok" for x in st["batch"]), st
    assert res["small_P"] <= 1e-4 and res["small_pr1"] <= 1e-3, res
