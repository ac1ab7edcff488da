"""The C ABI library: builds, loads, exports every symbol of include/vsaogm.h,
and validates its arguments on the host (no GPU needed for any of this)."""
import ctypes
import os
import re

import pytest

from paper_2408_09066_gb300 import build as build_mod
from paper_2408_09066_gb300 import vsaogm as V

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vsaogm.h")


@pytest.fixture(scope="module")
def L():
    build_mod.build()
    return V.lib()


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vsaogm_\w+)\s*\(", src)))


def test_header_declares_the_hot_path_entry_points():
    names = _declared_functions()
    for must in ("vsaogm_create", "vsaogm_encode_bundle", "vsaogm_decode", "vsaogm_entropy",
                 "vsaogm_destroy", "vsaogm_last_error"):
        assert must in names


def test_every_declaration_cites_its_passage():
    """Each entry point's comment cites the passage that defines it (an equation,
    section or algorithm of the paper) or says that the paper has no counterpart."""
    src = open(HEADER).read()
    pat = re.compile(r"/\*((?:(?!\*/).)*)\*/\s*\n(?:int|void|const char)\s*\*?\s*(vsaogm_\w+)\s*\(",
                     re.S)
    seen = {}
    for m in pat.finditer(src):
        seen[m.group(2)] = m.group(1)
    assert set(seen) == set(_declared_functions())
    for name, comment in seen.items():
        text = re.sub(r"\s*\n\s*\*\s*", " ", comment)   # join the comment's lines
        assert re.search(r"Eqs?\.|Sec\.|Algorithm|no counterpart", text, re.I), name


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert set(V._SIGNATURES) >= set(_declared_functions())


def test_config_layout_and_defaults(L):
    assert ctypes.sizeof(V.Config) == 72
    c = V.default_config()
    assert (c.D, c.grid_w, c.grid_h, c.tiles_x, c.tiles_y, c.r_occ, c.r_emp) == (8192, 400, 400, 4, 4, 3, 3)
    assert abs(c.resolution - 0.1) < 1e-7 and abs(c.length_scale - 0.1) < 1e-7
    assert c.decode_prec == V.DECODE_FP32 and c.flags == 0


@pytest.mark.parametrize("field,value,msg", [
    ("D", 0, "D must"), ("grid_w", 0, "grid_w"), ("resolution", 0.0, "resolution"),
    ("resolution", float("nan"), "resolution"), ("tiles_x", 0, "tiles"),
    ("tiles_x", 401, "tiles"), ("length_scale", -1.0, "length_scale"), ("r_occ", -1, "radii"),
    ("r_emp", 17, "radii"), ("decode_prec", 9, "decode_prec"), ("flags", 64, "flags"),
    ("x_min", float("inf"), "x_min")])
def test_create_rejects_bad_config_before_touching_the_gpu(L, field, value, msg):
    c = V.default_config(**{field: value})
    h = ctypes.c_void_p()
    rc = L.vsaogm_create(ctypes.byref(c), ctypes.byref(h))
    assert rc == V.E_INVAL and not h.value
    assert msg in L.vsaogm_last_error().decode()


def test_too_many_tiles_rejected(L):
    c = V.default_config(grid_w=2048, grid_h=2048, tiles_x=64, tiles_y=32)
    h = ctypes.c_void_p()
    assert L.vsaogm_create(ctypes.byref(c), ctypes.byref(h)) == V.E_INVAL


def test_null_arguments_rejected(L):
    assert L.vsaogm_create(None, None) == V.E_INVAL
    assert L.vsaogm_encode_bundle(None, None, None, 0, None) == V.E_INVAL
    assert L.vsaogm_decode(None, None, None) == V.E_INVAL
    assert L.vsaogm_entropy(None, None, None, None, None, None) == V.E_INVAL
    assert L.vsaogm_query(None, None, None, None, None, None) == V.E_INVAL
    assert L.vsaogm_fuse(None, None, None) == V.E_INVAL
    assert L.vsaogm_destroy(None) == V.OK


def test_create_without_a_gpu_fails_cleanly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    c = V.default_config(D=64, grid_w=8, grid_h=8, tiles_x=1, tiles_y=1)
    h = ctypes.c_void_p()
    rc = L.vsaogm_create(ctypes.byref(c), ctypes.byref(h))
    assert rc in (V.E_CUDA, V.E_NOMEM) and not h.value
    assert L.vsaogm_last_error().decode()


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    monkeypatch.setattr(V, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(V, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        V.lib()


def test_batch_create_rejects_bad_arguments_before_touching_the_gpu(L):
    h = ctypes.c_void_p()
    maps = (ctypes.c_void_p * (V.MAX_BATCH + 1))()
    for count in (0, V.MAX_BATCH + 1):
        assert L.vsaogm_batch_create(maps, count, ctypes.byref(h)) == V.E_INVAL
        assert "batch holds" in L.vsaogm_last_error().decode()
    assert L.vsaogm_batch_create(maps, 1, ctypes.byref(h)) == V.E_INVAL  # NULL map
    assert not h.value
    assert L.vsaogm_batch_destroy(None) == V.OK
    assert L.vsaogm_batch_replay(None, None) == V.E_INVAL


def test_bounds_checked_build_compiles_and_exports_the_same_symbols():
    """The checked variant (the library's sanitizer stand-in) builds for sm_103a
    and exports every declared entry point."""
    lib = build_mod.build(checked=True)
    L2 = ctypes.CDLL(lib)
    missing = [n for n in _declared_functions() if not hasattr(L2, n)]
    assert not missing, missing


@pytest.mark.parametrize("name", ["alu_rates", "mufu_range", "f32x2_rates"])
def test_microbenchmarks_compile_for_sm103a(tmp_path, name):
    """The microbenchmarks behind the encode's ALU roofline and phase tiers build
    for sm_103a."""
    import subprocess
    src = os.path.join(ROOT, "paper_2408_09066_gb300", "microbench", name + ".cu")
    out = tmp_path / (name + ".o")
    r = subprocess.run([build_mod.nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                        "-c", src, "-o", str(out)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert out.stat().st_size > 0
