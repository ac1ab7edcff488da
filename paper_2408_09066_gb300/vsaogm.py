"""Thin ctypes binding of libvsaogm.so (C ABI in include/vsaogm.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch supplies device memory and the current CUDA stream.
If the library has not been built, loading it raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# VSAOGM_CHECKED=1 loads the bounds-checked build (build.py --checked) instead
LIB_PATH = os.path.join(_HERE, "libvsaogm_checked.so" if os.environ.get("VSAOGM_CHECKED") == "1"
                        else "libvsaogm.so")

STAGES = ("sort", "encode", "reduce", "norms", "decode", "nonlinear", "entropy")
OK, E_INVAL, E_NOMEM, E_CUDA, E_TIMEOUT, E_DATA = 0, -1, -2, -3, -4, -5
DECODE_FP32, DECODE_BF16X3, DECODE_FP16X3, DECODE_FP8X3 = 0, 1, 2, 3
FLAG_CHECKED, FLAG_ATOMIC, FLAG_WINDOW_MAP_MAX = 1, 2, 4
MODE_NO_NORM, MODE_NO_SQUARE = 1, 2
ACT_ENTROPY, ACT_RELU, ACT_TANH, ACT_SIGMOID, ACT_NONE = 0, 16, 32, 48, 64
MAX_BATCH = 64


class VsaogmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"vsaogm error {code}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    """Mirror of ``vsaogm_config``."""
    _fields_ = [("D", ctypes.c_int32), ("grid_w", ctypes.c_int32), ("grid_h", ctypes.c_int32),
                ("resolution", ctypes.c_float), ("x_min", ctypes.c_float),
                ("y_min", ctypes.c_float), ("tiles_x", ctypes.c_int32),
                ("tiles_y", ctypes.c_int32), ("length_scale", ctypes.c_float),
                ("r_occ", ctypes.c_int32), ("r_emp", ctypes.c_int32), ("rho", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("decode_prec", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("decode_mode", ctypes.c_uint32)]


_lib = None
_lock = threading.Lock()
_V = ctypes.c_void_p
_SIGNATURES = {
    "vsaogm_config_default": (None, [_V]),
    "vsaogm_create": (ctypes.c_int, [_V, _V]),
    "vsaogm_destroy": (ctypes.c_int, [_V]),
    "vsaogm_reset": (ctypes.c_int, [_V, _V]),
    "vsaogm_encode_bundle": (ctypes.c_int, [_V, _V, _V, ctypes.c_int64, _V]),
    "vsaogm_encode_bundle_noalloc": (ctypes.c_int, [_V, _V, _V, ctypes.c_int64, _V]),
    "vsaogm_decode": (ctypes.c_int, [_V, _V, _V]),
    "vsaogm_entropy": (ctypes.c_int, [_V, _V, _V, _V, _V, _V]),
    "vsaogm_query": (ctypes.c_int, [_V, _V, _V, _V, _V, _V]),
    "vsaogm_update_query_host": (ctypes.c_int, [_V, _V, _V, ctypes.c_int64, _V, _V]),
    "vsaogm_query_window": (ctypes.c_int, [_V, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, _V, _V, _V, _V, _V]),
    "vsaogm_window_scratch": (ctypes.c_int, [_V, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int32, _V]),
    "vsaogm_decode_window": (ctypes.c_int, [_V, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, _V, _V]),
    "vsaogm_rejected": (ctypes.c_int, [_V, _V, _V]),
    "vsaogm_reserve": (ctypes.c_int, [_V, ctypes.c_int64]),
    "vsaogm_get_memory": (ctypes.c_int, [_V, _V, _V]),
    "vsaogm_set_memory": (ctypes.c_int, [_V, _V, _V]),
    "vsaogm_fuse": (ctypes.c_int, [_V, _V, _V]),
    "vsaogm_get_axis_frequencies": (ctypes.c_int, [_V, _V, _V]),
    "vsaogm_get_shape": (ctypes.c_int, [_V, _V, _V]),
    "vsaogm_status": (ctypes.c_int, [_V, _V]),
    "vsaogm_set_timing": (ctypes.c_int, [_V, ctypes.c_int]),
    "vsaogm_stage_times": (ctypes.c_int, [_V, _V, _V, ctypes.c_int]),
    "vsaogm_last_error": (ctypes.c_char_p, []),
    "vsaogm_device_bytes": (ctypes.c_int, [_V]),
    "vsaogm_batch_create": (ctypes.c_int, [_V, ctypes.c_int32, _V]),
    "vsaogm_batch_destroy": (ctypes.c_int, [_V]),
    "vsaogm_batch_step": (ctypes.c_int, [_V, _V, _V, _V, _V, _V, _V, ctypes.c_int32, _V]),
    "vsaogm_batch_capture": (ctypes.c_int, [_V, _V, _V, _V, _V, _V, _V, ctypes.c_int32, _V]),
    "vsaogm_batch_replay": (ctypes.c_int, [_V, _V]),
    "vsaogm_batch_autotune": (ctypes.c_int, [_V, _V, _V, _V, _V, _V, _V, _V, _V, _V]),
    "vsaogm_batch_set_timing": (ctypes.c_int, [_V, ctypes.c_int32]),
    "vsaogm_batch_stage_times": (ctypes.c_int, [_V, _V, _V, ctypes.c_int32]),
}


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() or "
                                   "python paper_2408_09066_gb300/build.py")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc: int):
    if rc != OK:
        raise VsaogmError(rc, lib().vsaogm_last_error().decode())


def device_bytes() -> int:
    """Device memory the library holds right now (vsaogm_device_bytes)."""
    v = ctypes.c_int64()
    _check(lib().vsaogm_device_bytes(ctypes.byref(v)))
    return int(v.value)


def default_config(**kw) -> Config:
    c = Config()
    lib().vsaogm_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise AttributeError(k)
        setattr(c, k, v)
    return c


def _stream(stream):
    import torch
    if stream is None:
        return _V(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _V(stream)
    return _V(stream.cuda_stream)


def _dev(t, dtype, shape=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return _V(t.data_ptr())


class Map:
    """One occupancy map: memories, axis frequencies and scratch on the device."""

    def __init__(self, config: Config | None = None, **kw):
        self.config = config if config is not None else default_config(**kw)
        h = _V()
        _check(lib().vsaogm_create(ctypes.byref(self.config), ctypes.byref(h)))
        self._h = h
        self.W, self.H, self.D = self.config.grid_w, self.config.grid_h, self.config.D
        T, S = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().vsaogm_get_shape(self._h, ctypes.byref(T), ctypes.byref(S)))
        self.n_tiles, self.n_memories = T.value, S.value

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().vsaogm_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- hot path ---------------------------------------------------------
    def reset(self, stream=None):
        _check(lib().vsaogm_reset(self._h, _stream(stream)))

    def encode_bundle(self, xy, labels, stream=None):
        import torch
        n = labels.shape[0]
        _check(lib().vsaogm_encode_bundle(self._h, _dev(xy, torch.float32, (n, 2), "xy"),
                                          _dev(labels, torch.uint8, (n,), "labels"), n,
                                          _stream(stream)))

    def encode_bundle_noalloc(self, xy, labels, stream=None):
        """Like encode_bundle, without allocating (static library scratch; at
        most 262144 points per call; calls must not overlap on the GPU)."""
        import torch
        n = labels.shape[0]
        _check(lib().vsaogm_encode_bundle_noalloc(self._h, _dev(xy, torch.float32, (n, 2), "xy"),
                                                  _dev(labels, torch.uint8, (n,), "labels"), n,
                                                  _stream(stream)))

    def decode(self, heat, stream=None):
        import torch
        _check(lib().vsaogm_decode(self._h, _dev(heat, torch.float32, (2, self.H, self.W), "heat"),
                                   _stream(stream)))

    def entropy(self, heat, occ, ogm=None, cls=None, stream=None):
        import torch
        hw = (self.H, self.W)
        _check(lib().vsaogm_entropy(
            self._h, _dev(heat, torch.float32, (2,) + hw, "heat"), _dev(occ, torch.float32, hw, "occ"),
            _dev(ogm, torch.float32, hw, "ogm") if ogm is not None else None,
            _dev(cls, torch.uint8, hw, "cls") if cls is not None else None, _stream(stream)))

    def query(self, heat, occ, ogm=None, cls=None, stream=None):
        import torch
        hw = (self.H, self.W)
        _check(lib().vsaogm_query(
            self._h, _dev(heat, torch.float32, (2,) + hw, "heat"), _dev(occ, torch.float32, hw, "occ"),
            _dev(ogm, torch.float32, hw, "ogm") if ogm is not None else None,
            _dev(cls, torch.uint8, hw, "cls") if cls is not None else None, _stream(stream)))

    def window_scratch(self, x0: int, y0: int, w: int, h: int) -> int:
        """Floats of heat scratch query_window needs for that window."""
        v = ctypes.c_int64()
        _check(lib().vsaogm_window_scratch(self._h, x0, y0, w, h, ctypes.byref(v)))
        return v.value

    def query_window(self, x0: int, y0: int, w: int, h: int, heat, occ, ogm=None, cls=None,
                     stream=None):
        """Occupancy of the window [x0, x0+w) x [y0, y0+h) into occ [h][w]; heat is
        scratch of at least window_scratch(...) floats."""
        import torch
        need = self.window_scratch(x0, y0, w, h)
        if not (isinstance(heat, torch.Tensor) and heat.is_cuda and heat.dtype == torch.float32
                and heat.is_contiguous() and heat.numel() >= need):
            raise ValueError(f"heat must be a contiguous CUDA float32 tensor of >= {need} elements")
        _check(lib().vsaogm_query_window(
            self._h, x0, y0, w, h, _V(heat.data_ptr()), _dev(occ, torch.float32, (h, w), "occ"),
            _dev(ogm, torch.float32, (h, w), "ogm") if ogm is not None else None,
            _dev(cls, torch.uint8, (h, w), "cls") if cls is not None else None, _stream(stream)))

    def decode_window(self, x0: int, y0: int, w: int, h: int, heat, stream=None):
        """P_hat of both classes for the window [x0, x0+w) x [y0, y0+h) into heat [2][h][w]."""
        import torch
        _check(lib().vsaogm_decode_window(self._h, x0, y0, w, h,
                                          _dev(heat, torch.float32, (2, h, w), "heat"),
                                          _stream(stream)))

    def update_query_host(self, xy: np.ndarray, labels: np.ndarray, occ: np.ndarray, stream=None):
        """Host arrays in and out: xy float32 [n][2], labels uint8 [n], occ float32 [H][W]."""
        for a, dt in ((xy, np.float32), (labels, np.uint8), (occ, np.float32)):
            if a.dtype != dt or not a.flags.c_contiguous:
                raise TypeError("host arrays must be C-contiguous with the documented dtypes")
        if occ.shape != (self.H, self.W) or xy.shape != (len(labels), 2):
            raise ValueError("bad host array shapes")
        _check(lib().vsaogm_update_query_host(self._h, _V(xy.ctypes.data), _V(labels.ctypes.data),
                                              len(labels), _V(occ.ctypes.data), _stream(stream)))

    # -- state --------------------------------------------------------------
    def reserve(self, max_points: int):
        """Grow scratch now so that later calls with up to max_points points
        (and any query) allocate nothing."""
        _check(lib().vsaogm_reserve(self._h, int(max_points)))

    def rejected(self, stream=None) -> int:
        v = ctypes.c_int64()
        _check(lib().vsaogm_rejected(self._h, ctypes.byref(v), _stream(stream)))
        return v.value

    def get_memory(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.n_memories, self.D), dtype=torch.complex64, device="cuda")
        _check(lib().vsaogm_get_memory(self._h, _dev(out, torch.complex64,
                                                     (self.n_memories, self.D), "omega"),
                                       _stream(stream)))
        return out

    def set_memory(self, omega, stream=None):
        import torch
        _check(lib().vsaogm_set_memory(self._h, _dev(omega, torch.complex64,
                                                     (self.n_memories, self.D), "omega"),
                                       _stream(stream)))

    def fuse(self, other: "Map", stream=None):
        _check(lib().vsaogm_fuse(self._h, other._h, _stream(stream)))

    def status(self, stream=None):
        """Raises VsaogmError(E_TIMEOUT) if a kernel gave up on a bounded wait."""
        _check(lib().vsaogm_status(self._h, _stream(stream)))

    def set_timing(self, enable: bool = True):
        _check(lib().vsaogm_set_timing(self._h, 1 if enable else 0))

    def stage_times(self, reset: bool = False):
        """{stage: (milliseconds, kernel launches)} accumulated since the last reset."""
        ms = (ctypes.c_double * len(STAGES))()
        cnt = (ctypes.c_int64 * len(STAGES))()
        _check(lib().vsaogm_stage_times(self._h, ms, cnt, 1 if reset else 0))
        return {s: (ms[i], cnt[i]) for i, s in enumerate(STAGES)}

    def axis_frequencies(self):
        nx = np.empty(self.D, np.float32)
        ny = np.empty(self.D, np.float32)
        _check(lib().vsaogm_get_axis_frequencies(self._h, _V(nx.ctypes.data), _V(ny.ctypes.data)))
        return nx, ny


def _ptrs(values):
    arr = (_V * len(values))()
    for i, v in enumerate(values):
        arr[i] = v
    return arr


class Batch:
    """Up to MAX_BATCH maps stepped together: one launch per stage for all.

    The batch refers to its maps (keep them alive).  Per-map inputs and
    outputs are lists in the order of `maps`: xy (n_i, 2) float32, labels
    (n_i,) uint8, heat (2, H_i, W_i), occ and ogm (H_i, W_i) float32, all
    CUDA tensors.
    """

    def __init__(self, maps):
        self.maps = list(maps)
        h = _V()
        handles = _ptrs([m.handle for m in self.maps])
        _check(lib().vsaogm_batch_create(handles, len(self.maps), ctypes.byref(h)))
        self._h = h
        self._keep = None

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().vsaogm_batch_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _args(self, xy, labels, heat, occ, ogm):
        import torch
        k = len(self.maps)
        if not (len(xy) == len(labels) == len(heat) == len(occ) == k) or (
                ogm is not None and len(ogm) != k):
            raise ValueError(f"every per-map list needs {k} entries")
        n = (ctypes.c_int64 * k)()
        xs, ls, hs, os_, gs = [], [], [], [], []
        for i, m in enumerate(self.maps):
            n[i] = labels[i].shape[0]
            xs.append(_dev(xy[i], torch.float32, (n[i], 2), "xy"))
            ls.append(_dev(labels[i], torch.uint8, (n[i],), "labels"))
            hs.append(_dev(heat[i], torch.float32, (2, m.H, m.W), "heat"))
            os_.append(_dev(occ[i], torch.float32, (m.H, m.W), "occ"))
            if ogm is not None:
                gs.append(_dev(ogm[i], torch.float32, (m.H, m.W), "ogm"))
        return (_ptrs(xs), _ptrs(ls), n, _ptrs(hs), _ptrs(os_),
                _ptrs(gs) if ogm is not None else None)

    def step(self, xy, labels, heat, occ, ogm=None, reset=True, stream=None):
        a = self._args(xy, labels, heat, occ, ogm)
        _check(lib().vsaogm_batch_step(self._h, *a, 1 if reset else 0, _stream(stream)))

    def capture(self, xy, labels, heat, occ, ogm=None, reset=True, stream=None):
        """Runs one step and captures it in a CUDA graph; replay() re-runs it
        on the same buffers (refill the inputs in place, same point counts)."""
        a = self._args(xy, labels, heat, occ, ogm)
        self._keep = (xy, labels, heat, occ, ogm)  # the graph holds their addresses
        _check(lib().vsaogm_batch_capture(self._h, *a, 1 if reset else 0, _stream(stream)))

    def replay(self, stream=None):
        _check(lib().vsaogm_batch_replay(self._h, _stream(stream)))

    def autotune(self, xy, labels, heat, occ, stream=None):
        """Times candidate shapes on these inputs, keeps the fastest and
        returns it as a dict (overwrites the maps' memories)."""
        a = self._args(xy, labels, heat, occ, None)
        pw, ipc, dw = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().vsaogm_batch_autotune(self._h, *a[:5], _stream(stream), ctypes.byref(pw),
                                           ctypes.byref(ipc), ctypes.byref(dw)))
        return {"poly_warps": pw.value, "items_per_cta": ipc.value, "decode_waves": dw.value}

    def set_timing(self, enable: bool = True):
        _check(lib().vsaogm_batch_set_timing(self._h, 1 if enable else 0))

    def stage_times(self, reset: bool = False):
        """{stage: (milliseconds, kernel launches)} accumulated since the last reset."""
        ms = (ctypes.c_double * len(STAGES))()
        cnt = (ctypes.c_int64 * len(STAGES))()
        _check(lib().vsaogm_batch_stage_times(self._h, ms, cnt, 1 if reset else 0))
        return {s: (ms[i], cnt[i]) for i, s in enumerate(STAGES)}

    def status(self, stream=None):
        for m in self.maps:
            m.status(stream)
