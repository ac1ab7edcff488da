"""FP64 CPU oracle for the VSA-OGM hot path (arXiv 2408.09066).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library in ``paper_2408_09066_gb300``; neither imports the other.

The arithmetic lives in ``oracle.c`` (plain C, double precision, each function
citing the equation or algorithm it follows); this module builds it with gcc and
marshals NumPy arrays through ctypes.  ``oracle.mirror`` restates the same
definitions in NumPy for tiny inputs, as an independent cross-check.

Every function here is pinned by ``tests/test_oracle_pins.py`` against what the
paper and the mathematics fix (self-similarity, linearity, the sinc kernel, brute
force on tiny inputs, closed forms of the entropy stencil, softmax identities,
the paper's model-size table and the published SplitMix64 outputs).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def compile_source(src: str, out: str) -> str:
    """Compile the C source ``src`` into the shared library ``out`` with the
    oracle's flags (gcc, OpenMP, no FP contraction)."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` unless it is up to date."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    return compile_source(_SRC, _LIB)


class _Grid(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("H", ctypes.c_int32), ("res", ctypes.c_double),
                ("x_min", ctypes.c_double), ("y_min", ctypes.c_double),
                ("tiles_x", ctypes.c_int32), ("tiles_y", ctypes.c_int32)]


@dataclasses.dataclass(frozen=True)
class Grid:
    """Map geometry: W x H cells of edge ``res`` metres from (x_min, y_min),
    split into tiles_x x tiles_y evenly sized tiles (delta per axis)."""
    W: int
    H: int
    res: float
    x_min: float
    y_min: float
    tiles_x: int = 1
    tiles_y: int = 1

    @property
    def T(self) -> int:
        return self.tiles_x * self.tiles_y

    def c(self) -> _Grid:
        return _Grid(self.W, self.H, self.res, self.x_min, self.y_min, self.tiles_x, self.tiles_y)


def bind(path: str):
    """Load a library built from ``oracle.c`` (or a test's altered copy of it)
    and declare the C signatures of its entry points."""
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    lib.orc_num_threads.restype = ctypes.c_int32
    lib.orc_num_threads.argtypes = []
    lib.orc_splitmix64_at.restype = ctypes.c_uint64
    lib.orc_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    lib.orc_draw_nu.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_double,
                                ctypes.c_void_p, ctypes.c_void_p]
    lib.orc_tile_of.restype = ctypes.c_int32
    lib.orc_tile_of.argtypes = [P(_Grid), ctypes.c_double, ctypes.c_double]
    lib.orc_tile_centre.argtypes = [P(_Grid), ctypes.c_int32, P(ctypes.c_double),
                                    P(ctypes.c_double)]
    lib.orc_assign.argtypes = [P(_Grid), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    lib.orc_memories.restype = ctypes.c_int32
    lib.orc_memories.argtypes = [P(_Grid), ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                 ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                 ctypes.c_void_p, ctypes.c_void_p]
    lib.orc_norms.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                              ctypes.c_void_p]
    lib.orc_decode_cells.argtypes = [P(_Grid), ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                     ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                     ctypes.c_void_p]
    lib.orc_decode_map.argtypes = [P(_Grid), ctypes.c_int32, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.c_void_p, ctypes.c_void_p]
    lib.orc_direct_cells.argtypes = [P(_Grid), ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.orc_nonlinear.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_void_p]
    lib.orc_entropy.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                ctypes.c_int32, ctypes.c_void_p]
    lib.orc_softmax_psd.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.orc_classify_f32.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_float,
                                     ctypes.c_void_p]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = bind(_LIB)
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _frame(frame: str) -> int:
    if frame not in ("global", "tile"):
        raise ValueError("frame must be 'global' or 'tile'")
    return 0 if frame == "global" else 1


# --------------------------------------------------------------------------
def num_threads() -> int:
    """Threads the oracle's parallel loops use."""
    return int(_load().orc_num_threads())


def splitmix64_at(seed: int, i: int) -> int:
    """Output number ``i`` (0-based) of the SplitMix64 stream seeded with ``seed``."""
    return int(_load().orc_splitmix64_at(seed, i))


def draw_nu(seed: int, D: int, length_scale: float):
    """Axis frequencies (cycles per metre, float32), uniform on (-1/2l, 1/2l)."""
    nx = np.empty(D, np.float32)
    ny = np.empty(D, np.float32)
    _load().orc_draw_nu(seed, D, float(length_scale), _ptr(nx), _ptr(ny))
    return nx, ny


def tile_of(g: Grid, x: float, y: float) -> int:
    """Algorithm 1: index of the nearest tile centre (first minimum wins)."""
    return int(_load().orc_tile_of(ctypes.byref(g.c()), float(x), float(y)))


def tile_centre(g: Grid, beta: int):
    cx, cy = ctypes.c_double(), ctypes.c_double()
    _load().orc_tile_centre(ctypes.byref(g.c()), beta, ctypes.byref(cx), ctypes.byref(cy))
    return cx.value, cy.value


def _exact_tile(g: Grid, x: Fraction, y: Fraction) -> int:
    """Algorithm 1's argmin of the L2 distance in exact rational arithmetic."""
    tw = Fraction(g.W) * Fraction(g.res) / g.tiles_x
    th = Fraction(g.H) * Fraction(g.res) / g.tiles_y
    best, bd = 0, None
    for by in range(g.tiles_y):
        for bx in range(g.tiles_x):
            cx = Fraction(g.x_min) + (bx + Fraction(1, 2)) * tw
            cy = Fraction(g.y_min) + (by + Fraction(1, 2)) * th
            d = (x - cx) ** 2 + (y - cy) ** 2
            if bd is None or d < bd:
                best, bd = by * g.tiles_x + bx, d
    return best


def _near_boundary(g: Grid, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Coordinates within 1e-9 (relative) of a line halfway between adjacent tile
    centres, where rounding of FP64 distances could invert Algorithm 1's argmin."""
    mask = np.zeros(len(x), bool)
    for lo, cells, tiles, v in ((g.x_min, g.W, g.tiles_x, x), (g.y_min, g.H, g.tiles_y, y)):
        t = cells * g.res / tiles
        for a in range(1, tiles):
            b = lo + a * t
            mask |= np.abs(v - b) <= 1e-9 * max(1.0, abs(b), abs(t))
    return mask


def assign(g: Grid, xy: np.ndarray) -> np.ndarray:
    """Algorithm 1: tile of each point.  FP64 distances decide, except for points
    near a tile boundary, which are decided in exact rational arithmetic (FP64
    rounding can make a point 1e-16 m off a boundary look like a tie)."""
    xy = np.ascontiguousarray(xy, np.float32).reshape(-1, 2)
    out = np.empty(len(xy), np.int32)
    _load().orc_assign(ctypes.byref(g.c()), _ptr(xy), len(xy), _ptr(out))
    near = np.nonzero(_near_boundary(g, xy[:, 0].astype(np.float64), xy[:, 1].astype(np.float64)))[0]
    for p in near:
        out[p] = _exact_tile(g, Fraction(float(xy[p, 0])), Fraction(float(xy[p, 1])))
    return out


def assign_cells(g: Grid, cells: np.ndarray) -> np.ndarray:
    """Tile of each cell (i, j): Algorithm 1's rule at the cell centre
    (x_min + (i + 1/2) res, y_min + (j + 1/2) res), exact near boundaries."""
    cells = np.ascontiguousarray(cells, np.int32).reshape(-1, 2)
    out = np.empty(len(cells), np.int32)
    cx = g.x_min + (cells[:, 0] + 0.5) * g.res
    cy = g.y_min + (cells[:, 1] + 0.5) * g.res
    lib = _load()
    gc = g.c()
    for q in range(len(cells)):
        out[q] = lib.orc_tile_of(ctypes.byref(gc), float(cx[q]), float(cy[q]))
    near = np.nonzero(_near_boundary(g, cx, cy))[0]
    for q in near:
        x = Fraction(g.x_min) + (int(cells[q, 0]) + Fraction(1, 2)) * Fraction(g.res)
        y = Fraction(g.y_min) + (int(cells[q, 1]) + Fraction(1, 2)) * Fraction(g.res)
        out[q] = _exact_tile(g, x, y)
    return out


def memories(g: Grid, nu_x, nu_y, xy, labels, frame: str = "tile", ks=None) -> np.ndarray:
    """Tile memories omega, complex128 [2T][D] (or [2T][len(ks)]), index 2*beta + psi."""
    nu_x = np.ascontiguousarray(nu_x, np.float32)
    nu_y = np.ascontiguousarray(nu_y, np.float32)
    xy = np.ascontiguousarray(xy, np.float32).reshape(-1, 2)
    labels = np.ascontiguousarray(labels, np.uint8)
    D = len(nu_x)
    if ks is None:
        nk, kp = D, None
    else:
        ks = np.ascontiguousarray(ks, np.int32)
        nk, kp = len(ks), _ptr(ks)
    out = np.empty((2 * g.T, nk, 2), np.float64)
    if np.any(labels > 1):
        raise ValueError("labels must be 0 or 1")
    beta = assign(g, xy)
    rc = _load().orc_memories(ctypes.byref(g.c()), D, _ptr(nu_x), _ptr(nu_y), _ptr(xy),
                              _ptr(labels), len(xy), _frame(frame), kp, nk, _ptr(beta),
                              _ptr(out))
    if rc != 0:
        raise ValueError("labels must be 0 or 1")
    return out[..., 0] + 1j * out[..., 1]


def _as_ri(omega: np.ndarray) -> np.ndarray:
    o = np.ascontiguousarray(omega, np.complex128)
    return np.ascontiguousarray(np.stack([o.real, o.imag], -1))


def norms(omega: np.ndarray) -> np.ndarray:
    ri = _as_ri(omega)
    out = np.empty(ri.shape[0], np.float64)
    _load().orc_norms(_ptr(ri), ri.shape[0], ri.shape[1], _ptr(out))
    return out


def decode_cells(g: Grid, nu_x, nu_y, omega, cells, frame: str = "tile") -> np.ndarray:
    """Eq. loc-query on normalised memories at the given (i, j) cells -> [ncells][2]."""
    ri = _as_ri(omega)
    cells = np.ascontiguousarray(cells, np.int32).reshape(-1, 2)
    out = np.empty((len(cells), 2), np.float64)
    _load().orc_decode_cells(ctypes.byref(g.c()), ri.shape[1],
                             _ptr(np.ascontiguousarray(nu_x, np.float32)),
                             _ptr(np.ascontiguousarray(nu_y, np.float32)), _ptr(ri),
                             _frame(frame), _ptr(cells), len(cells),
                             _ptr(assign_cells(g, cells)), _ptr(out))
    return out


def _all_cells(g: Grid) -> np.ndarray:
    j, i = np.meshgrid(np.arange(g.H), np.arange(g.W), indexing="ij")
    return np.ascontiguousarray(np.stack([i.ravel(), j.ravel()], 1), np.int32)


def decode_map(g: Grid, nu_x, nu_y, omega, frame: str = "tile") -> np.ndarray:
    """Eq. loc-query over every cell -> P float64 [2][H][W]."""
    ri = _as_ri(omega)
    out = np.empty((2, g.H, g.W), np.float64)
    _load().orc_decode_map(ctypes.byref(g.c()), ri.shape[1],
                           _ptr(np.ascontiguousarray(nu_x, np.float32)),
                           _ptr(np.ascontiguousarray(nu_y, np.float32)), _ptr(ri),
                           _frame(frame), _ptr(assign_cells(g, _all_cells(g))), _ptr(out))
    return out


def direct_cells(g: Grid, nu_x, nu_y, xy, labels, cells) -> np.ndarray:
    """Direct per-cell sum over points (no memory vectors), O(n^2 D) -> [ncells][2]."""
    xy = np.ascontiguousarray(xy, np.float32).reshape(-1, 2)
    labels = np.ascontiguousarray(labels, np.uint8)
    cells = np.ascontiguousarray(cells, np.int32).reshape(-1, 2)
    out = np.empty((len(cells), 2), np.float64)
    _load().orc_direct_cells(ctypes.byref(g.c()), len(nu_x),
                             _ptr(np.ascontiguousarray(nu_x, np.float32)),
                             _ptr(np.ascontiguousarray(nu_y, np.float32)), _ptr(xy),
                             _ptr(labels), len(xy), _ptr(cells), len(cells),
                             _ptr(assign(g, xy)), _ptr(assign_cells(g, cells)), _ptr(out))
    return out


def nonlinear(P: np.ndarray):
    """Eq. non-linearities per class over the whole map -> (P_hat, maxima[2])."""
    P = np.ascontiguousarray(P, np.float64)
    ncell = P[0].size
    Ph = np.empty_like(P)
    mx = np.empty(2, np.float64)
    _load().orc_nonlinear(_ptr(P), ncell, _ptr(Ph), _ptr(mx))
    return Ph, mx


def entropy(Phat_c: np.ndarray, r: int) -> np.ndarray:
    """Algorithm 2 / Eq. entropy-mask for one class map [H][W] and disk radius r."""
    Phat_c = np.ascontiguousarray(Phat_c, np.float64)
    H, W = Phat_c.shape
    out = np.empty_like(Phat_c)
    _load().orc_entropy(_ptr(Phat_c), W, H, int(r), _ptr(out))
    return out


def softmax_psd(H0: np.ndarray, H1: np.ndarray):
    """Eq. softmax and Eq. psd -> (Pr1, Pr0, OGM)."""
    H0 = np.ascontiguousarray(H0, np.float64)
    H1 = np.ascontiguousarray(H1, np.float64)
    pr1, pr0, ogm = (np.empty_like(H0) for _ in range(3))
    _load().orc_softmax_psd(_ptr(H0), _ptr(H1), H0.size, _ptr(pr1), _ptr(pr0), _ptr(ogm))
    return pr1, pr0, ogm


def classify_f32(ogm_f32: np.ndarray, rho: float) -> np.ndarray:
    """Eq. classification decided in float32: 1 (occupied) iff OGM >= rho."""
    o = np.ascontiguousarray(ogm_f32, np.float32)
    out = np.empty(o.shape, np.uint8)
    _load().orc_classify_f32(_ptr(o), o.size, np.float32(rho), _ptr(out))
    return out


def decode_variant(P: np.ndarray, norm: bool, square: bool, act: str, r_occ: int, r_emp: int):
    """The decoding ablation of Sec. IV-D1, P_hat = f_ACT(f_NL(f_N(P))), followed by
    Eq. softmax and Eq. psd.  f_N divides each class map by its maximum (0 if the
    maximum is not positive), f_NL squares, f_ACT is 'entropy' (Algorithm 2),
    'relu', 'tanh', 'sigmoid' or 'none'.  Returns (Pr1, Pr0, OGM)."""
    v = np.array(P, np.float64)
    if norm:
        for c in range(2):
            m = v[c].max()
            v[c] = v[c] / m if m > 0 else 0.0
    if square:
        v = v * v
    if act == "entropy":
        a0, a1 = entropy(v[0], r_emp), entropy(v[1], r_occ)
    elif act == "relu":
        a0, a1 = np.maximum(v[0], 0.0), np.maximum(v[1], 0.0)
    elif act == "tanh":
        a0, a1 = np.tanh(v[0]), np.tanh(v[1])
    elif act == "sigmoid":
        a0, a1 = 1.0 / (1.0 + np.exp(-v[0])), 1.0 / (1.0 + np.exp(-v[1]))
    elif act == "none":
        a0, a1 = v[0], v[1]
    else:
        raise ValueError(act)
    return softmax_psd(a0, a1)


def query_window(g: Grid, nu_x, nu_y, omega, x0: int, y0: int, w: int, h: int, r_occ: int,
                 r_emp: int, frame: str = "tile") -> dict:
    """A local map query (reading of the paper for windows): the window grown by
    R = max(r_occ, r_emp) cells and clipped to the map is decoded (Eq. loc-query),
    Eq. non-linearities normalises by the maximum over that region, Algorithm 2
    runs on the region (zero outside it), then Eqs. softmax and psd.  Returns the
    window's Pr(psi=1), OGM and the region's maxima."""
    R = max(r_occ, r_emp)
    rx0, ry0 = max(0, x0 - R), max(0, y0 - R)
    rx1, ry1 = min(g.W, x0 + w + R), min(g.H, y0 + h + R)
    jj, ii = np.meshgrid(np.arange(ry0, ry1), np.arange(rx0, rx1), indexing="ij")
    cells = np.stack([ii.ravel(), jj.ravel()], 1)
    P = decode_cells(g, nu_x, nu_y, omega, cells, frame).T.reshape(2, ry1 - ry0, rx1 - rx0)
    Ph, mx = nonlinear(P)
    H0 = entropy(Ph[0], r_emp)
    H1 = entropy(Ph[1], r_occ)
    pr1, pr0, ogm = softmax_psd(H0, H1)
    sy, sx = slice(y0 - ry0, y0 - ry0 + h), slice(x0 - rx0, x0 - rx0 + w)
    return dict(pr1=pr1[sy, sx], ogm=ogm[sy, sx], maxima=mx, P=P)


def pipeline(g: Grid, nu_x, nu_y, xy, labels, r_occ: int, r_emp: int, rho: float = 0.0,
             frame: str = "tile") -> dict:
    """The whole hot path in the paper's order: memories -> P -> P_hat -> H -> Pr, OGM."""
    om = memories(g, nu_x, nu_y, xy, labels, frame)
    P = decode_map(g, nu_x, nu_y, om, frame)
    Ph, mx = nonlinear(P)
    H0 = entropy(Ph[0], r_emp)
    H1 = entropy(Ph[1], r_occ)
    pr1, pr0, ogm = softmax_psd(H0, H1)
    return dict(omega=om, P=P, Phat=Ph, maxima=mx, H0=H0, H1=H1, pr1=pr1, pr0=pr0, ogm=ogm,
                cls=classify_f32(ogm.astype(np.float32), rho))
