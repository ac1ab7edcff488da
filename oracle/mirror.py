"""NumPy restatement of the oracle for tiny inputs (test infrastructure only).

Written separately from ``oracle.c`` from the same definitions, so that a slip
in one of the two shows up as a disagreement.  Vectorised, double precision,
no blocking.  Used only by the oracle's own pin tests.
"""
from __future__ import annotations

import numpy as np

_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64_at(seed: int, i: int) -> int:
    """SplitMix64 (Steele, Lea, Flood 2014), output number i of the stream."""
    z = (seed + (i + 1) * _GAMMA) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def draw_nu(seed: int, D: int, length_scale: float):
    ux = np.array([(splitmix64_at(seed, 2 * k) >> 11) for k in range(D)], np.float64) / 2.0**53
    uy = np.array([(splitmix64_at(seed, 2 * k + 1) >> 11) for k in range(D)], np.float64) / 2.0**53
    s = 0.5 / float(length_scale)
    return ((2.0 * ux - 1.0) * s).astype(np.float32), ((2.0 * uy - 1.0) * s).astype(np.float32)


def centres(g):
    """Tile centres mu, shape [T][2], tile index beta = by * tiles_x + bx."""
    tw = g.W * g.res / g.tiles_x
    th = g.H * g.res / g.tiles_y
    by, bx = np.meshgrid(np.arange(g.tiles_y), np.arange(g.tiles_x), indexing="ij")
    return np.stack([g.x_min + (bx.ravel() + 0.5) * tw, g.y_min + (by.ravel() + 0.5) * th], 1)


def assign(g, xy):
    mu = centres(g)
    p = np.asarray(xy, np.float64).reshape(-1, 2)
    d2 = ((p[:, None, :] - mu[None, :, :]) ** 2).sum(-1)
    beta = np.argmin(d2, axis=1)  # first minimum wins, as in Algorithm 1
    # where the two smallest FP64 distances are (nearly) equal, rounding may have
    # made the tie: decide those points with exact rational distances
    srt = np.sort(d2, axis=1)
    close = np.nonzero(srt[:, 1] - srt[:, 0] <= 1e-9 * np.maximum(srt[:, 1], 1e-300))[0] \
        if d2.shape[1] > 1 else []
    if len(close):
        from fractions import Fraction as F
        tw = F(g.W) * F(g.res) / g.tiles_x
        th = F(g.H) * F(g.res) / g.tiles_y
        cen = [(F(g.x_min) + (bx + F(1, 2)) * tw, F(g.y_min) + (by + F(1, 2)) * th)
               for by in range(g.tiles_y) for bx in range(g.tiles_x)]
        for q in close:
            x, y = F(float(p[q, 0])), F(float(p[q, 1]))
            d = [(x - cx) ** 2 + (y - cy) ** 2 for cx, cy in cen]
            beta[q] = d.index(min(d))
    return beta


def memories(g, nu_x, nu_y, xy, labels, frame="tile"):
    p = np.asarray(xy, np.float64).reshape(-1, 2)
    beta = assign(g, p)
    if frame == "tile":
        p = p - centres(g)[beta]
    nu = np.stack([np.asarray(nu_x, np.float64), np.asarray(nu_y, np.float64)], 0)  # [2][D]
    phi = np.exp(2j * np.pi * (p @ nu))  # [n][D]
    om = np.zeros((2 * g.T, len(nu_x)), np.complex128)
    np.add.at(om, 2 * beta + np.asarray(labels, np.int64), phi)
    return om


def cell_centres(g):
    j, i = np.meshgrid(np.arange(g.H), np.arange(g.W), indexing="ij")
    return np.stack([g.x_min + (i.ravel() + 0.5) * g.res, g.y_min + (j.ravel() + 0.5) * g.res], 1)


def decode_map(g, nu_x, nu_y, omega, frame="tile"):
    c = cell_centres(g)
    beta = assign(g, c)
    if frame == "tile":
        c = c - centres(g)[beta]
    nu = np.stack([np.asarray(nu_x, np.float64), np.asarray(nu_y, np.float64)], 0)
    phi = np.exp(2j * np.pi * (c @ nu))  # [cells][D]
    nrm = np.linalg.norm(omega, axis=1)
    P = np.zeros((2, g.H * g.W))
    for psi in range(2):
        w = omega[2 * beta + psi]  # [cells][D]
        n = nrm[2 * beta + psi]
        val = np.real((np.conj(w) * phi).sum(1))
        P[psi] = np.where(n > 0, val / np.where(n > 0, n, 1.0), 0.0)
    return P.reshape(2, g.H, g.W)


def nonlinear(P):
    out = np.zeros_like(P)
    mx = P.reshape(2, -1).max(1)
    for c in range(2):
        if mx[c] > 0:
            out[c] = (P[c] / mx[c]) ** 2
    return out, mx


def entropy(Ph, r):
    H, W = Ph.shape
    with np.errstate(divide="ignore", invalid="ignore"):
        h = np.where(Ph > 0, -Ph * np.log(np.where(Ph > 0, Ph, 1.0)), 0.0)
    out = np.zeros_like(Ph)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            if dx * dx + dy * dy > r * r:
                continue
            # out[y, x] += h[y + dy, x + dx] where in range
            ys = slice(max(0, -dy), min(H, H - dy))
            xs = slice(max(0, -dx), min(W, W - dx))
            yd = slice(max(0, dy), min(H, H + dy))
            xd = slice(max(0, dx), min(W, W + dx))
            out[ys, xs] += h[yd, xd]
    return out


def softmax_psd(H0, H1):
    e = np.exp(np.stack([H0, H1]) - np.maximum(H0, H1)[None])
    pr = e / e.sum(0, keepdims=True)
    return pr[1], pr[0], pr[1] - pr[0]
