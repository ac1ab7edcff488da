"""Pins for the FP64 oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks it against a closed
form, a published value, a library routine, an exact (rational) computation or
an independent brute-force formulation, chosen so that a dropped term, a wrong
sign or index, or a transposed operand fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import Grid, mirror

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ----------------------------------------------------------------- generator
def test_splitmix64_published_outputs():
    """SplitMix64, seed 0: the reference implementation's first three outputs."""
    want = [int(r[0], 16) for r in _read_golden("splitmix64_seed0.txt")]
    assert [oracle.splitmix64_at(0, i) for i in range(3)] == want
    assert [mirror.splitmix64_at(0, i) for i in range(3)] == want


def test_axis_frequencies_uniform_on_band():
    """Initialization (Sec. III-B2) with theta ~ U(-pi, pi): nu ~ U(-1/2l, 1/2l)."""
    from scipy import stats
    l = 0.1
    nx, ny = oracle.draw_nu(7, 20000, l)
    assert nx.dtype == np.float32 and ny.dtype == np.float32
    assert np.all(np.abs(nx) < 0.5 / l) and np.all(np.abs(ny) < 0.5 / l)
    for v in (nx, ny):
        assert stats.kstest(v.astype(np.float64), stats.uniform(loc=-5.0, scale=10.0).cdf).pvalue > 1e-3
    assert not np.array_equal(nx, ny)
    # prefix-stable: a shorter draw is the head of a longer one
    sx, sy = oracle.draw_nu(7, 100, l)
    assert np.array_equal(sx, nx[:100]) and np.array_equal(sy, ny[:100])


# ------------------------------------------------------------------- tiling
def _exact_argmin(g, x, y):
    """Algorithm 1 in exact rational arithmetic: first nearest tile centre."""
    tw = Fraction(g.W) * Fraction(g.res) / g.tiles_x
    th = Fraction(g.H) * Fraction(g.res) / g.tiles_y
    best, bd = None, None
    for by in range(g.tiles_y):
        for bx in range(g.tiles_x):
            cx = Fraction(g.x_min) + (bx + Fraction(1, 2)) * tw
            cy = Fraction(g.y_min) + (by + Fraction(1, 2)) * th
            d = (Fraction(x) - cx) ** 2 + (Fraction(y) - cy) ** 2
            if bd is None or d < bd:
                best, bd = by * g.tiles_x + bx, d
    return best


def test_tile_assignment_exact_including_ties_and_outside():
    g = Grid(W=64, H=48, res=0.125, x_min=-4.0, y_min=-3.0, tiles_x=4, tiles_y=3)
    rng = np.random.default_rng(3)
    pts = rng.uniform([-6, -5], [6, 5], size=(300, 2)).astype(np.float32)
    # exact boundaries (x = -2, 0, 2 ; y = -1, 1) and corners: ties go to the lower tile
    bnd = np.array([[-2, 0.3], [0, 0.3], [2, 0.3], [0.1, -1], [0.1, 1], [0, 1], [2, -1],
                    [-4, -3], [4, 3], [-100, 50], [100, -50],
                    # a hair off a boundary: FP64 distances to the two centres round to a tie
                    [5.4526174e-17, 0.3], [-3.0377352e-16, 0.7], [1e-38, -0.5], [-0.0, 0.2]],
                   np.float32)
    pts = np.concatenate([pts, bnd])
    got = oracle.assign(g, pts)
    want = [_exact_argmin(g, float(x), float(y)) for x, y in pts]
    assert got.tolist() == want
    assert mirror.assign(g, pts).tolist() == want
    # a tie at x = 0 between bx = 1 and bx = 2 resolves to bx = 1
    assert oracle.tile_of(g, 0.0, 0.3) % g.tiles_x == 1


def test_cell_assignment_exact_including_centres_on_boundaries():
    """Algorithm 1's rule at cell centres x_min + (i + 1/2) res, decided against an
    exact rational argmin: with 50 cells over 4 tiles a tile is 12.5 cells wide, so
    the centres of cells 12 and 37 lie exactly on a boundary and go to the lower
    tile; the decode's cell-to-tile map (shared by the memory and direct forms)
    is pinned here rather than through them."""
    g = Grid(W=50, H=30, res=0.1, x_min=-2.5, y_min=-1.5, tiles_x=4, tiles_y=3)
    cells = np.array([(i, j) for j in range(g.H) for i in range(g.W)], np.int32)
    got = oracle.assign_cells(g, cells)
    tw = Fraction(g.W) * Fraction(g.res) / g.tiles_x
    th = Fraction(g.H) * Fraction(g.res) / g.tiles_y
    for (i, j), b in zip(cells, got):
        x = Fraction(g.x_min) + (int(i) + Fraction(1, 2)) * Fraction(g.res)
        y = Fraction(g.y_min) + (int(j) + Fraction(1, 2)) * Fraction(g.res)
        best, bd = None, None
        for by in range(g.tiles_y):
            for bx in range(g.tiles_x):
                cx = Fraction(g.x_min) + (bx + Fraction(1, 2)) * tw
                cy = Fraction(g.y_min) + (by + Fraction(1, 2)) * th
                d = (x - cx) ** 2 + (y - cy) ** 2
                if bd is None or d < bd:
                    best, bd = by * g.tiles_x + bx, d
        assert b == best, (i, j, b, best)
    row = got[:g.W]
    assert row[12] == 0 and row[13] == 1 and row[37] == 2 and row[38] == 3


# ---------------------------------------------------------- encode / bundle
def test_self_similarity_is_D_and_index_is_2beta_plus_psi():
    """|phi_k| = 1, so <phi(p), phi(p)> = D; the point lands in memory 2*beta + psi."""
    g = Grid(W=40, H=40, res=0.1, x_min=-2.0, y_min=-2.0, tiles_x=2, tiles_y=2)
    D = 512
    nx, ny = oracle.draw_nu(11, D, 0.1)
    for (x, y, beta) in [(-1.3, -0.7, 0), (1.1, -1.9, 1), (-0.2, 1.7, 2), (0.9, 0.4, 3)]:
        for psi in (0, 1):
            om = oracle.memories(g, nx, ny, np.array([[x, y]], np.float32), np.array([psi], np.uint8))
            nz = [m for m in range(2 * g.T) if np.any(om[m] != 0)]
            assert nz == [2 * beta + psi]
            assert np.allclose(np.abs(om[2 * beta + psi]), 1.0, atol=1e-14)
            assert abs(np.vdot(om[2 * beta + psi], om[2 * beta + psi]).real - D) < 1e-12 * D


@pytest.mark.parametrize("frame", ["global", "tile"])
def test_bundling_is_linear(frame):
    """Eq. bundling: memories of a union equal the sum of memories (also Algorithm 3)."""
    g = Grid(W=32, H=32, res=0.1, x_min=-1.6, y_min=-1.6, tiles_x=2, tiles_y=2)
    nx, ny = oracle.draw_nu(5, 256, 0.1)
    rng = np.random.default_rng(0)
    A = rng.uniform(-1.8, 1.8, (40, 2)).astype(np.float32)
    B = rng.uniform(-1.8, 1.8, (25, 2)).astype(np.float32)
    la = rng.integers(0, 2, 40).astype(np.uint8)
    lb = rng.integers(0, 2, 25).astype(np.uint8)
    oa = oracle.memories(g, nx, ny, A, la, frame)
    ob = oracle.memories(g, nx, ny, B, lb, frame)
    oab = oracle.memories(g, nx, ny, np.concatenate([A, B]), np.concatenate([la, lb]), frame)
    assert np.max(np.abs(oab - (oa + ob))) < 1e-11


def test_similarity_is_sinc_kernel():
    """Quasi-KDE (Sec. III-A, Fig. 1B): with theta ~ U(-pi/l, pi/l),
    E[Re<phi(p), phi(q)>] / D = sinc(dx/l) sinc(dy/l), sinc(u) = sin(pi u)/(pi u).
    The per-draw spread is <= 1/sqrt(2D); M independent draws are averaged."""
    l, D, M = 0.1, 16384, 8
    g = Grid(W=64, H=64, res=0.1, x_min=-3.2, y_min=-3.2)
    p = np.array([[0.013, -0.021]], np.float32)
    deltas = [(0.0, 0.0), (0.05, 0.0), (0.0, 0.05), (0.1, 0.0), (0.05, 0.03), (0.13, -0.07),
              (0.02, 0.2), (0.25, 0.25)]
    for dx, dy in deltas:
        q = (p + np.array([[dx, dy]], np.float32)).astype(np.float32)
        ddx = float(q[0, 0]) - float(p[0, 0])
        ddy = float(q[0, 1]) - float(p[0, 1])
        est = 0.0
        for s in range(M):
            nx, ny = oracle.draw_nu(1000 + s, D, l)
            wp = oracle.memories(g, nx, ny, p, np.array([1], np.uint8), "global")[1]
            wq = oracle.memories(g, nx, ny, q, np.array([1], np.uint8), "global")[1]
            est += np.vdot(wp, wq).real / D
        est /= M
        want = np.sinc(ddx / l) * np.sinc(ddy / l)
        assert abs(est - want) < 5.0 / math.sqrt(2 * D * M), (dx, dy, est, want)


# ------------------------------------------------------------------- decode
def _tiny_case(tiles, seed, D=64, n=20):
    tx, ty = tiles
    g = Grid(W=8, H=8, res=0.25, x_min=-1.0, y_min=-1.0, tiles_x=tx, tiles_y=ty)
    rng = np.random.default_rng(seed)
    xy = rng.uniform(-1.1, 1.1, (n, 2)).astype(np.float32)
    lab = rng.integers(0, 2, n).astype(np.uint8)
    nx, ny = oracle.draw_nu(seed, D, 0.3)
    return g, nx, ny, xy, lab


@pytest.mark.parametrize("tiles", [(1, 1), (2, 2), (2, 1)])
@pytest.mark.parametrize("frame", ["global", "tile"])
def test_memory_form_equals_direct_point_sum(tiles, frame):
    """Brute force: Eq. loc-query through Eq. bundling, summed point by point with
    no memory vector, equals the memory-vector decode at every cell."""
    g, nx, ny, xy, lab = _tiny_case(tiles, seed=sum(tiles))
    om = oracle.memories(g, nx, ny, xy, lab, frame)
    P = oracle.decode_map(g, nx, ny, om, frame)
    cells = np.array([(i, j) for j in range(g.H) for i in range(g.W)], np.int32)
    Pd = oracle.direct_cells(g, nx, ny, xy, lab, cells)
    for c in range(2):
        assert np.max(np.abs(P[c].ravel() - Pd[:, c])) < 1e-12 * max(1.0, np.abs(Pd).max())


def test_single_point_at_cell_centre_decodes_to_sqrt_D():
    """One point exactly on cell (i0, j0)'s centre: P = D / ||omega|| = sqrt(D) there,
    and by Cauchy-Schwarz nowhere larger; the empty class stays zero.  The
    asymmetric cell pins the [class][row j][column i] layout and x/y roles."""
    g = Grid(W=16, H=12, res=0.125, x_min=-1.0, y_min=-0.75, tiles_x=2, tiles_y=2)
    D = 1024
    nx, ny = oracle.draw_nu(3, D, 0.1)
    i0, j0 = 11, 2
    x = g.x_min + (i0 + 0.5) * g.res
    y = g.y_min + (j0 + 0.5) * g.res
    for frame in ("global", "tile"):
        om = oracle.memories(g, nx, ny, np.array([[x, y]], np.float32), np.array([1], np.uint8), frame)
        P = oracle.decode_map(g, nx, ny, om, frame)
        assert abs(P[1, j0, i0] - math.sqrt(D)) < 1e-10 * math.sqrt(D)
        assert np.unravel_index(np.argmax(P[1]), P[1].shape) == (j0, i0)
        assert P[1].max() <= math.sqrt(D) * (1 + 1e-12)
        assert np.all(P[0] == 0.0)


def test_tile_frame_equals_global_frame():
    """Centring a tile's coordinates multiplies its memories by a unit phasor that
    cancels in Eq. loc-query: the decoded map is the same."""
    g = Grid(W=24, H=20, res=0.2, x_min=-2.4, y_min=-2.0, tiles_x=3, tiles_y=2)
    rng = np.random.default_rng(9)
    xy = rng.uniform(-2.5, 2.5, (150, 2)).astype(np.float32)
    lab = rng.integers(0, 2, 150).astype(np.uint8)
    nx, ny = oracle.draw_nu(21, 300, 0.2)
    Pg = oracle.decode_map(g, nx, ny, oracle.memories(g, nx, ny, xy, lab, "global"), "global")
    Pt = oracle.decode_map(g, nx, ny, oracle.memories(g, nx, ny, xy, lab, "tile"), "tile")
    assert np.max(np.abs(Pg - Pt)) < 1e-10 * np.abs(Pg).max()


def test_sampled_k_equals_full_memories():
    g, nx, ny, xy, lab = _tiny_case((2, 2), seed=4, D=96)
    full = oracle.memories(g, nx, ny, xy, lab, "tile")
    ks = np.array([0, 5, 95, 17, 17], np.int32)
    sub = oracle.memories(g, nx, ny, xy, lab, "tile", ks=ks)
    assert np.array_equal(sub, full[:, ks])


def test_labels_outside_0_1_rejected():
    g = Grid(W=8, H=8, res=0.1, x_min=0.0, y_min=0.0)
    nx, ny = oracle.draw_nu(1, 8, 0.1)
    with pytest.raises(ValueError):
        oracle.memories(g, nx, ny, np.zeros((1, 2), np.float32), np.array([2], np.uint8))


# ------------------------------------------------------------ non-linearity
def test_nonlinearity_born_rule():
    """Eq. non-linearities: (P / max P)^2 per class; the maximum maps to 1;
    a class with no positive value decodes to zeros."""
    rng = np.random.default_rng(1)
    P = rng.normal(size=(2, 6, 7))
    P[0] = -np.abs(P[0])  # class 0 never positive
    Ph, mx = oracle.nonlinear(P)
    assert mx[1] == P[1].max()
    assert np.all(Ph[0] == 0)
    assert np.allclose(Ph[1], (P[1] / P[1].max()) ** 2, rtol=0, atol=1e-15)
    assert Ph[1].ravel()[np.argmax(P[1])] == 1.0


# ------------------------------------------------------------------ entropy
def _lattice_disk_count(r):
    return sum(1 for a in range(-r, r + 1) for b in range(-r, r + 1) if a * a + b * b <= r * r)


def test_entropy_constant_field_gauss_circle():
    """Constant field c: an interior cell sums |disk(r)| equal terms -c ln c.
    |disk(r)| is the Gauss circle count 1, 5, 13, 29, 49, 81 for r = 0..5."""
    c = 0.37
    gauss = [1, 5, 13, 29, 49, 81]
    for r, n_r in enumerate(gauss):
        assert _lattice_disk_count(r) == n_r
        H = oracle.entropy(np.full((24, 30), c), r)
        interior = H[r:24 - r, r:30 - r]
        assert np.allclose(interior, -n_r * c * math.log(c), rtol=1e-14)
        # the corner sees only the quarter disk inside the grid
        q = sum(1 for a in range(0, r + 1) for b in range(0, r + 1) if a * a + b * b <= r * r)
        assert abs(H[0, 0] - (-q * c * math.log(c))) < 1e-13


@pytest.mark.parametrize("r", [0, 1, 2, 3, 5, 7])
def test_entropy_equals_disk_correlation_with_zero_padding(r):
    """Eq. entropy-mask with d <= r (inclusive) equals scipy's correlation of the
    summand -P ln P with a disk footprint, zero outside the grid."""
    from scipy import ndimage
    rng = np.random.default_rng(r)
    Ph = rng.uniform(0, 1.3, (19, 23))
    Ph[rng.uniform(size=Ph.shape) < 0.2] = 0.0
    h = np.zeros_like(Ph)
    nz = Ph != 0
    h[nz] = -Ph[nz] * np.log(Ph[nz])
    yy, xx = np.mgrid[-r:r + 1, -r:r + 1]
    disk = (xx * xx + yy * yy <= r * r).astype(np.float64)
    want = ndimage.correlate(h, disk, mode="constant", cval=0.0)
    assert np.allclose(oracle.entropy(Ph, r), want, rtol=1e-13, atol=1e-13)


def test_entropy_delta_field_is_disk_shaped():
    Ph = np.zeros((21, 21))
    v = 0.25
    Ph[10, 10] = v
    for r in (1, 3, 4):
        H = oracle.entropy(Ph, r)
        yy, xx = np.mgrid[0:21, 0:21]
        inside = (xx - 10) ** 2 + (yy - 10) ** 2 <= r * r
        assert np.allclose(H[inside], -v * math.log(v)) and np.all(H[~inside] == 0)


# ------------------------------------------------------- softmax / PSD / cls
def test_softmax_psd_identities():
    """Eq. softmax and Eq. psd for two classes: Pr1 = sigma(H1 - H0),
    OGM = tanh((H1 - H0) / 2); equal entropies give Pr = 1/2, OGM = 0."""
    from scipy.special import softmax
    rng = np.random.default_rng(2)
    H0 = rng.normal(scale=4, size=500)
    H1 = rng.normal(scale=4, size=500)
    H1[:10] = H0[:10]
    pr1, pr0, ogm = oracle.softmax_psd(H0, H1)
    sm = softmax(np.stack([H0, H1]), axis=0)
    assert np.allclose(pr1, sm[1], rtol=1e-14, atol=1e-15)
    assert np.allclose(pr0, sm[0], rtol=1e-14, atol=1e-15)
    assert np.allclose(ogm, np.tanh((H1 - H0) / 2), atol=1e-14)
    assert np.all(pr1[:10] == 0.5) and np.all(ogm[:10] == 0.0)
    big0, big1 = np.array([-3e4, 800.0]), np.array([5.0, -900.0])
    p1, p0, o = oracle.softmax_psd(big0, big1)
    assert np.all(np.isfinite(p1)) and p1[0] == 1.0 and p1[1] == 0.0


def test_classification_threshold_inclusive_in_float32():
    """Eq. classification: occupied iff OGM >= rho, decided in float32."""
    ogm = np.array([-0.5, 0.0, 0.1, 0.09999999, np.float32(0.1)], np.float32)
    assert oracle.classify_f32(ogm, 0.1).tolist() == [0, 0, 1, 0, 1]
    assert oracle.classify_f32(ogm, 0.0).tolist() == [0, 1, 1, 1, 1]


def test_decoding_ablation_variants():
    """Sec. IV-D1 toggles: all on with the entropy is the paper's pipeline; with no
    activation the two-class softmax is sigma(P_hat_1 - P_hat_0); ReLU of a
    non-negative square is the identity; the entropy ignores negative values."""
    from scipy.special import expit
    rng = np.random.default_rng(12)
    P = rng.normal(size=(2, 9, 11))
    Ph, mx = oracle.nonlinear(P)
    full = oracle.softmax_psd(oracle.entropy(Ph[0], 2), oracle.entropy(Ph[1], 3))
    var = oracle.decode_variant(P, True, True, "entropy", 3, 2)
    for u, v in zip(full, var):
        assert np.allclose(u, v, atol=1e-15)
    pr1, _, ogm = oracle.decode_variant(P, True, True, "none", 3, 2)
    assert np.allclose(pr1, expit(Ph[1] - Ph[0]), atol=1e-15)
    relu = oracle.decode_variant(P, True, True, "relu", 3, 2)
    assert np.allclose(relu[0], pr1, atol=1e-15)
    pr1t, _, _ = oracle.decode_variant(P, False, False, "tanh", 3, 2)
    assert np.allclose(pr1t, expit(np.tanh(P[1]) - np.tanh(P[0])), atol=1e-15)
    neg = -np.abs(P[0])
    assert np.all(oracle.entropy(neg, 2) == 0.0)


def test_window_query_over_the_whole_map_is_the_map_query():
    """A window covering the map decodes the map: it reduces to the full pipeline."""
    g = Grid(W=20, H=14, res=0.2, x_min=-2.0, y_min=-1.4, tiles_x=2, tiles_y=2)
    rng = np.random.default_rng(8)
    xy = rng.uniform(-2.0, 2.0, (80, 2)).astype(np.float32)
    lab = rng.integers(0, 2, 80).astype(np.uint8)
    nx, ny = oracle.draw_nu(4, 128, 0.2)
    full = oracle.pipeline(g, nx, ny, xy, lab, 2, 3)
    win = oracle.query_window(g, nx, ny, full["omega"], 0, 0, g.W, g.H, 2, 3)
    assert np.allclose(win["pr1"], full["pr1"], atol=1e-14)
    assert np.allclose(win["ogm"], full["ogm"], atol=1e-14)
    # an interior window whose region holds the global maxima equals the map query there
    j, i = np.unravel_index(np.argmax(full["P"][1]), full["P"][1].shape)
    k, l = np.unravel_index(np.argmax(full["P"][0]), full["P"][0].shape)
    x0, y0 = max(0, min(i, l) - 1), max(0, min(j, k) - 1)
    x1, y1 = min(g.W, max(i, l) + 2), min(g.H, max(j, k) + 2)
    part = oracle.query_window(g, nx, ny, full["omega"], x0, y0, x1 - x0, y1 - y0, 2, 3)
    assert np.allclose(part["pr1"], full["pr1"][y0:y1, x0:x1], atol=1e-13)


# ----------------------------------------------- the paper's printed numbers
def test_model_size_matches_paper_tables():
    """delta^2 tiles x 2 classes memories (Sec. III-B3) of d float32 elements
    reproduce the model sizes printed in the paper's tables."""
    for name, d, delta, val, unit in _read_golden("paper_model_sizes.txt"):
        d, delta, val = int(d), int(delta), float(val)
        g = Grid(W=4 * delta, H=4 * delta, res=1.0, x_min=0.0, y_min=0.0,
                 tiles_x=delta, tiles_y=delta)
        nx, ny = oracle.draw_nu(0, 2, 1.0)
        n_mem = oracle.memories(g, nx, ny, np.zeros((0, 2), np.float32),
                                np.zeros(0, np.uint8)).shape[0]
        assert n_mem == 2 * delta ** 2
        params = n_mem * d
        if unit == "MB":
            size_mb = params * 4 / 1e6
            assert abs(size_mb - val) / val < 0.01, (name, size_mb, val)
        else:
            assert abs(params / 1000 - val) / val < 0.01, (name, params, val)


# -------------------------------------------- C oracle equals NumPy mirror
@pytest.mark.parametrize("seed", [0, 1])
def test_c_oracle_equals_numpy_mirror(seed):
    g = Grid(W=12, H=10, res=0.2, x_min=-1.2, y_min=-1.0, tiles_x=2, tiles_y=2)
    rng = np.random.default_rng(seed)
    xy = rng.uniform(-1.3, 1.3, (30, 2)).astype(np.float32)
    lab = rng.integers(0, 2, 30).astype(np.uint8)
    nx, ny = oracle.draw_nu(seed, 48, 0.25)
    mx_, my_ = mirror.draw_nu(seed, 48, 0.25)
    assert np.array_equal(nx, mx_) and np.array_equal(ny, my_)
    for frame in ("global", "tile"):
        oc = oracle.memories(g, nx, ny, xy, lab, frame)
        om = mirror.memories(g, nx, ny, xy, lab, frame)
        assert np.max(np.abs(oc - om)) < 1e-11
        Pc = oracle.decode_map(g, nx, ny, oc, frame)
        Pm = mirror.decode_map(g, nx, ny, om, frame)
        assert np.max(np.abs(Pc - Pm)) < 1e-11
    Phc, mxc = oracle.nonlinear(Pc)
    Phm, mxm = mirror.nonlinear(Pm)
    assert np.allclose(Phc, Phm, atol=1e-10)
    for r in (0, 1, 3):
        assert np.allclose(oracle.entropy(Phc[1], r), mirror.entropy(Phm[1], r), atol=1e-10)
    H0, H1 = oracle.entropy(Phc[0], 2), oracle.entropy(Phc[1], 1)
    a = oracle.softmax_psd(H0, H1)
    b = mirror.softmax_psd(H0, H1)
    for u, v in zip(a, b):
        assert np.allclose(u, v, atol=1e-14)
