"""Seeded synthetic 2D lidar data shaped like the paper's workloads.

Input generator only: it builds worlds, scans and trajectories and labels the
points with the raycast heuristic of Sec. III-B1 (a beam that ends before its
maximum range gives an occupied point; the max-range end point and points
interpolated along the beam are empty).  It holds none of the mapping
method's arithmetic and is used by the tests, the benchmark and the examples
to feed both the CUDA path and the oracle the same arrays.

The paper's datasets (ToySim, Intel Map, EviLOG) are not available, so these
seeded stand-ins follow the workload shapes named for this library:
  * small   : 64 x 64 cells at 0.1 m (6.4 m square), one tile, D = 1024,
              one 360-beam scan from the centre, max range 6 m, sigma 0.02 m,
              10 empty samples per beam (about 3.96k points);
  * paper   : 400 x 400 cells at 0.1 m (40 m square), 4 x 4 tiles, D = 8192,
              100 scans along a 0.5 m-step random walk, 1080 beams, max range
              30 m, sigma 0.03 m, 20 empty samples per beam (about 2.27M points).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class World:
    half: float            # the world is the square [-half, half]^2, walled
    rects: np.ndarray      # [n][4] axis-aligned boxes (x0, y0, x1, y1)
    discs: np.ndarray      # [n][3] discs (cx, cy, r)

    def inside_obstacle(self, p: np.ndarray, margin: float = 0.0) -> np.ndarray:
        p = np.atleast_2d(p)
        x, y = p[:, 0:1], p[:, 1:2]
        r = self.rects
        in_r = ((x >= r[:, 0] - margin) & (x <= r[:, 2] + margin)
                & (y >= r[:, 1] - margin) & (y <= r[:, 3] + margin)).any(1)
        d = self.discs
        in_d = (((x - d[:, 0]) ** 2 + (y - d[:, 1]) ** 2) <= (d[:, 2] + margin) ** 2).any(1)
        out = (np.abs(p[:, 0]) > self.half - margin) | (np.abs(p[:, 1]) > self.half - margin)
        return in_r | in_d | out


def make_world(rng: np.random.Generator, half: float, n_rect: int, n_disc: int,
               rect_size: tuple, disc_r: tuple, keep_free=(0.0, 0.0), free_r: float = 0.5) -> World:
    """Random axis-aligned rectangles and discs; none covers the disc of radius
    ``free_r`` around ``keep_free`` (rejection sampling)."""
    kx, ky = keep_free
    rects, discs = [], []
    while len(rects) < n_rect:
        w, h = rng.uniform(*rect_size, size=2)
        cx, cy = rng.uniform(-half + w / 2, half - w / 2), rng.uniform(-half + h / 2, half - h / 2)
        box = (cx - w / 2, cy - h / 2, cx + w / 2, cy + h / 2)
        nx = min(max(kx, box[0]), box[2])
        ny = min(max(ky, box[1]), box[3])
        if (nx - kx) ** 2 + (ny - ky) ** 2 > free_r ** 2:
            rects.append(box)
    while len(discs) < n_disc:
        r = rng.uniform(*disc_r)
        cx, cy = rng.uniform(-half + r, half - r, size=2)
        if (cx - kx) ** 2 + (cy - ky) ** 2 > (r + free_r) ** 2:
            discs.append((cx, cy, r))
    return World(half, np.array(rects, np.float64).reshape(-1, 4),
                 np.array(discs, np.float64).reshape(-1, 3))


def raycast(world: World, origin, angles: np.ndarray) -> np.ndarray:
    """Distance from ``origin`` to the first surface along each angle."""
    ox, oy = float(origin[0]), float(origin[1])
    dx, dy = np.cos(angles)[:, None], np.sin(angles)[:, None]
    best = np.full((len(angles), 1), np.inf)
    with np.errstate(divide="ignore", invalid="ignore"):
        # boundary walls and rectangles: slab test against each box
        boxes = np.concatenate([world.rects,
                                np.array([[-world.half, -world.half, world.half, world.half]])])
        tx0 = (boxes[:, 0] - ox) / dx
        tx1 = (boxes[:, 2] - ox) / dx
        ty0 = (boxes[:, 1] - oy) / dy
        ty1 = (boxes[:, 3] - oy) / dy
        tmin = np.maximum(np.minimum(tx0, tx1), np.minimum(ty0, ty1))
        tmax = np.minimum(np.maximum(tx0, tx1), np.maximum(ty0, ty1))
        # entering hit for obstacles; the wall box is hit from the inside (tmax)
        t_obs = np.where((tmax >= tmin) & (tmin > 0), tmin, np.inf)[:, :-1]
        t_wall = tmax[:, -1:]
        best = np.minimum(best, t_wall)
        if t_obs.shape[1]:
            best = np.minimum(best, t_obs.min(1, keepdims=True))
        if len(world.discs):
            fx = ox - world.discs[:, 0]
            fy = oy - world.discs[:, 1]
            b = fx * dx + fy * dy
            c = fx * fx + fy * fy - world.discs[:, 2] ** 2
            disc = b * b - c
            t = -b - np.sqrt(np.where(disc >= 0, disc, np.nan))
            t = np.where((disc >= 0) & (t > 0), t, np.inf)
            best = np.minimum(best, t.min(1, keepdims=True))
    return best[:, 0]


def scan(world: World, origin, n_beams: int, max_range: float, sigma: float, n_empty: int,
         rng: np.random.Generator):
    """One labelled scan: per beam the end point (occupied if the beam hit a
    surface within max range, else the empty max-range point) followed by
    ``n_empty`` empty points at u * range, u ~ U(0, 1)."""
    ang = np.arange(n_beams) * (2 * np.pi / n_beams)
    rng_true = raycast(world, origin, ang)
    hit = rng_true <= max_range
    meas = np.where(hit, rng_true + rng.normal(0.0, sigma, n_beams), max_range)
    meas = np.maximum(meas, 0.0)
    u = rng.uniform(0.0, 1.0, (n_beams, n_empty))
    rr = np.concatenate([meas[:, None], u * meas[:, None]], 1)  # [beams][1 + n_empty]
    lab = np.zeros(rr.shape, np.uint8)
    lab[:, 0] = hit.astype(np.uint8)
    x = origin[0] + rr * np.cos(ang)[:, None]
    y = origin[1] + rr * np.sin(ang)[:, None]
    xy = np.stack([x.ravel(), y.ravel()], 1).astype(np.float32)
    return xy, lab.ravel()


def trajectory(world: World, start, n_steps: int, step: float, rng: np.random.Generator,
               margin: float = 0.3) -> np.ndarray:
    """Random walk of ``n_steps`` poses with fixed step length, rejecting steps
    that end inside an obstacle (or within ``margin`` of one)."""
    poses = [np.asarray(start, np.float64)]
    heading = rng.uniform(0, 2 * np.pi)
    while len(poses) < n_steps:
        for _ in range(64):
            h = heading + rng.normal(0.0, 0.6)
            cand = poses[-1] + step * np.array([np.cos(h), np.sin(h)])
            if not world.inside_obstacle(cand, margin)[0]:
                heading = h
                poses.append(cand)
                break
        else:
            heading = rng.uniform(0, 2 * np.pi)
    return np.array(poses)


@dataclasses.dataclass
class Workload:
    name: str
    xy: np.ndarray          # float32 [n][2]
    labels: np.ndarray      # uint8 [n]
    W: int
    H: int
    res: float
    x_min: float
    y_min: float
    tiles_x: int
    tiles_y: int
    D: int
    length_scale: float
    seed: int
    world: World

    @property
    def n(self) -> int:
        return len(self.labels)


def small_scan(seed: int = 1001, D: int = 1024) -> Workload:
    """One 360-beam scan in a walled 6.4 m square with 5 boxes and 3 discs."""
    rng = np.random.default_rng(seed)
    w = make_world(rng, 3.2, 5, 3, (0.3, 1.5), (0.2, 0.6))
    xy, lab = scan(w, (0.0, 0.0), 360, 6.0, 0.02, 10, rng)
    return Workload("small_64x64_1tile", xy, lab, 64, 64, 0.1, -3.2, -3.2, 1, 1, D, 0.1, seed, w)


def paper_trajectory(seed: int = 1002, D: int = 8192, n_scans: int = 100) -> Workload:
    """100 scans of 1080 beams along a random walk in a walled 40 m square
    with 40 obstacles (25 boxes of 1-5 m, 15 discs of radius 0.5-2 m)."""
    rng = np.random.default_rng(seed)
    w = make_world(rng, 20.0, 25, 15, (1.0, 5.0), (0.5, 2.0), free_r=1.0)
    poses = trajectory(w, (0.0, 0.0), n_scans, 0.5, rng)
    parts = [scan(w, p, 1080, 30.0, 0.03, 20, rng) for p in poses]
    xy = np.concatenate([p[0] for p in parts])
    lab = np.concatenate([p[1] for p in parts])
    return Workload("paper_400x400_4x4tiles", xy, lab, 400, 400, 0.1, -20.0, -20.0, 4, 4, D,
                    0.1, seed, w)


def _walk_workload(name, seed, half, n_rect, n_disc, rect_size, disc_r, n_scans, beams,
                   max_range, n_empty, cells, res, tiles, D, length_scale, step=0.5,
                   sigma=0.03, cells_y=None):
    rng = np.random.default_rng(seed)
    w = make_world(rng, half, n_rect, n_disc, rect_size, disc_r, free_r=1.0)
    poses = trajectory(w, (0.0, 0.0), n_scans, step, rng)
    parts = [scan(w, p, beams, max_range, sigma, n_empty, rng) for p in poses]
    xy = np.concatenate([p[0] for p in parts])
    lab = np.concatenate([p[1] for p in parts])
    ch = cells_y or cells
    return Workload(name, xy, lab, cells, ch, res, -cells * res / 2, -ch * res / 2, tiles[0],
                    tiles[1], D, length_scale, seed, w)


def toysim_like(seed: int = 2001, D: int = 16000, n_scans: int = 90) -> Workload:
    """Shaped like the ToySim row of the paper's dataset table: a 100 m x 100 m
    world, 90 scans of 50 beams, about as many occupied as empty points; with
    the ToySim parameters d = 32000 (D = 16000), l = 1, delta = 2; 0.25 m cells."""
    return _walk_workload("toysim_like_400x400_2x2tiles", seed, 50.0, 30, 15, (2.0, 10.0),
                          (1.0, 4.0), n_scans, 50, 40.0, 1, 400, 0.25, (2, 2), D, 1.0, step=1.0)


def intel_like(seed: int = 2002, D: int = 16000, n_scans: int = 910) -> Workload:
    """Shaped like the Intel Map row: a 38 m x 38 m building-sized world, 910 scans
    of 421 beams, a little more occupied than empty; d = 32000, l = 0.2,
    delta = 8, 0.1 m cells."""
    return _walk_workload("intel_like_380x380_8x8tiles", seed, 19.0, 40, 10, (0.5, 4.0),
                          (0.3, 1.0), n_scans, 421, 20.0, 1, 380, 0.1, (8, 8), D, 0.2, step=0.25)


def evilog_like(seed: int = 2003, D: int = 16000) -> Workload:
    """Shaped like the EviLOG row: one 48,000-point frame (2400 beams x 20 points)
    over 56.32 m x 81.92 m at 0.16 m (352 x 512 cells), d = 32000, l = 0.2,
    delta = 1."""
    rng = np.random.default_rng(seed)
    w = make_world(rng, 41.0, 40, 20, (1.0, 5.0), (0.5, 2.0), free_r=1.0)
    xy, lab = scan(w, (0.0, 0.0), 2400, 40.0, 0.03, 19, rng)
    return Workload("evilog_like_352x512_1tile", xy, lab, 352, 512, 0.16, -352 * 0.16 / 2,
                    -512 * 0.16 / 2, 1, 1, D, 0.2, seed, w)


@dataclasses.dataclass
class Robot:
    """One robot of a serving fleet: a square map of `cells` x `cells` cells of
    0.1 m centred on its world, tiles of 128 cells, and a pool of scans."""
    world: World
    cells: int
    res: float
    tiles: int
    scans: list            # [(xy float32 [n][2], labels uint8 [n])]


def robot_fleet(n_robots: int, seed: int = 1005, min_cells: int = 256, max_cells: int = 1024,
                scans_per_robot: int = 4, beams: int = 1080, n_empty: int = 20) -> list:
    """Robots with maps of 256^2 to 1024^2 cells (log-uniform, multiples of 128),
    each with a random-walk pool of scans of `beams` beams and `n_empty` empty
    samples per beam (1080 x 21 = 22,680 points per scan)."""
    rng = np.random.default_rng(seed)
    fleet = []
    for _ in range(n_robots):
        cells = int(np.exp(rng.uniform(np.log(min_cells), np.log(max_cells))) // 128 * 128)
        cells = max(min_cells, min(max_cells, cells))
        half = cells * 0.1 / 2
        w = make_world(rng, half, max(2, cells // 40), max(1, cells // 80), (1.0, 4.0),
                       (0.4, 1.5), free_r=1.0)
        poses = trajectory(w, (0.0, 0.0), scans_per_robot, 0.5, rng)
        rmax = min(30.0, half)
        scans = [scan(w, p, beams, rmax, 0.03, n_empty, rng) for p in poses]
        fleet.append(Robot(w, cells, 0.1, cells // 128, scans))
    return fleet


def batch_maps(n_maps: int = 64, seed: int = 1004, min_cells: int = 64, max_cells: int = 1024,
               min_points: int = 10_000, max_points: int = 500_000, max_tiles: int = 8,
               dims=(2048, 4096, 8192)) -> list:
    """Independent maps of uneven size for batched stepping: cells per side
    log-uniform in [min_cells, max_cells] at 0.1 m, tiles per axis uniform in
    1..max_tiles (independently, at least 8 cells a tile), D drawn from
    ``dims``, and a log-uniform number of labelled points in [min_points,
    max_points] from the small-scan generator (360 beams, 10 empty samples per
    beam, sigma 0.02 m) along a 0.5 m-step random walk, max range
    min(30 m, half the world)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_maps):
        cells = int(round(np.exp(rng.uniform(np.log(min_cells), np.log(max_cells)))))
        cells = max(min_cells, min(max_cells, cells))
        tx = int(rng.integers(1, max_tiles + 1))
        ty = int(rng.integers(1, max_tiles + 1))
        tx, ty = max(1, min(tx, cells // 8)), max(1, min(ty, cells // 8))
        D = int(dims[int(rng.integers(len(dims)))])
        n = int(round(np.exp(rng.uniform(np.log(min_points), np.log(max_points)))))
        half = cells * 0.1 / 2
        sc = min(1.0, half / 3.2)   # obstacles and steps shrink with worlds below 6.4 m
        w = make_world(rng, half, max(5, cells // 40), max(3, cells // 80),
                       (0.3 * sc, 3.0 * sc), (0.2 * sc, 1.2 * sc), free_r=0.6 * sc)
        per_scan = 360 * 11
        poses = trajectory(w, (0.0, 0.0), (n + per_scan - 1) // per_scan, 0.5 * sc, rng,
                           margin=0.3 * sc)
        parts = [scan(w, p, 360, min(30.0, half), 0.02, 10, rng) for p in poses]
        xy = np.concatenate([q[0] for q in parts])[:n]
        lab = np.concatenate([q[1] for q in parts])[:n]
        out.append(Workload(f"batch{k}_{cells}x{cells}_{tx}x{ty}_D{D}", np.ascontiguousarray(xy),
                            np.ascontiguousarray(lab), cells, cells, 0.1, -half, -half, tx, ty, D,
                            0.1, seed * 1000 + k, w))
    return out


def window_sizes(rng: np.random.Generator, cells: int, lo: int = 128, hi: int = 512):
    """A random query window (x0, y0, w, h) of lo..hi cells per side inside the map."""
    w = int(min(cells, rng.integers(lo, hi + 1)))
    h = int(min(cells, rng.integers(lo, hi + 1)))
    return (int(rng.integers(0, cells - w + 1)), int(rng.integers(0, cells - h + 1)), w, h)


def ground_truth(world: World, W: int, H: int, res: float, x_min: float, y_min: float) -> np.ndarray:
    """Occupancy of each cell centre (1 inside an obstacle or outside the walls)."""
    j, i = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    c = np.stack([x_min + (i.ravel() + 0.5) * res, y_min + (j.ravel() + 0.5) * res], 1)
    return world.inside_obstacle(c).reshape(H, W).astype(np.uint8)
