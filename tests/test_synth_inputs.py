"""The seeded input generator produces the workloads its recipe states.

The paper's datasets are not available, so every measurement and parity test
runs on ``synth`` stand-ins.  These CPU tests check the stated shapes, sizes and
structure: point counts, the raycast labelling of Sec. III-B1 (an occupied end
point lies on a surface, empty points lie in free space), a free sensor origin,
the size ranges of the batch and the serving fleet, and determinism per seed.
"""
import numpy as np
import pytest

from paper_2408_09066_gb300 import synth


def _surface_distance(world, p):
    """Distance from each point to the nearest surface: the walls, a box edge or a
    disc's circle (inside or outside the shape)."""
    x, y = p[:, 0:1].astype(np.float64), p[:, 1:2].astype(np.float64)
    d = np.abs(world.half - np.maximum(np.abs(x), np.abs(y)))[:, 0]
    r = world.rects
    if len(r):
        cx, cy = (r[:, 0] + r[:, 2]) / 2, (r[:, 1] + r[:, 3]) / 2
        hx, hy = (r[:, 2] - r[:, 0]) / 2, (r[:, 3] - r[:, 1]) / 2
        qx, qy = np.abs(x - cx) - hx, np.abs(y - cy) - hy
        outside = np.hypot(np.maximum(qx, 0), np.maximum(qy, 0))
        inside = -np.minimum(np.maximum(qx, qy), 0)
        d = np.minimum(d, (outside + inside).min(1))
    c = world.discs
    if len(c):
        d = np.minimum(d, np.abs(np.hypot(x - c[:, 0], y - c[:, 1]) - c[:, 2]).min(1))
    return d


def test_small_scan_recipe():
    w = synth.small_scan()
    assert (w.n, w.W, w.H, w.tiles_x, w.tiles_y, w.D, w.res) == (3960, 64, 64, 1, 1, 1024, 0.1)
    assert w.xy.dtype == np.float32 and w.labels.dtype == np.uint8
    # one end point and 10 empty samples per beam; every beam of the walled
    # 6.4 m square ends on a surface within the 6 m range (the corners are 4.53 m away)
    lab = w.labels.reshape(360, 11)
    assert np.all(lab[:, 0] == 1) and np.all(lab[:, 1:] == 0)
    again = synth.small_scan()
    assert np.array_equal(again.xy, w.xy) and np.array_equal(again.labels, w.labels)
    other = synth.small_scan(seed=7)
    assert not np.array_equal(other.xy, w.xy)
    # empty samples are uniform along each beam, so their density per unit area
    # falls as 1 / range: twice as dense in the ring 0.5-1 m as in the ring 1-2 m
    # (more than twice where beams end before 2 m)
    r = np.hypot(*w.xy[w.labels == 0].astype(np.float64).T)
    inner = np.count_nonzero((r >= 0.5) & (r < 1.0)) / (np.pi * (1.0 - 0.25))
    outer = np.count_nonzero((r >= 1.0) & (r < 2.0)) / (np.pi * (4.0 - 1.0))
    assert inner > 1.5 * outer


@pytest.mark.parametrize("make,sigma", [(synth.small_scan, 0.02), (synth.evilog_like, 0.03)])
def test_labels_follow_the_raycast_heuristic(make, sigma):
    """Sec. III-B1: a beam that stops before max range marks an occupied point on
    the surface it hit (here within 5 sigma of range noise); the samples along
    the beam are in free space (past a surface by at most the same noise)."""
    w = make()
    occ = w.xy[w.labels == 1]
    emp = w.xy[w.labels == 0]
    assert len(occ) > 0 and len(emp) > 0
    assert _surface_distance(w.world, occ).max() <= 5 * sigma
    assert not w.world.inside_obstacle(emp.astype(np.float64), margin=-5 * sigma).any()
    # the sensor at the origin stands in free space (kept clear by rejection sampling)
    assert not w.world.inside_obstacle(np.zeros((1, 2)), margin=0.35)[0]


def test_paper_trajectory_recipe():
    w = synth.paper_trajectory()
    assert w.n == 100 * 1080 * 21 == 2_268_000
    assert (w.W, w.H, w.tiles_x, w.tiles_y, w.D, w.res, w.x_min) == (400, 400, 4, 4, 8192, 0.1, -20.0)
    frac = w.labels.mean()
    assert 0.04 < frac < 0.055          # about 4.7 % occupied
    # tile occupancy is heavily skewed: the busiest 10 m tile holds many times the emptiest
    tx = np.clip(((w.xy[:, 0] + 20.0) // 10.0).astype(int), 0, 3)
    ty = np.clip(((w.xy[:, 1] + 20.0) // 10.0).astype(int), 0, 3)
    per_tile = np.bincount(ty * 4 + tx, minlength=16)
    assert per_tile.max() > 4 * max(1, per_tile.min())
    assert np.all(np.abs(w.xy) <= 20.0 + 5 * 0.03)


def test_trajectory_steps_avoid_obstacles():
    rng = np.random.default_rng(3)
    world = synth.make_world(rng, 20.0, 25, 15, (1.0, 5.0), (0.5, 2.0), free_r=1.0)
    poses = synth.trajectory(world, (0.0, 0.0), 60, 0.5, rng)
    assert poses.shape == (60, 2)
    assert np.allclose(np.hypot(*np.diff(poses, axis=0).T), 0.5)
    assert not world.inside_obstacle(poses, margin=0.3).any()


def test_batch_maps_recipe():
    maps = synth.batch_maps()
    assert len(maps) == 64
    assert sum(m.n for m in maps) == 7_890_257
    assert sum(m.W * m.H for m in maps) == 10_524_304
    for m in maps:
        assert 64 <= m.W <= 1024 and m.W == m.H and m.res == 0.1
        assert 1 <= m.tiles_x <= 8 and 1 <= m.tiles_y <= 8
        assert m.W // m.tiles_x >= 8 and m.H // m.tiles_y >= 8
        assert m.D in (2048, 4096, 8192)
        assert 10_000 <= m.n <= 500_000
        assert m.xy.flags.c_contiguous and m.labels.flags.c_contiguous
    # uneven sizes: the largest map has many times the cells and points of the smallest
    cells = [m.W * m.H for m in maps]
    pts = [m.n for m in maps]
    assert max(cells) > 20 * min(cells) and max(pts) > 10 * min(pts)
    assert len({m.D for m in maps}) == 3


def test_robot_fleet_recipe():
    fleet = synth.robot_fleet(32)
    assert len(fleet) == 32
    for r in fleet:
        assert r.cells % 128 == 0 and 256 <= r.cells <= 1024 and r.tiles == r.cells // 128
        for xy, lab in r.scans:
            assert xy.shape == (1080 * 21, 2) and lab.shape == (1080 * 21,)
    assert len({r.cells for r in fleet}) > 2


def test_window_sizes_stay_inside_the_map():
    rng = np.random.default_rng(0)
    for cells in (256, 300, 1024):
        for _ in range(200):
            x0, y0, w, h = synth.window_sizes(rng, cells)
            assert 128 <= w <= min(cells, 512) and 128 <= h <= min(cells, 512)
            assert 0 <= x0 and x0 + w <= cells and 0 <= y0 and y0 + h <= cells


def test_ground_truth_marks_obstacles_and_outside():
    world = synth.World(1.0, np.array([[0.0, 0.0, 0.5, 0.5]]), np.zeros((0, 3)))
    gt = synth.ground_truth(world, 24, 24, 0.1, -1.2, -1.2)
    assert gt.shape == (24, 24)
    # cell (i, j) has centre (-1.2 + (i + 0.5) 0.1, -1.2 + (j + 0.5) 0.1), row j first
    assert gt[15, 15] == 1                       # centre (0.35, 0.35): in the box
    assert gt[5, 5] == 0                         # centre (-0.65, -0.65): free
    assert gt[0, 5] == 1 and gt[5, 23] == 1      # beyond the walls at |x|, |y| = 1
