"""The serving loop's admission and ordering rules, on the CPU.

``serving.Server.run`` is host logic: it admits requests to execution slots as
they arrive and as slots free up, keeps each robot's requests in arrival order
and never runs two requests of one robot at once (a map is used by one stream
at a time).  Here the server's CUDA streams, events and maps are host fakes:
a fake map applies an update or answers a query when it is launched and marks
its robot busy until the slot's completion event, which completes after a
random number of polls.  The rules are then checked on the record of launches
and completions, with several robots and fewer slots than requests.
"""
import contextlib
import time

import numpy as np
import pytest
import torch

from paper_2408_09066_gb300 import serving


class World:
    def __init__(self, seed):
        self.rng = np.random.default_rng(seed)
        self.busy = set()          # robots with work launched and not yet completed
        self.launches = []         # (robot, kind, payload) in launch order
        self.max_in_flight = 0
        self.max_busy_robots = 0
        self.work_s = 0.0          # least wall time a slot's work takes


class FakeStream:
    def __init__(self):
        self.ops = []              # robots whose work was enqueued since the last event


class FakeEvent:
    def __init__(self, world):
        self.world = world
        self.t_rec = None
        self.t_done = None
        self.polls = 0
        self.robots = []

    def record(self, stream=None):
        self.t_rec = time.perf_counter()
        self.t_done = None
        self.polls = int(self.world.rng.integers(0, 6))
        self.robots = list(stream.ops) if stream is not None else []
        if stream is not None:
            stream.ops.clear()

    def query(self):
        if self.t_done is not None:
            return True
        if self.polls > 0 or time.perf_counter() - self.t_rec < self.world.work_s:
            self.polls = max(0, self.polls - 1)
            return False
        self.t_done = time.perf_counter()
        for r in self.robots:
            self.world.busy.discard(r)
        return True

    def elapsed_time(self, other):
        return (other.t_done - self.t_rec) * 1e3


class FakeTorch:
    class cuda:
        @staticmethod
        def stream(s):
            return contextlib.nullcontext()

        @staticmethod
        def synchronize():
            pass


class FakeMap:
    def __init__(self, world, robot, n_slots):
        self.world, self.robot, self.n_slots = world, robot, n_slots
        self.updates = 0

    def _launch(self, stream, kind, payload):
        w = self.world
        assert self.robot not in w.busy, "two requests of one robot in flight"
        w.busy.add(self.robot)
        assert len(w.busy) <= self.n_slots
        w.max_busy_robots = max(w.max_busy_robots, len(w.busy))
        stream.ops.append(self.robot)
        w.launches.append((self.robot, kind, payload))

    def encode_bundle(self, xy, lab, stream=None):
        self._launch(stream, "update", (len(lab), float(xy[:, 0].sum()), int(lab.sum())))
        self.updates += 1

    def query_window(self, x0, y0, w, h, heat, occ, stream=None):
        self._launch(stream, "query", (x0, y0, w, h))
        occ.fill_(float(self.updates))  # the answer: how many updates the map has seen


class FakeSlot:
    def __init__(self, world, max_points, max_cells):
        self.stream = FakeStream()
        self.xy = torch.empty((max_points, 2), dtype=torch.float32)
        self.lab = torch.empty(max_points, dtype=torch.uint8)
        self.heat = torch.empty(4 * max_cells, dtype=torch.float32)
        self.occ = torch.empty(max_cells, dtype=torch.float32)
        self.xy_h = torch.empty((max_points, 2), dtype=torch.float32)
        self.lab_h = torch.empty(max_points, dtype=torch.uint8)
        self.occ_h = torch.empty(max_cells, dtype=torch.float32)
        self.done = FakeEvent(world)
        self.req = None


def make_server(world, n_robots, n_slots, max_points=64, max_window=8):
    srv = serving.Server.__new__(serving.Server)
    srv.torch = FakeTorch
    srv.maps = [FakeMap(world, i, n_slots) for i in range(n_robots)]
    srv.max_points, srv.max_window = max_points, max_window
    srv.n_slots = n_slots
    srv.slots = [FakeSlot(world, max_points, max_window * max_window) for _ in range(n_slots)]
    srv.t0_event = FakeEvent(world)
    return srv


def make_requests(rng, n_robots, n, span):
    reqs, t = [], 0.0
    for _ in range(n):
        t += rng.exponential(span / n)
        rb = int(rng.integers(n_robots))
        if rng.uniform() < 0.5:
            w, h = (int(v) for v in rng.integers(1, 9, 2))
            reqs.append(serving.Request("query", rb, t, window=(int(rng.integers(0, 4)), 0, w, h)))
        else:
            k = int(rng.integers(1, 65))
            xy = rng.normal(size=(k, 2)).astype(np.float32)
            lab = rng.integers(0, 2, k).astype(np.uint8)
            reqs.append(serving.Request("update", rb, t, xy=xy, labels=lab))
    return reqs


@pytest.mark.parametrize("realtime", [False, True])
@pytest.mark.parametrize("n_slots", [1, 3, 8])
def test_admission_and_per_robot_order(realtime, n_slots):
    world = World(seed=n_slots)
    n_robots = 5
    reqs = make_requests(np.random.default_rng(10 + n_slots), n_robots, 120, span=0.03)
    srv = make_server(world, n_robots, n_slots)
    done = srv.run(reqs, realtime=realtime)

    # every request is served once
    assert len(done) == len(reqs) and len({id(r) for r in done}) == len(reqs)
    assert not world.busy
    # each robot's requests were launched in arrival order, with their own data
    for rb in range(n_robots):
        mine = [r for r in reqs if r.robot == rb]
        launched = [(k, p) for (r, k, p) in world.launches if r == rb]
        want = []
        for r in mine:
            if r.kind == "update":
                want.append(("update", (len(r.labels), float(r.xy[:, 0].sum()), int(r.labels.sum()))))
            else:
                want.append(("query", r.window))
        assert len(launched) == len(want)
        for (k, p), (wk, wp) in zip(launched, want):
            assert k == wk
            if k == "update":
                assert p[0] == wp[0] and p[2] == wp[2] and abs(p[1] - wp[1]) < 1e-4
            else:
                assert p == wp
        # a query answers with exactly the updates of its robot that arrived before it
        seen = 0
        for r in mine:
            if r.kind == "update":
                seen += 1
            else:
                x0, y0, w, h = r.window
                assert r.result.shape == (h, w)
                assert np.all(r.result == seen)
    # timing fields are consistent; with realtime, nothing starts before it arrives
    for r in done:
        assert r.done >= r.start - 1e-3
        if realtime:
            assert r.start >= r.arrival
    # with more than one slot, requests of different robots overlap
    if n_slots > 1:
        assert world.max_busy_robots > 1


def _check_order(world, reqs, n_robots):
    """Every request ends once, done or expired; an expired one never launched;
    each robot's launched requests ran in arrival order and each query saw
    exactly the robot's earlier updates that ran."""
    for r in reqs:
        assert r.status in ("done", "expired")
    for rb in range(n_robots):
        ran = [r for r in reqs if r.robot == rb and r.status == "done"]
        launched = [(k, p) for (q, k, p) in world.launches if q == rb]
        assert [k for k, _ in launched] == [r.kind for r in ran]
        seen = 0
        for r, (k, p) in zip(ran, launched):
            if k == "update":
                assert p[0] == len(r.labels)
                seen += 1
            else:
                assert p == r.window and np.all(r.result == seen)


def test_deadline_zero_expires_before_launch_and_none_waits():
    world = World(seed=4)
    reqs = make_requests(np.random.default_rng(4), 3, 60, span=0.01)
    for i, r in enumerate(reqs):
        r.deadline = 0.0 if i % 2 else None
    srv = make_server(world, 3, 2)
    done = srv.run(reqs, realtime=False)
    assert len(done) == len(reqs)
    assert all(r.status == ("expired" if i % 2 else "done") for i, r in enumerate(reqs))
    assert all(np.isnan(r.start) for r in reqs if r.status == "expired")
    _check_order(world, reqs, 3)
    s = serving.summarize(done, duration=1e-3)
    n_exp = sum(v.get("expired", 0) for k, v in s.items() if k in ("update", "query"))
    assert n_exp == len(reqs) // 2
    assert sum(v["count"] for k, v in s.items() if k in ("update", "query")) == len(reqs) - n_exp


def test_generous_deadlines_expire_nothing():
    world = World(seed=5)
    reqs = make_requests(np.random.default_rng(5), 4, 80, span=0.02)
    for r in reqs:
        r.deadline = 1e3
    srv = make_server(world, 4, 3)
    srv.run(reqs, realtime=True)
    assert all(r.status == "done" for r in reqs)
    _check_order(world, reqs, 4)


def test_overload_drops_late_requests_and_keeps_order():
    """One slot whose work takes 2 ms, requests arriving every 0.2 ms with a 3 ms
    start deadline: most expire, the rest run in order with the right data."""
    world = World(seed=6)
    world.work_s = 2e-3
    rng = np.random.default_rng(6)
    reqs = make_requests(rng, 3, 40, span=0.008)
    for r in reqs:
        r.deadline = 3e-3
    srv = make_server(world, 3, 1)
    srv.run(reqs, realtime=True)
    n_done = sum(r.status == "done" for r in reqs)
    assert 0 < n_done < len(reqs)
    for r in reqs:
        if r.status == "done":
            assert r.start <= r.arrival + r.deadline + 1e-3
    _check_order(world, reqs, 3)


def test_update_larger_than_the_slot_buffers_is_refused():
    world = World(seed=0)
    srv = make_server(world, 1, 2, max_points=16)
    big = serving.Request("update", 0, 0.0, xy=np.zeros((17, 2), np.float32),
                          labels=np.zeros(17, np.uint8))
    with pytest.raises(ValueError):
        srv.run([big], realtime=False)


def test_summary_percentiles_and_rate():
    rs = []
    for i, lat in enumerate([1.0, 2.0, 3.0, 4.0]):
        r = serving.Request("update" if i % 2 == 0 else "query", 0, 0.0)
        r.done = lat / 1e3
        rs.append(r)
    s = serving.summarize(rs, duration=1.0)
    assert s["update"]["count"] == 2 and s["query"]["count"] == 2
    assert s["update"]["p50_ms"] == pytest.approx(2.0) and s["query"]["max_ms"] == pytest.approx(4.0)
    assert s["requests_per_s"] == pytest.approx(4.0)


def test_garbage_collector_is_paused_while_serving_and_restored():
    """The loop runs with Python's cyclic garbage collector off (its pauses
    showed up as isolated ~10 ms latencies) and leaves it as it found it."""
    import gc
    world = World(seed=5)
    srv = make_server(world, n_robots=2, n_slots=2)
    seen = []
    orig = FakeEvent.query

    def spy(self):
        seen.append(gc.isenabled())
        return orig(self)

    reqs = make_requests(world.rng, 2, 12, 0.001)
    try:
        FakeEvent.query = spy
        assert gc.isenabled()
        srv.run(reqs, realtime=False)
        assert seen and not any(seen)
        assert gc.isenabled()
        gc.disable()
        srv.run(make_requests(world.rng, 2, 4, 0.001), realtime=False)
        assert not gc.isenabled()
    finally:
        FakeEvent.query = orig
        gc.enable()
