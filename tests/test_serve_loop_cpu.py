"""The serving loop's host logic (serve.run) with stand-ins for the library: a fake server
that admits requests into a fixed number of slots and retires each after three steps.
Every Poisson arrival is either completed or refused, refusals happen only with a
bounded queue and only when it is full, no microstructure ever has two requests in
flight (the library refuses that), and latencies are measured from arrival."""
import collections
import time
import types

import numpy as np
import pytest

from paper_2001_04789_gb300 import serve


class FakeCtx:
    def __init__(self, device=0, budget_bytes=0):
        self.used = 0

    def bytes_in_use(self):
        return self.used

    def close(self):
        pass


class FakeGrid:
    def __init__(self, ctx, p):
        self.ctx = ctx
        ctx.used += 1

    def close(self):
        self.ctx.used -= 1


class FakeServer:
    steps_per_request = 3

    def __init__(self, ctx, max_active):
        self.max_active = max_active
        self.waiting = collections.deque()
        self.active = {}
        self.done = {}
        self.held = set()
        self.next = 1
        self.submitted = 0

    def submit(self, g, **kw):
        assert g not in self.held, "a grid with a pending request was submitted again"
        t = self.next
        self.next += 1
        self.waiting.append((t, g))
        self.held.add(g)
        self.submitted += 1
        return t

    submit_amr = submit

    def step(self):
        time.sleep(0.002)
        while self.waiting and len(self.active) < self.max_active:
            t, g = self.waiting.popleft()
            self.active[t] = [g, self.steps_per_request]
        for t in list(self.active):
            self.active[t][1] -= 1
            if self.active[t][1] == 0:
                self.held.discard(self.active.pop(t)[0])
                self.done[t] = {"status": 0, "cycles": self.steps_per_request}
        return len(self.active), len(self.waiting)

    def poll(self, t):
        return (self.done.pop(t), 0.0) if t in self.done else None

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    servers = []

    def make_server(ctx, max_active):
        s = FakeServer(ctx, max_active)
        servers.append(s)
        return s

    fake_lib = types.SimpleNamespace(elas_grid_bytes_estimate=lambda d: 1)
    fake_E = types.SimpleNamespace(Context=FakeCtx, Server=make_server, MIXED=1, lib=lambda: fake_lib,
                                   desc_for=lambda p, mixed=True: p,
                                   grid_from_problem=lambda ctx, p, mixed=True: FakeGrid(ctx, p), Amr=None)
    monkeypatch.setattr(serve, "E", fake_E)
    monkeypatch.setattr(serve, "make_entry", lambda mid: types.SimpleNamespace(mid=mid))
    monkeypatch.setattr(serve, "scale_entry", lambda g, p, sc: None)
    return servers


def poisson_arrivals(seed, rate, seconds, catalogue_len):
    """Arrivals before `seconds`, replaying the loop's draws (time, microstructure, scale)."""
    rng = np.random.default_rng(seed)
    t = rng.exponential(1.0 / rate)
    count = 0
    while t < seconds:
        rng.integers(catalogue_len)
        rng.uniform(0.5, 1.5)
        t += rng.exponential(1.0 / rate)
        count += 1
    return count


def test_overloaded_loop_refuses_beyond_its_queue_bound(fake):
    kw = dict(seconds=0.4, rate=1500.0, sizes=(17,), kinds=("sphere", "crack"), variants=3, max_active=2,
              budget=1 << 30, seed=4)
    out = serve.run(max_queue=5, **kw)
    arrivals = poisson_arrivals(4, 1500.0, 0.4, 2 * 3)
    assert out["completed"] + out["refused"] == arrivals
    assert out["refused"] > 0 and out["completed"] == fake[0].submitted
    assert out["converged"] == out["completed"] and out["mean_cycles"] == FakeServer.steps_per_request
    assert 0 < out["latency_ms"]["p50"] <= out["latency_ms"]["p99"]
    assert out["mean_active"] <= 2


def test_unbounded_loop_serves_every_arrival(fake):
    out = serve.run(seconds=0.3, rate=300.0, sizes=(17,), kinds=("sphere",), variants=4, max_active=4,
                    budget=1 << 30, seed=7, max_queue=None)
    assert out["refused"] == 0
    assert out["completed"] == poisson_arrivals(7, 300.0, 0.3, 4) == fake[0].submitted
