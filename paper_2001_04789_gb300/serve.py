"""Request loop around the native continuous-batching engine (elas_server_*).

Requests arrive as a Poisson stream.  Each names a microstructure (Eshelby
sphere, penny crack or polycrystal at one of several sizes) and a load scale.
Hierarchies stay resident on the device between requests, up to an HBM budget
(least recently used idle grids are evicted to admit a new one), and every solve
is warm-started from the previous displacement of the same microstructure.  A
request waits while its grid is busy with an earlier request; otherwise it is
submitted at once and joins the batch at the next refinement step.

``python -m paper_2001_04789_gb300.serve --seconds 20`` prints one JSON line with
completed solves, solves/s and p50/p99 latency measured from arrival.
"""
from __future__ import annotations

import argparse
import collections
import json
import time

import numpy as np

from . import elas as E
from . import microstructure as M


def make_problem(kind, n, seed=0):
    if kind == "sphere":
        return M.eshelby_sphere(n)
    if kind == "crack":
        return M.penny_crack(n, width=3.0 / (n - 1), clamp_lateral=True)
    return M.polycrystal(n, grains=12, seed=seed)


def scale_loads(grid, problem, s):
    """Same microstructure, loads scaled by s (boundary data and eigenstrain)."""
    for f in range(6):
        if problem.periodic[f // 2]:
            continue
        for c in range(3):
            kind, val = problem.bc[f][c]
            grid.set_bc(f, c, kind, s * val)
    if problem.eigenstrain is not None:
        grid.set_eigenstrain(s * problem.eigenstrain)


class ResidentCache:
    """Grids kept on the device, keyed by microstructure id, evicted LRU when the
    context's HBM budget would be exceeded."""

    def __init__(self, ctx, budget):
        self.ctx = ctx
        self.budget = budget
        self.grids = collections.OrderedDict()     # id -> (grid, problem)
        self.busy = set()

    def get(self, mid, factory):
        if mid in self.grids:
            self.grids.move_to_end(mid)
            return self.grids[mid]
        p = factory()
        need = E.lib().elas_grid_bytes_estimate(E.desc_for(p, mixed=True))
        while self.ctx.bytes_in_use() + need > self.budget:
            victim = next((k for k in self.grids if k not in self.busy), None)
            if victim is None:
                return None
            g, _ = self.grids.pop(victim)
            g.close()
        g = E.grid_from_problem(self.ctx, p, mixed=True)
        self.grids[mid] = (g, p)
        return self.grids[mid]

    def close(self):
        for g, _ in self.grids.values():
            g.close()
        self.grids.clear()


def run(seconds=20.0, rate=200.0, sizes=(65, 129), kinds=("sphere", "crack", "polycrystal"),
        variants=2, budget=150 << 30, max_active=16, seed=0, rel_tol=1e-8, device=0):
    rng = np.random.default_rng(seed)
    ctx = E.Context(device, budget_bytes=budget)
    server = E.Server(ctx, max_active=max_active)
    cache = ResidentCache(ctx, budget)
    catalogue = [(k, n, v) for k in kinds for n in sizes for v in range(variants)]
    pending = collections.deque()          # (arrival, mid, scale) waiting for a free grid
    inflight = {}                          # ticket -> (arrival, mid)
    latencies, results = [], []
    t0 = time.perf_counter()
    next_arrival = rng.exponential(1.0 / rate)
    steps = 0
    active_sum = 0
    while True:
        now = time.perf_counter() - t0
        while next_arrival <= now and next_arrival < seconds:
            mid = catalogue[int(rng.integers(len(catalogue)))]
            pending.append((next_arrival, mid, float(rng.uniform(0.5, 1.5))))
            next_arrival += rng.exponential(1.0 / rate)
        # submit every pending request whose grid is resident and idle
        keep = collections.deque()
        for arr, mid, sc in pending:
            if mid in cache.busy:
                keep.append((arr, mid, sc))
                continue
            entry = cache.get(mid, lambda mid=mid: make_problem(mid[0], mid[1], seed=mid[2]))
            if entry is None:
                keep.append((arr, mid, sc))
                continue
            g, p = entry
            scale_loads(g, p, sc)
            t = server.submit(g, rel_tol=rel_tol, max_cycles=200, warm_start=True)
            inflight[t] = (arr, mid)
            cache.busy.add(mid)
        pending = keep
        act, _ = server.step()
        steps += 1
        active_sum += act
        done_now = time.perf_counter() - t0
        for t in list(inflight):
            r = server.poll(t)
            if r is None:
                continue
            info, _ = r
            arr, mid = inflight.pop(t)
            cache.busy.discard(mid)
            latencies.append(done_now - arr)
            results.append(info)
        if now >= seconds and not inflight and not pending:
            break
        if now > 4 * seconds + 60:
            break
    elapsed = time.perf_counter() - t0
    server.close()
    cache.close()
    ctx.close()
    lat = np.sort(np.array(latencies)) if latencies else np.array([np.nan])
    return {
        "completed": len(results), "seconds": elapsed, "solves_per_s": len(results) / elapsed,
        "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3)},
        "rate": rate, "steps": steps, "mean_active": active_sum / max(steps, 1),
        "converged": sum(1 for r in results if r["status"] == 0),
        "mean_cycles": float(np.mean([r["cycles"] for r in results])) if results else None,
        "sizes": list(sizes), "kinds": list(kinds), "max_active": max_active,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seconds", type=float, default=20.0)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--sizes", default="65,129")
    ap.add_argument("--max-active", type=int, default=16)
    a = ap.parse_args()
    out = run(seconds=a.seconds, rate=a.rate, sizes=tuple(int(v) for v in a.sizes.split(",")),
              max_active=a.max_active)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
