"""Request loop around the native continuous-batching engine (elas_server_*).

Requests arrive as a Poisson stream.  Each names a microstructure (Eshelby
sphere, penny crack or polycrystal) at one of several sizes, either on one grid
(mixed precision) or as a two-level block-structured AMR layout (composite FP64
cycles, one per server step), and a load scale.  Hierarchies stay resident on
the device between requests, up to an HBM budget (least recently used idle ones
are evicted to admit a new one), and every solve is warm-started from the
previous displacement of the same microstructure.  A request waits while its
hierarchy is busy with an earlier request; otherwise it is submitted at once and
joins the batch at the next step.  Admission is bounded: an arrival that finds
``max_queue`` requests already waiting is refused (and counted), so the reported
latencies are those of a load the device sustains.

``python -m paper_2001_04789_gb300.serve --seconds 20`` prints one JSON line with
completed and refused requests, solves/s and p50/p99 latency from arrival.
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


def amr_bytes(specs):
    """Device bytes of a composite solve: each level's grid plus five work fields."""
    total = 0
    for sp in specs:
        d = E.desc_for(sp.problem, mixed=False, max_levels=0 if sp.level == 0 else 1)
        total += E.lib().elas_grid_bytes_estimate(d) + 5 * 3 * 8 * int(np.prod(sp.problem.n))
    return total


class ResidentCache:
    """Hierarchies kept on the device, keyed by microstructure id: a single grid
    (value (grid, problem)) or a composite AMR solve (value (amr, specs)); evicted LRU
    when the context's HBM budget would be exceeded."""

    def __init__(self, ctx, budget):
        self.ctx = ctx
        self.budget = budget
        self.grids = collections.OrderedDict()     # id -> (grid or amr, problem or specs)
        self.busy = set()

    def get(self, mid, factory):
        if mid in self.grids:
            self.grids.move_to_end(mid)
            return self.grids[mid]
        p = factory()
        amr = isinstance(p, list)
        need = amr_bytes(p) if amr else E.lib().elas_grid_bytes_estimate(E.desc_for(p, mixed=True))
        while self.ctx.bytes_in_use() + need > self.budget:
            victim = next((k for k in self.grids if k not in self.busy), None)
            if victim is None:
                return None
            g, _ = self.grids.pop(victim)
            g.close()
        g = E.Amr(self.ctx, p, mixed=True) if amr else E.grid_from_problem(self.ctx, p, mixed=True)
        self.grids[mid] = (g, p)
        return self.grids[mid]

    def close(self):
        for g, _ in self.grids.values():
            g.close()
        self.grids.clear()


def make_entry(mid):
    kind, n, seed = mid
    if kind.startswith("amr_"):
        return M.amr_request_layout(kind[4:], n, seed=seed)
    return make_problem(kind, n, seed=seed)


def scale_entry(g, p, sc):
    if isinstance(p, list):
        for grid, sp in zip(g.grids, p):
            scale_loads(grid, sp.problem, sc)
    else:
        scale_loads(g, p, sc)


def run(seconds=20.0, rate=200.0, sizes=(65, 129), kinds=("sphere", "crack", "polycrystal"),
        variants=2, budget=150 << 30, max_active=16, seed=0, rel_tol=1e-8, device=0,
        amr_kinds=(), amr_sizes=(65,), max_queue=None, prewarm=False):
    rng = np.random.default_rng(seed)
    ctx = E.Context(device, budget_bytes=budget)
    server = E.Server(ctx, max_active=max_active)
    cache = ResidentCache(ctx, budget)
    catalogue = [(k, n, v) for k in kinds for n in sizes for v in range(variants)]
    catalogue += [("amr_" + k, n, v) for k in amr_kinds for n in amr_sizes for v in range(variants)]
    pending = collections.deque()          # (arrival, mid, scale) waiting for a free grid
    inflight = {}                          # ticket -> (arrival, mid)
    latencies, results = [], []
    refused = 0
    t_prewarm = 0.0
    if prewarm:
        # resident hierarchies: every microstructure of the catalogue is generated and set
        # up on the device before the stream starts (as far as the budget allows)
        t = time.perf_counter()
        for mid in catalogue:
            cache.get(mid, lambda mid=mid: make_entry(mid))
        t_prewarm = time.perf_counter() - t
    t0 = time.perf_counter()
    next_arrival = rng.exponential(1.0 / rate)
    steps = 0
    active_sum = 0
    while True:
        now = time.perf_counter() - t0
        while next_arrival <= now and next_arrival < seconds:
            mid = catalogue[int(rng.integers(len(catalogue)))]
            sc = float(rng.uniform(0.5, 1.5))
            if max_queue is not None and len(pending) >= max_queue:
                refused += 1
            else:
                pending.append((next_arrival, mid, sc))
            next_arrival += rng.exponential(1.0 / rate)
        # submit every pending request whose grid is resident and idle
        keep = collections.deque()
        for arr, mid, sc in pending:
            if mid in cache.busy:
                keep.append((arr, mid, sc))
                continue
            entry = cache.get(mid, lambda mid=mid: make_entry(mid))
            if entry is None:
                keep.append((arr, mid, sc))
                continue
            g, p = entry
            scale_entry(g, p, sc)
            if isinstance(p, list):
                t = server.submit_amr(g, precision=E.MIXED, rel_tol=rel_tol, max_cycles=200, warm_start=True)
            else:
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
        "completed": len(results), "refused": refused, "max_queue": max_queue,
        "prewarm_seconds": t_prewarm,
        "seconds": elapsed, "solves_per_s": len(results) / elapsed,
        "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3)},
        "rate": rate, "steps": steps, "mean_active": active_sum / max(steps, 1),
        "converged": sum(1 for r in results if r["status"] == 0),
        "mean_cycles": float(np.mean([r["cycles"] for r in results])) if results else None,
        "sizes": list(sizes), "kinds": list(kinds), "amr_kinds": list(amr_kinds), "amr_sizes": list(amr_sizes),
        "max_active": max_active,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seconds", type=float, default=20.0)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--sizes", default="65,129")
    ap.add_argument("--max-active", type=int, default=16)
    ap.add_argument("--amr", default="", help="AMR request kinds, e.g. sphere,crack,polycrystal")
    ap.add_argument("--amr-sizes", default="65", help="base node counts of the AMR requests")
    ap.add_argument("--kinds", default="sphere,crack,polycrystal", help="single-grid request kinds")
    ap.add_argument("--max-queue", type=int, default=None, help="refuse arrivals beyond this many waiting")
    ap.add_argument("--prewarm", action="store_true", help="create every hierarchy before the stream starts")
    a = ap.parse_args()
    out = run(seconds=a.seconds, rate=a.rate, sizes=tuple(int(v) for v in a.sizes.split(",")),
              max_active=a.max_active, kinds=tuple(k for k in a.kinds.split(",") if k),
              amr_kinds=tuple(k for k in a.amr.split(",") if k),
              amr_sizes=tuple(int(v) for v in a.amr_sizes.split(",")), max_queue=a.max_queue,
              prewarm=a.prewarm)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
