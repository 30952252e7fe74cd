"""Batched RVE solves timed through the C ABI.

The members are periodic ellipsoid RVEs of uneven sizes drawn from {33, 65, 97, 129}^3
node planes (1-8 random ellipsoids each, random symmetric mean strain), all on one
context. ``elas_batch_solve`` runs each phase of a refinement step (the double-float
refinement residual, each level's half-sweeps, residual, transfers and bottom solve, the
corrections) as one launch over a device work list of all members, replays two steps at a
time from a captured CUDA graph, and stops each member on its own tolerance (FP32 V-cycles
inside FP64 refinement, relative residual 1e-8). For comparison, the same members are then
solved one after another with ``elas_solve``.

``python -m paper_2001_04789_gb300.batch --count 256`` prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import elas as E
from . import microstructure as M


def run(count=256, seed=0, rel_tol=1e-8, device=0):
    sizes = M.batch_sizes(count, seed=seed)
    t0 = time.perf_counter()
    ctx = E.Context(device)
    grids, dof = [], 0
    for i, n in enumerate(sizes):
        p = M.ellipsoid_rve(n, seed=seed * 100000 + i)
        grids.append(E.grid_from_problem(ctx, p, mixed=True))
        dof += 3 * int(np.prod(p.n))
    t_setup = time.perf_counter() - t0
    # smoother launch shapes: one tuning pass per distinct size
    tuned = set()
    for n, g in zip(sizes, grids):
        if n not in tuned:
            g.autotune()
            tuned.add(n)
    # first call (includes graph capture), then a timed call from zero
    E.batch_solve(grids, precision=E.MIXED, rel_tol=rel_tol, max_cycles=200)
    torch.cuda.synchronize()
    t = time.perf_counter()
    infos = E.batch_solve(grids, precision=E.MIXED, rel_tol=rel_tol, max_cycles=200)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t
    t = time.perf_counter()
    seq = [g.solve(precision=E.MIXED, rel_tol=rel_tol, max_cycles=200) for g in grids]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t
    out = {
        "members": count, "sizes": {str(s): sizes.count(s) for s in sorted(set(sizes))}, "dof": dof,
        "hbm_bytes": ctx.bytes_in_use(),
        "batch_solves_per_s": count / t_batch, "batch_seconds": t_batch,
        "sequential_solves_per_s": count / t_seq, "sequential_seconds": t_seq,
        "batch_over_sequential": t_seq / t_batch,
        "converged": sum(1 for i in infos if i["status"] == 0),
        "max_rel_residual": max(i["rel_residual"] for i in infos),
        "mean_cycles": float(np.mean([i["cycles"] for i in infos])),
        "sequential_converged": sum(1 for i in seq if i["status"] == 0),
        "setup_seconds": t_setup,
    }
    for g in grids:
        g.close()
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=256)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    print(json.dumps(run(count=a.count, seed=a.seed)), flush=True)


if __name__ == "__main__":
    main()
