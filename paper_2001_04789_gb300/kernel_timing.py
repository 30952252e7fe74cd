"""Time one finest-level kernel of the polycrystal workload through the C ABI.

``python -m paper_2001_04789_gb300.kernel_timing --n 129 --kernel sweep32 --shape 3``
builds the n^3 polycrystal grid (finest level only), pins the smoother's launch shape
(autotuner index) for that level, runs ``--reps`` launches of the chosen kernel on
random fields, and prints one JSON line with the mean device time per launch (CUDA
events on the library's stream) and the algorithmic and issued bandwidth.  Kernels:
``sweep32`` (one FP32 red-black sweep = two half-sweep launches), ``resid32`` (FP32
residual), ``resid64`` (FP64 residual), ``residdf`` (the double-float refinement
residual; each call also splits u and f into double-float copies, two more launches),
``restrict32`` (FP32 full-weighting restriction of level 0 to level 1) and ``prolong32``
(FP32 trilinear prolongation of a level-1 correction added to level 0).  It is also the
small profiling target for ncu captures of these kernels.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=129)
    ap.add_argument("--kernel", default="sweep32", choices=["sweep32", "resid32", "resid64", "residdf", "restrict32", "prolong32"])
    ap.add_argument("--shape", type=int, default=3, help="smoother launch shape (autotuner index)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--grains", type=int, default=10)
    a = ap.parse_args()
    import torch
    from . import build as B
    B.build()
    from . import elas as E
    from . import microstructure as M
    p = M.polycrystal(a.n, grains=a.grains, seed=0)
    ctx = E.Context(0)
    # the double-float residual and the transfers need the hierarchy; the others time level 0 alone
    hier = a.kernel in ("residdf", "restrict32", "prolong32")
    g = E.grid_from_problem(ctx, p, mixed=True, max_levels=0 if hier else 1)
    for flag in (0, 1, 2):
        E.autotune_load(f"{a.n} {a.n} {a.n} 21 4 {flag} {a.shape}")
    rng = np.random.default_rng(0)
    dt = torch.float64 if a.kernel in ("resid64", "residdf") else torch.float32
    prec = {"resid64": E.FP64, "residdf": E.OP_DF}.get(a.kernel, E.MIXED)
    u = torch.as_tensor(rng.normal(size=(3,) + g.shape) * 1e-3, dtype=dt, device="cuda:0")
    f = torch.as_tensor(rng.normal(size=(3,) + g.shape), dtype=dt, device="cuda:0")
    ec = None
    if a.kernel == "prolong32":
        nc = g.level_dims(1)
        ec = torch.as_tensor(rng.normal(size=(3, nc[2], nc[1], nc[0])) * 1e-3, dtype=dt, device="cuda:0")
    torch.cuda.synchronize()

    def once():
        if a.kernel == "sweep32":
            g.op_sweep(0, prec, u, f)
        elif a.kernel == "restrict32":
            g.op_restrict(0, prec, f)
        elif a.kernel == "prolong32":
            g.op_prolong_add(0, prec, ec, u)
        else:
            g.op_residual(0, prec, u, f)

    once()          # through the binding: its argument checks run here, untimed
    # the timed calls go to the library directly with the same pointers, so the binding's
    # host-side checks add nothing between back-to-back launches
    import ctypes
    L = E.lib()
    r = torch.empty_like(u, dtype=torch.float32 if prec == E.OP_DF else u.dtype)
    fc = g.op_restrict(0, prec, f) if a.kernel == "restrict32" else None
    pu, pf, pr = E._ptr(u), E._ptr(f), E._ptr(r)
    ss = ctypes.c_double()

    def direct():
        if a.kernel == "sweep32":
            rc = L.elas_op_sweep(g.h, 0, prec, pu, pf)
        elif a.kernel == "restrict32":
            rc = L.elas_op_restrict(g.h, 0, prec, pf, E._ptr(fc))
        elif a.kernel == "prolong32":
            rc = L.elas_op_prolong_add(g.h, 0, prec, E._ptr(ec), pu)
        else:
            rc = L.elas_op_residual(g.h, 0, prec, pu, pf, pr, ctypes.byref(ss))
        if rc:
            raise E.ElasError(rc, ctx.error())

    s = ctx.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(a.reps):
        direct()
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    N = int(np.prod(p.n))
    launches = 2 if a.kernel == "sweep32" else 1
    # algorithmic bytes per finest node and pass: each array read once, written once (a
    # coarse node per 8 fine ones)
    alg = {"sweep32": 120.0, "resid32": 120.0, "resid64": 240.0, "residdf": 240.0,
           "restrict32": 12.0 + 12.0 / 8, "prolong32": 12.0 / 8 + 24.0}[a.kernel]
    print(json.dumps({"kernel": a.kernel, "n": a.n, "nodes": N, "shape": a.shape, "reps": a.reps,
                      "ms_per_launch": ms / launches, "ms_per_pass": ms,
                      "alg_GBs": alg * N / (ms * 1e-3) / 1e9}), flush=True)
    g.close()
    ctx.close()


if __name__ == "__main__":
    main()
