"""Composite (block-structured AMR) cycle of the oracle, reflux-free (Section 3.2).

Test infrastructure (see the package docstring).

Levels 0..L: level 0 covers the domain and carries the geometric-multigrid
hierarchy of Section 3.1 (levels below 0); level l >= 1 is one box at spacing
h_0 / 2^l, properly nested, with one ghost layer on each coarse/fine face.

Reading of Section 3.2 and Appendix A taken here (listed in the design notes):

* the valid nodes of a fine level include its coarse/fine boundary nodes, which
  are relaxed with the ordinary stencil; the ghost layer beyond them is a
  Dirichlet boundary whose values are the trilinear interpolation I_nm of the
  coarser level (Section 3.2, "interpolation operator");
* a coarse node that coincides with a valid fine node is covered: it takes the
  fine value (injection; Appendix A, where the coarse node at the coarse/fine
  boundary equals the fine one), so the ghost interpolation sees the fine
  solution and no flux correction (reflux) is needed;
* composite equations: fine rows on valid fine nodes, coarse rows on uncovered
  coarse nodes.  Coarse rows next to the fine region read covered neighbours,
  i.e. the injected fine values;
* the residual of a covered coarse node is the restriction R_mn of the fine
  residual: the single-grid weights (1/4, 1/2, 1/4) / (1/2, 1/2) per direction,
  truncated to valid fine nodes and renormalised;
* cycle (correction scheme, finest to coarsest and back): relax the correction on
  each fine level with zero ghosts, pass its remaining residual down, run the
  level-0 V-cycle on the composite residual, then on the way up add the
  interpolated coarse correction on all valid fine nodes, set the ghosts from it,
  and relax again; finally add the corrections and inject fine values into covered
  coarse nodes.

Reading R2 (``reading="R2"``), the other reading of Section 3.2 ("N + 1 ghost
nodes" with N = 1): fine grids carry two ghost layers on each coarse/fine face.  The
inner layer is relaxed with the valid nodes (it is the epsilon-neighbourhood of the
valid region); only the outer layer is a Dirichlet boundary filled by interpolation.
Every covered coarse node then has its whole restriction footprint among relaxed
fine nodes, so residuals, moduli and the solution itself pass down by the untruncated
full-weighting restriction (no injection).  Covered Dirichlet coarse rows keep their
boundary values.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from paper_2001_04789_gb300.microstructure import DIRICHLET
from . import multigrid as MG
from . import stencil as S


@dataclasses.dataclass
class AmrData:
    spec: object                 # microstructure.AmrLevel
    L: MG.LevelData              # smoother data of the level's grid
    f: np.ndarray
    levels0: list = None         # level 0 only: its multigrid hierarchy
    ghost_mask: np.ndarray = None   # Dirichlet ghost nodes (filled by interpolation)
    valid_mask: np.ndarray = None
    covered: np.ndarray = None   # nodes covered by the next finer level
    relax_mask: np.ndarray = None   # relaxed nodes: valid (R1), valid + inner ghost layer (R2)
    relax_spec: object = None       # the spec with its valid box grown to the relaxed nodes
    reading: str = "R1"


def _single_level(level):
    types = S.row_types(level)
    B = S.block_diagonal(level, types)
    Binv = np.linalg.inv(np.moveaxis(B, (0, 1), (-2, -1)))
    k, j, i = np.meshgrid(*[np.arange(s) for s in level.shape], indexing="ij")
    return MG.LevelData(level, types, Binv, (i + j + k) % 2, np.zeros((0, 3) + level.shape))


def _coords_1d(spec, d):
    return spec.grid_lo[d] + np.arange(spec.problem.n[d])


def relaxed_spec(sp, reading):
    """The spec with its valid box grown to the nodes that are relaxed: the valid box
    itself (R1), or the valid box and the inner ghost layer of each coarse/fine face (R2)."""
    if reading == "R1" or sp.level == 0:
        return sp
    lo = tuple(sp.valid_lo[d] - (1 if sp.ghost[2 * d] else 0) for d in range(3))
    hi = tuple(sp.valid_hi[d] + (1 if sp.ghost[2 * d + 1] else 0) for d in range(3))
    return dataclasses.replace(sp, valid_lo=lo, valid_hi=hi)


def coarse_moduli(specs, reading="R1"):
    """Operator equivalence across AMR levels (Section 3.1): a covered coarse node
    takes the restriction of the finer level's moduli, exactly as the multigrid
    levels below 0 take restricted moduli.  Returns one moduli array per level."""
    mods = [np.array(sp.problem.moduli, dtype=np.float64) for sp in specs]
    n0 = specs[0].problem.n
    for l in range(len(specs) - 1, 0, -1):
        counts = tuple((n0[d] - 1) * 2 ** l + 1 for d in range(3))
        restrict_field(relaxed_spec(specs[l], reading), mods[l], specs[l - 1], mods[l - 1], counts)
    return mods


def build(specs, reading="R1"):
    if reading not in ("R1", "R2"):
        raise ValueError(reading)
    out = []
    mods = coarse_moduli(specs, reading)
    specs = [dataclasses.replace(sp, problem=dataclasses.replace(sp.problem, moduli=mod))
             for sp, mod in zip(specs, mods)]
    for sp in specs:
        lev = S.level_from_problem(sp.problem)
        if sp.level == 0:
            levels0 = MG.build_hierarchy(lev)
            Ld = levels0[0]
        else:
            levels0 = None
            Ld = _single_level(lev)
        f = S.rhs(lev, sp.problem)
        rsp = relaxed_spec(sp, reading)
        masks = []
        for box in (sp, rsp):
            m = np.ones(lev.shape, dtype=bool)
            for d in range(3):
                g = _coords_1d(sp, d)
                ok = (g >= box.valid_lo[d]) & (g <= box.valid_hi[d])
                shape = [1, 1, 1]
                shape[2 - d] = -1
                m &= ok.reshape(shape)
            masks.append(m)
        valid, relax = masks
        out.append(AmrData(sp, Ld, f, levels0, ~relax, valid, relax_mask=relax, relax_spec=rsp, reading=reading))
    for l in range(len(out) - 1):
        c, fn = out[l], out[l + 1]
        cov = np.ones(c.L.level.shape, dtype=bool)
        for d in range(3):
            g = _coords_1d(c.spec, d)
            ok = (2 * g >= fn.spec.valid_lo[d]) & (2 * g <= fn.spec.valid_hi[d])
            shape = [1, 1, 1]
            shape[2 - d] = -1
            cov &= ok.reshape(shape)
        c.covered = cov
    out[-1].covered = np.zeros(out[-1].L.level.shape, dtype=bool)
    return out


# --------------------------------------------------------------------------
# transfers between AMR levels
# --------------------------------------------------------------------------

def interpolate(coarse: AmrData, cfield, fine: AmrData):
    """I_nm: trilinear interpolation of a coarse field at every node of the fine grid
    (fine global node g sits on coarse node g/2, or between (g-1)/2 and (g+1)/2)."""
    idx, wts = [], []
    for d in range(3):
        g = _coords_1d(fine.spec, d)
        i0 = g // 2 - coarse.spec.grid_lo[d]
        i1 = (g + 1) // 2 - coarse.spec.grid_lo[d]
        w1 = np.where(g % 2 == 1, 0.5, 0.0)
        idx.append((i0, i1))
        wts.append((1.0 - w1, w1))
    out = np.zeros((3,) + fine.L.level.shape)
    for a in range(2):
        for b in range(2):
            for c in range(2):
                w = (wts[2][c][:, None, None] * wts[1][b][None, :, None] * wts[0][a][None, None, :])
                vals = cfield[:, idx[2][c][:, None, None], idx[1][b][None, :, None], idx[0][a][None, None, :]]
                out += w[None] * vals
    return out


def fill_ghosts(coarse: AmrData, cfield, fine: AmrData, ffield):
    """Ghost layer of the fine level = interpolated coarse field (Dirichlet data)."""
    interp = interpolate(coarse, cfield, fine)
    ffield[:] = np.where(fine.ghost_mask[None], interp, ffield)


def inject(fine: AmrData, ffield, coarse: AmrData, cfield):
    """Covered coarse nodes take the value of the coincident fine node."""
    gi = [_coords_1d(coarse.spec, d) for d in range(3)]
    fi = [2 * gi[d] - fine.spec.grid_lo[d] for d in range(3)]
    ok = [(2 * gi[d] >= fine.spec.valid_lo[d]) & (2 * gi[d] <= fine.spec.valid_hi[d]) for d in range(3)]
    zc, yc, xc = [np.flatnonzero(ok[d]) for d in (2, 1, 0)]
    cfield[:, zc[:, None, None], yc[None, :, None], xc[None, None, :]] = \
        ffield[:, fi[2][zc][:, None, None], fi[1][yc][None, :, None], fi[0][xc][None, None, :]]


def _restrict_weights_1d(gc, fine_spec, d, n_level_fine):
    """Per-direction weights of fine offsets -1, 0, +1 for coarse global node gc."""
    fc = 2 * gc
    if fc == 0:
        w = {0: 0.5, 1: 0.5}
    elif fc == n_level_fine - 1:
        w = {-1: 0.5, 0: 0.5}
    else:
        w = {-1: 0.25, 0: 0.5, 1: 0.25}
    w = {o: v for o, v in w.items() if fine_spec.valid_lo[d] <= fc + o <= fine_spec.valid_hi[d]}
    s = sum(w.values())
    return {o: v / s for o, v in w.items()}


def restrict_residual(fine: AmrData, fres, coarse: AmrData, cres, n_level_fine):
    """R_mn at covered coarse nodes: weights truncated to relaxed fine nodes (the valid
    ones in R1) and renormalised (applied direction by direction: the weights are a
    tensor product)."""
    restrict_field(fine.relax_spec, fres, coarse.spec, cres, n_level_fine)
    cres[:] = np.where(coarse.L.types == DIRICHLET, 0.0, cres)


def sync_covered(fine: AmrData, ffield, coarse: AmrData, cfield, n_level_fine):
    """Covered coarse nodes from the fine solution: injection (R1), or the full-weighting
    restriction over the relaxed fine nodes on non-Dirichlet coarse rows (R2)."""
    if fine.reading == "R1":
        inject(fine, ffield, coarse, cfield)
        return
    tmp = cfield.copy()
    restrict_field(fine.relax_spec, ffield, coarse.spec, tmp, n_level_fine)
    cfield[:] = np.where(coarse.L.types == DIRICHLET, cfield, tmp)


def restrict_field(sp, fres, csp, cres, n_level_fine):
    """The same restriction for any field given on the fine grid (written in place at
    the covered nodes of the coarse grid)."""
    coarse_spec = csp
    mats, sel = [], []
    for d in range(3):
        gcs = _coords_1d(coarse_spec, d)
        ok = (2 * gcs >= sp.valid_lo[d]) & (2 * gcs <= sp.valid_hi[d])
        W = np.zeros((int(ok.sum()), sp.problem.n[d]))
        for r, gc in enumerate(gcs[ok]):
            for o, w in _restrict_weights_1d(int(gc), sp, d, n_level_fine[d]).items():
                W[r, 2 * gc + o - sp.grid_lo[d]] = w
        mats.append(W)
        sel.append(np.flatnonzero(ok))
    vals = np.einsum("zZ,yY,xX,cZYX->czyx", mats[2], mats[1], mats[0], fres, optimize=True)
    cres[:, sel[2][:, None, None], sel[1][None, :, None], sel[0][None, None, :]] = vals


# --------------------------------------------------------------------------
# composite residual and cycle
# --------------------------------------------------------------------------

def fine_level_counts(data):
    """Global node counts per direction of every level (level-l index space)."""
    n0 = data[0].spec.problem.n
    return [tuple((n0[d] - 1) * 2 ** l + 1 for d in range(3)) for l in range(len(data))]


def composite_residual(data, u):
    """Residual on every level: fine rows on valid nodes (ghosts from the coarser
    level), coarse rows elsewhere, restricted fine residual on covered nodes."""
    nl = len(data)
    counts = fine_level_counts(data)
    for l in range(nl - 1, 0, -1):
        fill_ghosts(data[l - 1], u[l - 1], data[l], u[l])
    res = []
    for l in range(nl):
        r = S.residual(data[l].L.level, u[l], data[l].f, data[l].L.types)
        r = np.where(data[l].relax_mask[None], r, 0.0)
        res.append(r)
    for l in range(nl - 1, 0, -1):
        restrict_residual(data[l], res[l], data[l - 1], res[l - 1], counts[l])
    return res


def composite_norm(data, res):
    tot = 0.0
    for l, d in enumerate(data):
        mask = d.valid_mask & ~d.covered
        tot += float(np.sum(np.where(mask[None], res[l], 0.0) ** 2))
    return np.sqrt(tot)


def initial_state(data):
    u = []
    for d in data:
        uD = S.dirichlet_values(d.L.level)
        u.append(np.where(d.ghost_mask[None], 0.0, uD))
    counts = fine_level_counts(data)
    for l in range(len(data) - 1, 0, -1):
        sync_covered(data[l], u[l], data[l - 1], u[l - 1], counts[l])
    return u


def cycle(data, u, nu1=2, nu2=2):
    """One composite correction cycle (finest to coarsest and back)."""
    nl = len(data)
    counts = fine_level_counts(data)
    res = composite_residual(data, u)
    res_pass = [r.copy() for r in res]
    cor = [np.zeros_like(x) for x in u]
    for l in range(nl - 1, 0, -1):
        Ld = data[l].L
        for _ in range(nu1):
            MG.sweep(Ld, cor[l], res[l])
        rr = S.residual(Ld.level, cor[l], res[l], Ld.types)
        res_pass[l] = np.where(data[l].relax_mask[None], rr, 0.0)
        restrict_residual(data[l], res_pass[l], data[l - 1], res_pass[l - 1], counts[l])
        if l - 1 > 0:
            res[l - 1] = np.where(data[l - 1].covered[None], res_pass[l - 1], res[l - 1])
    levels0 = data[0].levels0
    r0 = res_pass[0] if nl > 1 else res[0]
    MG.vcycle(levels0, 0, cor[0], r0, nu1, nu2)
    for l in range(1, nl):
        Ld = data[l].L
        interp = interpolate(data[l - 1], cor[l - 1], data[l])
        nonD = Ld.types != DIRICHLET
        cor[l] = np.where(data[l].relax_mask[None] & nonD, cor[l] + interp, cor[l])
        cor[l] = np.where(data[l].ghost_mask[None], interp, cor[l])
        for _ in range(nu2):
            MG.sweep(Ld, cor[l], res[l])
    for l in range(nl):
        u[l] += np.where(data[l].ghost_mask[None], 0.0, cor[l])
    for l in range(nl - 1, 0, -1):
        sync_covered(data[l], u[l], data[l - 1], u[l - 1], counts[l])


def solve(specs, tol=1e-8, max_cycles=100, nu1=2, nu2=2, data=None, fixed_cycles=None, reading="R1"):
    if data is None:
        data = build(specs, reading)
    u = initial_state(data)
    r0 = composite_norm(data, composite_residual(data, u))
    hist = []
    k = 0
    while True:
        rel = composite_norm(data, composite_residual(data, u)) / r0
        hist.append(rel)
        if fixed_cycles is not None:
            if k >= fixed_cycles:
                break
        elif rel <= tol or k >= max_cycles:
            break
        cycle(data, u, nu1, nu2)
        k += 1
    return u, {"cycles": k, "rel_history": hist, "rel_residual": hist[-1], "r0": r0,
               "converged": hist[-1] <= tol}
