"""Geometric multigrid of the oracle: hierarchy, transfers, smoother, bottom, cycle.

Test infrastructure (see the package docstring).  Follows Section 3.1 (the
multigrid hierarchy of levels below AMR level 0, operator equivalence through
rediscretisation on every level) and Section 3.2 (trilinear interpolation
I_nm, restriction R_mn by the standard power-of-two weights).

Readings where the paper is silent or where this solver departs from it on
purpose (each is listed in the design notes):

* cycle: V(nu1, nu2) with a red-black nodal block Gauss-Seidel smoother (the
  paper's runs use F-cycles with Jacobi sweeps, Section 3.1).  Within one colour
  every row is evaluated with the values from before that half-sweep
  (Jacobi-within-colour), so the result does not depend on evaluation order;
  red = (i + j + k) even is swept first, omega = 1;
* coarsening: node count (n - 1) / 2 + 1 per non-periodic direction, n / 2 per
  periodic one, while every direction stays coarsenable and some direction has
  more than 5 nodes; coarse operators are rediscretised with moduli restricted by
  the same weights as residuals; boundary types carry over, Dirichlet values 0;
* restriction = V_c^-1 P^T V_f with node control volumes V (half volumes on
  boundary planes): (1/4, 1/2, 1/4) in the interior, (1/2, 1/2) at a boundary
  node; prolongation = trilinear interpolation, added on non-Dirichlet rows;
* bottom: dense solve of the coarsest operator assembled column by column;
* rigid-body modes left free by the boundary conditions (translations of a
  periodic grid, rigid motions of traction-free parts) make the operator
  singular.  The product-rule operator is not in divergence form, so the
  discrete right-hand side is in general not in its range.  The solve therefore
  adds an equilibrating load W lambda (W = the free rigid modes) that absorbs the
  incompatible part of the residual, and removes the rigid-mode part of u at the
  end;
* convergence test: the residual after the pre-smoothing of a cycle, relative to
  the residual of the Dirichlet-only initial field; when it is at or below the
  tolerance the solve stops with that field.

Options beside the default (the comparison with the paper's own cycle):

* smoother "gs8": eight colours (i mod 2, j mod 2, k mod 2), swept in the order
  c = (i mod 2) + 2 (j mod 2) + 4 (k mod 2), each colour Jacobi within itself.  No
  two nodes of one colour are neighbours in the 19-point interior stencil, so on
  interior rows this is block Gauss-Seidel in the colour ordering;
* smoother "jacobi": damped nodal block Jacobi, u <- u + omega B^-1 r on every node
  at once.  The paper smooths with Jacobi iterations (Section 3.1) and states no
  weight; the reading is omega = 2/3, the usual damping of Jacobi as a smoother;
* cycle "F" (Section 3.1: the paper's runs use F-cycles only): the coarse-grid
  correction of level l is an F-cycle on level l + 1 from zero followed by a
  V-cycle on level l + 1 from that result; the coarsest level is solved exactly.
  The paper's schedule, two Jacobi iterations per smoothing operation and four
  smoothing operations per level, is read as F(4, 4) with Jacobi: four iterations
  before and four after each coarse-grid correction.
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np

from paper_2001_04789_gb300.microstructure import DIRICHLET, Problem
from . import stencil as S


# --------------------------------------------------------------------------
# transfers (Section 3.2)
# --------------------------------------------------------------------------

def restrict_axis(a, d, periodic):
    ax = a.ndim - 1 - d
    a = np.moveaxis(a, ax, -1)
    e = a[..., 0::2]
    o = a[..., 1::2]
    if periodic:
        c = 0.5 * e + 0.25 * o + 0.25 * np.roll(o, 1, axis=-1)
    else:
        c = 0.5 * e
        c[..., 1:-1] += 0.25 * o[..., 1:] + 0.25 * o[..., :-1]
        c[..., 0] += 0.5 * o[..., 0]
        c[..., -1] += 0.5 * o[..., -1]
    return np.moveaxis(c, -1, ax)


def prolong_axis(c, d, periodic):
    ax = c.ndim - 1 - d
    c = np.moveaxis(c, ax, -1)
    nc = c.shape[-1]
    nf = 2 * nc if periodic else 2 * nc - 1
    f = np.zeros(c.shape[:-1] + (nf,))
    f[..., 0::2] = c
    if periodic:
        f[..., 1::2] = 0.5 * (c + np.roll(c, -1, axis=-1))
    else:
        f[..., 1::2] = 0.5 * (c[..., :-1] + c[..., 1:])
    return np.moveaxis(f, -1, ax)


def restrict(a, level):
    for d in range(3):
        a = restrict_axis(a, d, level.periodic[d])
    return a


def prolong(c, fine_level):
    for d in range(3):
        c = prolong_axis(c, d, fine_level.periodic[d])
    return c


# --------------------------------------------------------------------------
# hierarchy (Section 3.1, levels below 0)
# --------------------------------------------------------------------------

def coarsenable(level):
    ok = True
    for d in range(3):
        n = level.n[d]
        if level.periodic[d]:
            ok &= (n % 2 == 0) and (n // 2 >= 4)
        else:
            ok &= ((n - 1) % 2 == 0) and ((n - 1) // 2 + 1 >= 3)
    return ok and max(level.n) > 5


def coarsen(level):
    n = tuple(level.n[d] // 2 if level.periodic[d] else (level.n[d] - 1) // 2 + 1 for d in range(3))
    h = tuple(2.0 * level.h[d] for d in range(3))
    return S.Level(n=n, periodic=level.periodic, h=h, moduli_kind=level.moduli_kind,
                   moduli=restrict(level.moduli, level), bc_types=level.bc_types.copy(),
                   bc_values=np.zeros_like(level.bc_values), lo=level.lo, face_values=None)


@dataclasses.dataclass
class LevelData:
    level: S.Level
    types: np.ndarray
    Binv: np.ndarray          # (nz, ny, nx, 3, 3)
    colour: np.ndarray        # (nz, ny, nx) 0 = red, 1 = black
    null: np.ndarray          # (m, 3, nz, ny, nx) free rigid modes
    dense: object = None      # bottom: (free mask, matrix)


def rigid_modes(level, types):
    """Rigid motions (3 translations, 3 rotations about the grid centre) that vanish on
    every Dirichlet row and are periodic in every periodic direction."""
    sh = level.shape
    h = level.h
    ax = [level.lo[d] + h[d] * np.arange(level.n[d]) for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    ctr = [0.5 * (ax[d][0] + ax[d][-1]) for d in range(3)]
    x = [X - ctr[0], Y - ctr[1], Z - ctr[2]]
    modes = []
    for c in range(3):
        m = np.zeros((3,) + sh)
        m[c] = 1.0
        modes.append(m)
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        if level.periodic[b] or level.periodic[c]:
            continue
        m = np.zeros((3,) + sh)
        m[b] = -x[c]          # e_a x x
        m[c] = x[b]
        modes.append(m)
    modes = np.stack(modes)
    dmask = types == DIRICHLET
    M = np.stack([mo[dmask] for mo in modes], axis=1) if dmask.any() else np.zeros((0, len(modes)))
    if M.shape[0] == 0:
        basis = np.eye(len(modes))
    else:
        _, sv, vt = np.linalg.svd(M, full_matrices=True)
        rank = int(np.sum(sv > 1e-10 * max(sv.max(), 1.0)))
        basis = vt[rank:].T
    out = np.einsum("mq,m...->q...", basis, modes)
    for q in range(out.shape[0]):
        out[q] = np.where(dmask, 0.0, out[q])
    return out


def assemble_dense(level, types):
    """Matrix of the operator over the non-Dirichlet rows, one column per unit vector."""
    free = types != DIRICHLET
    idx = np.flatnonzero(free)
    A = np.zeros((idx.size, idx.size))
    for col, q in enumerate(idx):
        e = np.zeros(free.size)
        e[q] = 1.0
        A[:, col] = S.apply(level, e.reshape(free.shape), types)[free]
    return free, A


def build_hierarchy(level0):
    levels = [level0]
    while coarsenable(levels[-1]):
        levels.append(coarsen(levels[-1]))
    out = []
    for lv in levels:
        types = S.row_types(lv)
        B = S.block_diagonal(lv, types)
        Binv = np.linalg.inv(np.moveaxis(B, (0, 1), (-2, -1)))
        k, j, i = np.meshgrid(*[np.arange(s) for s in lv.shape], indexing="ij")
        colour = (i + j + k) % 2
        out.append(LevelData(lv, types, Binv, colour, rigid_modes(lv, types)))
    out[-1].dense = assemble_dense(out[-1].level, out[-1].types)
    return out


# --------------------------------------------------------------------------
# smoother, bottom, cycle
# --------------------------------------------------------------------------

def half_sweep(L: LevelData, u, f, colour):
    """One colour of the red-black nodal block smoother (Jacobi within the colour):
    u_p <- u_p + B_p^-1 r_p for every node p of that colour."""
    r = S.residual(L.level, u, f, L.types)
    delta = np.einsum("...ik,k...->i...", L.Binv, r)
    u += np.where(L.colour == colour, delta, 0.0)


def colour8(shape):
    """Eight-colour index (i mod 2) + 2 (j mod 2) + 4 (k mod 2) of every node."""
    k, j, i = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    return (i % 2) + 2 * (j % 2) + 4 * (k % 2)


def colour_pass(L: LevelData, u, f, mask, omega=1.0):
    """u_p <- u_p + omega B_p^-1 r_p on the nodes of `mask`, every row evaluated with
    the values from before the pass."""
    r = S.residual(L.level, u, f, L.types)
    delta = np.einsum("...ik,k...->i...", L.Binv, r)
    u += np.where(mask, omega * delta, 0.0)


@dataclasses.dataclass(frozen=True)
class Smoother:
    """Smoother of the cycle: "rb" (red-black, the default), "gs8" (eight colours) or
    "jacobi" (damped block Jacobi with weight omega).  One sweep is red + black, the
    eight colours, or one Jacobi iteration."""
    kind: str = "rb"
    omega: float = 2.0 / 3.0


RB = Smoother()


def sweep(L, u, f, sm: Smoother = RB):
    if sm.kind == "rb":
        half_sweep(L, u, f, 0)
        half_sweep(L, u, f, 1)
    elif sm.kind == "gs8":
        c8 = colour8(L.level.shape)
        for c in range(8):
            colour_pass(L, u, f, c8 == c)
    elif sm.kind == "jacobi":
        colour_pass(L, u, f, np.ones(L.level.shape, dtype=bool), sm.omega)
    else:
        raise ValueError(sm.kind)


def bottom_solve(L: LevelData, f):
    """Exact solve of the coarsest level.  With free rigid modes N the bordered system
    [A N; N^T 0][e; mu] = [f; 0] is solved, which absorbs any incompatible part of f."""
    free, A = L.dense
    rhs = f[free]
    m = L.null.shape[0]
    if m:
        N = np.stack([nm[free] for nm in L.null], axis=1)
        K = np.block([[A, N], [N.T, np.zeros((m, m))]])
        x = np.linalg.solve(K, np.concatenate([rhs, np.zeros(m)]))[: rhs.size]
    else:
        x = np.linalg.solve(A, rhs)
    e = np.zeros(f.shape)
    e[free] = x
    return e


def vcycle(levels, l, u, f, nu1, nu2, sm: Smoother = RB, cycle="V"):
    """One cycle on level l from the current u: nu1 sweeps, the coarse-grid correction
    (of the V or F kind), nu2 sweeps; the coarsest level is solved exactly."""
    L = levels[l]
    if l == len(levels) - 1:
        u[...] = bottom_solve(L, f)
        return
    for _ in range(nu1):
        sweep(L, u, f, sm)
    r = S.residual(L.level, u, f, L.types)
    correct(levels, l, u, r, nu1, nu2, sm, cycle)
    for _ in range(nu2):
        sweep(L, u, f, sm)


def correct(levels, l, u, r, nu1, nu2, sm: Smoother = RB, cycle="V"):
    """Coarse-grid correction: restrict r, cycle on the next level from zero (for an F
    cycle: an F-cycle, then a V-cycle from its result), add the interpolated
    correction on non-Dirichlet rows."""
    L = levels[l]
    if l == len(levels) - 1:
        # a single-level hierarchy: the correction is the exact (bordered) solve
        u += bottom_solve(L, r)
        return
    fc = restrict(r, L.level)
    Lc = levels[l + 1]
    fc = np.where(Lc.types == DIRICHLET, 0.0, fc)
    uc = np.zeros_like(fc)
    if cycle == "F":
        vcycle(levels, l + 1, uc, fc, nu1, nu2, sm, "F")
        vcycle(levels, l + 1, uc, fc, nu1, nu2, sm, "V")
    else:
        vcycle(levels, l + 1, uc, fc, nu1, nu2, sm, "V")
    u += np.where(L.types == DIRICHLET, 0.0, prolong(uc, L.level))


def norm2(a):
    return float(np.sqrt(np.sum(a * a)))


@dataclasses.dataclass
class SolveInfo:
    cycles: int
    rel_history: list
    rel_residual: float
    converged: bool
    lam: np.ndarray
    r0: float


def equilibrate(null, r, lam):
    """Absorb the rigid-mode part of the residual into the equilibrating load."""
    m = null.shape[0]
    if m == 0:
        return r, lam
    Nf = null.reshape(m, -1)
    dl = np.linalg.solve(Nf @ Nf.T, Nf @ r.reshape(-1))
    return r - np.einsum("p,p...->...", dl, null), lam + dl


def solve(problem: Problem, tol=1e-8, max_cycles=100, nu1=2, nu2=2, u0=None, levels=None,
          f=None, fixed_cycles=None, smoother: Smoother = RB, cycle="V"):
    """FP64 V(nu1, nu2) (or F(nu1, nu2)) solve.  Returns (u, info).  With
    ``fixed_cycles`` the solve runs exactly that many coarse-grid corrections and stops
    after the next pre-smoothing."""
    if levels is None:
        levels = build_hierarchy(S.level_from_problem(problem))
    L0 = levels[0]
    if f is None:
        f = S.rhs(L0.level, problem)
    uD = S.dirichlet_values(L0.level, problem.dirichlet_values)
    u = uD.copy()
    if u0 is not None:
        u = np.where(L0.types == DIRICHLET, uD, u0)
    r0 = norm2(S.residual(L0.level, uD, f, L0.types))
    lam = np.zeros(L0.null.shape[0])
    hist = []
    converged = False
    cycles = 0
    while True:
        feff = f - np.einsum("p,p...->...", lam, L0.null) if lam.size else f
        for _ in range(nu1):
            sweep(L0, u, feff, smoother)
        r = S.residual(L0.level, u, feff, L0.types)
        r, lam = equilibrate(L0.null, r, lam)
        rel = norm2(r) / r0 if r0 > 0 else 0.0
        hist.append(rel)
        if fixed_cycles is None:
            if rel <= tol:
                converged = True
                break
            if cycles >= max_cycles:
                break
        elif cycles >= fixed_cycles:
            converged = rel <= tol
            break
        feff = f - np.einsum("p,p...->...", lam, L0.null) if lam.size else f
        correct(levels, 0, u, r, nu1, nu2, smoother, cycle)
        for _ in range(nu2):
            sweep(L0, u, feff, smoother)
        cycles += 1
    u = remove_rigid(L0.null, u)
    return u, SolveInfo(cycles, hist, hist[-1], converged, lam, r0)


def remove_rigid(null, u):
    m = null.shape[0]
    if m == 0:
        return u
    Nf = null.reshape(m, -1)
    c = np.linalg.solve(Nf @ Nf.T, Nf @ u.reshape(-1))
    return u - np.einsum("p,p...->...", c, null)
