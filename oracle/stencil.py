"""Discrete operator of the oracle: interior stencil, boundary-operator rows, RHS.

Test infrastructure (see the package docstring).  Follows Section 2.1:

* the governing equations, Eq. (1a)-(1d): interior equilibrium with eigenstrain,
  and the displacement, traction and Neumann boundary conditions;
* the partitioned boundary operator (Section 2.1, text after Eq. 1d): every
  boundary node carries the row of its boundary operator and the boundary data
  enters only through the right-hand side;
* the product-rule split of Section 2.1.1:
  D(u)_i = C_ijkl,j (u_k,l - eps0_kl) + C_ijkl (u_k,lj - eps0_kl,j);
* the homogeneous / inhomogeneous split D_H(u) = D(u) - D(0), with the solution
  of D_H(u) = -(D(0) + b) (Section 2.1.1);
* the stress output sigma = C (grad u - eps0) of Eq. (1c), with the operator's first
  differences.

Readings where the paper is silent (each is listed in the design notes):

* derivatives: central first differences, compact three-point second
  differences, four-corner mixed differences, central differences of the nodal
  moduli for C_ijkl,j;
* boundary rows: first derivatives normal to a boundary plane are one-sided and
  second order, (-3 u0 + 4 u1 - u2) / 2h inward; every other first derivative at
  a boundary node is central unless that node also lies on a boundary plane of
  that direction, where it is one-sided too;
* a traction row (Eq. 1c) is the equilibrium balance of the node's half (quarter,
  eighth) control cell: the product-rule terms of the directions along which the
  node is not on a boundary, plus for each boundary direction a the difference
  between the stress at the half-cell face and the prescribed traction, divided
  by h_a / 2.  Written out, this is the traction operator C (grad u - eps0) n with
  its normal derivative corrected back to the boundary by the field equation, a
  second-order discretisation of Eq. (1c) whose diagonal block is as strong as
  an interior one.  (Rows built from one-sided normal and central tangential
  derivatives alone have a local relaxation gain above 1 for rotated cubic moduli
  and make every point or block smoother diverge.)  All rows are force densities;
* Neumann rows are  -(2/h_a) C_iaia s d_a u_i = -(2/h_a) C_iaia du0_i;
* per component, a node on several faces takes Dirichlet if any of its faces is
  Dirichlet for that component (value of the lowest-numbered such face), else
  Neumann over its Neumann faces, else the sum of the traction rows of its faces;
* periodic directions wrap indices (no boundary rows).
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import Optional

import numpy as np

from paper_2001_04789_gb300.microstructure import (DIRICHLET, MODULI_GEN21, MODULI_ISO,
                                                   NEUMANN, TRACTION, Problem)

INTERIOR = 0
VOIGT = ((0, 5, 4), (5, 1, 3), (4, 3, 2))


def upper_index(a, b):
    """Position of Voigt entry (a, b) in the 21-entry row-major upper triangle."""
    if a > b:
        a, b = b, a
    return a * (11 - a) // 2 + b


@dataclasses.dataclass
class Level:
    n: tuple
    periodic: tuple
    h: tuple
    moduli_kind: int
    moduli: np.ndarray
    bc_types: np.ndarray        # (6, 3) int
    bc_values: np.ndarray       # (6, 3) float
    lo: tuple = (0.0, 0.0, 0.0)
    face_values: Optional[dict] = None     # per-node boundary data, face -> (3, nz, ny, nx)

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])


def level_from_problem(p: Problem) -> Level:
    t = np.zeros((6, 3), dtype=np.int64)
    v = np.zeros((6, 3))
    for f in range(6):
        d = f // 2
        for c in range(3):
            if p.periodic[d]:
                continue
            t[f, c], v[f, c] = p.bc[f][c]
    return Level(n=tuple(p.n), periodic=tuple(p.periodic), h=p.h, moduli_kind=p.moduli_kind,
                 moduli=np.asarray(p.moduli, dtype=np.float64), bc_types=t, bc_values=v,
                 lo=tuple(p.lo), face_values=p.face_values)


# --------------------------------------------------------------------------
# moduli
# --------------------------------------------------------------------------

def modulus(level: Level, i, j, k, l):
    """C_ijkl at every node, or None where it is identically zero."""
    if level.moduli_kind == MODULI_ISO:
        lam, mu = level.moduli[0], level.moduli[1]
        a = 1.0 if (i == j and k == l) else 0.0
        b = (1.0 if (i == k and j == l) else 0.0) + (1.0 if (i == l and j == k) else 0.0)
        if a == 0.0 and b == 0.0:
            return None
        return a * lam + b * mu
    return level.moduli[upper_index(VOIGT[i][j], VOIGT[k][l])]


def strain_tensor(e6, k, l):
    return e6[VOIGT[k][l]]


# --------------------------------------------------------------------------
# finite differences (direction d: 0 = x, 1 = y, 2 = z)
# --------------------------------------------------------------------------

def shift(a, d, s):
    """b[p] = a[p + s e_d], wrapping at the ends (wrapped values are only used in
    periodic directions; boundary rows never read them)."""
    return np.roll(a, -s, axis=a.ndim - 1 - d)


def d1(a, d, h):
    return (shift(a, d, 1) - shift(a, d, -1)) / (2.0 * h[d])


def d2(a, d, e, h):
    if d == e:
        return (shift(a, d, 1) - 2.0 * a + shift(a, d, -1)) / (h[d] * h[d])
    pp = shift(shift(a, d, 1), e, 1)
    pm = shift(shift(a, d, 1), e, -1)
    mp = shift(shift(a, d, -1), e, 1)
    mm = shift(shift(a, d, -1), e, -1)
    return (pp - pm - mp + mm) / (4.0 * h[d] * h[e])


def plane(shape, d, idx):
    """Boolean mask of the node plane index == idx in direction d."""
    m = np.zeros(shape, dtype=bool)
    sl = [slice(None)] * 3
    sl[2 - d] = idx
    m[tuple(sl)] = True
    return m


def boundary_plane_masks(level: Level):
    """lo[d], hi[d]: masks of the boundary planes of direction d (all False if periodic)."""
    lo, hi = [], []
    for d in range(3):
        if level.periodic[d]:
            lo.append(np.zeros(level.shape, dtype=bool))
            hi.append(np.zeros(level.shape, dtype=bool))
        else:
            lo.append(plane(level.shape, d, 0))
            hi.append(plane(level.shape, d, level.n[d] - 1))
    return lo, hi


def grad_boundary(a, d, level: Level):
    """First derivative in direction d: central, except one-sided second order on the
    boundary planes of a non-periodic direction d."""
    g = d1(a, d, level.h)
    if level.periodic[d]:
        return g
    h = level.h[d]
    ax = a.ndim - 1 - d
    n = level.n[d]
    take = lambda i: np.take(a, i, axis=ax)
    sl0 = [slice(None)] * a.ndim
    sl0[ax] = 0
    g[tuple(sl0)] = (-3.0 * take(0) + 4.0 * take(1) - take(2)) / (2.0 * h)
    sl1 = [slice(None)] * a.ndim
    sl1[ax] = n - 1
    g[tuple(sl1)] = (3.0 * take(n - 1) - 4.0 * take(n - 2) + take(n - 3)) / (2.0 * h)
    return g


# --------------------------------------------------------------------------
# row classification
# --------------------------------------------------------------------------

def face_mask(level: Level, f):
    d = f // 2
    if level.periodic[d]:
        return np.zeros(level.shape, dtype=bool)
    return plane(level.shape, d, 0 if f % 2 == 0 else level.n[d] - 1)


def row_types(level: Level):
    """(3, nz, ny, nx) row type of every (component, node)."""
    types = np.full((3,) + level.shape, INTERIOR, dtype=np.int64)
    masks = [face_mask(level, f) for f in range(6)]
    on_boundary = np.zeros(level.shape, dtype=bool)
    for m in masks:
        on_boundary |= m
    for c in range(3):
        has = {DIRICHLET: np.zeros(level.shape, bool), NEUMANN: np.zeros(level.shape, bool)}
        for f in range(6):
            t = level.bc_types[f, c]
            if t in has:
                has[t] |= masks[f]
        tc = np.where(on_boundary, TRACTION, INTERIOR)
        tc = np.where(has[NEUMANN], NEUMANN, tc)
        tc = np.where(has[DIRICHLET], DIRICHLET, tc)
        types[c] = tc
    return types


def face_value(level: Level, f, c):
    """Boundary datum of face f, component c: the per-node array if one was given,
    else the face's uniform value."""
    if level.face_values is not None and f in level.face_values:
        return level.face_values[f][c]
    return level.bc_values[f, c]


def dirichlet_values(level: Level, override: Optional[np.ndarray] = None):
    """Prescribed displacement at Dirichlet rows (Eq. 1b), 0 elsewhere; the lowest
    numbered Dirichlet face wins where faces meet."""
    types = row_types(level)
    u = np.zeros((3,) + level.shape)
    for c in range(3):
        for f in reversed(range(6)):
            if level.bc_types[f, c] == DIRICHLET:
                u[c] = np.where(face_mask(level, f), face_value(level, f, c), u[c])
        if override is not None:
            u[c] = np.where(types[c] == DIRICHLET, override[c], u[c])
        u[c] = np.where(types[c] == DIRICHLET, u[c], 0.0)
    return u


# --------------------------------------------------------------------------
# the operator
# --------------------------------------------------------------------------

def centre_coefficients(level: Level):
    """c[l]: weight of the node itself in the boundary derivative of direction l,
    -3/(2h) on a low boundary plane, +3/(2h) on a high one, 0 elsewhere."""
    lo, hi = boundary_plane_masks(level)
    h = level.h
    return [np.where(lo[l], -1.5 / h[l], 0.0) + np.where(hi[l], 1.5 / h[l], 0.0) for l in range(3)]


def pde_rows(level: Level, u):
    """Interior and traction rows.

    At a node p with boundary directions B(p) (the non-periodic boundary planes it
    lies on) component i of the row is

      sum_{j not in B} sum_kl (d_j C_ijkl)(D_l u_k) + C_ijkl D_j D_l u_k      (product rule)
      - sum_{a in B} (2/h_a) s_a sum_kl Cbar_iakl Dbar_l u_k                 (half cell)

    D_l is central, or one-sided second order where p lies on a boundary plane of l;
    D_j D_j is the compact second difference.  The half-cell term closes the normal
    flux of direction a with the traction (whose data go to the right-hand side):
    Cbar is the mean of C at p and at its inward neighbour, Dbar_a u is the one-cell
    difference between them, Dbar_l u (l != a) the mean of D_l u at the two nodes.
    At interior nodes B(p) is empty and the row is D_H(u) of Section 2.1.1."""
    h = level.h
    lo, hi = boundary_plane_masks(level)
    bnd = [lo[d] | hi[d] for d in range(3)]
    g = {(k, l): grad_boundary(u[k], l, level) for k in range(3) for l in range(3)}
    out = np.zeros_like(u)
    for i, j, k, l in itertools.product(range(3), repeat=4):
        C = modulus(level, i, j, k, l)
        if C is None:
            continue
        if l == j:
            second = d2(u[k], j, j, h)
        else:
            second = grad_boundary(d1(u[k], j, h), l, level)
        out[i] += np.where(bnd[j], 0.0, d1(C, j, h) * g[(k, l)] + C * second)
    for f in range(6):
        a = f // 2
        if level.periodic[a]:
            continue
        s = -1.0 if f % 2 == 0 else 1.0
        inward = 1 if f % 2 == 0 else -1
        m = face_mask(level, f)
        for i in range(3):
            acc = np.zeros(level.shape)
            for k, l in itertools.product(range(3), repeat=2):
                C = modulus(level, i, a, k, l)
                if C is None:
                    continue
                Cbar = 0.5 * (C + shift(C, a, inward))
                if l == a:
                    Dbar = inward * (shift(u[k], a, inward) - u[k]) / h[a]
                else:
                    Dbar = 0.5 * (g[(k, l)] + shift(g[(k, l)], a, inward))
                acc += Cbar * Dbar
            out[i] += np.where(m, -(2.0 / h[a]) * s * acc, 0.0)
    return out


def neumann_rows(level: Level, u):
    """Neumann rows (Eq. 1d) in force-density form: -(2/h_a) C_iaia s D_a u_i,
    summed over the node's Neumann faces for component i."""
    h = level.h
    out = np.zeros_like(u)
    for f in range(6):
        a = f // 2
        if level.periodic[a]:
            continue
        s = -1.0 if f % 2 == 0 else 1.0
        m = face_mask(level, f)
        for i in range(3):
            if level.bc_types[f, i] != NEUMANN:
                continue
            C = modulus(level, i, a, i, a)
            out[i] += np.where(m, -(2.0 / h[a]) * C * s * grad_boundary(u[i], a, level), 0.0)
    return out


def apply(level: Level, u, types=None):
    """A u: interior / traction rows, Neumann rows, identity on Dirichlet rows."""
    if types is None:
        types = row_types(level)
    out = np.where((types == INTERIOR) | (types == TRACTION), pde_rows(level, u), 0.0)
    out = np.where(types == NEUMANN, neumann_rows(level, u), out)
    out = np.where(types == DIRICHLET, u, out)
    return out


def residual(level: Level, u, f, types=None):
    """r = f - A u on non-Dirichlet rows, 0 on Dirichlet rows."""
    if types is None:
        types = row_types(level)
    r = f - apply(level, u, types)
    return np.where(types == DIRICHLET, 0.0, r)


def rhs(level: Level, p: Problem):
    """Right-hand side: -(D(0) + b) of Section 2.1.1 on interior rows; on traction rows
    the same terms for the non-boundary directions plus, per boundary face, the
    prescribed traction of Eq. (1c) and the eigenstrain part of the half-cell stress;
    the prescribed normal derivative of Eq. (1d) on Neumann rows.  A mean strain E
    of a periodic grid enters as u = E x + u~, like an eigenstrain -E in the
    modulus-gradient term."""
    h = level.h
    types = row_types(level)
    sh = level.shape
    lo, hi = boundary_plane_masks(level)
    bnd = [lo[d] | hi[d] for d in range(3)]
    eps0 = p.eigenstrain if p.eigenstrain is not None else np.zeros((6,) + sh)
    ebar = p.mean_strain if p.mean_strain is not None else np.zeros(6)
    f = np.zeros((3,) + sh)
    if p.body_force is not None:
        f -= p.body_force
    for i, j, k, l in itertools.product(range(3), repeat=4):
        C = modulus(level, i, j, k, l)
        if C is None:
            continue
        e = strain_tensor(eps0, k, l)
        term = d1(C, j, h) * (e - strain_tensor(ebar, k, l)) + C * d1(e, j, h)
        f[i] += np.where(bnd[j], 0.0, term)
    ne = np.zeros((3,) + sh)
    for fc in range(6):
        a = fc // 2
        if level.periodic[a]:
            continue
        s = -1.0 if fc % 2 == 0 else 1.0
        inward = 1 if fc % 2 == 0 else -1
        m = face_mask(level, fc)
        for i in range(3):
            t = level.bc_types[fc, i]
            val = face_value(level, fc, i)
            if t == TRACTION:
                acc = np.zeros(sh)
                for k, l in itertools.product(range(3), repeat=2):
                    C = modulus(level, i, a, k, l)
                    if C is None:
                        continue
                    e = strain_tensor(eps0, k, l)
                    acc += 0.5 * (C + shift(C, a, inward)) * 0.5 * (e + shift(e, a, inward))
                f[i] -= np.where(m, (2.0 / h[a]) * (val + s * acc), 0.0)
            elif t == NEUMANN:
                C = modulus(level, i, a, i, a)
                ne[i] += np.where(m, -(2.0 / h[a]) * C * val, 0.0)
    out = np.where((types == INTERIOR) | (types == TRACTION), f, 0.0)
    out = np.where(types == NEUMANN, ne, out)
    return out


def block_diagonal(level: Level, types=None):
    """B[i, k] = d(A u)_i / d u_k at the same node: the 3x3 diagonal block of the
    nodal block smoother.  Identity rows on Dirichlet components."""
    if types is None:
        types = row_types(level)
    h = level.h
    sh = level.shape
    lo, hi = boundary_plane_masks(level)
    bnd = [lo[d] | hi[d] for d in range(3)]
    cl = centre_coefficients(level)
    B = np.zeros((3, 3) + sh)
    for i, j, k, l in itertools.product(range(3), repeat=4):
        C = modulus(level, i, j, k, l)
        if C is None:
            continue
        term = d1(C, j, h) * cl[l]
        if l == j:
            term = term + C * (-2.0 / (h[j] * h[j]))
        B[i, k] += np.where(bnd[j], 0.0, term)
    for f in range(6):
        a = f // 2
        if level.periodic[a]:
            continue
        s = -1.0 if f % 2 == 0 else 1.0
        inward = 1 if f % 2 == 0 else -1
        m = face_mask(level, f)
        for i, k, l in itertools.product(range(3), repeat=3):
            C = modulus(level, i, a, k, l)
            if C is None:
                continue
            Cbar = 0.5 * (C + shift(C, a, inward))
            coef = (s / h[a]) if l == a else 0.5 * cl[l]
            B[i, k] += np.where(m, -(2.0 / h[a]) * s * Cbar * coef, 0.0)
    ne = np.zeros((3, 3) + sh)
    for f in range(6):
        a = f // 2
        if level.periodic[a]:
            continue
        s = -1.0 if f % 2 == 0 else 1.0
        m = face_mask(level, f)
        for i in range(3):
            if level.bc_types[f, i] == NEUMANN:
                C = modulus(level, i, a, i, a)
                ne[i, i] += np.where(m, -(2.0 / h[a]) * C * s * cl[a], 0.0)
    for i in range(3):
        for k in range(3):
            B[i, k] = np.where(types[i] == NEUMANN, ne[i, k], B[i, k])
            B[i, k] = np.where(types[i] == DIRICHLET, 1.0 if i == k else 0.0, B[i, k])
    return B


# --------------------------------------------------------------------------
# stress (output)
# --------------------------------------------------------------------------

def stress(level: Level, u, eps0=None, ebar=None):
    """Stress sigma = C : (grad u + ebar - eps0) at every node, the quantity whose normal
    component the traction condition Eq. (1c) prescribes.  Returns the six tensor
    components 11, 22, 33, 23, 31, 12 (shape (6, nz, ny, nx)).

    grad u uses the operator's first derivatives: central, one-sided second order on
    the boundary planes of a non-periodic direction.  ebar is the mean strain of a
    periodic cell (u is then the fluctuation u~ of u = ebar x + u~), eps0 the
    eigenstrain field (6 tensor components), both optional."""
    sh = level.shape
    g = [[grad_boundary(u[k], l, level) for l in range(3)] for k in range(3)]
    eps = np.zeros((6,) + sh)
    for a, (k, l) in enumerate(((0, 0), (1, 1), (2, 2), (1, 2), (2, 0), (0, 1))):
        eps[a] = 0.5 * (g[k][l] + g[l][k])
        if ebar is not None:
            eps[a] += ebar[a]
        if eps0 is not None:
            eps[a] -= eps0[a]
    out = np.zeros((6,) + sh)
    for a, (i, j) in enumerate(((0, 0), (1, 1), (2, 2), (1, 2), (2, 0), (0, 1))):
        for k, l in itertools.product(range(3), repeat=2):
            C = modulus(level, i, j, k, l)
            if C is None:
                continue
            out[a] += C * eps[VOIGT[k][l]]
    return out
