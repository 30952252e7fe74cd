"""Pins of the CPU oracle against facts fixed by the paper or by the mathematics.

None of these re-types the oracle's own formulas: each compares it with a closed
form (polynomial fields that the second-order stencil differentiates exactly, the
analytic stress of a manufactured field, the Eshelby sphere), a brute-force
matrix (assembled column by column from the oracle and checked for symmetry,
definiteness, the smoother's matrix splitting, exact dense solves), or an
invariant (restriction = scaled transpose of interpolation, rotation invariance).
"""
import itertools

import numpy as np
import pytest

from paper_2001_04789_gb300 import microstructure as M
from oracle import multigrid as MG
from oracle import stencil as S


# --------------------------------------------------------------------------
# helpers: closed-form fields
# --------------------------------------------------------------------------

def random_general_C(rng, scale=1.0):
    """A symmetric positive-definite 6x6 Voigt matrix (random rotated cubic + iso)."""
    base = M.voigt_to_tensor(M.cubic_voigt(1.68, 1.21, 0.75))
    T = M.rotate_tensor(base, M.random_rotation(rng))
    lam, mu = M.lame(1.0, 0.25)
    T = T + M.voigt_to_tensor(M.cubic_voigt(lam + 2 * mu, lam, mu))
    return scale * T


def upper21_field(T, shape):
    v = M.tensor_to_upper21(T)
    return np.broadcast_to(v[:, None, None, None], (21,) + shape).copy()


def make_problem(n, kind, C_tensor=None, lamu=None, periodic=(False, False, False),
                 bc=None, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    p = M.Problem(n=n, periodic=periodic, lo=lo, hi=hi)
    shape = (n[2], n[1], n[0])
    if kind == M.MODULI_ISO:
        p.moduli_kind = M.MODULI_ISO
        p.moduli = np.stack([np.broadcast_to(lamu[0], shape), np.broadcast_to(lamu[1], shape)]).astype(float)
    else:
        p.moduli_kind = M.MODULI_GEN21
        p.moduli = upper21_field(C_tensor, shape)
    p.bc = bc if bc is not None else M.all_faces(M.DIRICHLET, 0.0)
    return p


def quadratic_field(rng, X, Y, Z):
    Q = rng.normal(size=(3, 3, 3))
    L = rng.normal(size=(3, 3))
    c = rng.normal(size=3)
    x = [X, Y, Z]
    u = np.zeros((3,) + X.shape)
    for k in range(3):
        u[k] = c[k]
        for a in range(3):
            u[k] += L[k, a] * x[a]
            for b in range(3):
                u[k] += Q[k, a, b] * x[a] * x[b]
    grad = np.zeros((3, 3) + X.shape)      # grad[k, l] = d u_k / d x_l
    for k, l in itertools.product(range(3), repeat=2):
        grad[k, l] = L[k, l]
        for b in range(3):
            grad[k, l] += (Q[k, l, b] + Q[k, b, l]) * x[b]
    hess = np.zeros((3, 3, 3))            # hess[k, j, l]
    for k, j, l in itertools.product(range(3), repeat=3):
        hess[k, j, l] = Q[k, j, l] + Q[k, l, j]
    return u, grad, hess


def iso_tensor(lam, mu):
    d = np.eye(3)
    T = np.zeros((3, 3, 3, 3) + np.shape(lam))
    for i, j, k, l in itertools.product(range(3), repeat=4):
        T[i, j, k, l] = lam * d[i, j] * d[k, l] + mu * (d[i, k] * d[j, l] + d[i, l] * d[j, k])
    return T


# --------------------------------------------------------------------------
# interior stencil: exact on quadratic u with affine moduli (Section 2.1.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", [M.MODULI_ISO, M.MODULI_GEN21])
def test_interior_rows_exact_for_quadratic_u_affine_moduli(kind):
    rng = np.random.default_rng(1)
    n = (7, 6, 8)
    p = make_problem(n, M.MODULI_ISO, lamu=(1.0, 1.0), lo=(0.1, -0.2, 0.3), hi=(0.9, 0.7, 1.5))
    X, Y, Z = p.coords()
    x = [X, Y, Z]
    if kind == M.MODULI_ISO:
        gl, gm = rng.normal(size=3) * 0.2, rng.normal(size=3) * 0.2
        lam = 1.0 + sum(gl[a] * x[a] for a in range(3))
        mu = 1.0 + sum(gm[a] * x[a] for a in range(3))
        p.moduli = np.stack([lam, mu])
        C = iso_tensor(lam, mu)
        dC = np.zeros((3, 3, 3, 3, 3))  # dC[i,j,k,l,m] = d C_ijkl / d x_m
        d = np.eye(3)
        for i, j, k, l in itertools.product(range(3), repeat=4):
            dC[i, j, k, l] = gl * d[i, j] * d[k, l] + gm * (d[i, k] * d[j, l] + d[i, l] * d[j, k])
    else:
        T0 = random_general_C(rng)
        G = [0.1 * random_general_C(rng) for _ in range(3)]
        Cfield = T0[..., None, None, None] + sum(G[a][..., None, None, None] * x[a] for a in range(3))
        p.moduli_kind = M.MODULI_GEN21
        p.moduli = np.stack([M.tensor_to_upper21(Cfield[..., kk, jj, ii])
                             for kk, jj, ii in itertools.product(*[range(s) for s in X.shape])],
                            axis=-1).reshape((21,) + X.shape)
        C = Cfield
        dC = np.stack(G, axis=-1)
    u, grad, hess = quadratic_field(rng, X, Y, Z)
    expect = np.zeros((3,) + X.shape)
    for i, j, k, l in itertools.product(range(3), repeat=4):
        expect[i] += dC[i, j, k, l][j] * grad[k, l] + C[i, j, k, l] * hess[k, j, l]
    lev = S.level_from_problem(p)
    got = S.pde_rows(lev, u)
    inner = (slice(None), slice(1, -1), slice(1, -1), slice(1, -1))
    assert np.allclose(got[inner], expect[inner], rtol=0, atol=1e-10 * np.abs(expect).max())


# --------------------------------------------------------------------------
# traction rows: exact for quadratic u with constant moduli (Eq. 1c)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", [M.MODULI_ISO, M.MODULI_GEN21])
def test_traction_rows_exact_for_quadratic_u_constant_moduli(kind):
    """At a boundary node with constant C and quadratic u the half-cell row must equal
    D(u) - sum_a (2/h_a) t_a with t_a = s_a sigma_ia the exact traction on face a."""
    rng = np.random.default_rng(2)
    n = (6, 7, 5)
    if kind == M.MODULI_ISO:
        p = make_problem(n, kind, lamu=(1.3, 0.7), bc=M.all_faces(M.TRACTION, 0.0),
                         lo=(-0.3, 0.0, 0.2), hi=(0.6, 1.1, 0.9))
        C = iso_tensor(1.3, 0.7)
    else:
        C = random_general_C(rng)
        p = make_problem(n, kind, C_tensor=C, bc=M.all_faces(M.TRACTION, 0.0),
                         lo=(-0.3, 0.0, 0.2), hi=(0.6, 1.1, 0.9))
    X, Y, Z = p.coords()
    u, grad, hess = quadratic_field(rng, X, Y, Z)
    sigma = np.einsum("ijkl,kl...->ij...", C, grad)
    Du = np.einsum("ijkl,kjl->i", C, hess)[:, None, None, None] * np.ones(X.shape)
    lev = S.level_from_problem(p)
    expect = Du.copy()
    h = p.h
    for f in range(6):
        a, s = f // 2, (-1.0 if f % 2 == 0 else 1.0)
        m = S.face_mask(lev, f)
        expect -= np.where(m, (2.0 / h[a]) * s * sigma[:, a], 0.0)
    got = S.pde_rows(lev, u)
    scale = np.abs(expect).max()
    assert np.allclose(got, expect, rtol=0, atol=1e-10 * scale)


def test_rhs_traction_and_eigenstrain_linear_field_has_zero_residual():
    """A uniform strain with constant C and a uniform eigenstrain is an exact solution
    when every face carries the matching uniform traction C (grad u - eps0) n."""
    rng = np.random.default_rng(3)
    C = random_general_C(rng)
    E = rng.normal(size=(3, 3)) * 1e-3
    eps0 = rng.normal(size=(3, 3)) * 1e-3
    eps0 = 0.5 * (eps0 + eps0.T)
    sigma = np.einsum("ijkl,kl->ij", C, 0.5 * (E + E.T) - eps0)
    bc = []
    for f in range(6):
        a, s = f // 2, (-1.0 if f % 2 == 0 else 1.0)
        bc.append([(M.TRACTION, s * sigma[i, a]) for i in range(3)])
    p = make_problem((7, 7, 7), M.MODULI_GEN21, C_tensor=C, bc=bc)
    X, Y, Z = p.coords()
    x = [X, Y, Z]
    u = np.stack([sum(E[k, l] * x[l] for l in range(3)) for k in range(3)])
    e6 = np.array([eps0[0, 0], eps0[1, 1], eps0[2, 2], eps0[1, 2], eps0[2, 0], eps0[0, 1]])
    p.eigenstrain = np.broadcast_to(e6[:, None, None, None], (6,) + X.shape).copy()
    lev = S.level_from_problem(p)
    r = S.residual(lev, u, S.rhs(lev, p))
    f = S.rhs(lev, p)
    assert np.abs(r).max() <= 1e-12 * max(np.abs(f).max(), 1e-3)


def test_neumann_rows_exact_for_quadratic_component():
    rng = np.random.default_rng(4)
    n = (6, 6, 6)
    bc = M.all_faces(M.NEUMANN, 0.0)
    p = make_problem(n, M.MODULI_ISO, lamu=(1.0, 0.5), bc=bc)
    X, Y, Z = p.coords()
    u, grad, _ = quadratic_field(rng, X, Y, Z)
    lev = S.level_from_problem(p)
    got = S.neumann_rows(lev, u)
    h = p.h
    C = iso_tensor(1.0, 0.5)
    expect = np.zeros_like(u)
    for f in range(6):
        a, s = f // 2, (-1.0 if f % 2 == 0 else 1.0)
        m = S.face_mask(lev, f)
        for i in range(3):
            expect[i] += np.where(m, -(2.0 / h[a]) * C[i, a, i, a] * s * grad[i, a], 0.0)
    assert np.allclose(got, expect, atol=1e-10 * np.abs(expect).max())


# --------------------------------------------------------------------------
# block diagonal = the operator's own diagonal block, found by probing
# --------------------------------------------------------------------------

def test_block_diagonal_matches_probing():
    rng = np.random.default_rng(5)
    n = (7, 6, 8)
    bc = [[(M.TRACTION, 0.0), (M.DIRICHLET, 0.0), (M.NEUMANN, 0.0)],
          [(M.TRACTION, 0.0)] * 3,
          [(M.NEUMANN, 0.0), (M.TRACTION, 0.0), (M.TRACTION, 0.0)],
          [(M.TRACTION, 0.0)] * 3,
          [(M.DIRICHLET, 0.0), (M.TRACTION, 0.0), (M.TRACTION, 0.0)],
          [(M.TRACTION, 0.0)] * 3]
    p = make_problem(n, M.MODULI_GEN21, C_tensor=random_general_C(rng), bc=bc,
                     hi=(1.0, 0.8, 1.3))
    X, Y, Z = p.coords()
    p.moduli = p.moduli * (1.0 + 0.3 * np.sin(3 * X + 2 * Y - Z))[None]
    lev = S.level_from_problem(p)
    types = S.row_types(lev)
    B = S.block_diagonal(lev, types)
    kk, jj, ii = np.meshgrid(*[np.arange(s) for s in lev.shape], indexing="ij")
    probed = np.zeros_like(B)
    for cls in itertools.product(range(3), repeat=3):
        sel = (ii % 3 == cls[0]) & (jj % 3 == cls[1]) & (kk % 3 == cls[2])
        for k in range(3):
            e = np.zeros((3,) + lev.shape)
            e[k] = np.where(sel, 1.0, 0.0)
            Ae = S.apply(lev, e, types)
            for i in range(3):
                probed[i, k] = np.where(sel, Ae[i], probed[i, k])
    assert np.allclose(B, probed, atol=1e-9 * np.abs(B).max())


# --------------------------------------------------------------------------
# brute-force matrix properties
# --------------------------------------------------------------------------

def test_constant_moduli_dirichlet_operator_symmetric_negative_definite():
    rng = np.random.default_rng(6)
    p = make_problem((5, 5, 5), M.MODULI_GEN21, C_tensor=random_general_C(rng))
    lev = S.level_from_problem(p)
    free, A = MG.assemble_dense(lev, S.row_types(lev))
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.max() < 0


def test_periodic_constant_moduli_three_zero_modes():
    lam, mu = M.lame(1.0, 0.3)
    p = make_problem((4, 4, 4), M.MODULI_ISO, lamu=(lam, mu), periodic=(True, True, True), bc=[])
    lev = S.level_from_problem(p)
    free, A = MG.assemble_dense(lev, S.row_types(lev))
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    ev = np.sort(np.linalg.eigvalsh(A))
    scale = np.abs(ev).max()
    assert np.all(np.abs(ev[-3:]) < 1e-10 * scale)
    assert ev[-4] < -1e-6 * scale


def test_variable_moduli_operator_is_stable():
    """The product-rule operator is not symmetric for varying moduli; its eigenvalues
    must still have negative real parts (Dirichlet rows eliminated)."""
    p = M.eshelby_sphere(7)
    lev = S.level_from_problem(p)
    free, A = MG.assemble_dense(lev, S.row_types(lev))
    ev = np.linalg.eigvals(A)
    assert ev.real.max() < 0
    asym = np.abs(A - A.T).max() / np.abs(A).max()
    assert asym > 1e-6          # genuinely non-symmetric


# --------------------------------------------------------------------------
# transfers (Section 3.2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("periodic", [False, True])
def test_restriction_is_volume_scaled_transpose_of_interpolation(periodic):
    nf = 8 if periodic else 9
    nc = 4 if periodic else 5
    P = np.zeros((nf, nc))
    for c in range(nc):
        e = np.zeros(nc)
        e[c] = 1.0
        P[:, c] = MG.prolong_axis(e, 0, periodic)
    R = np.zeros((nc, nf))
    for q in range(nf):
        e = np.zeros(nf)
        e[q] = 1.0
        R[:, q] = MG.restrict_axis(e, 0, periodic)
    Vf = np.ones(nf)
    Vc = 2.0 * np.ones(nc)
    if not periodic:
        Vf[[0, -1]] = 0.5
        Vc[[0, -1]] = 1.0
    assert np.allclose(R, np.diag(1.0 / Vc) @ P.T @ np.diag(Vf))
    assert np.allclose(R.sum(axis=1), 1.0)          # constants restrict to constants
    xc = np.arange(nc) * 2.0
    assert np.allclose(P @ (3.0 * xc + 1.0), 3.0 * np.arange(nf) + 1.0) or periodic


def test_trilinear_interpolation_reproduces_affine_3d():
    rng = np.random.default_rng(7)
    g = rng.normal(size=3)
    fine = S.Level(n=(9, 5, 7), periodic=(False, False, False), h=(1, 1, 1), moduli_kind=2,
                   moduli=np.zeros((2, 7, 5, 9)), bc_types=np.zeros((6, 3), int),
                   bc_values=np.zeros((6, 3)))
    kc, jc, ic = np.meshgrid(np.arange(4), np.arange(3), np.arange(5), indexing="ij")
    coarse = g[0] * 2 * ic + g[1] * 2 * jc + g[2] * 2 * kc
    kf, jf, i_f = np.meshgrid(np.arange(7), np.arange(5), np.arange(9), indexing="ij")
    assert np.allclose(MG.prolong(coarse, fine), g[0] * i_f + g[1] * jf + g[2] * kf)


# --------------------------------------------------------------------------
# smoother = its matrix splitting; bottom and cycle = dense solve
# --------------------------------------------------------------------------

def test_red_black_sweep_equals_matrix_splitting():
    p = M.polycrystal(5, grains=3, seed=2)
    levels = MG.build_hierarchy(S.level_from_problem(p))
    L = levels[0]
    free, A = MG.assemble_dense(L.level, L.types)
    rng = np.random.default_rng(8)
    u0 = np.where(L.types == M.DIRICHLET, 0.0, rng.normal(size=(3,) + L.level.shape))
    f = np.where(L.types == M.DIRICHLET, 0.0, rng.normal(size=(3,) + L.level.shape))
    u = u0.copy()
    MG.sweep(L, u, f)
    # explicit splitting with the assembled matrix
    idx = np.flatnonzero(free)
    comp, node = np.unravel_index(idx, free.shape)[0], np.ravel_multi_index(
        np.unravel_index(idx, free.shape)[1:], free.shape[1:])
    colour = L.colour.reshape(-1)[node]
    x = u0[free].copy()
    b = f[free]
    for c in (0, 1):
        r = b - A @ x
        dx = np.zeros_like(x)
        for q in np.unique(node[colour == c]):
            rows = np.flatnonzero(node == q)
            dx[rows] = np.linalg.solve(A[np.ix_(rows, rows)], r[rows])
        x = x + dx
    assert np.allclose(u[free], x, atol=1e-12 * np.abs(x).max())


def test_vcycle_solve_matches_dense_solve_dirichlet():
    p = M.eshelby_sphere(9)
    lev = S.level_from_problem(p)
    types = S.row_types(lev)
    free, A = MG.assemble_dense(lev, types)
    f = S.rhs(lev, p)
    u_ref = np.zeros_like(f)
    u_ref[free] = np.linalg.solve(A, f[free])
    u, info = MG.solve(p, tol=1e-13, max_cycles=60)
    assert info.converged
    assert np.abs(u - u_ref).max() <= 1e-10 * np.abs(u_ref).max()


def test_singular_problem_solve_matches_bordered_dense_solve():
    """Traction-free faces leave rigid modes; the solve must return the dense bordered
    solution: A u + W lam = f, W^T u = 0, with W the free rigid modes."""
    p = M.polycrystal(9, grains=3, seed=4)
    levels = MG.build_hierarchy(S.level_from_problem(p))
    L = levels[0]
    assert L.null.shape[0] == 3
    free, A = MG.assemble_dense(L.level, L.types)
    f = S.rhs(L.level, p)
    uD = S.dirichlet_values(L.level)
    b = (f - S.apply(L.level, uD, L.types))[free]
    W = np.stack([w[free] for w in L.null], axis=1)
    m = W.shape[1]
    K = np.block([[A, W], [W.T, np.zeros((m, m))]])
    sol = np.linalg.solve(K, np.concatenate([b, np.zeros(m)]))
    u_ref = uD.copy()
    u_ref[free] = sol[: b.size]
    u, info = MG.solve(p, tol=1e-13, max_cycles=200, levels=levels)
    assert info.converged
    assert np.abs(u - u_ref).max() <= 1e-9 * np.abs(u_ref).max()
    assert np.allclose(info.lam, sol[b.size:], rtol=1e-6, atol=1e-12 * np.abs(b).max())


def test_periodic_rve_solve_matches_bordered_dense_solve():
    p = M.ellipsoid_rve(9, seed=5)
    levels = MG.build_hierarchy(S.level_from_problem(p))
    L = levels[0]
    assert L.null.shape[0] == 3
    free, A = MG.assemble_dense(L.level, L.types)
    b = S.rhs(L.level, p)[free]
    W = np.stack([w[free] for w in L.null], axis=1)
    K = np.block([[A, W], [W.T, np.zeros((3, 3))]])
    sol = np.linalg.solve(K, np.concatenate([b, np.zeros(3)]))
    u, info = MG.solve(p, tol=1e-13, max_cycles=200, levels=levels)
    assert np.abs(u[free] - sol[:-3]).max() <= 1e-9 * np.abs(sol[:-3]).max()


# --------------------------------------------------------------------------
# convergence under refinement
# --------------------------------------------------------------------------

def manufactured_sine(n):
    """u = sin products, smooth isotropic moduli, body force b = -D(u) from the
    analytic derivatives, u = exact on all faces."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    X3 = (x, y, z)
    lam = 1.0 + 0.3 * sp.sin(2 * x + y) * sp.cos(z)
    mu = 0.8 + 0.2 * sp.cos(x - 2 * y + z)
    U = [sp.sin(sp.pi * x) * sp.sin(2 * y) * (1 + z), sp.cos(x + y) * sp.sin(sp.pi * z),
         x * y * sp.exp(z) + sp.sin(y)]
    eps = [[(sp.diff(U[k], X3[l]) + sp.diff(U[l], X3[k])) / 2 for l in range(3)] for k in range(3)]
    tr = eps[0][0] + eps[1][1] + eps[2][2]
    sig = [[lam * tr * (1 if i == j else 0) + 2 * mu * eps[i][j] for j in range(3)] for i in range(3)]
    D = [sum(sp.diff(sig[i][j], X3[j]) for j in range(3)) for i in range(3)]
    fn = sp.lambdify((x, y, z), [lam, mu] + U + D, "numpy")
    p = M.Problem(n=(n, n, n))
    X, Y, Z = p.coords()
    vals = [np.broadcast_to(np.asarray(v, dtype=float), X.shape) for v in fn(X, Y, Z)]
    p.moduli_kind = M.MODULI_ISO
    p.moduli = np.stack(vals[:2])
    u_exact = np.stack(vals[2:5])
    p.body_force = -np.stack(vals[5:8])
    p.bc = M.all_faces(M.DIRICHLET, 0.0)
    p.dirichlet_values = u_exact
    return p, u_exact


def test_second_order_convergence_manufactured_solution():
    errs = []
    for n in (9, 17, 33):
        p, ue = manufactured_sine(n)
        u, info = MG.solve(p, tol=1e-12, max_cycles=80)
        assert info.converged
        errs.append(np.abs(u - ue).max())
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert 1.8 < orders[-1] < 2.3, (errs, orders)


def test_traction_boundary_second_order_convergence():
    """Manufactured smooth field with Dirichlet data on the -x face and its exact
    traction sigma(u) n, node by node, on the five other faces: second order."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    X3 = (x, y, z)
    lam = 1.0 + 0.3 * sp.sin(2 * x + y) * sp.cos(z)
    mu = 0.8 + 0.2 * sp.cos(x - 2 * y + z)
    U = [sp.sin(sp.pi * x) * sp.sin(2 * y) * (1 + z), sp.cos(x + y) * sp.sin(2 * z),
         x * y * sp.exp(z) + sp.sin(y)]
    eps = [[(sp.diff(U[k], X3[l]) + sp.diff(U[l], X3[k])) / 2 for l in range(3)] for k in range(3)]
    tr = eps[0][0] + eps[1][1] + eps[2][2]
    sig = [[lam * tr * (1 if i == j else 0) + 2 * mu * eps[i][j] for j in range(3)] for i in range(3)]
    D = [sum(sp.diff(sig[i][j], X3[j]) for j in range(3)) for i in range(3)]
    flat = [lam, mu] + U + D + [sig[i][j] for i in range(3) for j in range(3)]
    fn = sp.lambdify((x, y, z), flat, "numpy")
    errs = []
    for n in (9, 17, 33):
        p = M.Problem(n=(n, n, n))
        X, Y, Z = p.coords()
        v = [np.broadcast_to(np.asarray(q, dtype=float), X.shape) for q in fn(X, Y, Z)]
        p.moduli_kind = M.MODULI_ISO
        p.moduli = np.stack(v[:2])
        ue = np.stack(v[2:5])
        p.body_force = -np.stack(v[5:8])
        S_ = np.stack(v[8:17]).reshape((3, 3) + X.shape)
        bc = M.all_faces(M.TRACTION, 0.0)
        bc[0] = [(M.DIRICHLET, 0.0)] * 3
        p.bc = bc
        p.face_values = {0: ue}
        for f in range(1, 6):
            a, s = f // 2, (-1.0 if f % 2 == 0 else 1.0)
            p.face_values[f] = s * S_[:, a]
        u, info = MG.solve(p, tol=1e-12, max_cycles=150)
        assert info.converged
        errs.append(np.abs(u - ue).max())
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert 1.8 < orders[-1] < 2.4, (errs, orders)


def eshelby_sphere_closed_form(X, Y, Z, a, eps_star, E_i, E_m, nu):
    """Sharp spherical inhomogeneity with dilatational eigenstrain eps_star I in an
    infinite matrix: u = A x inside, A a^3 x / r^3 outside, with
    A = 3 K_i eps_star / (3 K_i + 4 mu_m) (continuity of u and of radial traction)."""
    K_i = E_i / (3 * (1 - 2 * nu))
    mu_m = E_m / (2 * (1 + nu))
    A = 3 * K_i * eps_star / (3 * K_i + 4 * mu_m)
    x = [X - 0.5, Y - 0.5, Z - 0.5]
    r = np.sqrt(x[0] ** 2 + x[1] ** 2 + x[2] ** 2)
    fac = np.where(r <= a, A, A * a ** 3 / np.maximum(r, 1e-30) ** 3)
    return np.stack([fac * xi for xi in x]), r


def test_eshelby_sphere_far_field_converges_to_closed_form():
    errs = []
    for n in (17, 33):
        p = M.eshelby_sphere(n, radius=0.2)
        X, Y, Z = p.coords()
        ue, r = eshelby_sphere_closed_form(X, Y, Z, 0.2, 1e-3, 2.0, 1.0, 0.3)
        p.dirichlet_values = ue
        u, info = MG.solve(p, tol=1e-11, max_cycles=80)
        assert info.converged
        far = r >= 0.3
        errs.append(np.abs(u - ue)[:, far].max() / np.abs(ue).max())
    assert errs[1] < 0.6 * errs[0], errs
    assert errs[1] < 0.05, errs


# --------------------------------------------------------------------------
# input generators (Section 4.3)
# --------------------------------------------------------------------------

def test_rotation_invariance_of_moduli():
    rng = np.random.default_rng(9)
    lam, mu = M.lame(2.0, 0.3)
    iso = M.voigt_to_tensor(M.cubic_voigt(lam + 2 * mu, lam, mu))
    R = M.random_rotation(rng)
    assert np.allclose(R @ R.T, np.eye(3)) and np.isclose(np.linalg.det(R), 1.0)
    assert np.allclose(M.rotate_tensor(iso, R), iso)
    cub = M.voigt_to_tensor(M.cubic_voigt(1.68, 1.21, 0.75))
    R90 = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    assert np.allclose(M.rotate_tensor(cub, R90), cub)
    T = M.rotate_tensor(cub, R)
    assert np.allclose(T, np.transpose(T, (2, 3, 0, 1)))
    assert np.allclose(T, np.transpose(T, (1, 0, 2, 3)))


# --------------------------------------------------------------------------
# mean strain of a periodic cell: laminate closed form
# --------------------------------------------------------------------------

def laminate_closed_form(C0, ebar, a, x_a, alpha, beta):
    """Continuum fluctuation of a periodic laminate under the mean strain ebar.

    Moduli C(x) = C0 / (alpha + beta cos(2 pi x_a)) vary along direction a only, so
    the fluctuation u~ depends on x_a alone.  Equilibrium makes the traction on the
    layer planes, sigma_ia = C_iakl (ebar_kl + u~_k,a delta_la), uniform; with
    A_ik = C0_iaka and b_i = C0_iakl ebar_kl (tensor ebar, shears not doubled) and
    a zero-mean u~_,a this gives u~_,a = (beta / alpha) cos(2 pi x_a) A^-1 b, hence
    u~ = (beta / alpha) sin(2 pi x_a) / (2 pi) A^-1 b; the homogenised traction is
    sigma_ia = b_i / alpha."""
    E = np.array([[ebar[0], ebar[5], ebar[4]], [ebar[5], ebar[1], ebar[3]], [ebar[4], ebar[3], ebar[2]]])
    A = C0[:, a, :, a]
    b = np.einsum("ikl,kl->i", C0[:, a, :, :], E)
    amp = np.linalg.solve(A, b) * beta / alpha
    return np.einsum("k,...->k...", amp, np.sin(2 * np.pi * x_a) / (2 * np.pi)), b / alpha


def laminate_problem(n, a, kind, C0, ebar, alpha, beta):
    p = M.Problem(n=n, periodic=(True, True, True))
    X, Y, Z = p.coords()
    xa = (X, Y, Z)[a]
    scale = 1.0 / (alpha + beta * np.cos(2 * np.pi * xa))
    if kind == M.MODULI_ISO:
        lam = C0[0, 0, 1, 1]
        mu = C0[0, 1, 0, 1]
        p.moduli_kind = M.MODULI_ISO
        p.moduli = np.stack([lam * scale, mu * scale])
    else:
        p.moduli_kind = M.MODULI_GEN21
        p.moduli = M.tensor_to_upper21(C0)[:, None, None, None] * scale[None]
    p.mean_strain = np.asarray(ebar, dtype=float)
    p.bc = []
    return p, xa


@pytest.mark.parametrize("a,kind", [(0, M.MODULI_ISO), (2, M.MODULI_GEN21), (1, M.MODULI_GEN21)])
def test_periodic_laminate_mean_strain_matches_closed_form(a, kind):
    """Pins the mean-strain part of the right-hand side (u = ebar x + u~, Section
    2.1.1 product rule) against the laminate closed form: the solved fluctuation
    converges to it at second order, with the right sign and the tensor (not
    engineering) shear components, for normal and shear mean strains."""
    if kind == M.MODULI_ISO:
        lam, mu = M.lame(1.0, 0.3)
        C0 = iso_tensor(float(lam), float(mu))
    else:
        rng = np.random.default_rng(11)
        C0 = M.voigt_to_tensor(M.cubic_voigt(1.68, 1.21, 0.75))
        C0 = M.rotate_tensor(C0, M.random_rotation(rng))
    ebar = np.array([0.7, -0.4, 0.25, 0.5, -0.35, 0.6]) * 1e-3
    alpha, beta = 1.0, 0.5
    errs = []
    for na in (16, 32, 64):
        n = [8, 8, 8]
        n[a] = na
        p, xa = laminate_problem(tuple(n), a, kind, C0, ebar, alpha, beta)
        u, info = MG.solve(p, tol=1e-12, max_cycles=200)
        assert info.converged
        ue, _ = laminate_closed_form(C0, ebar, a, xa, alpha, beta)
        # the fluctuation is defined up to a translation: compare zero-mean fields
        u = u - u.mean(axis=(1, 2, 3), keepdims=True)
        errs.append(np.abs(u - ue).max() / np.abs(ue).max())
    assert errs[-1] < 2e-3, errs
    orders = [np.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]
    assert all(1.8 < o < 2.2 for o in orders), (errs, orders)


def test_periodic_laminate_homogenised_traction():
    """The mean traction on the layer planes of the discrete solution (central
    differences of u = ebar x + u~) equals the closed-form homogenised traction
    b / alpha to second order."""
    lam, mu = M.lame(1.0, 0.3)
    C0 = iso_tensor(float(lam), float(mu))
    ebar = np.array([0.7, -0.4, 0.25, 0.5, -0.35, 0.6]) * 1e-3
    alpha, beta = 1.0, 0.5
    p, xa = laminate_problem((64, 8, 8), 0, M.MODULI_ISO, C0, ebar, alpha, beta)
    u, info = MG.solve(p, tol=1e-12, max_cycles=200)
    _, t_exact = laminate_closed_form(C0, ebar, 0, xa, alpha, beta)
    h = p.h[0]
    E = np.array([[ebar[0], ebar[5], ebar[4]], [ebar[5], ebar[1], ebar[3]], [ebar[4], ebar[3], ebar[2]]])
    # strain = ebar + sym grad u~ (u~ varies along x only)
    dux = (np.roll(u, -1, axis=3) - np.roll(u, 1, axis=3)) / (2 * h)
    eps = np.broadcast_to(E[:, :, None, None, None], (3, 3) + u.shape[1:]).copy()
    for k in range(3):
        eps[k, 0] += 0.5 * dux[k]
        eps[0, k] += 0.5 * dux[k]
    scale = 1.0 / (alpha + beta * np.cos(2 * np.pi * xa))
    sig_x = np.einsum("ikl,kl...->i...", C0[:, 0], eps) * scale[None]
    t_num = sig_x.mean(axis=(1, 2, 3))
    assert np.allclose(t_num, t_exact, rtol=2e-3, atol=2e-3 * np.abs(t_exact).max()), (t_num, t_exact)


# --------------------------------------------------------------------------
# the paper's own cycle: eight-colour Gauss-Seidel, damped Jacobi, F-cycles
# --------------------------------------------------------------------------

def _periodic_varied(n=8, seed=2):
    rng = np.random.default_rng(seed)
    p = make_problem((n, n, n), M.MODULI_GEN21, C_tensor=random_general_C(rng), periodic=(True, True, True))
    X, Y, Z = p.coords()
    p.moduli = p.moduli * (1.0 + 0.3 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * (Y + Z)))[None]
    p.bc = []
    return p


def test_eight_colour_sweep_is_block_gauss_seidel_in_colour_order():
    """On a periodic grid of even size no two nodes of one colour share a stencil, so
    one eight-colour sweep must equal block Gauss-Seidel in colour order, written as
    x_new = (D + L)^-1 (f - U x_old) with D, L, U from the assembled matrix permuted
    colour by colour."""
    p = _periodic_varied()
    L = MG.build_hierarchy(S.level_from_problem(p))[0]
    free, A = MG.assemble_dense(L.level, L.types)
    assert free.all()
    rng = np.random.default_rng(3)
    u = rng.normal(size=(3,) + L.level.shape)
    f = rng.normal(size=(3,) + L.level.shape) * 50
    c8 = np.broadcast_to(MG.colour8(L.level.shape)[None], u.shape).reshape(-1)
    order = np.argsort(c8, kind="stable")
    Ap = A[np.ix_(order, order)]
    cp = c8[order]
    lower = cp[:, None] > cp[None, :]
    same = cp[:, None] == cp[None, :]
    DL = np.where(lower | same, Ap, 0.0)
    U = np.where(~(lower | same), Ap, 0.0)
    x_old = u.reshape(-1)[order]
    x_new = np.linalg.solve(DL, f.reshape(-1)[order] - U @ x_old)
    expect = np.empty_like(x_new)
    expect[order] = x_new
    MG.sweep(L, u, f, MG.Smoother("gs8"))
    assert np.allclose(u.reshape(-1), expect, rtol=0, atol=1e-11 * np.abs(expect).max())


def test_jacobi_sweep_is_damped_block_splitting():
    """One damped Jacobi sweep equals u + omega D^-1 (f - A u) with D the 3x3 node
    blocks of the assembled matrix (Dirichlet rows included as identity)."""
    p = make_problem((5, 4, 5), M.MODULI_GEN21, C_tensor=random_general_C(np.random.default_rng(4)),
                     bc=[[(M.TRACTION, 0.0)] * 3 if f_ != 4 else [(M.DIRICHLET, 0.0)] * 3 for f_ in range(6)])
    L = MG.build_hierarchy(S.level_from_problem(p))[0]
    n = L.level.shape
    N = n[0] * n[1] * n[2]
    A = np.zeros((3 * N, 3 * N))
    for col in range(3 * N):
        e = np.zeros(3 * N)
        e[col] = 1.0
        A[:, col] = S.apply(L.level, e.reshape((3,) + n), L.types).reshape(-1)
    rng = np.random.default_rng(6)
    u = rng.normal(size=(3,) + n)
    f = rng.normal(size=(3,) + n)
    f = np.where(L.types == M.DIRICHLET, 0.0, f)
    omega = 0.6
    r = np.where(L.types.reshape(-1) == M.DIRICHLET, 0.0, f.reshape(-1) - A @ u.reshape(-1))
    expect = u.reshape(-1).copy()
    for q in range(N):
        idx = [q, N + q, 2 * N + q]
        expect[idx] += omega * np.linalg.solve(A[np.ix_(idx, idx)], r[idx])
    MG.sweep(L, u, f, MG.Smoother("jacobi", omega))
    assert np.allclose(u.reshape(-1), expect, rtol=0, atol=1e-12 * np.abs(expect).max())


def test_f_cycle_is_its_definition_on_three_levels():
    """With three levels the F-cycle's correction of level 1 is V(1) from zero, then V(1)
    from that result (the level-1 F-cycle ends in the exact coarsest solve); written
    out with the V-cycle, one F-cycle must give the same field."""
    p = M.polycrystal(17, grains=4, seed=7)
    levels = MG.build_hierarchy(S.level_from_problem(p))
    assert len(levels) == 3
    L0, L1 = levels[0], levels[1]
    rng = np.random.default_rng(8)
    f = np.where(L0.types == M.DIRICHLET, 0.0, rng.normal(size=(3,) + L0.level.shape))
    uF = np.zeros_like(f)
    MG.vcycle(levels, 0, uF, f, 2, 2, MG.RB, "F")
    u = np.zeros_like(f)
    for _ in range(2):
        MG.sweep(L0, u, f)
    r = S.residual(L0.level, u, f, L0.types)
    fc = np.where(L1.types == M.DIRICHLET, 0.0, MG.restrict(r, L0.level))
    e = np.zeros_like(fc)
    MG.vcycle(levels, 1, e, fc, 2, 2)
    MG.vcycle(levels, 1, e, fc, 2, 2)
    u += np.where(L0.types == M.DIRICHLET, 0.0, MG.prolong(e, L0.level))
    for _ in range(2):
        MG.sweep(L0, u, f)
    assert np.allclose(uF, u, rtol=0, atol=1e-14 * np.abs(u).max())


@pytest.mark.parametrize("sm,cycle,nu", [("gs8", "V", 2), ("jacobi", "F", 4), ("rb", "F", 2)])
def test_other_smoothers_and_cycles_reach_the_dense_solution(sm, cycle, nu):
    p = M.eshelby_sphere(9)
    levels = MG.build_hierarchy(S.level_from_problem(p))
    L = levels[0]
    free, A = MG.assemble_dense(L.level, L.types)
    f = S.rhs(L.level, p)
    u_ref = np.zeros_like(f)
    u_ref[free] = np.linalg.solve(A, f[free])
    u, info = MG.solve(p, tol=1e-13, max_cycles=200, nu1=nu, nu2=nu, levels=levels,
                       smoother=MG.Smoother(sm), cycle=cycle)
    assert info.converged
    assert np.abs(u - u_ref).max() <= 1e-10 * np.abs(u_ref).max()


# --------------------------------------------------------------------------
# stress output
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", [M.MODULI_ISO, M.MODULI_GEN21])
def test_stress_exact_for_quadratic_u_affine_moduli_and_eigenstrain(kind):
    """Central and one-sided second-order first differences are exact on quadratics, so
    the stress output equals C(x) : (grad u - eps0) evaluated analytically, on every
    node including faces, edges and corners."""
    rng = np.random.default_rng(21)
    p = M.Problem(n=(6, 5, 7), lo=(0.1, -0.2, 0.3), hi=(1.0, 0.6, 1.4))
    X, Y, Z = p.coords()
    u, grad, _ = quadratic_field(rng, X, Y, Z)
    e0 = rng.normal(size=6) * 1e-3
    eps0 = np.zeros((6,) + X.shape)
    for a in range(6):
        eps0[a] = e0[a] * (1 + 0.5 * X - 0.3 * Z)
    if kind == M.MODULI_ISO:
        lam = 1.0 + 0.2 * X + 0.1 * Y
        mu = 0.7 - 0.1 * Z + 0.05 * X
        p.moduli_kind = M.MODULI_ISO
        p.moduli = np.stack([lam, mu])
        T = iso_tensor(lam, mu)
    else:
        T0 = random_general_C(rng)
        w = 1.0 + 0.3 * X - 0.2 * Y + 0.1 * Z
        p.moduli_kind = M.MODULI_GEN21
        p.moduli = M.tensor_to_upper21(T0)[:, None, None, None] * w[None]
        T = T0[..., None, None, None] * w
    p.bc = M.all_faces(M.TRACTION, 0.0)
    lev = S.level_from_problem(p)
    got = S.stress(lev, u, eps0=eps0)
    E0 = np.zeros((3, 3) + X.shape)
    for a, (k, l) in enumerate(((0, 0), (1, 1), (2, 2), (1, 2), (2, 0), (0, 1))):
        E0[k, l] = E0[l, k] = eps0[a]
    strain = 0.5 * (grad + np.swapaxes(grad, 0, 1)) - E0
    sig = np.einsum("ijkl...,kl...->ij...", T, strain)
    expect = np.stack([sig[0, 0], sig[1, 1], sig[2, 2], sig[1, 2], sig[2, 0], sig[0, 1]])
    assert np.allclose(got, expect, rtol=0, atol=1e-11 * np.abs(expect).max())


def test_stress_inside_eshelby_sphere_converges_to_closed_form():
    """Inside a spherical inhomogeneity with a dilatational eigenstrain the strain is
    uniform, A I with A = 3 K_i eps* / (3 K_i + 4 mu_m), and the stress hydrostatic,
    3 K_i (A - eps*) I (Eshelby's solution); with the closed form as Dirichlet data the
    stress near the centre approaches it as the grid and interface width shrink."""
    errs = []
    for n in (17, 33):
        p = M.eshelby_sphere(n, radius=0.2)
        X, Y, Z = p.coords()
        ue, r = eshelby_sphere_closed_form(X, Y, Z, 0.2, 1e-3, 2.0, 1.0, 0.3)
        p.dirichlet_values = ue
        u, info = MG.solve(p, tol=1e-11, max_cycles=80)
        lev = S.level_from_problem(p)
        sig = S.stress(lev, u, eps0=p.eigenstrain)
        lam_i, mu_i = M.lame(2.0, 0.3)
        _, mu_m = M.lame(1.0, 0.3)
        K_i = lam_i + 2.0 * mu_i / 3.0
        A = 3 * K_i * 1e-3 / (3 * K_i + 4 * mu_m)
        s_exact = 3 * K_i * (A - 1e-3)
        core = r <= 0.08
        errs.append(max(np.abs(sig[a][core] - s_exact).max() for a in range(3)) / abs(s_exact))
        assert max(np.abs(sig[a][core]).max() for a in range(3, 6)) < 0.05 * abs(s_exact)
    # first order in h (the interface is 3h wide on a sphere of radius 3.2 - 6.4 h); a
    # dropped or sign-flipped eigenstrain would be off by the whole stress
    assert errs[1] < 0.6 * errs[0] and errs[1] < 0.25, errs


def test_eshelby_tensor_helper_sphere_limit_and_identities():
    """The ellipsoid closed form used to validate the stress: its sphere limit is
    S_1111 = (7 - 5 nu) / (15 (1 - nu)), S_1122 = (5 nu - 1) / (15 (1 - nu)), and the
    integrals satisfy I_1 + I_2 + I_3 = 4 pi and 3 I_11 + I_12 + I_13 = 4 pi / a_1^2."""
    import eshelby_closed_form as EC
    nu = 0.3
    S = EC.normal_eshelby_block((0.7, 0.7, 0.7), nu)
    assert np.isclose(S[0, 0], (7 - 5 * nu) / (15 * (1 - nu)), rtol=1e-7)
    assert np.isclose(S[0, 1], (5 * nu - 1) / (15 * (1 - nu)), rtol=1e-7)
    a = (1.0, 0.75, 0.5)
    I, Iij = EC.eshelby_integrals(a)
    assert np.isclose(I.sum(), 4 * np.pi, rtol=1e-8)
    for i in range(3):
        assert np.isclose(3 * Iij[i, i] + sum(Iij[i, j] for j in range(3) if j != i), 4 * np.pi / a[i] ** 2,
                          rtol=1e-8)


def test_ellipsoid_indicator_reading():
    """The Section 4.1 indicator as read: 1 at the centre, 1/2 on the sharp ellipsoid,
    0 far outside, and the eigenstrain dilatational."""
    p = M.eshelby_ellipsoid(33)
    X, Y, Z = p.coords()
    e = p.eigenstrain[0] / 1e-3
    c = p.n[0] // 2
    assert e[c, c, c] == pytest.approx(1.0)
    assert e[0, 0, 0] == pytest.approx(0.0, abs=1e-12)
    q = (X / 1.0) ** 2 + (Y / 0.75) ** 2 + (Z / 0.5) ** 2
    on = np.isclose(q, 1.0, atol=1e-12)
    assert on.any() and np.allclose(e[on], 0.5)
    assert np.array_equal(p.eigenstrain[0], p.eigenstrain[2]) and not p.eigenstrain[3:].any()
