"""Pins of the oracle's composite (reflux-free) AMR treatment, Section 3.2 and
Appendix A: the effective coarse/fine stencil printed in Appendix A, exactness on
affine fields, and convergence of the composite cycle."""
import json
import os

import numpy as np
import pytest

from paper_2001_04789_gb300 import microstructure as M
from oracle import amr as A
from oracle import stencil as S

GOLD = os.path.join(os.path.dirname(__file__), "golden", "appendix_a_stencil.json")


def laplacian_box(mu=0.7):
    """lambda = -mu: the elastic operator becomes mu * Laplacian on each component,
    the scalar setting of Appendix A."""
    def mk(n3, lo3, hi3):
        p = M.Problem(n=tuple(n3), lo=tuple(lo3), hi=tuple(hi3))
        shape = (n3[2], n3[1], n3[0])
        p.moduli_kind = M.MODULI_ISO
        p.moduli = np.stack([np.full(shape, -mu), np.full(shape, mu)])
        p.bc = M.all_faces(M.DIRICHLET, 0.0)
        return p
    return mk


def two_level(mu=0.7):
    ind = lambda X, Y, Z: np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) / 0.02)
    specs = M.amr_layout(laplacian_box(mu), 17, 2, ind, thresh=0.3, block=8)
    assert len(specs) == 2 and all(specs[1].ghost)
    return specs, A.build(specs)


def test_appendix_a_one_d_effective_stencil():
    gold = json.load(open(GOLD))["one_d"]["coefficients_times_dxf2"]
    mu = 0.7
    specs, data = two_level(mu)
    c, f = data
    rng = np.random.default_rng(0)
    # fields varying in x only
    uc = np.broadcast_to(rng.normal(size=c.L.level.n[0])[None, None, None, :], (3,) + c.L.level.shape).copy()
    uf = np.broadcast_to(rng.normal(size=f.L.level.n[0])[None, None, None, :], (3,) + f.L.level.shape).copy()
    A.inject(f, uf, c, uc)
    A.fill_ghosts(c, uc, f, uf)
    sp = f.spec
    lo = sp.valid_lo[0]
    ix = lo - sp.grid_lo[0]                     # grid index of the C/F node in x
    jy = (sp.valid_lo[1] + sp.valid_hi[1]) // 2 - sp.grid_lo[1]
    kz = (sp.valid_lo[2] + sp.valid_hi[2]) // 2 - sp.grid_lo[2]
    row = S.pde_rows(f.L.level, uf)[0, kz, jy, ix]
    h = f.L.level.h[0]
    cI = lo // 2 - c.spec.grid_lo[0]            # coarse node coincident with the C/F node
    expect = mu * (gold["fine_inward"] * uf[0, kz, jy, ix + 1] + gold["fine_node"] * uf[0, kz, jy, ix]
                   + gold["coarse_outward"] * uc[0, 0, 0, cI - 1]) / h ** 2
    assert np.isclose(row, expect, rtol=1e-12, atol=1e-12 * abs(expect))
    kc = (sp.grid_lo[2] + kz) // 2 - c.spec.grid_lo[2]
    jc = (sp.grid_lo[1] + jy) // 2 - c.spec.grid_lo[1]
    assert np.isclose(uc[0, kc, jc, cI], uf[0, kz, jy, ix])      # injection


def test_appendix_a_two_d_corner_effective_stencil():
    gold = json.load(open(GOLD))["two_d_corner"]
    gx, gy = gold["x_part_times_dxf2"], gold["y_part_times_dyf2"]
    mu = 0.7
    specs, data = two_level(mu)
    c, f = data
    rng = np.random.default_rng(1)
    ny_c, nx_c = c.L.level.shape[1:]
    ny_f, nx_f = f.L.level.shape[1:]
    uc = np.broadcast_to(rng.normal(size=(ny_c, nx_c))[None, None], (3,) + c.L.level.shape).copy()
    uf = np.broadcast_to(rng.normal(size=(ny_f, nx_f))[None, None], (3,) + f.L.level.shape).copy()
    A.inject(f, uf, c, uc)
    A.fill_ghosts(c, uc, f, uf)
    sp = f.spec
    ix, jy = sp.valid_lo[0] - sp.grid_lo[0], sp.valid_lo[1] - sp.grid_lo[1]
    kz = (sp.valid_lo[2] + sp.valid_hi[2]) // 2 - sp.grid_lo[2]
    row = S.pde_rows(f.L.level, uf)[1, kz, jy, ix]
    hx, hy = f.L.level.h[0], f.L.level.h[1]
    cI, cJ = sp.valid_lo[0] // 2 - c.spec.grid_lo[0], sp.valid_lo[1] // 2 - c.spec.grid_lo[1]
    expect = mu * ((gx["fine_inward"] * uf[1, kz, jy, ix + 1] + gx["fine_node"] * uf[1, kz, jy, ix]
                    + gx["coarse_outward"] * uc[1, 0, cJ, cI - 1]) / hx ** 2
                   + (gy["fine_inward"] * uf[1, kz, jy + 1, ix] + gy["fine_node"] * uf[1, kz, jy, ix]
                      + gy["coarse_outward"] * uc[1, 0, cJ - 1, cI]) / hy ** 2)
    assert np.isclose(row, expect, rtol=1e-12, atol=1e-12 * abs(expect))


def test_composite_solve_reproduces_affine_field_exactly():
    G = np.array([[1.0, 0.3, -0.2], [0.1, -0.5, 0.4], [0.2, 0.0, 0.7]]) * 1e-3
    b = np.array([1e-4, -2e-4, 3e-4])

    def mk(n3, lo3, hi3):
        p = M.Problem(n=tuple(n3), lo=tuple(lo3), hi=tuple(hi3))
        X, Y, Z = p.coords()
        lam, mu = M.lame(np.ones(X.shape), 0.3)
        p.moduli_kind = M.MODULI_ISO
        p.moduli = np.stack([lam, mu])
        x = [X, Y, Z]
        ue = np.stack([sum(G[k, l] * x[l] for l in range(3)) + b[k] for k in range(3)])
        p.bc = M.all_faces(M.DIRICHLET, 0.0)
        p.face_values = {f_: ue for f_ in range(6)}
        return p

    ind = lambda X, Y, Z: np.exp(-((X - 0.4) ** 2 + (Y - 0.6) ** 2 + (Z - 0.5) ** 2) / 0.02)
    specs = M.amr_layout(mk, 17, 3, ind, thresh=0.15, block=8)
    assert len(specs) == 3
    u, info = A.solve(specs, tol=1e-12, max_cycles=60)
    assert info["converged"]
    for sp, ul in zip(specs, u):
        X, Y, Z = sp.problem.coords()
        x = [X, Y, Z]
        ue = np.stack([sum(G[k, l] * x[l] for l in range(3)) + b[k] for k in range(3)])
        assert np.abs(ul - ue).max() < 1e-11


def test_composite_cycle_converges_on_penny_crack():
    specs = M.amr_penny_crack(base_n=17, nlevels=2, block=8, width=3.0 / 32)
    u, info = A.solve(specs, tol=1e-9, max_cycles=60)
    assert info["converged"], info["rel_history"][-5:]


def test_composite_solution_approaches_uniform_fine_solution():
    """With the refined box around the only structure of the field, the composite
    solution on the fine box approaches the uniform fine-grid solution as the box
    grows: the error of a 2-level solve stays far below the coarse-grid error."""
    from oracle import multigrid as MG

    def mk(n3, lo3, hi3):
        p = M.Problem(n=tuple(n3), lo=tuple(lo3), hi=tuple(hi3))
        X, Y, Z = p.coords()
        E = 1.0 + 0.8 * np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) / 0.01)
        lam, mu = M.lame(E, 0.3)
        p.moduli_kind = M.MODULI_ISO
        p.moduli = np.stack([lam, mu])
        e = np.zeros((6,) + X.shape)
        e[0] = e[1] = e[2] = 1e-3 * np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) / 0.01)
        p.eigenstrain = e
        p.bc = M.all_faces(M.DIRICHLET, 0.0)
        return p

    ind = lambda X, Y, Z: np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) / 0.01)
    specs = M.amr_layout(mk, 17, 2, ind, thresh=0.05, block=8)
    u, info = A.solve(specs, tol=1e-11, max_cycles=80)
    assert info["converged"]
    fine = mk((33, 33, 33), (0, 0, 0), (1, 1, 1))
    uf, _ = MG.solve(fine, tol=1e-11, max_cycles=80)
    coarse = mk((17, 17, 17), (0, 0, 0), (1, 1, 1))
    uc, _ = MG.solve(coarse, tol=1e-11, max_cycles=80)
    sp = specs[1]
    sl = tuple(slice(sp.valid_lo[d], sp.valid_hi[d] + 1) for d in (2, 1, 0))
    ul = u[1][(slice(None),) + tuple(slice(sp.valid_lo[d] - sp.grid_lo[d], sp.valid_hi[d] - sp.grid_lo[d] + 1)
                                     for d in (2, 1, 0))]
    err_amr = np.abs(ul - uf[(slice(None),) + sl]).max()
    err_coarse = np.abs(uc - uf[:, ::2, ::2, ::2]).max()
    assert err_amr < 0.5 * err_coarse, (err_amr, err_coarse)


# --------------------------------------------------------------------------
# restriction to covered coarse nodes: truncated, renormalised weights
# --------------------------------------------------------------------------

def _box(grid_lo, n, valid_lo=None, valid_hi=None):
    from types import SimpleNamespace
    return SimpleNamespace(grid_lo=grid_lo, valid_lo=valid_lo, valid_hi=valid_hi,
                           problem=SimpleNamespace(n=n))


def test_restriction_weights_truncated_and_renormalised_by_hand():
    """Section 3.2's R_mn at covered coarse nodes, weights worked out by hand: the
    single-grid (1/4, 1/2, 1/4) (interior) and (1/2, 1/2) (domain boundary) weights,
    cut to the valid fine nodes and scaled to sum to one."""
    fine = _box((3, 3, 3), (11, 11, 11), (4, 4, 4), (12, 12, 12))   # 17 fine nodes per direction
    w = lambda gc: A._restrict_weights_1d(gc, fine, 0, 17)
    assert w(2) == pytest.approx({0: 2 / 3, 1: 1 / 3})          # footprint 3, 4, 5; 3 is a ghost
    assert w(4) == pytest.approx({-1: 0.25, 0: 0.5, 1: 0.25})
    assert w(6) == pytest.approx({-1: 1 / 3, 0: 2 / 3})
    edge = _box((0, 0, 0), (10, 10, 10), (0, 0, 0), (8, 8, 8))     # valid box on the low domain face
    we = lambda gc: A._restrict_weights_1d(gc, edge, 1, 17)
    assert we(0) == pytest.approx({0: 0.5, 1: 0.5})                 # domain boundary node, untouched
    assert we(4) == pytest.approx({-1: 1 / 3, 0: 2 / 3})            # fine node 9 is outside the box


def test_restriction_of_a_point_value_and_of_a_constant():
    fine = _box((3, 3, 3), (11, 11, 11), (4, 4, 4), (12, 12, 12))
    coarse = _box((0, 0, 0), (9, 9, 9))
    # a unit value at fine global node (x, y, z) = (4, 5, 12) reaches coarse (2, 2, 6) with
    # 2/3 * 1/3 * 2/3 and coarse (2, 3, 6) with 2/3 * 1/4 * 2/3; nothing else
    fres = np.zeros((1, 11, 11, 11))
    fres[0, 12 - 3, 5 - 3, 4 - 3] = 1.0
    cres = np.full((1, 9, 9, 9), -7.0)
    A.restrict_field(fine, fres, coarse, cres, (17, 17, 17))
    expect = np.full((1, 9, 9, 9), -7.0)
    expect[0, 2:7, 2:7, 2:7] = 0.0                                  # every covered node is written
    expect[0, 6, 2, 2] = 4 / 27
    expect[0, 6, 3, 2] = 1 / 9
    assert np.allclose(cres, expect, rtol=0, atol=1e-15)
    # renormalised weights conserve constants on every covered node, including the
    # truncated ones next to the coarse/fine boundary
    fres = np.full((2, 11, 11, 11), 5.0)
    cres = np.zeros((2, 9, 9, 9))
    A.restrict_field(fine, fres, coarse, cres, (17, 17, 17))
    assert np.allclose(cres[:, 2:7, 2:7, 2:7], 5.0, rtol=0, atol=1e-14)
    assert np.all(cres[:, :2] == 0) and np.all(cres[:, 7:] == 0)


# --------------------------------------------------------------------------
# reading R2: N + 1 = 2 ghost layers, inner layer relaxed, full weighting
# --------------------------------------------------------------------------

def test_r2_restriction_weights_are_untruncated_at_the_coarse_fine_boundary():
    """In R2 the inner ghost layer is relaxed, so a covered coarse node on the
    coarse/fine boundary restricts with the full (1/4, 1/2, 1/4) footprint."""
    from types import SimpleNamespace
    sp = SimpleNamespace(level=1, grid_lo=(2, 2, 2), valid_lo=(4, 4, 4), valid_hi=(12, 12, 12),
                         ghost=(True,) * 6, problem=SimpleNamespace(n=(13, 13, 13)))
    import dataclasses as dc

    @dc.dataclass
    class Spec:
        level: int
        grid_lo: tuple
        valid_lo: tuple
        valid_hi: tuple
        ghost: tuple
        problem: object
    spec = Spec(sp.level, sp.grid_lo, sp.valid_lo, sp.valid_hi, sp.ghost, sp.problem)
    rsp = A.relaxed_spec(spec, "R2")
    assert rsp.valid_lo == (3, 3, 3) and rsp.valid_hi == (13, 13, 13)
    assert A._restrict_weights_1d(2, rsp, 0, 17) == pytest.approx({-1: 0.25, 0: 0.5, 1: 0.25})
    assert A.relaxed_spec(spec, "R1") is spec


def test_r2_composite_solve_reproduces_affine_field_exactly():
    G = np.array([[1.0, 0.3, -0.2], [0.1, -0.5, 0.4], [0.2, 0.0, 0.7]]) * 1e-3
    b = np.array([1e-4, -2e-4, 3e-4])

    def field(p):
        X, Y, Z = p.coords()
        x = [X, Y, Z]
        return np.stack([sum(G[k, l] * x[l] for l in range(3)) + b[k] for k in range(3)])

    def mk(n3, lo3, hi3):
        p = M.Problem(n=tuple(n3), lo=tuple(lo3), hi=tuple(hi3))
        X, _, _ = p.coords()
        lam, mu = M.lame(np.ones(X.shape), 0.3)
        p.moduli_kind = M.MODULI_ISO
        p.moduli = np.stack([lam, mu])
        p.bc = M.all_faces(M.DIRICHLET, 0.0)
        p.face_values = {f_: field(p) for f_ in range(6)}
        return p

    ind = lambda X, Y, Z: np.exp(-((X - 0.4) ** 2 + (Y - 0.6) ** 2 + (Z - 0.5) ** 2) / 0.02)
    specs = M.amr_layout(mk, 17, 3, ind, thresh=0.15, block=8, ghost_layers=2)
    assert len(specs) == 3
    u, info = A.solve(specs, tol=1e-12, max_cycles=60, reading="R2")
    assert info["converged"]
    for sp, ul in zip(specs, u):
        assert np.abs(ul - field(sp.problem)).max() < 1e-11


def test_r2_is_closer_to_the_uniform_fine_solution_than_r1():
    """Both readings on the same smooth problem: the R2 composite solution lies closer
    to the uniform fine-grid solution than R1's, and both far below the coarse error."""
    from oracle import multigrid as MG

    def mk(n3, lo3, hi3):
        p = M.Problem(n=tuple(n3), lo=tuple(lo3), hi=tuple(hi3))
        X, Y, Z = p.coords()
        g = np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) / 0.01)
        lam, mu = M.lame(1.0 + 0.8 * g, 0.3)
        p.moduli_kind = M.MODULI_ISO
        p.moduli = np.stack([lam, mu])
        e = np.zeros((6,) + X.shape)
        e[0] = e[1] = e[2] = 1e-3 * g
        p.eigenstrain = e
        p.bc = M.all_faces(M.DIRICHLET, 0.0)
        return p

    ind = lambda X, Y, Z: np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) / 0.01)
    uf, _ = MG.solve(mk((33, 33, 33), (0, 0, 0), (1, 1, 1)), tol=1e-11, max_cycles=80)
    uc, _ = MG.solve(mk((17, 17, 17), (0, 0, 0), (1, 1, 1)), tol=1e-11, max_cycles=80)
    err = {}
    for reading, layers in (("R1", 1), ("R2", 2)):
        specs = M.amr_layout(mk, 17, 2, ind, thresh=0.05, block=8, ghost_layers=layers)
        u, info = A.solve(specs, tol=1e-11, max_cycles=80, reading=reading)
        assert info["converged"]
        sp = specs[1]
        sl = tuple(slice(sp.valid_lo[d], sp.valid_hi[d] + 1) for d in (2, 1, 0))
        ul = u[1][(slice(None),) + tuple(slice(sp.valid_lo[d] - sp.grid_lo[d], sp.valid_hi[d] - sp.grid_lo[d] + 1)
                                         for d in (2, 1, 0))]
        err[reading] = np.abs(ul - uf[(slice(None),) + sl]).max()
    err_coarse = np.abs(uc - uf[:, ::2, ::2, ::2]).max()
    assert err["R2"] < err["R1"] < 0.5 * err_coarse, (err, err_coarse)
