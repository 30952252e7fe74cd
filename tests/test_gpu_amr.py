"""Composite (reflux-free) AMR solve through the C ABI against the oracle's
composite cycle: same layout, same cycles, every level element by element
(FP64, 1e-9 relative), and exactness on an affine field."""
import numpy as np
import pytest

from paper_2001_04789_gb300 import microstructure as M
from oracle import amr as A

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2001_04789_gb300 import build as B
    B.build()
    from paper_2001_04789_gb300 import elas
    return elas


@pytest.fixture(scope="module")
def ctx(E):
    c = E.Context(0)
    yield c
    c.close()


def layouts():
    return {
        "crack2": lambda: M.amr_penny_crack(base_n=17, nlevels=2, block=8, width=3.0 / 32),
        "crack3": lambda: M.amr_penny_crack(base_n=17, nlevels=3, block=8, width=3.0 / 64),
    }


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("name", list(layouts()))
def test_amr_fixed_cycles_match_oracle(E, ctx, name):
    specs = layouts()[name]()
    amr = E.Amr(ctx, specs)
    info = amr.solve(fixed_cycles=3)
    got = amr.displacements()
    ref, rinfo = A.solve(specs, fixed_cycles=3)
    for l, (g, r) in enumerate(zip(got, ref)):
        valid = np.ones(g.shape[1:], bool)
        sp = specs[l]
        sl = (slice(None),) + tuple(slice(sp.valid_lo[d] - sp.grid_lo[d], sp.valid_hi[d] - sp.grid_lo[d] + 1)
                                    for d in (2, 1, 0))
        assert rel_err(g[sl], r[sl]) < 1e-9, (name, l)
    assert np.allclose(info["rel_history"], rinfo["rel_history"], rtol=1e-7)
    amr.close()


def test_amr_converged_solve_matches_oracle(E, ctx):
    specs = layouts()["crack2"]()
    amr = E.Amr(ctx, specs)
    info = amr.solve(rel_tol=1e-8)
    ref, rinfo = A.solve(specs, tol=1e-8)
    assert info["status"] == 0 and info["cycles"] == rinfo["cycles"]
    for g, r in zip(amr.displacements(), ref):
        assert rel_err(g, r) < 1e-9
    amr.close()


def test_amr_affine_field_is_exact(E, ctx):
    G = np.array([[1.0, 0.3, -0.2], [0.1, -0.5, 0.4], [0.2, 0.0, 0.7]]) * 1e-3

    def mk(n3, lo3, hi3):
        p = M.Problem(n=tuple(n3), lo=tuple(lo3), hi=tuple(hi3))
        X, Y, Z = p.coords()
        lam, mu = M.lame(np.ones(X.shape), 0.3)
        p.moduli_kind = M.MODULI_ISO
        p.moduli = np.stack([lam, mu])
        x = [X, Y, Z]
        ue = np.stack([sum(G[k, l] * x[l] for l in range(3)) for k in range(3)])
        p.bc = M.all_faces(M.DIRICHLET, 0.0)
        p.face_values = {f: ue for f in range(6)}
        return p

    ind = lambda X, Y, Z: np.exp(-((X - 0.4) ** 2 + (Y - 0.6) ** 2 + (Z - 0.5) ** 2) / 0.02)
    specs = M.amr_layout(mk, 17, 3, ind, thresh=0.15, block=8)
    amr = E.Amr(ctx, specs)
    info = amr.solve(rel_tol=1e-12, max_cycles=80)
    assert info["status"] == 0
    for sp, ul in zip(specs, amr.displacements()):
        X, Y, Z = sp.problem.coords()
        x = [X, Y, Z]
        ue = np.stack([sum(G[k, l] * x[l] for l in range(3)) for k in range(3)])
        sl = (slice(None),) + tuple(slice(sp.valid_lo[d] - sp.grid_lo[d], sp.valid_hi[d] - sp.grid_lo[d] + 1)
                                    for d in (2, 1, 0))
        assert np.abs(ul[sl] - ue[sl]).max() < 1e-11
    amr.close()


def r2_layouts():
    return {
        "crack2_r2": lambda: M.amr_penny_crack(base_n=17, nlevels=2, block=8, width=3.0 / 32, ghost_layers=2),
        "crack3_r2": lambda: M.amr_penny_crack(base_n=17, nlevels=3, block=8, width=3.0 / 64, ghost_layers=2),
    }


@pytest.mark.parametrize("name", list(r2_layouts()))
def test_amr_r2_fixed_cycles_match_oracle(E, ctx, name):
    """Reading R2 (two ghost layers, inner relaxed, full-weighting restriction) on the
    GPU against the oracle's R2 cycle: every level's valid and inner-ghost nodes."""
    specs = r2_layouts()[name]()
    amr = E.Amr(ctx, specs, reading="R2")
    info = amr.solve(fixed_cycles=3)
    got = amr.displacements()
    ref, rinfo = A.solve(specs, fixed_cycles=3, reading="R2")
    for l, (g, r) in enumerate(zip(got, ref)):
        sp = specs[l]
        grow = [(1 if sp.ghost[2 * d] else 0, 1 if sp.ghost[2 * d + 1] else 0) if l > 0 else (0, 0) for d in range(3)]
        sl = (slice(None),) + tuple(slice(sp.valid_lo[d] - grow[d][0] - sp.grid_lo[d],
                                          sp.valid_hi[d] + grow[d][1] - sp.grid_lo[d] + 1) for d in (2, 1, 0))
        assert rel_err(g[sl], r[sl]) < 1e-9, (name, l)
    assert np.allclose(info["rel_history"], rinfo["rel_history"], rtol=1e-7)
    amr.close()


def test_amr_r2_needs_two_ghost_layers(E, ctx):
    specs = layouts()["crack2"]()
    with pytest.raises(E.ElasError):
        E.Amr(ctx, specs, reading="R2")


def test_amr_config3_at_stated_size_matches_oracle(E, ctx):
    """The penny-crack layout at its stated size (base 65^3, three levels, 32-cell blocks;
    levels of 65^3, 129 x 129 x 67 and 195 x 195 x 67 nodes): one composite cycle on the
    GPU against the oracle's on every level's valid nodes, then a converged GPU solve."""
    specs = M.amr_penny_crack(base_n=65, nlevels=3, block=32)
    assert len(specs) == 3
    amr = E.Amr(ctx, specs)
    info = amr.solve(fixed_cycles=1)
    got = amr.displacements()
    ref, rinfo = A.solve(specs, fixed_cycles=1)
    for l, (g, r) in enumerate(zip(got, ref)):
        sp = specs[l]
        sl = (slice(None),) + tuple(slice(sp.valid_lo[d] - sp.grid_lo[d], sp.valid_hi[d] - sp.grid_lo[d] + 1)
                                    for d in (2, 1, 0))
        assert rel_err(g[sl], r[sl]) < 1e-9, l
    assert np.allclose(info["rel_history"], rinfo["rel_history"], rtol=1e-7)
    full = amr.solve(rel_tol=1e-8, max_cycles=200)
    assert full["status"] == 0 and full["rel_residual"] <= 1e-8
    amr.close()


@pytest.mark.parametrize("reading,name", [("R1", "crack2"), ("R1", "crack3"), ("R2", "crack2_r2")])
def test_amr_mixed_composite_solve_reaches_the_oracle(E, ctx, reading, name):
    """FP32 composite cycles inside FP64 refinement: at a relative composite residual of
    1e-8 (checked in FP64) every level is within 1e-7 of the oracle's FP64 solution."""
    specs = (layouts() if reading == "R1" else r2_layouts())[name]()
    amr = E.Amr(ctx, specs, reading=reading, mixed=True)
    info = amr.solve(rel_tol=1e-8, max_cycles=200, precision=E.MIXED)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-8
    ref, rinfo = A.solve(specs, tol=1e-8, max_cycles=200, reading=reading)
    for l, (g, r) in enumerate(zip(amr.displacements(), ref)):
        sp = specs[l]
        sl = (slice(None),) + tuple(slice(sp.valid_lo[d] - sp.grid_lo[d], sp.valid_hi[d] - sp.grid_lo[d] + 1)
                                    for d in (2, 1, 0))
        assert rel_err(g[sl], r[sl]) < 1e-7, (name, l)
    amr.close()


def test_amr_config3_at_stated_size_mixed(E, ctx):
    """Config 3 in mixed precision: converges to 1e-8 (FP64 composite norm) and agrees
    with the FP64 composite solve of the same layout."""
    specs = M.amr_penny_crack(base_n=65, nlevels=3, block=32)
    amr = E.Amr(ctx, specs, mixed=True)
    i64 = amr.solve(rel_tol=1e-9, max_cycles=200)
    u64 = amr.displacements()
    imx = amr.solve(rel_tol=1e-8, max_cycles=200, precision=E.MIXED)
    assert i64["status"] == 0 and imx["status"] == 0 and imx["rel_residual"] <= 1e-8
    for l, (a_, b_) in enumerate(zip(amr.displacements(), u64)):
        assert rel_err(a_, b_) < 1e-6, l
    amr.close()
