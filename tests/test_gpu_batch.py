"""Batched solves (one CUDA graph over many grids) through the C ABI: every member's
result equals its solve alone (same kernels, same order: identical to rounding),
and matches the FP64 oracle at a relative residual of 1e-8 within 1e-7."""
import numpy as np
import pytest

from paper_2001_04789_gb300 import microstructure as M
from oracle import multigrid as MG

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


def members():
    return [M.ellipsoid_rve(17, seed=1), M.ellipsoid_rve(33, seed=2), M.ellipsoid_rve(17, seed=3),
            M.eshelby_sphere(17), M.polycrystal(17, grains=4, seed=5)]


def test_batch_equals_individual_solves_fixed_cycles(E, ctx):
    probs = members()
    grids = [E.grid_from_problem(ctx, p, mixed=True) for p in probs]
    infos = E.batch_solve(grids, precision=E.MIXED, rel_tol=0.0, fixed_cycles=3)
    batch_u = [g.displacement() for g in grids]
    for p, g, info, ub in zip(probs, grids, infos, batch_u):
        assert info["cycles"] == 3
        alone = g.solve(precision=E.MIXED, rel_tol=0.0, fixed_cycles=3)
        ua = g.displacement()
        assert np.abs(ua - ub).max() <= 1e-14 * np.abs(ua).max()
        assert np.allclose(alone["rel_history"], info["rel_history"], rtol=1e-12)
    for g in grids:
        g.close()


def test_batch_converges_to_oracle_solution(E, ctx):
    probs = members()
    grids = [E.grid_from_problem(ctx, p, mixed=True) for p in probs]
    infos = E.batch_solve(grids, precision=E.MIXED, rel_tol=1e-8, max_cycles=200)
    for p, g, info in zip(probs, grids, infos):
        assert info["status"] == 0 and info["rel_residual"] <= 1e-8
        ref, rinfo = MG.solve(p, tol=1e-8, max_cycles=300)
        err = np.abs(g.displacement() - ref).max() / np.abs(ref).max()
        assert err < 1e-7, (p.name, err)
    for g in grids:
        g.close()


def test_batch_warm_start_from_converged_members_stops_at_once(E, ctx):
    probs = members()[:3]
    grids = [E.grid_from_problem(ctx, p, mixed=True) for p in probs]
    E.batch_solve(grids, precision=E.MIXED, rel_tol=1e-10, max_cycles=200)
    infos = E.batch_solve(grids, precision=E.MIXED, rel_tol=1e-8, warm_start=True)
    assert all(i["cycles"] == 0 for i in infos)
    for g in grids:
        g.close()
