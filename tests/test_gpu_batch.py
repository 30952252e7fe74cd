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


# --------------------------------------------------------------------------
# the per-phase engine: batches of one moduli kind and FP32 layout
# --------------------------------------------------------------------------

def iso_members():
    return [M.ellipsoid_rve(17, seed=1), M.ellipsoid_rve(33, seed=2), M.eshelby_sphere(17),
            M.penny_crack(17, width=3.0 / 16, clamp_lateral=True), M.ellipsoid_rve(33, seed=7)]


def gen_members():
    from test_gpu_parity import mixed_bc_problem
    return [M.polycrystal(17, grains=4, seed=5), M.polycrystal(33, grains=5, seed=6), mixed_bc_problem()]


@pytest.mark.parametrize("family", ["iso", "gen21_split"])
@pytest.mark.parametrize("cycle", [0, 1])
def test_engine_members_are_bitwise_their_lone_solves(E, ctx, family, cycle):
    """One launch per phase over all members: each member runs exactly the kernels of
    its lone solve, so results and residual histories are identical bit for bit."""
    probs = iso_members() if family == "iso" else gen_members()
    grids = [E.grid_from_problem(ctx, p, mixed=True) for p in probs]
    infos = E.batch_solve(grids, precision=E.MIXED, rel_tol=1e-8, max_cycles=100, inner_cycles=2, cycle=cycle)
    batch_u = [g.displacement() for g in grids]
    for g, info, ub in zip(grids, infos, batch_u):
        assert info["status"] == 0
        alone = g.solve(precision=E.MIXED, rel_tol=1e-8, max_cycles=100, inner_cycles=2, cycle=cycle)
        assert np.array_equal(g.displacement(), ub)
        assert alone["rel_history"] == info["rel_history"] and alone["cycles"] == info["cycles"]
    for g in grids:
        g.close()


def test_engine_launches_do_not_grow_with_member_count(E, ctx):
    """Launches per refinement step depend on the levels, not on how many members (the
    initial state and the final rigid-mode removal are per member, once per call)."""
    per_step = {}
    for m in (2, 6):
        grids = [E.grid_from_problem(ctx, M.ellipsoid_rve(33, seed=10 + i), mixed=True) for i in range(m)]
        counts = {}
        for steps in (2, 6):
            E.batch_solve(grids, precision=E.MIXED, rel_tol=0.0, fixed_cycles=steps)   # plan and graph
            l0 = E.launch_count()
            E.batch_solve(grids, precision=E.MIXED, rel_tol=0.0, fixed_cycles=steps)
            counts[steps] = E.launch_count() - l0
        per_step[m] = counts[6] - counts[2]
        for g in grids:
            g.close()
    assert per_step[2] == per_step[6] > 0, per_step


def test_engine_plan_follows_new_loads(E, ctx):
    """A cached plan is rebuilt when a member's loads (and so its r0) change."""
    probs = iso_members()[:3]
    grids = [E.grid_from_problem(ctx, p, mixed=True) for p in probs]
    E.batch_solve(grids, precision=E.MIXED, rel_tol=1e-8)
    p2 = M.ellipsoid_rve(17, seed=1)
    p2.mean_strain = -2.0 * p2.mean_strain
    grids[0].set_mean_strain(p2.mean_strain)
    infos = E.batch_solve(grids, precision=E.MIXED, rel_tol=1e-8)
    ub = grids[0].displacement()
    alone = grids[0].solve(precision=E.MIXED, rel_tol=1e-8)
    assert np.array_equal(grids[0].displacement(), ub) and alone["cycles"] == infos[0]["cycles"]
    for g in grids:
        g.close()


def test_a_grid_listed_twice_is_refused(E, ctx):
    """Members share nothing: a grid listed twice (its two solves would share one set of
    buffers) is an invalid argument, refused before any launch; the grid stays usable."""
    g = E.grid_from_problem(ctx, M.ellipsoid_rve(17, seed=3), mixed=True)
    with pytest.raises(E.ElasError) as err:
        E.batch_solve([g, g], precision=E.MIXED, rel_tol=1e-8)
    assert err.value.code == E.ERR_INVALID_ARG
    info = E.batch_solve([g], precision=E.MIXED, rel_tol=1e-8)[0]
    assert info["status"] == 0 and info["rel_residual"] <= 1e-8
    g.close()
