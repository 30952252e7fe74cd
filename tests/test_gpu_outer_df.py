"""Double-float refinement residual of mixed solves against the oracle.

The residual r = f - A u of the finest level evaluated in double-float arithmetic
(FP32 pairs, about 48 bits) must (1) agree with the oracle's FP64 residual to the FP32
rounding of its output when r is of the size of f, and (2) cancel to its own rounding
level, about 1e-13 of the row scale, when f = A u: the regime of a converged solve,
where an FP32 evaluation is left with errors near 1e-7 of the row scale.  Mixed solves
with the double-float residual reach the oracle's solution as the FP64 residual does,
and their batched, graph-replayed and served forms stay bitwise equal to the lone solve.
"""
import numpy as np
import pytest

from paper_2001_04789_gb300 import microstructure as M
from oracle import multigrid as MG
from oracle import stencil as S

from test_gpu_parity import CASES, dev, rel_err

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


def smooth_field(shape, seed):
    rng = np.random.default_rng(seed)
    n = np.array(shape[1:])
    X = np.meshgrid(*[np.linspace(0, 1, k) for k in n], indexing="ij")
    u = np.zeros(shape)
    for i in range(3):
        a = rng.normal(size=4)
        u[i] = a[0] + a[1] * np.sin(2 * X[0] + a[2]) * np.cos(X[1] - a[3] * X[2]) + 0.3 * X[i] ** 2
    return 1e-3 * u


@pytest.mark.parametrize("case", list(CASES))
def test_df_residual_matches_oracle(E, ctx, case):
    p = CASES[case]()
    g = E.grid_from_problem(ctx, p, mixed=True)
    lev = S.level_from_problem(p)
    rng = np.random.default_rng(2)
    u = rng.normal(size=(3,) + g.shape) * 1e-3
    f = rng.normal(size=(3,) + g.shape)
    r, ss = g.op_residual(0, E.OP_DF, dev(u), dev(f))
    got = r.cpu().numpy()
    ref = S.residual(lev, u, f)
    # FP32 output of a double-float evaluation: the rounding of the written values
    assert got.dtype == np.float32
    assert rel_err(got, ref) < 1e-6
    assert abs(ss - float((got.astype(np.float64) ** 2).sum())) <= 1e-5 * ss
    g.close()


@pytest.mark.parametrize("case", list(CASES))
def test_df_residual_cancels_to_its_rounding(E, ctx, case):
    p = CASES[case]()
    g = E.grid_from_problem(ctx, p, mixed=True)
    lev = S.level_from_problem(p)
    scale = np.abs(S.apply(lev, np.random.default_rng(5).normal(size=(3,) + g.shape) * 1e-3)).max()
    for u in (np.random.default_rng(3).normal(size=(3,) + g.shape) * 1e-3, smooth_field((3,) + g.shape, 4)):
        f = S.apply(lev, u)            # A u (u itself on Dirichlet rows): r = 0 exactly
        r_df = g.op_residual(0, E.OP_DF, dev(u), dev(f))[0].cpu().numpy().astype(np.float64)
        r64 = g.op_residual(0, E.FP64, dev(u), dev(f))[0].cpu().numpy()
        r32 = g.op_residual(0, E.MIXED, dev(u, torch.float32), dev(f, torch.float32))[0].cpu().numpy()
        err_df = np.abs(r_df).max() / scale
        err32 = np.abs(r32).max() / scale
        assert np.abs(r64).max() / scale < 1e-14
        assert err_df < 1e-11, err_df
        # the test separates the arithmetics: FP32 leaves errors four orders larger
        assert err32 > 1e3 * max(err_df, 1e-15), (err32, err_df)
    g.close()


@pytest.mark.parametrize("case", ["eshelby", "polycrystal", "mixed_gen"])
def test_mixed_solve_with_df_residual_reaches_oracle_solution(E, ctx, case):
    p = CASES[case]()
    ref, rinfo = MG.solve(p, tol=1e-8, max_cycles=300)
    g = E.grid_from_problem(ctx, p, mixed=True)
    idf = g.solve(precision=E.MIXED, rel_tol=1e-8, outer=E.OUTER_DF)
    assert idf["status"] == 0 and idf["rel_residual"] <= 1e-8
    rel64, _ = g.query_residual()
    assert rel64 <= 1.01e-8
    u_df = g.displacement()
    assert rel_err(u_df, ref) < 1e-7
    i64 = g.solve(precision=E.MIXED, rel_tol=1e-8, outer=E.OUTER_FP64)
    assert i64["status"] == 0
    # same cycle count and the same refinement history to the residual's FP32 output
    assert idf["cycles"] == i64["cycles"]
    assert np.allclose(idf["rel_history"], i64["rel_history"], rtol=1e-4, atol=1e-12)
    assert rel_err(u_df, g.displacement()) < 1e-9
    # AUTO takes the double-float residual at this tolerance: the same bits
    iau = g.solve(precision=E.MIXED, rel_tol=1e-8)
    assert iau["rel_history"] == idf["rel_history"]
    assert np.array_equal(g.displacement(), u_df)
    g.close()


def test_tight_tolerance_takes_fp64_residual(E, ctx):
    p = M.eshelby_sphere(17)
    g = E.grid_from_problem(ctx, p, mixed=True)
    a = g.solve(precision=E.MIXED, rel_tol=1e-12)
    b = g.solve(precision=E.MIXED, rel_tol=1e-12, outer=E.OUTER_FP64)
    assert a["status"] == 0 and a["rel_residual"] <= 1e-12
    assert a["rel_history"] == b["rel_history"]
    g.close()


def test_df_residual_batched_graph_and_served_equal_lone(E, ctx):
    probs = [M.polycrystal(17, grains=5, seed=s) for s in (1, 2)]
    lone = []
    for p in probs:
        g = E.grid_from_problem(ctx, p, mixed=True)
        info = g.solve(precision=E.MIXED, rel_tol=1e-8, outer=E.OUTER_DF)
        lone.append((info["cycles"], g.displacement()))
        g.close()
    grids = [E.grid_from_problem(ctx, p, mixed=True) for p in probs]
    infos = E.batch_solve(grids, rel_tol=1e-8, outer=E.OUTER_DF)
    for (cyc, u), info, g in zip(lone, infos, grids):
        assert info["cycles"] == cyc
        assert np.array_equal(g.displacement(), u)
    for (cyc, u), g in zip(lone, grids):
        info = g.solve(precision=E.MIXED, rel_tol=1e-8, outer=E.OUTER_DF, use_graph=True)
        assert info["cycles"] == cyc
        assert np.array_equal(g.displacement(), u)
    srv = E.Server(ctx, max_active=4)
    tickets = [srv.submit(g, rel_tol=1e-8, outer=E.OUTER_DF) for g in grids]
    done = {}
    for _ in range(500):
        srv.step()
        for t in tickets:
            if t not in done:
                r = srv.poll(t)
                if r is not None:
                    done[t] = r
        if len(done) == len(tickets):
            break
    for (cyc, u), t, g in zip(lone, tickets, grids):
        assert done[t][0]["status"] == 0
        assert np.array_equal(g.displacement(), u)
    srv.close()
    for g in grids:
        g.close()
