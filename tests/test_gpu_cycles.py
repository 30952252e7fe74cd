"""The paper's own cycle and the stronger smoother (Section 3.1) on the CUDA path,
through the C ABI, against the CPU oracle: one sweep of the eight-colour and the damped
Jacobi smoothers element by element (FP64 to 1e-12, FP32 to 5e-5 of the row scale),
and F-cycle solves (the paper's F(4,4) Jacobi schedule and F(2,2) red-black) with the
oracle's residual history and solution after the same number of cycles (FP64 to 1e-9),
the mixed path to 1e-7 at a relative residual of 1e-8."""
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


SMOOTHERS = {"gs8": (1, MG.Smoother("gs8")), "jacobi": (2, MG.Smoother("jacobi", 0.6))}


@pytest.mark.parametrize("smoother", list(SMOOTHERS))
@pytest.mark.parametrize("case", list(CASES))
def test_one_sweep_matches_oracle(E, ctx, case, smoother):
    code, sm = SMOOTHERS[smoother]
    p = CASES[case]()
    g = E.grid_from_problem(ctx, p, mixed=True)
    L = MG.build_hierarchy(S.level_from_problem(p))[0]
    rng = np.random.default_rng(12)
    u = np.where(L.types == M.DIRICHLET, 0.0, rng.normal(size=(3,) + g.shape))
    f = np.where(L.types == M.DIRICHLET, 0.0, rng.normal(size=(3,) + g.shape)) * 100
    ref = u.copy()
    MG.sweep(L, ref, f, sm)
    ud = dev(u)
    g.op_smooth(0, E.FP64, code, ud, dev(f), omega=sm.omega)
    assert rel_err(ud.cpu().numpy(), ref) < 1e-12
    u32 = dev(u, torch.float32)
    g.op_smooth(0, E.MIXED, code, u32, dev(f, torch.float32), omega=sm.omega)
    assert rel_err(u32.cpu().numpy(), ref) < 5e-5
    g.close()


CYCLES = {
    "F44_jacobi": dict(smoother=2, cycle=1, nu=4, sm=MG.Smoother("jacobi"), kind="F"),
    "F22_rb": dict(smoother=0, cycle=1, nu=2, sm=MG.RB, kind="F"),
    "V22_gs8": dict(smoother=1, cycle=0, nu=2, sm=MG.Smoother("gs8"), kind="V"),
}


@pytest.mark.parametrize("cyc", list(CYCLES))
@pytest.mark.parametrize("case", ["mixed_gen", "polycrystal", "periodic_iso"])
def test_fixed_cycles_match_oracle(E, ctx, case, cyc):
    c = CYCLES[cyc]
    p = CASES[case]()
    g = E.grid_from_problem(ctx, p)
    info = g.solve(precision=E.FP64, fixed_cycles=3, nu1=c["nu"], nu2=c["nu"], smoother=c["smoother"],
                   cycle=c["cycle"])
    ref, rinfo = MG.solve(p, fixed_cycles=3, nu1=c["nu"], nu2=c["nu"], smoother=c["sm"], cycle=c["kind"])
    assert rel_err(g.displacement(), ref) < 1e-9
    assert np.allclose(info["rel_history"][:4], rinfo.rel_history, rtol=1e-7, atol=0)
    g.close()


@pytest.mark.parametrize("cyc", ["F44_jacobi", "F22_rb"])
def test_f_cycle_fp64_and_mixed_solves_reach_the_oracle(E, ctx, cyc):
    c = CYCLES[cyc]
    p = CASES["polycrystal"]()
    g = E.grid_from_problem(ctx, p, mixed=True)
    kw = dict(nu1=c["nu"], nu2=c["nu"], smoother=c["smoother"], cycle=c["cycle"])
    ref, rinfo = MG.solve(p, tol=1e-8, max_cycles=200, nu1=c["nu"], nu2=c["nu"], smoother=c["sm"],
                          cycle=c["kind"])
    i64 = g.solve(precision=E.FP64, rel_tol=1e-8, max_cycles=200, **kw)
    assert i64["status"] == 0 and i64["cycles"] == rinfo.cycles
    assert rel_err(g.displacement(), ref) < 1e-9
    imx = g.solve(precision=E.MIXED, rel_tol=1e-8, max_cycles=200, **kw)
    assert imx["status"] == 0
    rel_fp64, _ = g.query_residual()
    assert rel_fp64 <= 1.01e-8
    assert rel_err(g.displacement(), ref) < 1e-7
    g.close()


def test_invalid_smoother_options_are_errors(E, ctx):
    g = E.grid_from_problem(ctx, CASES["eshelby"]())
    for kw in (dict(smoother=7), dict(cycle=3), dict(smoother=2, omega=1.5)):
        with pytest.raises(E.ElasError):
            g.solve(precision=E.FP64, fixed_cycles=1, **kw)
    g.close()
