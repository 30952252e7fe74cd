"""Stress output (elas_get_stress, the stress of Eq. 1c) through the C ABI: element by
element against the oracle on the same displacement (FP64 to 1e-12), and the
ellipsoidal Eshelby inclusion of Section 4.1 solved on the GPU: the stress inside the
inclusion approaches Eshelby's uniform interior stress as the grid is refined."""
import numpy as np
import pytest

from paper_2001_04789_gb300 import microstructure as M
from oracle import stencil as S

from test_gpu_parity import CASES, rel_err

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


@pytest.mark.parametrize("case", list(CASES))
def test_stress_matches_oracle(E, ctx, case):
    p = CASES[case]()
    g = E.grid_from_problem(ctx, p)
    rng = np.random.default_rng(31)
    u = rng.normal(size=(3,) + g.shape) * 1e-3
    g.set_displacement(u)
    got = g.stress()
    ref = S.stress(S.level_from_problem(p), u, eps0=p.eigenstrain, ebar=p.mean_strain)
    assert rel_err(got, ref) < 1e-12
    g.close()


def test_ellipsoid_interior_stress_approaches_eshelby(E, ctx):
    import eshelby_closed_form as EC
    s_exact = EC.interior_stress_dilatational((1.0, 0.75, 0.5), 210.0, 0.3, 1e-3)
    errs = []
    for n in (65, 129):
        p = M.eshelby_ellipsoid(n)
        g = E.grid_from_problem(ctx, p)
        info = g.solve(precision=E.FP64, rel_tol=1e-10, max_cycles=200)
        assert info["status"] == 0
        sig = g.stress()
        X, Y, Z = p.coords()
        core = (X / 1.0) ** 2 + (Y / 0.75) ** 2 + (Z / 0.5) ** 2 <= 0.3 ** 2
        mean = np.array([sig[a][core].mean() for a in range(3)])
        errs.append(np.abs(mean - s_exact).max() / np.abs(s_exact).max())
        assert max(np.abs(sig[a][core]).max() for a in range(3, 6)) < 0.05 * np.abs(s_exact).max()
        g.close()
    assert errs[1] < errs[0] and errs[1] < 0.05, (errs, s_exact)
