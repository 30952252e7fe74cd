"""The residual entry point that allocates nothing (for callers that cannot call
cudaMalloc while they run), checked through the C ABI against the ordinary
residual entry point on two calls in a row.  Collected last on purpose."""
import numpy as np
import pytest

from paper_2001_04789_gb300 import microstructure as M

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


def test_noalloc_residual_matches_residual_on_two_calls(E):
    ctx = E.Context(0)
    p = M.polycrystal(17, grains=4, seed=3)
    g = E.grid_from_problem(ctx, p, mixed=True)
    rng = np.random.default_rng(11)
    for call in range(2):                     # two calls in a row share the static scratch
        for precision, dtype, tol in ((E.FP64, torch.float64, 1e-12), (E.MIXED, torch.float32, 1e-6)):
            u = torch.as_tensor(rng.normal(size=(3,) + g.shape), dtype=dtype, device="cuda:0")
            f = torch.as_tensor(rng.normal(size=(3,) + g.shape), dtype=dtype, device="cuda:0")
            r_ref, ss_ref = g.op_residual(0, precision, u, f)
            r = torch.empty_like(u)
            ss = g.op_residual_noalloc(0, precision, u, f, r)
            assert torch.allclose(r, r_ref, rtol=0, atol=tol * float(r_ref.abs().max()))
            assert ss == pytest.approx(ss_ref, rel=1e-12)
    g.close()
    ctx.close()
