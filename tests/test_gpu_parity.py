"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Sizes span several 256-thread blocks with ragged tails; every row type occurs
(interior, Dirichlet, traction faces/edges/corners, Neumann, periodic wrap).
Tolerances: FP64 operations agree to rounding (1e-12 relative); FP32 operations
to 2e-5 relative of the row scale; FP64 solves after the same number of cycles
to 1e-9 in the relative inf-norm, mixed solves at a relative residual of 1e-8
to 1e-7 against the oracle's converged FP64 solution.
"""
import numpy as np
import pytest

from paper_2001_04789_gb300 import microstructure as M
from oracle import multigrid as MG
from oracle import stencil as S

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


def mixed_bc_problem(n=(13, 9, 11), kind=M.MODULI_GEN21, seed=0):
    rng = np.random.default_rng(seed)
    p = M.Problem(n=n, hi=(1.0, 0.7, 0.9), name="mixed_bc")
    X, Y, Z = p.coords()
    if kind == M.MODULI_GEN21:
        base = M.voigt_to_tensor(M.cubic_voigt(1.68, 1.21, 0.75))
        c1 = M.tensor_to_upper21(M.rotate_tensor(base, M.random_rotation(rng)))
        c2 = M.tensor_to_upper21(M.rotate_tensor(base, M.random_rotation(rng)))
        w = 0.5 * (1 + np.tanh(4 * (X - 0.5 + 0.2 * np.sin(3 * Y + Z))))
        p.moduli_kind = M.MODULI_GEN21
        p.moduli = c1[:, None, None, None] * (1 - w) + c2[:, None, None, None] * w
    else:
        lam, mu = M.lame(1.0 + 0.5 * np.sin(2 * X + Y) * np.cos(Z), 0.3)
        p.moduli_kind = M.MODULI_ISO
        p.moduli = np.stack([lam, mu])
    e = np.zeros((6,) + X.shape)
    e[0] = 1e-3 * np.exp(-10 * ((X - 0.4) ** 2 + (Y - 0.3) ** 2))
    e[5] = 5e-4 * np.sin(2 * Z)
    p.eigenstrain = e
    p.body_force = np.stack([np.sin(Y), X * Z, np.cos(X + Y)]) * 1e-2
    bc = M.all_faces(M.TRACTION, 0.0)
    bc[0] = [(M.DIRICHLET, 1e-3), (M.TRACTION, 0.01), (M.NEUMANN, 0.002)]
    bc[1] = [(M.TRACTION, -0.02), (M.DIRICHLET, 0.0), (M.TRACTION, 0.0)]
    bc[2] = [(M.NEUMANN, 0.0), (M.TRACTION, 0.0), (M.TRACTION, 0.03)]
    bc[5] = [(M.DIRICHLET, 0.0)] * 3
    p.bc = bc
    return p


def periodic_problem(n=16):
    return M.ellipsoid_rve(n + 1, seed=3)


CASES = {
    "mixed_gen": lambda: mixed_bc_problem(kind=M.MODULI_GEN21),
    "mixed_iso": lambda: mixed_bc_problem(kind=M.MODULI_ISO, n=(9, 13, 7)),
    "periodic_iso": lambda: periodic_problem(16),
    "eshelby": lambda: M.eshelby_sphere(17),
    "polycrystal": lambda: M.polycrystal(17, grains=5, seed=1),
}


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


def rel_err(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("case", list(CASES))
def test_apply_fp64_matches_oracle(E, ctx, case):
    p = CASES[case]()
    g = E.grid_from_problem(ctx, p, mixed=True)
    rng = np.random.default_rng(1)
    u = rng.normal(size=(3,) + g.shape)
    got = g.op_apply(0, E.FP64, dev(u)).cpu().numpy()
    ref = S.apply(S.level_from_problem(p), u)
    assert rel_err(got, ref) < 1e-12
    # FP32 moduli and field, same rows
    got32 = g.op_apply(0, E.MIXED, dev(u, torch.float32)).cpu().numpy()
    assert rel_err(got32, ref) < 2e-5
    g.close()


@pytest.mark.parametrize("case", list(CASES))
def test_rhs_matches_oracle(E, ctx, case):
    p = CASES[case]()
    g = E.grid_from_problem(ctx, p)
    got = g.op_rhs().cpu().numpy()
    ref = S.rhs(S.level_from_problem(p), p)
    assert rel_err(got, ref) < 1e-12
    g.close()


@pytest.mark.parametrize("case", list(CASES))
def test_sweep_matches_oracle(E, ctx, case):
    p = CASES[case]()
    g = E.grid_from_problem(ctx, p, mixed=True)
    levels = MG.build_hierarchy(S.level_from_problem(p))
    L = levels[0]
    rng = np.random.default_rng(2)
    u = np.where(L.types == M.DIRICHLET, 0.0, rng.normal(size=(3,) + g.shape))
    f = np.where(L.types == M.DIRICHLET, 0.0, rng.normal(size=(3,) + g.shape)) * 100
    ud = dev(u)
    g.op_sweep(0, E.FP64, ud, dev(f))
    ref = u.copy()
    MG.sweep(L, ref, f)
    assert rel_err(ud.cpu().numpy(), ref) < 1e-12
    u32 = dev(u, torch.float32)
    g.op_sweep(0, E.MIXED, u32, dev(f, torch.float32))
    assert rel_err(u32.cpu().numpy(), ref) < 5e-5
    g.close()


@pytest.mark.parametrize("n,sweep", [((71, 69, 67), True), ((103, 103, 99), False)])
def test_face_row_paths_match_oracle_at_size(E, ctx, n, sweep):
    """Face rows take different code paths by level size: levels of 300000 to 2^20 nodes
    evaluate every face row in the face kernels (FP64 and FP32), larger ones take the x
    faces from stored coefficients and the y and z faces from the face kernels.  One level
    of each band, general moduli and mixed boundary types: operator rows against the
    oracle, and one sweep on the first (the oracle's sweep of a million nodes takes
    minutes)."""
    p = mixed_bc_problem(n=n)
    g = E.grid_from_problem(ctx, p, mixed=True, max_levels=1)
    lev = S.level_from_problem(p)
    types = S.row_types(lev)
    rng = np.random.default_rng(7)
    u = np.where(types == M.DIRICHLET, 0.0, rng.normal(size=(3,) + g.shape))
    f = np.where(types == M.DIRICHLET, 0.0, rng.normal(size=(3,) + g.shape)) * 100
    ref = S.apply(lev, u, types)
    assert rel_err(g.op_apply(0, E.FP64, dev(u)).cpu().numpy(), ref) < 1e-12
    assert rel_err(g.op_apply(0, E.MIXED, dev(u, torch.float32)).cpu().numpy(), ref) < 2e-5
    if not sweep:
        g.close()
        return
    B = S.block_diagonal(lev, types)
    k, j, i = np.meshgrid(*[np.arange(s) for s in lev.shape], indexing="ij")
    L = MG.LevelData(lev, types, np.linalg.inv(np.moveaxis(B, (0, 1), (-2, -1))), (i + j + k) % 2,
                     MG.rigid_modes(lev, types))
    sw = u.copy()
    MG.sweep(L, sw, f)
    ud = dev(u)
    g.op_sweep(0, E.FP64, ud, dev(f))
    assert rel_err(ud.cpu().numpy(), sw) < 1e-12
    u32 = dev(u, torch.float32)
    g.op_sweep(0, E.MIXED, u32, dev(f, torch.float32))
    assert rel_err(u32.cpu().numpy(), sw) < 5e-5
    g.close()


@pytest.mark.parametrize("case", list(CASES))
def test_transfers_match_oracle(E, ctx, case):
    p = CASES[case]()
    g = E.grid_from_problem(ctx, p)
    if g.levels() < 2:
        pytest.skip("single level")
    levels = MG.build_hierarchy(S.level_from_problem(p))
    rng = np.random.default_rng(3)
    r = np.where(levels[0].types == M.DIRICHLET, 0.0, rng.normal(size=(3,) + g.shape))
    fc = g.op_restrict(0, E.FP64, dev(r)).cpu().numpy()
    ref = np.where(levels[1].types == M.DIRICHLET, 0.0, MG.restrict(r, levels[0].level))
    assert rel_err(fc, ref) < 1e-13
    nc = g.level_dims(1)
    ec = rng.normal(size=(3, nc[2], nc[1], nc[0]))
    u = rng.normal(size=(3,) + g.shape)
    got = g.op_prolong_add(0, E.FP64, dev(ec), dev(u)).cpu().numpy()
    ref = u + np.where(levels[0].types == M.DIRICHLET, 0.0, MG.prolong(ec, levels[0].level))
    assert rel_err(got, ref) < 1e-13
    g.close()


@pytest.mark.parametrize("case", list(CASES))
def test_bottom_matches_oracle(E, ctx, case):
    p = CASES[case]()
    g = E.grid_from_problem(ctx, p)
    levels = MG.build_hierarchy(S.level_from_problem(p))
    Lb = levels[-1]
    rng = np.random.default_rng(4)
    f = np.where(Lb.types == M.DIRICHLET, 0.0, rng.normal(size=(3,) + Lb.level.shape))
    got = g.op_bottom(E.FP64, dev(f)).cpu().numpy()
    ref = MG.bottom_solve(Lb, f)
    assert rel_err(got, ref) < 1e-10
    g.close()


@pytest.mark.parametrize("case", list(CASES))
def test_fp64_cycles_match_oracle(E, ctx, case):
    p = CASES[case]()
    g = E.grid_from_problem(ctx, p)
    info = g.solve(precision=E.FP64, fixed_cycles=3)
    got = g.displacement()
    ref, rinfo = MG.solve(p, fixed_cycles=3)
    assert rel_err(got, ref) < 1e-9
    assert np.allclose(info["rel_history"], rinfo.rel_history, rtol=1e-7, atol=0)
    g.close()


@pytest.mark.parametrize("case", ["eshelby", "polycrystal", "periodic_iso"])
def test_fp64_and_mixed_solves_reach_oracle_solution(E, ctx, case):
    p = CASES[case]()
    truth, tinfo = MG.solve(p, tol=1e-13, max_cycles=300)
    assert tinfo.converged
    g = E.grid_from_problem(ctx, p, mixed=True)
    i64 = g.solve(precision=E.FP64, rel_tol=1e-8)
    assert i64["status"] == 0 and i64["rel_residual"] <= 1e-8
    ref, rinfo = MG.solve(p, tol=1e-8, max_cycles=300)
    assert i64["cycles"] == rinfo.cycles
    assert rel_err(g.displacement(), ref) < 1e-9
    imx = g.solve(precision=E.MIXED, rel_tol=1e-8)
    assert imx["status"] == 0 and imx["rel_residual"] <= 1e-8
    rel_fp64, _ = g.query_residual()
    assert rel_fp64 <= 1.01e-8
    # both at a relative residual of 1e-8: the mixed result against the oracle's
    assert rel_err(g.displacement(), ref) < 1e-7
    # and both within the same distance of the converged discrete solution
    assert rel_err(g.displacement(), truth) < 10 * max(rel_err(ref, truth), 1e-9)
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_residual_max_norm_matches_oracle(E, ctx, precision):
    """||r||_inf of the residual kernels (solve info and query) against the oracle's
    residual of the returned displacement (all rigid modes held by Dirichlet rows)."""
    p = CASES["mixed_gen"]()
    lev = S.level_from_problem(p)
    f = S.rhs(lev, p)
    g = E.grid_from_problem(ctx, p, mixed=True)
    prec = E.FP64 if precision == "fp64" else E.MIXED
    info = g.solve(precision=prec, rel_tol=1e-7)
    assert info["status"] == 0 and info["nlam"] == 0
    ref = np.abs(S.residual(lev, g.displacement(), f)).max()
    ref0 = np.abs(S.residual(lev, S.dirichlet_values(lev), f)).max()
    rel_q, abs_q = g.query_residual_inf()
    assert abs(abs_q - ref) <= 1e-6 * ref + 1e-13 * np.abs(f).max()
    assert abs(rel_q - ref / ref0) <= 1e-6 * rel_q + 1e-13
    # the solve's own last evaluation: FP64 (bitwise the query's) or double-float (FP32 output)
    tol = 0.0 if precision == "fp64" else 1e-6 * abs_q
    assert abs(info["residual_inf"] - abs_q) <= tol
    assert info["rel_residual_inf"] > 0
    g.close()


def test_warm_start_from_solution_converges_immediately(E, ctx):
    p = M.eshelby_sphere(17)
    g = E.grid_from_problem(ctx, p, mixed=True)
    g.solve(precision=E.MIXED, rel_tol=1e-10)
    info = g.solve(precision=E.MIXED, rel_tol=1e-8, warm_start=True)
    assert info["cycles"] == 0
    g.close()


def test_smallest_grid_is_single_level(E, ctx):
    p = M.eshelby_sphere(5)
    g = E.grid_from_problem(ctx, p)
    assert g.levels() == 1
    info = g.solve(precision=E.FP64, rel_tol=1e-12)
    ref, _ = MG.solve(p, tol=1e-12)
    assert rel_err(g.displacement(), ref) < 1e-9
    g.close()


def test_invalid_arguments_are_errors(E, ctx):
    d = E.desc_for(M.eshelby_sphere(9))
    d.n[0] = 2
    with pytest.raises(E.ElasError):
        E.Grid(ctx, d)
    d = E.desc_for(M.eshelby_sphere(9))
    d.moduli_kind = 7
    with pytest.raises(E.ElasError):
        E.Grid(ctx, d)
    g = E.Grid(ctx, E.desc_for(M.eshelby_sphere(9)))
    with pytest.raises(E.ElasError):
        g.solve()                    # moduli not set
    with pytest.raises(E.ElasError):
        g.set_bc(6, 0, M.DIRICHLET)
    g.close()


def test_budget_refuses_oversized_grid(E):
    c = E.Context(0, budget_bytes=1 << 20)
    with pytest.raises(E.ElasError) as ei:
        E.Grid(c, E.desc_for(M.eshelby_sphere(33)))
    assert ei.value.code == -2
    c.close()


def test_autotuned_launch_shapes_do_not_change_results(E, ctx):
    p = CASES["mixed_gen"]()
    g = E.grid_from_problem(ctx, p, mixed=True)
    before = g.solve(precision=E.MIXED, rel_tol=0.0, fixed_cycles=3)
    ub = g.displacement()
    times = g.autotune()
    # the untiled shapes always apply; a tiled one reports -1 where it does not
    assert len(times) == E.NUM_SWEEP_VARIANTS and all(times[v] > 0 for v in E.UNTILED_VARIANTS)
    assert all(t > 0 or t == -1 for t in times)
    assert len(E.autotune_dump().strip().splitlines()) >= 1
    after = g.solve(precision=E.MIXED, rel_tol=0.0, fixed_cycles=3)
    assert np.array_equal(ub, g.displacement())
    assert before["rel_history"] == after["rel_history"]
    g.close()


def test_two_inner_fp32_cycles_per_refinement_step(E, ctx):
    p = CASES["polycrystal"]()
    g = E.grid_from_problem(ctx, p, mixed=True)
    one = g.solve(precision=E.MIXED, rel_tol=1e-8)
    two = g.solve(precision=E.MIXED, rel_tol=1e-8, inner_cycles=2)
    assert two["status"] == 0 and two["cycles"] < one["cycles"]
    ref, _ = MG.solve(p, tol=1e-8, max_cycles=300)
    assert rel_err(g.displacement(), ref) < 1e-7
    g.close()


def test_graph_replayed_mixed_solve_equals_direct_solve(E, ctx):
    p = CASES["polycrystal"]()
    g = E.grid_from_problem(ctx, p, mixed=True)
    direct = g.solve(precision=E.MIXED, rel_tol=1e-8, inner_cycles=2)
    ud = g.displacement()
    graph = g.solve(precision=E.MIXED, rel_tol=1e-8, inner_cycles=2, use_graph=True)
    assert graph["cycles"] == direct["cycles"]
    assert np.abs(g.displacement() - ud).max() <= 1e-14 * np.abs(ud).max()
    g.close()


@pytest.mark.parametrize("case", ["polycrystal", "eshelby", "periodic_iso"])
def test_half_moduli_v_cycle_reaches_the_oracle_solution(E, ctx, case):
    """FP16 moduli only precondition: the FP64 refinement still reaches the oracle."""
    p = CASES[case]()
    g = E.grid_from_problem(ctx, p, mixed=True, half_moduli=True)
    info = g.solve(precision=E.MIXED, rel_tol=1e-8, inner_cycles=2)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-8
    ref, _ = MG.solve(p, tol=1e-8, max_cycles=300)
    assert rel_err(g.displacement(), ref) < 1e-7
    g.close()


def force_variant(E, p, v):
    """Tuning-table entries that pin interior smoother shape v on every FP32 level (keys
    of blocked and of colour-split moduli; a shape that does not apply to a level falls
    back to shape 0 there)."""
    n = list(p.n)
    lines = []
    for _ in range(12):
        k = 21 if p.moduli_kind == M.MODULI_GEN21 else 2
        lines.append(f"{n[0]} {n[1]} {n[2]} {k} 4 0 {v}")
        lines.append(f"{n[0]} {n[1]} {n[2]} {k} 4 2 {v}")
        if min(n) < 5:
            break
        n = [(m - 1) // 2 + 1 if not per else m // 2 for m, per in zip(n, p.periodic)]
    assert E.autotune_load("\n".join(lines)) == len(lines)


TILE_CASES = {
    # interior 68 x 35 x 21: two full 32-wide tiles and a ragged one, ragged rows, z chunks
    "gen21_ragged": lambda: mixed_bc_problem(n=(70, 37, 23), kind=M.MODULI_GEN21),
    "iso_ragged": lambda: mixed_bc_problem(n=(41, 19, 13), kind=M.MODULI_ISO),
    "periodic_iso": lambda: periodic_problem(32),
    "polycrystal": lambda: M.polycrystal(33, grains=5, seed=2),
    # odd nx, ny: colour-split moduli; interior 67 x 35 x 21 (ragged tiles, z chunks)
    "split_ragged": lambda: mixed_bc_problem(n=(69, 37, 23), kind=M.MODULI_GEN21),
}


@pytest.mark.parametrize("case", list(TILE_CASES))
def test_tiled_smoother_is_bitwise_equal_to_untiled(E, ctx, case):
    """The shared-memory tiled interior half-sweep runs the same arithmetic as the
    one-thread-per-pair kernel: a sweep from the same state gives identical bits."""
    p = TILE_CASES[case]()
    g = E.grid_from_problem(ctx, p, mixed=True, max_levels=1)
    rng = np.random.default_rng(5)
    u = rng.normal(size=(3,) + g.shape)
    f = rng.normal(size=(3,) + g.shape) * 100
    out = {}
    for v in range(E.NUM_SWEEP_VARIANTS):
        force_variant(E, p, v)
        u32 = dev(u, torch.float32)
        g.op_sweep(0, E.MIXED, u32, dev(f, torch.float32))
        out[v] = u32.cpu().numpy()
    for v in range(1, E.NUM_SWEEP_VARIANTS):
        assert np.array_equal(out[v], out[0]), f"shape {v}"
    force_variant(E, p, 0)
    g.close()


@pytest.mark.parametrize("case", ["periodic_iso", "polycrystal"])
def test_tiled_smoother_mixed_solve_matches(E, ctx, case):
    """Whole mixed solves (equilibrating load included on the periodic cell) with the
    tiled smoother on every FP32 level repeat the untiled residual history exactly."""
    p = TILE_CASES[case]()
    g = E.grid_from_problem(ctx, p, mixed=True)
    hist = {}
    for v in (0,) + E.TILED_VARIANTS + E.SPLIT_TILED_VARIANTS:
        force_variant(E, p, v)
        info = g.solve(precision=E.MIXED, rel_tol=0.0, fixed_cycles=4, inner_cycles=2)
        hist[v] = (info["rel_history"], g.displacement())
    for v in E.TILED_VARIANTS + E.SPLIT_TILED_VARIANTS:
        assert hist[v][0] == hist[0][0]
        assert np.array_equal(hist[v][1], hist[0][1])
    force_variant(E, p, 0)
    g.close()


def test_inputs_written_by_async_kernels_on_the_current_stream(E, ctx):
    """Device inputs produced by kernels still queued on torch's current stream are
    read only after those kernels: the binding orders the library's stream after it."""
    p = mixed_bc_problem()
    g = E.grid_from_problem(ctx, p)
    rng = np.random.default_rng(5)
    u_host = rng.normal(size=(3,) + g.shape)
    u_sync = dev(u_host)
    ref = g.op_apply(0, E.FP64, u_sync).cpu().numpy()
    torch.cuda.synchronize()
    x = torch.full((4096, 4096), 1.0 / 4096, device="cuda:0")
    for _ in range(12):            # a queue of long kernels ahead of the input's producer
        x = x @ x
    u_async = torch.as_tensor(u_host, device="cuda:0") + x[0, 0] * 0.0
    out = g.op_apply(0, E.FP64, u_async).cpu().numpy()
    assert np.array_equal(out, ref)
    g.close()
