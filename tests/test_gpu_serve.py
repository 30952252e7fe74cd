"""Continuous batching (elas_server_*) through the C ABI: requests admitted into
slots while others run give the same result as each solve alone, and the request
loop completes a short Poisson stream with every solve converged."""
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


def problems():
    return [M.eshelby_sphere(17), M.penny_crack(17, width=3.0 / 16, clamp_lateral=True),
            M.polycrystal(17, grains=4, seed=2), M.ellipsoid_rve(17, seed=4), M.eshelby_sphere(33)]


def test_each_result_is_the_same_alone_and_in_the_mix(E):
    ctx = E.Context(0)
    probs = problems()
    grids = [E.grid_from_problem(ctx, p, mixed=True) for p in probs]
    alone = []
    for g in grids:
        info = g.solve(precision=E.MIXED, rel_tol=1e-8)
        alone.append((g.displacement(), info))
    server = E.Server(ctx, max_active=2)
    tickets = {}
    done = {}
    pending = list(range(len(grids)))
    steps = 0
    while len(done) < len(grids):
        # stagger arrivals: one new request every other step
        if pending and steps % 2 == 0:
            i = pending.pop(0)
            tickets[server.submit(grids[i], rel_tol=1e-8, warm_start=False)] = i
        act, wait = server.step()
        assert act <= 2
        for t, i in list(tickets.items()):
            r = server.poll(t)
            if r is not None:
                done[i] = r[0]
                del tickets[t]
        steps += 1
        assert steps < 2000
    for i, g in enumerate(grids):
        ua, ia = alone[i]
        ub = g.displacement()
        assert done[i]["cycles"] == ia["cycles"]
        assert np.abs(ua - ub).max() <= 1e-14 * np.abs(ua).max()
    server.close()
    for g in grids:
        g.close()
    ctx.close()


def test_request_loop_completes_short_stream(E):
    from paper_2001_04789_gb300 import serve
    out = serve.run(seconds=2.0, rate=40.0, sizes=(17, 33), max_active=8, budget=8 << 30)
    assert out["completed"] > 0
    assert out["converged"] == out["completed"]
    assert out["latency_ms"]["p99"] >= out["latency_ms"]["p50"] > 0


def test_duplicate_submission_refused_and_failed_setup_retires(E):
    """A grid with a request still waiting or active is refused; a request whose set-up
    fails at admission (no moduli) polls as done with that error and frees its slot for
    the next request."""
    ctx = E.Context(0)
    good = E.grid_from_problem(ctx, M.eshelby_sphere(17), mixed=True)
    bare = E.Grid(ctx, E.desc_for(M.eshelby_sphere(17), mixed=True))     # moduli never set
    server = E.Server(ctx, max_active=1)
    t_bad = server.submit(bare, rel_tol=1e-8)
    t_good = server.submit(good, rel_tol=1e-8)
    with pytest.raises(E.ElasError) as err:
        server.submit(good, rel_tol=1e-8)
    assert err.value.code == E.ERR_STATE
    results = {}
    for _ in range(500):
        server.step()
        for t in (t_bad, t_good):
            if t not in results:
                r = server.poll(t)
                if r is not None:
                    results[t] = r[0]
        if len(results) == 2:
            break
    assert results[t_bad]["status"] == E.ERR_STATE
    assert results[t_good]["status"] == 0 and results[t_good]["rel_residual"] <= 1e-8
    server.close()
    good.close()
    bare.close()
    ctx.close()


def test_amr_request_is_the_same_alone_and_in_the_mix(E):
    """A composite AMR solve served as a request (one composite cycle per step, beside
    single-grid requests) gives the same cycles and the same bits as elas_amr_solve."""
    from paper_2001_04789_gb300 import microstructure as M2
    ctx = E.Context(0)
    specs = M2.amr_penny_crack(base_n=17, nlevels=2, block=8, width=3.0 / 32)
    amr = E.Amr(ctx, specs)
    alone = amr.solve(rel_tol=1e-8)
    u_alone = amr.displacements()
    grids = [E.grid_from_problem(ctx, p, mixed=True) for p in problems()[:2]]
    server = E.Server(ctx, max_active=3)
    tickets = {server.submit(grids[0], rel_tol=1e-8): "g0", server.submit_amr(amr, rel_tol=1e-8): "amr",
               server.submit(grids[1], rel_tol=1e-8): "g1"}
    done = {}
    for _ in range(1000):
        server.step()
        for t, name in list(tickets.items()):
            r = server.poll(t)
            if r is not None:
                done[name] = r[0]
                del tickets[t]
        if not tickets:
            break
    assert done["amr"]["status"] == 0 and done["amr"]["cycles"] == alone["cycles"]
    assert np.allclose(done["amr"]["rel_history"], alone["rel_history"], rtol=1e-12)
    for ua, ub in zip(u_alone, amr.displacements()):
        assert np.array_equal(ua, ub)
    server.close()
    amr.close()
    for g in grids:
        g.close()
    ctx.close()


def test_request_loop_with_amr_requests_and_bounded_admission(E):
    """The request loop serves two-level AMR requests beside single-grid ones and refuses
    arrivals beyond its queue bound; every served solve converges."""
    from paper_2001_04789_gb300 import serve
    out = serve.run(seconds=2.0, rate=60.0, sizes=(17,), kinds=("sphere", "polycrystal"),
                    amr_kinds=("sphere", "crack", "polycrystal"), amr_sizes=(17,), max_active=4,
                    budget=8 << 30, max_queue=6)
    assert out["completed"] > 0 and out["converged"] == out["completed"]
    assert out["refused"] >= 0 and out["max_queue"] == 6
    assert out["latency_ms"]["p99"] >= out["latency_ms"]["p50"] > 0


def test_mixed_amr_request_is_the_same_alone_and_in_the_mix(E):
    from paper_2001_04789_gb300 import microstructure as M2
    ctx = E.Context(0)
    specs = M2.amr_penny_crack(base_n=17, nlevels=2, block=8, width=3.0 / 32)
    amr = E.Amr(ctx, specs, mixed=True)
    alone = amr.solve(rel_tol=1e-8, precision=E.MIXED)
    u_alone = amr.displacements()
    g = E.grid_from_problem(ctx, problems()[0], mixed=True)
    server = E.Server(ctx, max_active=2)
    ta = server.submit_amr(amr, precision=E.MIXED, rel_tol=1e-8)
    tg = server.submit(g, rel_tol=1e-8)
    done = {}
    for _ in range(1000):
        server.step()
        for t in (ta, tg):
            if t not in done:
                r = server.poll(t)
                if r is not None:
                    done[t] = r[0]
        if len(done) == 2:
            break
    assert done[ta]["status"] == 0 and done[ta]["cycles"] == alone["cycles"]
    for ua, ub in zip(u_alone, amr.displacements()):
        assert np.array_equal(ua, ub)
    server.close()
    amr.close()
    g.close()
    ctx.close()


def test_a_grid_held_by_a_request_refuses_solves_setters_and_queries(E):
    """While a request on a grid waits or runs, calls that would launch on the grid or
    change it are refused with ELAS_ERR_STATE before touching the device (the request keeps
    its activity flags and iterate in the grid between steps); reading the displacement
    stays allowed, and once the request retires the grid solves again, with the same
    result as the request."""
    ctx = E.Context(0)
    g = E.grid_from_problem(ctx, M.eshelby_sphere(17), mixed=True)
    server = E.Server(ctx, max_active=1)
    ticket = server.submit(g, rel_tol=1e-8)
    refused = (lambda: g.solve(precision=E.MIXED, rel_tol=1e-8),
               lambda: g.set_bc(0, 0, M.DIRICHLET, 0.0),
               lambda: g.query_residual())
    done = None
    for step in range(500):
        for call in refused:                    # waiting (step 0), then active
            with pytest.raises(E.ElasError) as err:
                call()
            assert err.value.code == E.ERR_STATE
        g.displacement()
        server.step()
        done = server.poll(ticket)
        if done is not None:
            break
    assert done is not None and done[0]["status"] == 0
    served = g.displacement()
    info = g.solve(precision=E.MIXED, rel_tol=1e-8)
    assert info["status"] == 0 and info["cycles"] == done[0]["cycles"]
    assert np.abs(g.displacement() - served).max() <= 1e-14 * np.abs(served).max()
    server.close()
    g.close()
    ctx.close()
