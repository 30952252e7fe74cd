"""Host-side logic that needs no GPU: the smoother's tuning table (text round trip,
rejection of unknown launch shapes), the HBM estimate used for admission by the serving
loop, the binding's checks of single-operation arguments, and the serving loop's
resident cache."""
import pytest

from paper_2001_04789_gb300 import microstructure as M

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def E():
    from paper_2001_04789_gb300 import build as B
    try:
        B.build()
    except RuntimeError as e:       # no nvcc on this machine
        pytest.skip(str(e))
    from paper_2001_04789_gb300 import elas
    return elas


def test_tuning_table_round_trip_and_unknown_shapes(E):
    bad = E.NUM_SWEEP_VARIANTS          # one past the last launch shape
    text = f"41 43 47 21 4 0 2\n23 29 31 2 8 1 1\n19 19 19 21 4 0 {bad}\n"
    assert E.autotune_load(text) == 2   # the unknown shape is refused
    dump = E.autotune_dump()
    lines = set(dump.strip().splitlines())
    assert "41 43 47 21 4 0 2" in lines and "23 29 31 2 8 1 1" in lines
    assert not any(l.startswith("19 19 19 21 4 0") for l in lines)
    # the dump reads back entry for entry
    assert E.autotune_load(dump) == len(lines)
    assert set(E.autotune_dump().strip().splitlines()) == lines


def test_hbm_estimate_orders_precisions_and_sizes(E):
    est = lambda p, **kw: E.lib().elas_grid_bytes_estimate(E.desc_for(p, **kw))
    small = M.polycrystal(33, grains=3, seed=0)
    fp64 = est(small)
    mixed = est(small, mixed=True)
    half = est(small, mixed=True, half_moduli=True)
    assert fp64 < half < mixed
    # FP64 general moduli: 21 planes + 18 divergence planes + 12 field planes per node,
    # summed over a hierarchy of about 8/7 of the finest level, plus 9 input planes
    # (eigenstrain, body force) and the stored rows (243 coefficients a node) of the edges
    # and corners (FP64 levels below 2^20 nodes)
    n0 = 33 ** 3
    base = 8 * (51 + 9) * n0
    assert base <= fp64 <= 1.5 * base
    # the FP32 copy of such a level of general moduli also stores every face node's row
    assert mixed - fp64 >= 4 * 243 * 6 * 31 * 31
    n1 = 129 ** 3
    large = M.Problem(n=(129, 129, 129), name="descriptor only")
    large.moduli_kind = M.MODULI_GEN21
    assert est(large) >= 8 * 60 * n1 + 8 * 243 * 2 * 129 * 129
    larger = M.Problem(n=(257, 257, 257), name="descriptor only")
    larger.moduli_kind = M.MODULI_GEN21
    ratio = est(larger, mixed=True) / est(large, mixed=True)
    assert 7.0 < ratio < 9.0            # node count grows 7.9x from 129^3 to 257^3


class _OnDevice0(torch.Tensor):
    """A host tensor that reports itself as a CUDA tensor on device 0, so the binding's
    argument checks can be exercised without a GPU (no pointer reaches the library)."""

    @property
    def is_cuda(self):
        return True

    def get_device(self):
        return 0


def test_single_operation_arguments_are_checked_before_the_library(E):
    """The single-operation wrappers refuse, before any pointer reaches the library, a
    field argument its kernels would address out of bounds: not a CUDA tensor (a numpy
    array, a host tensor, another device), the wrong element type, a strided view, or a
    size other than 3 x the level's nodes."""
    dims = (5, 4, 3)
    ok = torch.zeros((3, 3, 4, 5), dtype=torch.float64).as_subclass(_OnDevice0)
    assert E.check_field("u", ok, dims, torch.float64, 0) is ok
    assert E.check_field("u", ok, dims, None, 0) is ok        # dtype left to the library
    bad = {
        "numpy": torch.zeros(3 * 60, dtype=torch.float64).numpy(),
        "host": torch.zeros(3 * 60, dtype=torch.float64),
        "device 1": ok,
        "dtype": ok.to(torch.float32),
        "strided": torch.zeros((3, 3, 4, 10), dtype=torch.float64).as_subclass(_OnDevice0)[..., ::2],
        "short": ok.reshape(-1)[:-1],
        "long": torch.zeros(3 * 60 + 3, dtype=torch.float64).as_subclass(_OnDevice0),
    }
    for what, a in bad.items():
        device = 1 if what == "device 1" else 0
        with pytest.raises(ValueError):
            E.check_field("u", a, dims, torch.float64, device)
    # whole-grid copies (moduli in, displacement out): float64, contiguous, exact count;
    # host tensors are copied from host memory, device ones must be on the context's device
    host = torch.zeros(3 * 60, dtype=torch.float64)
    assert E.check_buffer("u", host, 180, 0) is host
    assert E.check_buffer("u", ok.reshape(-1), 180, 0) is not None
    for a, device in ((host.numpy(), 0), (host.to(torch.float32), 0), (host[:-1], 0),
                      (torch.zeros((3, 120), dtype=torch.float64)[:, ::2], 0), (ok, 1)):
        with pytest.raises(ValueError):
            E.check_buffer("u", a, 180, device)
    # element types: FP64 and FP32 fields; the double-float residual takes FP64 u and f
    # and writes FP32 r; a precision the library refuses has none
    assert E.op_dtype(E.FP64) == torch.float64 and E.op_dtype(E.FP64, output=True) == torch.float64
    assert E.op_dtype(E.MIXED) == torch.float32
    assert E.op_dtype(E.OP_DF) == torch.float64 and E.op_dtype(E.OP_DF, output=True) == torch.float32
    assert E.op_dtype(7) is None


def test_resident_cache_evicts_idle_hierarchies_least_recently_used(monkeypatch):
    """The serving loop's resident cache (host logic only, with stand-ins for the library):
    a hit moves the entry to the most recent end; admitting an entry that would exceed the
    HBM budget evicts idle entries, least recently used first, until it fits, and never a
    busy one; when only busy entries remain the new one waits (None)."""
    import types
    from paper_2001_04789_gb300 import serve

    closed = []

    class FakeGrid:
        def __init__(self, ctx, p):
            self.ctx, self.p = ctx, p
            ctx.used += p.bytes

        def close(self):
            closed.append(self.p.name)
            self.ctx.used -= self.p.bytes

    class FakeCtx:
        used = 0

        def bytes_in_use(self):
            return self.used

    fake_lib = types.SimpleNamespace(elas_grid_bytes_estimate=lambda d: d.bytes)
    fake_E = types.SimpleNamespace(lib=lambda: fake_lib, desc_for=lambda p, mixed=True: p,
                                   grid_from_problem=lambda ctx, p, mixed=True: FakeGrid(ctx, p),
                                   Amr=None)
    monkeypatch.setattr(serve, "E", fake_E)
    prob = lambda name, b: types.SimpleNamespace(name=name, bytes=b)
    ctx = FakeCtx()
    cache = serve.ResidentCache(ctx, budget=100)
    for name in "abc":
        assert cache.get(name, lambda name=name: prob(name, 30)) is not None
    assert ctx.used == 90 and closed == []
    cache.get("a", lambda: prob("a", 30))                 # hit: a becomes the most recent
    cache.busy.add("b")
    g, _ = cache.get("d", lambda: prob("d", 30))          # needs 30: evicts c (b is busy, a recent)
    assert closed == ["c"] and list(cache.grids) == ["b", "a", "d"] and ctx.used == 90
    g, _ = cache.get("e", lambda: prob("e", 40))          # needs 40: evicting a is enough
    assert closed == ["c", "a"] and list(cache.grids) == ["b", "d", "e"] and ctx.used == 100
    cache.busy.add("e")
    assert cache.get("f", lambda: prob("f", 50)) is None   # evicts idle d, then only busy ones: wait
    assert closed == ["c", "a", "d"] and list(cache.grids) == ["b", "e"] and ctx.used == 70
