"""Thin ctypes binding of the C ABI in ``include/elas.h``.

Argument marshalling only: every step of the solve runs in the CUDA library.
PyTorch supplies the device memory (through the caching allocator, passed to the
library as an allocator callback) and the CUDA stream.  Importing this module
does not need a GPU; creating a context does, and fails loudly when the library
or the device is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import microstructure as M

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libelas_gb300.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_NOT_CONVERGED = -3
ERR_DIVERGED = -4
ERR_STATE = -7
HOST, DEVICE = 0, 1
FP64, MIXED = 0, 1
SMOOTH_RB, SMOOTH_GS8, SMOOTH_JACOBI = 0, 1, 2
CYCLE_V, CYCLE_F = 0, 1
OUTER_AUTO, OUTER_FP64, OUTER_DF = 0, 1, 2   # arithmetic of a mixed solve's refinement residual
OP_DF = 2   # op_residual: the refinement residual in double-float arithmetic (FP64 u, f; FP32 r)
HISTORY = 128


class ElasError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"elas error {code}: {msg}")
        self.code = code


class GridDesc(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("periodic", C.c_int * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("moduli_kind", C.c_int), ("mixed", C.c_int),
                ("max_levels", C.c_int), ("half_moduli", C.c_int)]


class AmrLevelDesc(C.Structure):
    _fields_ = [("grid_lo", C.c_int * 3), ("valid_lo", C.c_int * 3), ("valid_hi", C.c_int * 3),
                ("ghost", C.c_int * 6)]


class SolveOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("rel_tol", C.c_double), ("max_cycles", C.c_int),
                ("nu1", C.c_int), ("nu2", C.c_int), ("warm_start", C.c_int),
                ("fixed_cycles", C.c_int), ("use_graph", C.c_int), ("inner_cycles", C.c_int),
                ("smoother", C.c_int), ("cycle", C.c_int), ("omega", C.c_double),
                ("outer_residual", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("cycles", C.c_int), ("rel_residual", C.c_double),
                ("r0", C.c_double), ("nlam", C.c_int), ("lam", C.c_double * 6),
                ("seconds", C.c_double), ("rel_history", C.c_double * HISTORY),
                ("residual_inf", C.c_double), ("rel_residual_inf", C.c_double)]

    def as_dict(self):
        n = min(self.cycles + 1, HISTORY)
        return {"status": self.status, "cycles": self.cycles, "rel_residual": self.rel_residual,
                "r0": self.r0, "nlam": self.nlam, "lam": list(self.lam[: self.nlam]),
                "seconds": self.seconds, "rel_history": list(self.rel_history[:n]),
                "residual_inf": self.residual_inf, "rel_residual_inf": self.rel_residual_inf}


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


_lib = None


def lib():
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, ip, dp = C.c_void_p, C.c_int, C.POINTER(C.c_double)
    sig = {
        "elas_ctx_create": (ip, [C.POINTER(vp), ip, C.c_size_t, C.POINTER(Allocator), vp]),
        "elas_ctx_destroy": (ip, [vp]),
        "elas_last_error": (C.c_char_p, [vp]),
        "elas_ctx_bytes_in_use": (C.c_size_t, [vp]),
        "elas_grid_create": (ip, [vp, C.POINTER(GridDesc), C.POINTER(vp)]),
        "elas_grid_destroy": (ip, [vp]),
        "elas_grid_levels": (ip, [vp, C.POINTER(ip)]),
        "elas_grid_level_dims": (ip, [vp, ip, C.POINTER(ip)]),
        "elas_grid_bytes": (C.c_size_t, [vp]),
        "elas_grid_bytes_estimate": (C.c_size_t, [C.POINTER(GridDesc)]),
        "elas_set_moduli": (ip, [vp, vp, ip]),
        "elas_set_eigenstrain": (ip, [vp, vp, ip]),
        "elas_set_body_force": (ip, [vp, vp, ip]),
        "elas_set_mean_strain": (ip, [vp, dp]),
        "elas_set_bc": (ip, [vp, ip, ip, ip, C.c_double]),
        "elas_set_face_values": (ip, [vp, ip, vp, ip]),
        "elas_solve_opts_default": (None, [C.POINTER(SolveOpts)]),
        "elas_solve": (ip, [vp, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
        "elas_get_displacement": (ip, [vp, vp, ip]),
        "elas_set_displacement": (ip, [vp, vp, ip]),
        "elas_get_stress": (ip, [vp, vp, ip]),
        "elas_query_residual": (ip, [vp, dp, dp]),
        "elas_query_residual_inf": (ip, [vp, dp, dp]),
        "elas_op_apply": (ip, [vp, ip, ip, vp, vp]),
        "elas_op_residual": (ip, [vp, ip, ip, vp, vp, vp, dp]),
        "elas_op_residual_noalloc": (ip, [vp, ip, ip, vp, vp, vp, dp]),
        "elas_op_sweep": (ip, [vp, ip, ip, vp, vp]),
        "elas_op_smooth": (ip, [vp, ip, ip, ip, C.c_double, vp, vp]),
        "elas_op_restrict": (ip, [vp, ip, ip, vp, vp]),
        "elas_op_prolong_add": (ip, [vp, ip, ip, vp, vp]),
        "elas_op_rhs": (ip, [vp, vp]),
        "elas_op_bottom": (ip, [vp, ip, vp, vp]),
        "elas_batch_solve": (ip, [C.POINTER(vp), ip, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
        "elas_profile_enable": (ip, [vp, ip]),
        "elas_amr_create": (ip, [C.POINTER(vp), C.POINTER(AmrLevelDesc), ip, C.POINTER(vp)]),
        "elas_server_create": (ip, [vp, ip, C.POINTER(vp)]),
        "elas_autotune": (ip, [vp, C.POINTER(C.c_float), ip]),
        "elas_autotune_dump": (ip, [C.c_char_p, ip]),
        "elas_autotune_load": (ip, [C.c_char_p]),
        "elas_server_destroy": (ip, [vp]),
        "elas_server_submit": (ip, [vp, vp, C.POINTER(SolveOpts), C.POINTER(C.c_longlong)]),
        "elas_server_submit_amr": (ip, [vp, vp, C.POINTER(SolveOpts), C.POINTER(C.c_longlong)]),
        "elas_server_step": (ip, [vp, C.POINTER(ip), C.POINTER(ip)]),
        "elas_server_poll": (ip, [vp, C.c_longlong, C.POINTER(SolveInfo), dp]),
        "elas_amr_destroy": (ip, [vp]),
        "elas_amr_set_reading": (ip, [vp, ip]),
        "elas_amr_solve": (ip, [vp, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
        "elas_profile_read": (ip, [vp, ip, dp, C.POINTER(C.c_longlong)]),
        "elas_launch_count": (C.c_ulonglong, []),
        "elas_measure_fma_peak": (ip, [ip, ip, dp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


PROF_SWEEP64_L0, PROF_SWEEP32_L0, PROF_RESID64_L0, PROF_RESID32_L0 = 0, 1, 2, 3


def launch_count():
    return int(lib().elas_launch_count())


def measure_fma_peak(device=0, precision=FP64):
    """Measured FMA throughput of the device in TFLOP/s (FP64 or FP32 chains)."""
    t = C.c_double()
    rc = lib().elas_measure_fma_peak(device, precision, C.byref(t))
    if rc != OK:
        raise ElasError(rc, "FMA peak measurement failed")
    return t.value


def exported_symbols():
    return [n for n in dir(lib()) if n.startswith("elas_")]


def check_field(name, a, dims, dtype, device):
    """Check a device field argument of a single operation before its pointer goes to the
    library, whose kernels address 3 x nx x ny x nz elements of it (dims = (nx, ny, nz),
    the level's nodes) unchecked: a contiguous CUDA tensor on `device`, of element type
    `dtype` (None: the library refuses the operation before reading it) and of that size."""
    import torch
    if not isinstance(a, torch.Tensor) or not a.is_cuda or a.get_device() != device:
        raise ValueError(f"{name}: a CUDA tensor on device {device} is required")
    if dtype is not None and a.dtype != dtype:
        raise ValueError(f"{name}: dtype {a.dtype}, the operation takes {dtype}")
    if not a.is_contiguous():
        raise ValueError(f"{name}: a contiguous tensor is required")
    nx, ny, nz = dims
    if a.numel() != 3 * nx * ny * nz:
        raise ValueError(f"{name}: {a.numel()} elements, the level holds 3 x {nx} x {ny} x {nz}")
    return a


def check_buffer(name, a, count, device):
    """Check a tensor the library copies `count` doubles from or into (host or device
    memory, by pointer and count alone): a contiguous float64 tensor of exactly that size,
    on `device` when it is a CUDA tensor."""
    import torch
    if not isinstance(a, torch.Tensor):
        raise ValueError(f"{name}: a torch tensor is required")
    if a.is_cuda and a.get_device() != device:
        raise ValueError(f"{name}: the tensor is on device {a.get_device()}, the context on {device}")
    if a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != count:
        raise ValueError(f"{name}: a contiguous float64 tensor of {count} elements is required "
                         f"({a.dtype}, {a.numel()} elements)")
    return a


def op_dtype(precision, output=False):
    """Element type of a single operation's fields: FP64, FP32 (MIXED), or for OP_DF FP64
    inputs and an FP32 output; None for a precision the library refuses."""
    import torch
    if precision == FP64:
        return torch.float64
    if precision == MIXED:
        return torch.float32
    if precision == OP_DF:
        return torch.float32 if output else torch.float64
    return None


def _ptr(a):
    """Device pointer of a torch tensor, or host pointer of a C-contiguous numpy array."""
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


class Context:
    """A solver context on one CUDA device with a torch-owned stream and allocator."""

    def __init__(self, device=0, budget_bytes=0, stream=None, torch_allocator=True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the solver has no CPU path")
        self.torch = torch
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        self._keep = []
        alloc_p = None
        if torch_allocator:
            dev = device
            strm = self.stream

            def _alloc(nbytes, user, stream):
                try:
                    return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, strm))
                except Exception:
                    return 0

            def _free(ptr, nbytes, user, stream):
                try:
                    torch.cuda.caching_allocator_delete(int(ptr))
                except Exception:
                    pass

            cb = Allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
            self._keep += [cb, _alloc, _free]
            alloc_p = C.pointer(cb)
        h = C.c_void_p()
        rc = lib().elas_ctx_create(C.byref(h), device, budget_bytes, alloc_p, C.c_void_p(self.stream.cuda_stream))
        if rc != OK:
            raise ElasError(rc, "context creation failed")
        self.h = h

    def error(self):
        return lib().elas_last_error(self.h).decode()

    def after_current(self, *tensors):
        """Order the context's stream after torch's current stream when any argument is
        a device tensor: inputs are usually produced by asynchronous kernels on the
        current stream, and the library reads them on its own stream."""
        if any(getattr(t, "is_cuda", False) for t in tensors):
            self.stream.wait_stream(self.torch.cuda.current_stream(self.device))

    def check(self, rc):
        if rc not in (OK,):
            raise ElasError(rc, self.error())

    def profile(self, enable=True):
        self.check(lib().elas_profile_enable(self.h, int(enable)))

    def profile_read(self, cls):
        ms, n = C.c_double(), C.c_longlong()
        self.check(lib().elas_profile_read(self.h, cls, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def bytes_in_use(self):
        return lib().elas_ctx_bytes_in_use(self.h)

    def close(self):
        """Destroy the context (its servers first: the library refuses while one is alive)."""
        if getattr(self, "h", None):
            self.check(lib().elas_ctx_destroy(self.h))
            self.h = None


def desc_for(problem: M.Problem, mixed=False, max_levels=0, half_moduli=False):
    d = GridDesc()
    d.max_levels = int(max_levels)
    d.half_moduli = int(bool(half_moduli))
    for k in range(3):
        d.n[k] = int(problem.n[k])
        d.periodic[k] = int(bool(problem.periodic[k]))
        d.lo[k] = float(problem.lo[k])
        d.hi[k] = float(problem.hi[k])
    d.moduli_kind = int(problem.moduli_kind)
    d.mixed = int(bool(mixed))
    return d


class Grid:
    """One node grid with its multigrid hierarchy."""

    def __init__(self, ctx: Context, desc: GridDesc):
        self.ctx = ctx
        self.desc = desc
        h = C.c_void_p()
        ctx.check(lib().elas_grid_create(ctx.h, C.byref(desc), C.byref(h)))
        self.h = h
        self.n = tuple(desc.n)
        self.N = self.n[0] * self.n[1] * self.n[2]
        self.shape = (self.n[2], self.n[1], self.n[0])

    # -- inputs ------------------------------------------------------------------
    def _host(self, a, count):
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.size != count:
            raise ValueError(f"expected {count} values, got {a.size}")
        return a

    def set_moduli(self, comps):
        a = self._host(comps, self.desc.moduli_kind * self.N)
        self.ctx.check(lib().elas_set_moduli(self.h, _ptr(a), HOST))

    def set_moduli_from(self, tensor):
        """Moduli from a torch tensor: pinned host memory or device memory."""
        check_buffer("moduli", tensor, self.desc.moduli_kind * self.N, self.ctx.device)
        self.ctx.after_current(tensor)
        space = DEVICE if tensor.is_cuda else HOST
        self.ctx.check(lib().elas_set_moduli(self.h, _ptr(tensor), space))

    def displacement_into(self, tensor):
        """Copy the displacement into a torch tensor (pinned host or device)."""
        check_buffer("displacement", tensor, 3 * self.N, self.ctx.device)
        self.ctx.after_current(tensor)
        space = DEVICE if tensor.is_cuda else HOST
        self.ctx.check(lib().elas_get_displacement(self.h, _ptr(tensor), space))
        return tensor

    def set_eigenstrain(self, eps6):
        if eps6 is None:
            self.ctx.check(lib().elas_set_eigenstrain(self.h, None, HOST))
            return
        a = self._host(eps6, 6 * self.N)
        self.ctx.check(lib().elas_set_eigenstrain(self.h, _ptr(a), HOST))

    def set_body_force(self, b3):
        if b3 is None:
            self.ctx.check(lib().elas_set_body_force(self.h, None, HOST))
            return
        a = self._host(b3, 3 * self.N)
        self.ctx.check(lib().elas_set_body_force(self.h, _ptr(a), HOST))

    def set_mean_strain(self, eps6):
        a = (C.c_double * 6)(*[float(v) for v in eps6])
        self.ctx.check(lib().elas_set_mean_strain(self.h, a))

    def set_bc(self, face, comp, kind, value=0.0):
        self.ctx.check(lib().elas_set_bc(self.h, face, comp, kind, float(value)))

    def set_face_values(self, face, values):
        if values is None:
            self.ctx.check(lib().elas_set_face_values(self.h, face, None, HOST))
            return
        a = self._host(values, 3 * self.N)
        self.ctx.check(lib().elas_set_face_values(self.h, face, _ptr(a), HOST))

    # -- solve -------------------------------------------------------------------
    def solve(self, precision=FP64, rel_tol=1e-8, max_cycles=100, nu1=2, nu2=2, warm_start=False,
              fixed_cycles=0, use_graph=False, raise_on_error=True, inner_cycles=1, smoother=None, cycle=None,
              omega=None, outer=None):
        o = _opts(precision, rel_tol, max_cycles, nu1, nu2, warm_start, fixed_cycles, use_graph, inner_cycles,
                  smoother, cycle, omega, outer)
        info = SolveInfo()
        rc = lib().elas_solve(self.h, C.byref(o), C.byref(info))
        if rc != OK and raise_on_error and rc not in (ERR_NOT_CONVERGED,):
            raise ElasError(rc, self.ctx.error())
        return info.as_dict()

    def displacement(self):
        out = np.empty((3,) + self.shape)
        self.ctx.check(lib().elas_get_displacement(self.h, _ptr(out), HOST))
        return out

    def set_displacement(self, u):
        a = self._host(u, 3 * self.N)
        self.ctx.check(lib().elas_set_displacement(self.h, _ptr(a), HOST))

    def stress(self):
        """Stress of the current displacement, (6, nz, ny, nx): 11, 22, 33, 23, 31, 12."""
        out = np.empty((6,) + self.shape)
        self.ctx.check(lib().elas_get_stress(self.h, _ptr(out), HOST))
        return out

    def query_residual(self):
        rel, ab = C.c_double(), C.c_double()
        self.ctx.check(lib().elas_query_residual(self.h, C.byref(rel), C.byref(ab)))
        return rel.value, ab.value

    def query_residual_inf(self):
        """Max norm of the FP64 residual: (||r||_inf / ||r_0||_inf, ||r||_inf)."""
        rel, ab = C.c_double(), C.c_double()
        self.ctx.check(lib().elas_query_residual_inf(self.h, C.byref(rel), C.byref(ab)))
        return rel.value, ab.value

    def levels(self):
        n = C.c_int()
        self.ctx.check(lib().elas_grid_levels(self.h, C.byref(n)))
        return n.value

    def level_dims(self, level):
        a = (C.c_int * 3)()
        self.ctx.check(lib().elas_grid_level_dims(self.h, level, a))
        return tuple(a)

    def bytes(self):
        return lib().elas_grid_bytes(self.h)

    # -- single operations (device tensors) -------------------------------------------
    def _sync(self):
        self.ctx.stream.synchronize()

    def _field(self, name, a, level, dtype):
        return check_field(name, a, self.level_dims(level), dtype, self.ctx.device)

    def _dtype(self, precision, output=False):
        return op_dtype(precision, output)

    def op_apply(self, level, precision, u):
        self._field("u", u, level, self._dtype(precision))
        out = self.ctx.torch.empty_like(u)
        self.ctx.after_current(u, out)
        self.ctx.check(lib().elas_op_apply(self.h, level, precision, _ptr(u), _ptr(out)))
        return out

    def op_residual(self, level, precision, u, f):
        """r = f - A u and sum r^2; precision OP_DF: double-float from FP64 u, f, r in FP32."""
        T = self.ctx.torch
        self._field("u", u, level, self._dtype(precision))
        self._field("f", f, level, self._dtype(precision))
        r = T.empty_like(u, dtype=T.float32) if precision == OP_DF else T.empty_like(u)
        self.ctx.after_current(u, f, r)
        ss = C.c_double()
        self.ctx.check(lib().elas_op_residual(self.h, level, precision, _ptr(u), _ptr(f), _ptr(r), C.byref(ss)))
        return r, ss.value

    def op_residual_noalloc(self, level, precision, u, f, r):
        """elas_op_residual without any allocation: the caller passes the output r;
        the reduction uses the library's static device scratch."""
        self._field("u", u, level, self._dtype(precision))
        self._field("f", f, level, self._dtype(precision))
        self._field("r", r, level, self._dtype(precision, output=True))
        ss = C.c_double()
        self.ctx.after_current(u, f, r)
        self.ctx.check(lib().elas_op_residual_noalloc(self.h, level, precision, _ptr(u), _ptr(f), _ptr(r),
                                                      C.byref(ss)))
        return ss.value

    def op_sweep(self, level, precision, u, f):
        self._field("u", u, level, self._dtype(precision))
        self._field("f", f, level, self._dtype(precision))
        self.ctx.after_current(u, f)
        self.ctx.check(lib().elas_op_sweep(self.h, level, precision, _ptr(u), _ptr(f)))
        return u

    def op_smooth(self, level, precision, smoother, u, f, omega=2.0 / 3.0):
        """One sweep of the given smoother (SMOOTH_RB, SMOOTH_GS8, SMOOTH_JACOBI), in place."""
        self._field("u", u, level, self._dtype(precision))
        self._field("f", f, level, self._dtype(precision))
        self.ctx.after_current(u, f)
        self.ctx.check(lib().elas_op_smooth(self.h, level, precision, smoother, omega, _ptr(u), _ptr(f)))
        return u

    def op_restrict(self, level, precision, r):
        self._field("r", r, level, self._dtype(precision))
        nc = self.level_dims(level + 1)
        fc = self.ctx.torch.empty((3, nc[2], nc[1], nc[0]), dtype=r.dtype, device=r.device)
        self.ctx.after_current(r, fc)
        self.ctx.check(lib().elas_op_restrict(self.h, level, precision, _ptr(r), _ptr(fc)))
        return fc

    def op_prolong_add(self, level, precision, ec, u):
        self._field("ec", ec, level + 1, self._dtype(precision))
        self._field("u", u, level, self._dtype(precision))
        self.ctx.after_current(ec, u)
        self.ctx.check(lib().elas_op_prolong_add(self.h, level, precision, _ptr(ec), _ptr(u)))
        return u

    def op_rhs(self):
        f = self.ctx.torch.empty((3,) + self.shape, dtype=self.ctx.torch.float64, device=f"cuda:{self.ctx.device}")
        self.ctx.after_current(f)
        self.ctx.check(lib().elas_op_rhs(self.h, _ptr(f)))
        return f

    def op_bottom(self, precision, f):
        self._field("f", f, self.levels() - 1, self._dtype(precision))
        u = self.ctx.torch.empty_like(f)
        self.ctx.after_current(f, u)
        self.ctx.check(lib().elas_op_bottom(self.h, precision, _ptr(f), _ptr(u)))
        return u

    def autotune(self):
        """Pick the fastest smoother launch shape per level; returns the finest
        level's FP32 timings (ms) per shape, -1 for a shape that does not apply."""
        t = (C.c_float * NUM_SWEEP_VARIANTS)()
        self.ctx.check(lib().elas_autotune(self.h, t, NUM_SWEEP_VARIANTS))
        return list(t)

    def close(self):
        """Destroy the grid; refused (ElasError, the grid stays usable) while a server holds a
        request on it or an AMR layout holds it as a level."""
        if getattr(self, "h", None):
            self.ctx.check(lib().elas_grid_destroy(self.h))
            self.h = None


# interior smoother launch shapes: 0-4 untiled (threads, min blocks per SM) = (256,1),
# (256,2), (256,3), (256,4), (128,8); 5-6 shared-memory tiled, 32x16 and 32x8 tiles
# (blocked FP32 moduli); 7-8 z-marching tiled with staged displacement, 32x16 and 32x8
# tiles (colour-split FP32 moduli).
# Levels with FP16 moduli use shapes 1 and 2 only (the others report -1 when tuned).
NUM_SWEEP_VARIANTS = 9
UNTILED_VARIANTS = tuple(range(5))
TILED_VARIANTS = (5, 6)
SPLIT_TILED_VARIANTS = (7, 8)


def autotune_dump():
    n = lib().elas_autotune_dump(None, 0)
    buf = C.create_string_buffer(n + 1)
    lib().elas_autotune_dump(buf, n + 1)
    return buf.value.decode()


def autotune_load(text):
    return lib().elas_autotune_load(text.encode())


def grid_from_problem(ctx: Context, p: M.Problem, mixed=False, max_levels=0, half_moduli=False) -> Grid:
    """Create a grid and load a Problem's moduli, loads and boundary conditions."""
    g = Grid(ctx, desc_for(p, mixed, max_levels, half_moduli))
    g.set_moduli(p.moduli)
    if p.eigenstrain is not None:
        g.set_eigenstrain(p.eigenstrain)
    if p.body_force is not None:
        g.set_body_force(p.body_force)
    if p.mean_strain is not None:
        g.set_mean_strain(p.mean_strain)
    for f in range(6):
        if p.periodic[f // 2]:
            continue
        for c in range(3):
            kind, val = p.bc[f][c]
            g.set_bc(f, c, kind, val)
    faces = dict(p.face_values or {})
    if p.dirichlet_values is not None:
        for f in range(6):
            if p.periodic[f // 2]:
                continue
            if any(p.bc[f][c][0] == M.DIRICHLET for c in range(3)):
                base = faces.get(f)
                arr = np.empty((3,) + g.shape)
                for c in range(3):
                    if p.bc[f][c][0] == M.DIRICHLET:
                        arr[c] = p.dirichlet_values[c]
                    elif base is not None:
                        arr[c] = base[c]
                    else:
                        arr[c] = p.bc[f][c][1]
                faces[f] = arr
    for f, arr in faces.items():
        g.set_face_values(f, arr)
    return g


def _opts(precision=FP64, rel_tol=1e-8, max_cycles=100, nu1=2, nu2=2, warm_start=False, fixed_cycles=0,
          use_graph=False, inner_cycles=1, smoother=None, cycle=None, omega=None, outer=None):
    o = SolveOpts()
    lib().elas_solve_opts_default(C.byref(o))
    o.precision, o.rel_tol, o.max_cycles = precision, rel_tol, max_cycles
    o.nu1, o.nu2, o.warm_start, o.fixed_cycles = nu1, nu2, int(warm_start), fixed_cycles
    o.use_graph = int(use_graph)
    o.inner_cycles = int(inner_cycles)
    if smoother is not None:
        o.smoother = int(smoother)
    if cycle is not None:
        o.cycle = int(cycle)
    if omega is not None:
        o.omega = float(omega)
    if outer is not None:
        o.outer_residual = int(outer)
    return o


class Amr:
    """Composite (reflux-free) AMR solve over the levels of an AMR layout
    (``microstructure.AmrLevel`` list): one grid per level, level 0 with its
    multigrid hierarchy, finer levels smoothed only."""

    def __init__(self, ctx: Context, specs, reading="R1", mixed=False):
        self.ctx = ctx
        self.specs = specs
        self.grids = [grid_from_problem(ctx, sp.problem, mixed=mixed, max_levels=0 if sp.level == 0 else 1)
                      for sp in specs]
        descs = (AmrLevelDesc * len(specs))()
        for i, sp in enumerate(specs):
            for d in range(3):
                descs[i].grid_lo[d] = sp.grid_lo[d]
                descs[i].valid_lo[d] = sp.valid_lo[d]
                descs[i].valid_hi[d] = sp.valid_hi[d]
            for f in range(6):
                descs[i].ghost[f] = int(sp.ghost[f])
        arr = (C.c_void_p * len(specs))(*[g.h for g in self.grids])
        h = C.c_void_p()
        try:
            ctx.check(lib().elas_amr_create(arr, descs, len(specs), C.byref(h)))
        except Exception:
            for g in self.grids:
                g.close()
            raise
        self.h = h
        try:
            ctx.check(lib().elas_amr_set_reading(self.h, {"R1": 1, "R2": 2}[reading]))
        except Exception:
            self.close()          # a refused reading leaves no layout or grids behind
            raise

    def solve(self, rel_tol=1e-8, max_cycles=200, nu1=2, nu2=2, fixed_cycles=0, raise_on_error=True,
              precision=FP64):
        info = SolveInfo()
        rc = lib().elas_amr_solve(self.h, C.byref(_opts(precision, rel_tol, max_cycles, nu1, nu2, False, fixed_cycles)),
                                  C.byref(info))
        if rc != OK and raise_on_error and rc != ERR_NOT_CONVERGED:
            raise ElasError(rc, self.ctx.error())
        return info.as_dict()

    def displacements(self):
        return [g.displacement() for g in self.grids]

    def close(self):
        """Destroy the layout, then its level grids; refused (ElasError) while a server holds
        a request on it."""
        if getattr(self, "h", None):
            self.ctx.check(lib().elas_amr_destroy(self.h))
            self.h = None
        for g in self.grids:
            g.close()


def batch_solve(grids, precision=MIXED, rel_tol=1e-8, max_cycles=100, nu1=2, nu2=2, warm_start=False,
                fixed_cycles=0, raise_on_error=True, inner_cycles=1, cycle=None, outer=None):
    """Solve every grid of one context together: one launch per phase of the cycle covers
    every member (grids of one moduli kind and layout; otherwise the members' own launches
    run as parallel branches), a captured CUDA graph replays refinement steps, and members
    stop on their own tolerance.  Returns one info dict per grid."""
    if not grids:
        return []
    n = len(grids)
    arr = (C.c_void_p * n)(*[g.h for g in grids])
    infos = (SolveInfo * n)()
    o = _opts(precision, rel_tol, max_cycles, nu1, nu2, warm_start, fixed_cycles, False, inner_cycles, None, cycle,
              None, outer)
    rc = lib().elas_batch_solve(arr, n, C.byref(o), infos)
    if rc != OK and raise_on_error and rc != ERR_NOT_CONVERGED:
        raise ElasError(rc, grids[0].ctx.error())
    return [infos[i].as_dict() for i in range(n)]


class Server:
    """Continuous-batching step engine of the C library (see elas_server_* in elas.h)."""

    def __init__(self, ctx: Context, max_active=16):
        self.ctx = ctx
        h = C.c_void_p()
        ctx.check(lib().elas_server_create(ctx.h, max_active, C.byref(h)))
        self.h = h

    def submit(self, grid: Grid, **kw):
        t = C.c_longlong()
        self.ctx.check(lib().elas_server_submit(self.h, grid.h, C.byref(_opts(MIXED, **kw)), C.byref(t)))
        return t.value

    def submit_amr(self, amr, precision=FP64, **kw):
        """A composite AMR solve (an ``Amr``) as a request: one composite cycle per step
        (MIXED: an FP32 correction cycle on the FP64 composite residual)."""
        t = C.c_longlong()
        self.ctx.check(lib().elas_server_submit_amr(self.h, amr.h, C.byref(_opts(precision, **kw)), C.byref(t)))
        return t.value

    def step(self):
        a, w = C.c_int(), C.c_int()
        self.ctx.check(lib().elas_server_step(self.h, C.byref(a), C.byref(w)))
        return a.value, w.value

    def poll(self, ticket):
        info = SolveInfo()
        lat = C.c_double()
        rc = lib().elas_server_poll(self.h, ticket, C.byref(info), C.byref(lat))
        if rc < 0:
            raise ElasError(rc, self.ctx.error())
        return (info.as_dict(), lat.value) if rc == 1 else None

    def close(self):
        if getattr(self, "h", None):
            lib().elas_server_destroy(self.h)
            self.h = None
