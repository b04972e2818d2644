"""ctypes marshalling for the C ABI of include/lexgb.h (no computation here)."""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

OK, E_INVAL, E_NOMEM, E_CUDA, E_NOCONV, E_NONFINITE, E_TIMEOUT, E_CALLBACK = range(8)
STATUS = {0: "LX_OK", 1: "LX_E_INVAL", 2: "LX_E_NOMEM", 3: "LX_E_CUDA", 4: "LX_E_NOCONV", 5: "LX_E_NONFINITE",
          6: "LX_E_TIMEOUT", 7: "LX_E_CALLBACK"}
ADVDIFF, BURGERS = 0, 1
ADVDIFF_UP3, BURGERS_UP3 = 2, 3  # the paper's discretisation: periodic [-1,1)^2, third-order upwind gradient
FP64, MIXED, DF64 = 0, 1, 2
ROS_EU, EXPRB32, EPIRK4S3A = 0, 1, 2

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_vp = C.c_void_p


class LxProblem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nu", C.c_double), ("a", C.c_double), ("kind", C.c_int),
                ("precision", C.c_int)]


class LxStats(C.Structure):
    _fields_ = [("loop_ms", C.c_double), ("loop_iterations", C.c_longlong), ("loop_launches", C.c_longlong),
                ("power_ms", C.c_double), ("kernels", C.c_longlong)]


class LxIntegrateInfo(C.Structure):
    _fields_ = [("t", C.c_double), ("h", C.c_double), ("steps", C.c_int), ("rejected", C.c_int),
                ("leja_iters", C.c_longlong), ("last_err", C.c_double), ("power_iters", C.c_int)]


class LxRhsStats(C.Structure):
    _fields_ = [("leja_iterations", C.c_longlong), ("rhs_calls", C.c_longlong), ("kernels", C.c_longlong)]


# lx_rhs_fn: int f(const double* in, double* out, void* user, void* stream)
RHS_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p)


class LexgbError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)} {lx_status_str(status)} {_cuda_err()}")


_lib = None
_lock = threading.Lock()


def lib():
    """Load _lexgb.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not _build.up_to_date():
                if os.environ.get("LEXGB_NO_BUILD"):
                    raise RuntimeError(f"{path} is missing or stale and LEXGB_NO_BUILD is set")
                _build.build()
            L = C.CDLL(path)
            L.lx_status_str.restype = C.c_char_p
            L.lx_status_str.argtypes = [C.c_int]
            L.lx_last_cuda_error.restype = C.c_char_p
            L.lx_leja_points.argtypes = [C.c_int, _dp]
            L.lx_leja_coeffs.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, _dp, C.c_int, _dp]
            L.lx_leja_coeff_count.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int]
            L.lx_leja_coeff_count.restype = C.c_int
            L.lx_spectral_interval.argtypes = [C.c_double, _dp, _dp]
            L.leja_setup.argtypes = [C.POINTER(LxProblem), C.c_int, C.c_int, _vp, C.POINTER(_vp)]
            L.leja_destroy.argtypes = [_vp]
            L.leja_destroy.restype = None
            L.power_bound.argtypes = [_vp, _vp, _vp, C.c_int, _dp, _ip]
            L.phi_l_apply.argtypes = [_vp, C.c_int, _vp, _vp, _vp, C.c_double, C.c_double, C.c_double, C.c_double,
                                      C.c_double, _ip]
            L.phi_l_apply_vertical.argtypes = [_vp, C.c_int, C.c_int, _dp, _vp, _vp, C.POINTER(C.c_void_p),
                                               C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, _ip]
            L.expint_step.argtypes = [_vp, _vp, _vp, _vp, C.c_double, C.c_double, C.c_double, C.c_double,
                                      C.c_double, _dp, _ip]
            L.expint_step_host.argtypes = [_vp, _vp, _vp, _vp, C.c_double, C.c_double, C.c_double, C.c_double,
                                           C.c_double, _dp, _ip]
            L.lx_ctx_stats.argtypes = [_vp, C.POINTER(LxStats), C.c_int]
            L.lx_ctx_kernel_name.argtypes = [_vp, C.c_char_p, C.c_int]
            L.lx_ctx_set_loop_mode.argtypes = [_vp, C.c_int]
            L.lx_ctx_set_graph_unroll.argtypes = [_vp, C.c_int]
            L.lx_ctx_set_source.argtypes = [_vp, _vp]
            L.lx_controller_classical.restype = C.c_double
            L.lx_controller_classical.argtypes = [C.c_double, C.c_double, C.c_double]
            L.lx_integrate.argtypes = [_vp, _vp, _vp, C.c_double, C.c_double, C.c_double, C.c_int,
                                       C.POINTER(LxIntegrateInfo)]
            L.batch_setup.argtypes = [C.c_int, C.POINTER(LxProblem), C.c_int, _vp, C.POINTER(_vp)]
            L.batch_step.argtypes = [_vp, C.c_int, C.POINTER(_vp), C.POINTER(_vp), _dp, _dp, _dp, C.c_double,
                                     C.c_double, _ip, _ip]
            L.batch_stats.argtypes = [_vp, C.POINTER(LxStats), C.c_int]
            L.batch_destroy.argtypes = [_vp]
            L.batch_destroy.restype = None
            _fp = C.POINTER(C.c_float)
            L.mlp_param_count.restype = C.c_int
            L.mlp_setup.argtypes = [C.c_int, _fp, _fp, _vp, C.POINTER(_vp)]
            L.mlp_get_weights.argtypes = [_vp, _fp]
            L.mlp_forward.argtypes = [_vp, _vp, _vp, C.c_int]
            L.mlp_forward_host.argtypes = [_vp, _fp, _fp, C.c_int]
            L.mlp_train_step.argtypes = [_vp, _vp, _vp, C.c_int, C.c_int, C.c_float, _fp, _fp]
            L.mlp_destroy.argtypes = [_vp]
            L.mlp_destroy.restype = None
            L.lx_integrate_learned.argtypes = [_vp, _vp, _vp, C.c_double, C.c_double, C.c_double, C.c_int, _vp,
                                               C.c_double, C.POINTER(LxIntegrateInfo)]
            L.lx_ctx_autotune.argtypes = [_vp, C.c_int, C.c_char_p, C.c_char_p, C.c_int]
            L.lx_ctx_select_kernel.argtypes = [_vp, C.c_char_p, C.c_int]
            L.lx_ctx_iters_per_launch.argtypes = [_vp]
            L.lx_ctx_iters_per_launch.restype = C.c_int
            L.phi_l_apply_noalloc.argtypes = [C.POINTER(LxProblem), C.c_int, _vp, _vp, C.c_double, C.c_double,
                                              C.c_double, C.c_double, C.c_double, _vp, _ip]
            L.lx_rhs_builtin.argtypes = [_vp, _vp, _vp, _vp]
            L.lx_rhs_builtin.restype = C.c_int
            L.leja_setup_rhs.argtypes = [C.c_longlong, _vp, _vp, C.c_double, C.c_int, C.c_int, _vp, C.POINTER(_vp)]
            L.leja_destroy_rhs.argtypes = [_vp]
            L.leja_destroy_rhs.restype = None
            L.power_bound_rhs.argtypes = [_vp, _vp, _vp, C.c_int, _dp, _ip]
            L.phi_l_apply_rhs.argtypes = [_vp, C.c_int, _vp, _vp, _vp, C.c_double, C.c_double, C.c_double,
                                          C.c_double, C.c_double, _ip]
            L.expint_step_rhs.argtypes = [_vp, _vp, _vp, _vp, C.c_double, C.c_double, C.c_double, C.c_double,
                                          C.c_double, _dp, _ip]
            L.lx_rhs_ctx_stats.argtypes = [_vp, C.POINTER(LxRhsStats), C.c_int]
            _lib = L
    return _lib


def _cuda_err():
    try:
        return lib().lx_last_cuda_error().decode()
    except Exception:  # pragma: no cover
        return ""


def lx_status_str(status: int) -> str:
    return lib().lx_status_str(int(status)).decode()


def _dev(t):
    """Device address of a torch CUDA float64 contiguous tensor, or an int."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _host(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):  # torch CPU tensor (e.g. pinned)
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("expected a contiguous CPU tensor")
        return a.data_ptr()
    if not (isinstance(a, np.ndarray) and a.flags.c_contiguous and a.dtype == np.float64):
        raise ValueError("expected a C-contiguous float64 numpy array")
    return a.ctypes.data


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ host numerics
def lx_leja_points(K: int) -> np.ndarray:
    xi = np.zeros(K)
    st = lib().lx_leja_points(K, xi.ctypes.data_as(_dp))
    if st != OK:
        raise LexgbError(st, "lx_leja_points")
    return xi


def lx_leja_coeffs(l: int, h: float, c: float, gamma: float, xi) -> np.ndarray:
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    d = np.zeros_like(xi)
    st = lib().lx_leja_coeffs(l, h, c, gamma, xi.ctypes.data_as(_dp), len(xi), d.ctypes.data_as(_dp))
    if st != OK:
        raise LexgbError(st, "lx_leja_coeffs")
    return d


def lx_leja_coeff_count(h: float, c: float, gamma: float, K: int) -> int:
    return lib().lx_leja_coeff_count(h, c, gamma, K)


def spectral_interval(rho: float):
    """(c, gamma) of the focal interval for a spectral-radius estimate, from
    lx_spectral_interval."""
    c, g = C.c_double(0.0), C.c_double(0.0)
    st = lib().lx_spectral_interval(float(rho), C.byref(c), C.byref(g))
    if st != OK:
        raise LexgbError(st, "lx_spectral_interval")
    return c.value, g.value


# ------------------------------------------------------------------ context
class Context:
    """Owns an lx_ctx*; leja_destroy runs on close() or garbage collection."""

    def __init__(self, handle, problem, integrator):
        self.handle = handle
        self.problem = problem
        self.integrator = integrator

    @property
    def n(self):
        return self.problem.nx * self.problem.ny

    def close(self):
        if self.handle:
            lib().leja_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def leja_setup(nx, ny, nu, a=0.0, kind=ADVDIFF, precision=FP64, integrator=ROS_EU, max_leja=1000,
               stream=None) -> Context:
    prob = LxProblem(nx, ny, nu, a, kind, precision)
    h = _vp()
    st = lib().leja_setup(C.byref(prob), integrator, max_leja, _stream_handle(stream), C.byref(h))
    if st != OK:
        raise LexgbError(st, "leja_setup")
    return Context(h.value, prob, integrator)


def leja_destroy(ctx: Context):
    ctx.close()


def power_bound(ctx: Context, u, v0, max_iters=10):
    """Returns (status, rho, passes)."""
    rho = C.c_double(0.0)
    it = C.c_int(0)
    st = lib().power_bound(ctx.handle, _dev(u), _dev(v0), max_iters, C.byref(rho), C.byref(it))
    return st, rho.value, it.value


def phi_l_apply(ctx: Context, l, u, w, out, c, gamma, h, rtol, atol):
    """Returns (status, iters)."""
    it = C.c_int(0)
    st = lib().phi_l_apply(ctx.handle, l, _dev(u), _dev(w), _dev(out), c, gamma, h, rtol, atol, C.byref(it))
    return st, it.value


def phi_l_apply_vertical(ctx: Context, l, alphas, u, w, outs, c, gamma, h, rtol, atol):
    """phi_l(alpha_j h J) w into outs[j] for every alpha_j, one Newton basis.
    Returns (status, iters)."""
    al = np.ascontiguousarray(alphas, dtype=np.float64)
    if len(outs) != al.size:
        raise ValueError("one output per alpha")
    ptrs = (C.c_void_p * al.size)(*[_dev(o) for o in outs])
    it = C.c_int(0)
    st = lib().phi_l_apply_vertical(ctx.handle, l, al.size, al.ctypes.data_as(_dp), _dev(u), _dev(w), ptrs, c,
                                    gamma, h, rtol, atol, C.byref(it))
    return st, it.value


def expint_step(ctx: Context, u, u_low, u_high, c, gamma, h, rtol, atol):
    """Returns (status, err, iters)."""
    err = C.c_double(0.0)
    it = C.c_int(0)
    st = lib().expint_step(ctx.handle, _dev(u), _dev(u_low), _dev(u_high), c, gamma, h, rtol, atol,
                           C.byref(err), C.byref(it))
    return st, err.value, it.value


def expint_step_host(ctx: Context, u, u_low, u_high, c, gamma, h, rtol, atol):
    """Host-buffer step (numpy float64 arrays or pinned CPU tensors).  Returns (status, err, iters)."""
    err = C.c_double(0.0)
    it = C.c_int(0)
    st = lib().expint_step_host(ctx.handle, _host(u), _host(u_low), _host(u_high), c, gamma, h, rtol, atol,
                                C.byref(err), C.byref(it))
    return st, err.value, it.value


def lx_ctx_stats(ctx: Context, reset=False) -> dict:
    s = LxStats()
    st = lib().lx_ctx_stats(ctx.handle, C.byref(s), 1 if reset else 0)
    if st != OK:
        raise LexgbError(st, "lx_ctx_stats")
    return {"loop_ms": s.loop_ms, "loop_iterations": s.loop_iterations, "loop_launches": s.loop_launches,
            "power_ms": s.power_ms, "kernels": s.kernels}


def lx_ctx_kernel_name(ctx: Context) -> str:
    buf = C.create_string_buffer(128)
    lib().lx_ctx_kernel_name(ctx.handle, buf, 128)
    return buf.value.decode()


def lx_ctx_set_loop_mode(ctx: Context, stream_loop: int) -> int:
    return lib().lx_ctx_set_loop_mode(ctx.handle, int(stream_loop))


def lx_ctx_set_graph_unroll(ctx: Context, unroll: int) -> int:
    return lib().lx_ctx_set_graph_unroll(ctx.handle, int(unroll))


def lx_ctx_set_source(ctx: Context, source) -> int:
    """Borrow a CUDA float64 tensor of nx*ny values as the source S (None
    removes it); the context keeps a reference so the tensor stays alive."""
    if source is None:
        ctx._source = None
        return lib().lx_ctx_set_source(ctx.handle, None)
    if hasattr(source, "numel") and source.numel() != ctx.n:
        raise ValueError("source must have nx*ny values")
    ctx._source = source
    return lib().lx_ctx_set_source(ctx.handle, _dev(source))


def phi_l_apply_noalloc(nx, ny, nu, a, l, w, out, c, gamma, h, rtol, atol, stream=None):
    """Allocation-free phi_l(hA)w (diffusion-advection, FP64).  Returns (status, iters)."""
    prob = LxProblem(nx, ny, nu, a, ADVDIFF, FP64)
    it = C.c_int(0)
    st = lib().phi_l_apply_noalloc(C.byref(prob), l, _dev(w), _dev(out), c, gamma, h, rtol, atol,
                                   _stream_handle(stream), C.byref(it))
    return st, it.value


def lx_ctx_autotune(ctx: Context, iters=10, cache_path=None):
    """Returns (status, report dict)."""
    import json

    buf = C.create_string_buffer(16384)
    st = lib().lx_ctx_autotune(ctx.handle, iters, cache_path.encode() if cache_path else None, buf, 16384)
    rep = json.loads(buf.value.decode()) if st == OK and buf.value else {}
    return st, rep


def lx_ctx_select_kernel(ctx: Context, name: str, strip_h: int) -> int:
    return lib().lx_ctx_select_kernel(ctx.handle, name.encode(), strip_h)


def lx_ctx_iters_per_launch(ctx: Context) -> int:
    return int(lib().lx_ctx_iters_per_launch(ctx.handle))


def lx_controller_classical(h, err, tol) -> float:
    return lib().lx_controller_classical(h, err, tol)


def lx_integrate(ctx: Context, u, v0, t_final, tol, leja_tol, max_attempts=100000, t0=0.0, h0=None,
                 power_iters=10):
    """Adaptive EXPRB32 run updating u in place.  Returns (status, info dict)."""
    info = LxIntegrateInfo(t0, h0, 0, 0, 0, 0.0, power_iters)
    st = lib().lx_integrate(ctx.handle, _dev(u), _dev(v0), t_final, tol, leja_tol, max_attempts, C.byref(info))
    return st, {"t": info.t, "h": info.h, "steps": info.steps, "rejected": info.rejected,
                "leja_iters": info.leja_iters, "last_err": info.last_err}


class Batch:
    """Owns an lx_batch*."""

    def __init__(self, handle, problems):
        self.handle = handle
        self.problems = problems

    @property
    def count(self):
        return len(self.problems)

    def close(self):
        if self.handle:
            lib().batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_setup(problems, max_leja=1000, stream=None, precision=FP64) -> Batch:
    """problems: list of (nx, ny, nu, a); precision FP64 or DF64 (every nx % 128 == 0)."""
    arr = (LxProblem * len(problems))(*[LxProblem(nx, ny, nu, a, ADVDIFF, precision)
                                        for (nx, ny, nu, a) in problems])
    h = _vp()
    st = lib().batch_setup(len(problems), arr, max_leja, _stream_handle(stream), C.byref(h))
    if st != OK:
        raise LexgbError(st, "batch_setup")
    return Batch(h.value, list(problems))


def batch_step(b: Batch, l, ws, outs, c, gamma, h, rtol, atol):
    """Returns (status, iters[list], statuses[list])."""
    B = b.count
    wp = (_vp * B)(*[_dev(x) for x in ws])
    op = (_vp * B)(*[_dev(x) for x in outs])
    ca = np.ascontiguousarray(c, dtype=np.float64)
    ga = np.ascontiguousarray(gamma, dtype=np.float64)
    ha = np.ascontiguousarray(h, dtype=np.float64)
    its = (C.c_int * B)()
    sts = (C.c_int * B)()
    st = lib().batch_step(b.handle, l, wp, op, ca.ctypes.data_as(_dp), ga.ctypes.data_as(_dp),
                          ha.ctypes.data_as(_dp), rtol, atol, its, sts)
    return st, list(its), list(sts)


def batch_stats(b: Batch, reset=False) -> dict:
    s = LxStats()
    lib().batch_stats(b.handle, C.byref(s), 1 if reset else 0)
    return {"loop_ms": s.loop_ms, "loop_iterations": s.loop_iterations, "loop_launches": s.loop_launches}


class Mlp:
    """Owns an lx_mlp*."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            lib().mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def mlp_param_count() -> int:
    return lib().mlp_param_count()


def mlp_setup(batch_max, w, norm, stream=None) -> Mlp:
    w, norm = _f32(w), _f32(norm)
    h = _vp()
    fp = C.POINTER(C.c_float)
    st = lib().mlp_setup(batch_max, w.ctypes.data_as(fp), norm.ctypes.data_as(fp), _stream_handle(stream),
                         C.byref(h))
    if st != OK:
        raise LexgbError(st, "mlp_setup")
    return Mlp(h.value)


def mlp_get_weights(m: Mlp) -> np.ndarray:
    w = np.zeros(mlp_param_count(), dtype=np.float32)
    st = lib().mlp_get_weights(m.handle, w.ctypes.data_as(C.POINTER(C.c_float)))
    if st != OK:
        raise LexgbError(st, "mlp_get_weights")
    return w


def mlp_forward(m: Mlp, x, y, B) -> int:
    """x, y: CUDA float32 tensors [B,5], [B,2]."""
    return lib().mlp_forward(m.handle, _dev(x), _dev(y), B)


def mlp_forward_host(m: Mlp, x) -> np.ndarray:
    x = _f32(x)
    B = x.shape[0]
    y = np.zeros((B, 2), dtype=np.float32)
    fp = C.POINTER(C.c_float)
    st = lib().mlp_forward_host(m.handle, x.ctypes.data_as(fp), y.ctypes.data_as(fp), B)
    if st != OK:
        raise LexgbError(st, "mlp_forward_host")
    return y


def mlp_train_step(m: Mlp, x, t, B, adam=True, lr=1e-3, want_grad=False):
    """Returns (status, loss, grad or None)."""
    fp = C.POINTER(C.c_float)
    g = np.zeros(mlp_param_count(), dtype=np.float32) if want_grad else None
    loss = C.c_float(0.0)
    st = lib().mlp_train_step(m.handle, _dev(x), _dev(t), B, 1 if adam else 0, lr,
                              g.ctypes.data_as(fp) if g is not None else None, C.byref(loss))
    return st, float(loss.value), g


def lx_integrate_learned(ctx: Context, u, v0, t_final, tol, leja_tol, model: "Mlp", dt_ref, max_attempts=100000,
                         t0=0.0, h0=None, power_iters=10):
    """Adaptive EXPRB32 run with the learned controller.  Returns (status, info dict)."""
    info = LxIntegrateInfo(t0, h0, 0, 0, 0, 0.0, power_iters)
    st = lib().lx_integrate_learned(ctx.handle, _dev(u), _dev(v0), t_final, tol, leja_tol, max_attempts,
                                    model.handle, dt_ref, C.byref(info))
    return st, {"t": info.t, "h": info.h, "steps": info.steps, "rejected": info.rejected,
                "leja_iters": info.leja_iters, "last_err": info.last_err}


# ------------------------------------------------------------------ unfused form (caller's right-hand side)
class _DevRange:
    """n doubles at a device address, described by __cuda_array_interface__
    so that torch can view them without a copy."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False), "version": 2,
                                         "strides": None}


def rhs_function(f, n):
    """Wrap a Python right-hand side f(x, out) -- x, out: torch CUDA float64
    views of n values (no copy); f writes f(x) into out with torch operations
    -- as an lx_rhs_fn.  It runs on the stream the engine passes.  An
    exception inside f is printed and reported to the engine as an error."""
    import sys
    import traceback

    import torch

    views = {}  # the engine passes a few fixed buffers; callers' vectors may vary

    def view(ptr):
        t = views.get(ptr)
        if t is None:
            if len(views) >= 32:
                views.clear()
            t = torch.as_tensor(_DevRange(ptr, n), device="cuda")
            views[ptr] = t
        return t

    def cb(inp, out, _user, stream):
        try:
            s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(s):
                f(view(inp), view(out))
            return 0
        except Exception:  # reported to the engine as LX_E_CALLBACK
            traceback.print_exc(file=sys.stderr)
            return 1

    return RHS_FN(cb)


class RhsContext:
    """Owns an lx_rhs_ctx* and keeps its right-hand side alive."""

    def __init__(self, handle, n, integrator, keep):
        self.handle = handle
        self.n = n
        self.integrator = integrator
        self._keep = keep

    def close(self):
        if self.handle:
            lib().leja_destroy_rhs(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def leja_setup_rhs(n, f=None, problem=None, eps0=0.0, integrator=ROS_EU, max_leja=1000, stream=None) -> RhsContext:
    """f: a Python f(x, out) (see rhs_function), or None with problem =
    (nx, ny, nu, a, kind) for the engine's own right-hand side
    (lx_rhs_builtin)."""
    if f is None:
        if problem is None:
            raise ValueError("need f or problem")
        nx, ny, nu, a, kind = problem
        prob = LxProblem(nx, ny, nu, a, kind, FP64)
        keep = (prob,)
        fn = C.cast(lib().lx_rhs_builtin, _vp).value
        user = C.addressof(prob)
    else:
        cb = rhs_function(f, n)
        keep = (cb,)
        fn = C.cast(cb, _vp).value
        user = None
    h = _vp()
    st = lib().leja_setup_rhs(n, fn, user, eps0, integrator, max_leja, _stream_handle(stream), C.byref(h))
    if st != OK:
        raise LexgbError(st, "leja_setup_rhs")
    return RhsContext(h.value, n, integrator, keep)


def leja_destroy_rhs(ctx: RhsContext):
    ctx.close()


def lx_rhs_builtin(problem, x, out, stream=None) -> int:
    """The engine's own f(x) into out for problem = (nx, ny, nu, a, kind)."""
    nx, ny, nu, a, kind = problem
    prob = LxProblem(nx, ny, nu, a, kind, FP64)
    return lib().lx_rhs_builtin(_dev(x), _dev(out), C.addressof(prob), _stream_handle(stream))


def power_bound_rhs(ctx: RhsContext, u, v0, max_iters=10):
    """Returns (status, rho, passes)."""
    rho = C.c_double(0.0)
    it = C.c_int(0)
    st = lib().power_bound_rhs(ctx.handle, _dev(u), _dev(v0), max_iters, C.byref(rho), C.byref(it))
    return st, rho.value, it.value


def phi_l_apply_rhs(ctx: RhsContext, l, u, w, out, c, gamma, h, rtol, atol):
    """Returns (status, iters)."""
    it = C.c_int(0)
    st = lib().phi_l_apply_rhs(ctx.handle, l, _dev(u), _dev(w), _dev(out), c, gamma, h, rtol, atol, C.byref(it))
    return st, it.value


def expint_step_rhs(ctx: RhsContext, u, u_low, u_high, c, gamma, h, rtol, atol):
    """Returns (status, err, iters)."""
    err = C.c_double(0.0)
    it = C.c_int(0)
    st = lib().expint_step_rhs(ctx.handle, _dev(u), _dev(u_low), _dev(u_high), c, gamma, h, rtol, atol,
                               C.byref(err), C.byref(it))
    return st, err.value, it.value


def lx_rhs_ctx_stats(ctx: RhsContext, reset=False) -> dict:
    s = LxRhsStats()
    st = lib().lx_rhs_ctx_stats(ctx.handle, C.byref(s), 1 if reset else 0)
    if st != OK:
        raise LexgbError(st, "lx_rhs_ctx_stats")
    return {"leja_iterations": s.leja_iterations, "rhs_calls": s.rhs_calls, "kernels": s.kernels}
