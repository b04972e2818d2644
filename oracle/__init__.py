"""Python access to the CPU oracle (oracle.c) through ctypes.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use this module; the product never imports it.

Every function takes and returns numpy float64 arrays and follows the passage
of arXiv 2310.08344 named in oracle.c.  Status codes: 0 ok, 1 invalid
argument, 2 out of memory, 4 no convergence within the point table,
5 non-finite value.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

OK, E_INVAL, E_NOMEM, E_NOCONV, E_NONFINITE = 0, 1, 2, 4, 5
ADVDIFF, BURGERS = 0, 1
# the paper's discretisation (periodic [-1,1]^2, third-order upwind gradient)
ADVDIFF_UP3, BURGERS_UP3 = 2, 3

_lib = None
_lib_omp = None
_lock = threading.Lock()
_leja_cache: dict[int, np.ndarray] = {}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
# a caller's right-hand side f(in, out, user) over n doubles (Sec. 2)
_RHS = C.CFUNCTYPE(None, _dp, _dp, C.c_void_p)


def _p(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def lib(parallel: bool = False):
    """The parity build (single-threaded), or with parallel=True the OpenMP
    build of the same source, which only times the CPU baseline."""
    global _lib, _lib_omp
    with _lock:
        if parallel:
            if _lib_omp is None:
                _lib_omp = _declare(C.CDLL(_build.build(openmp=True)))
            return _lib_omp
        if _lib is None:
            _lib = _declare(C.CDLL(_build.build()))
    return _lib


def threads(parallel: bool = False) -> int:
    """Threads the grid loops of that build use."""
    return lib(parallel).or_threads()


def _declare(L):
    """Declare the argument and result types of the exported functions."""
    L.or_threads.restype = C.c_int
    L.or_phi.restype = C.c_double
    L.or_phi.argtypes = [C.c_int, C.c_double]
    L.or_qreal_mant_dig.restype = C.c_int
    L.or_leja_points.argtypes = [C.c_int, _dp]
    L.or_divdiff_values.argtypes = [C.c_int, _dp, _dp, _dp]
    L.or_leja_coeffs.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, _dp, C.c_int, _dp]
    L.or_apply_advdiff.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp]
    L.or_burgers_f.argtypes = [C.c_int, C.c_int, C.c_double, _dp, _dp]
    L.or_burgers_J.argtypes = [C.c_int, C.c_int, C.c_double, _dp, _dp, _dp]
    L.or_apply_advdiff_up3.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp]
    L.or_burgers_up3_f.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp]
    L.or_burgers_up3_J.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp, _dp]
    L.or_power_iteration.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp,
                                     C.c_int, _dp, _ip]
    L.or_leja_phi.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _dp, C.c_int, _dp,
                              C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, _dp, C.c_int,
                              _dp, _ip]
    L.or_ros_eu.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _dp, C.c_double,
                            C.c_double, C.c_double, C.c_double, C.c_double, _dp, C.c_int, _dp, _ip]
    L.or_exprb32.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _dp, C.c_double,
                             C.c_double, C.c_double, C.c_double, C.c_double, _dp, C.c_int, _dp, _dp,
                             _dp, _ip]
    L.or_leja_phi_given.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp, C.c_double,
                                    C.c_double, C.c_double, C.c_double, _dp, _dp, C.c_int, _dp, _ip, _dp,
                                    C.c_int]
    L.or_leja_phi_vertical.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _dp, C.c_int,
                                       C.c_int, _dp, _dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                       C.c_double, _dp, C.c_int, _dp, _ip]
    L.or_ros_eu_src.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp,
                                C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, _dp, C.c_int,
                                _dp, _ip]
    L.or_exprb32_src.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp,
                                 C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, _dp, C.c_int,
                                 _dp, _dp, _dp, _ip]
    L.or_epirk4s3a_src.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp, C.c_double,
                                   C.c_double, C.c_double, C.c_double, C.c_double, _dp, C.c_int, _dp, _dp, _dp, _ip]
    L.or_controller.restype = C.c_double
    L.or_controller.argtypes = [C.c_double, C.c_double, C.c_double]
    L.or_integrate_exprb32.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp,
                                       C.c_double, C.c_double, C.c_double, C.c_double, _dp, C.c_int,
                                       C.c_int, _ip, _ip, C.POINTER(C.c_longlong), _dp, _dp]
    L.or_integrate_exprb32_log.argtypes = L.or_integrate_exprb32.argtypes + [_dp, C.c_int]
    L.or_fd_jv.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _RHS, C.c_void_p, C.c_double,
                           _dp, _dp, _dp]
    L.or_power_iteration_fd.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _RHS,
                                        C.c_void_p, C.c_double, _dp, _dp, C.c_int, _dp, _ip]
    L.or_leja_phi_fd.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _RHS, C.c_void_p,
                                 C.c_double, _dp, C.c_int, _dp, C.c_double, C.c_double, C.c_double,
                                 C.c_double, C.c_double, _dp, C.c_int, _dp, _ip]
    L.or_ros_eu_fd.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _RHS, C.c_void_p,
                               C.c_double, _dp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                               _dp, C.c_int, _dp, _ip]
    L.or_exprb32_fd.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _RHS, C.c_void_p,
                                C.c_double, _dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                C.c_double, _dp, C.c_int, _dp, _dp, _dp, _ip]
    return L


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def qreal_mant_dig() -> int:
    return lib().or_qreal_mant_dig()


def phi(l: int, z: float) -> float:
    """phi_l(z), evaluated in binary128 and rounded to double."""
    return lib().or_phi(l, z)


GOLDEN_LEJA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                           "leja_points_oracle_1000.txt")


def leja_points(K: int) -> np.ndarray:
    """The first K greedy Leja points on [-2, 2].

    Computed by the oracle (an exhaustive search over all node intervals);
    K <= 1000 is served from the table that tests/golden/make_golden.py wrote
    with this same oracle, so that the O(K^3) search runs once.
    """
    if K in _leja_cache:
        return _leja_cache[K].copy()
    if K <= 1000 and os.path.exists(GOLDEN_LEJA):
        tab = np.loadtxt(GOLDEN_LEJA, dtype=np.float64)
        if tab.shape[0] >= K:
            _leja_cache[K] = tab[:K].copy()
            return tab[:K].copy()
    return leja_points_compute(K)


def leja_points_compute(K: int) -> np.ndarray:
    """Run the oracle's greedy Leja search (slow for K in the hundreds)."""
    xi = np.zeros(K)
    st = lib().or_leja_points(K, _p(xi))
    if st != OK:
        raise RuntimeError(f"or_leja_points status {st}")
    _leja_cache[K] = xi.copy()
    return xi


def divdiff_values(x, f) -> np.ndarray:
    x, f = _f64(x), _f64(f)
    d = np.zeros_like(x)
    st = lib().or_divdiff_values(len(x), _p(x), _p(f), _p(d))
    if st != OK:
        raise RuntimeError(f"or_divdiff_values status {st}")
    return d


def leja_coeffs(l: int, h: float, c: float, gamma: float, xi) -> np.ndarray:
    xi = _f64(xi)
    d = np.zeros_like(xi)
    st = lib().or_leja_coeffs(l, h, c, gamma, _p(xi), len(xi), _p(d))
    if st != OK:
        raise RuntimeError(f"or_leja_coeffs status {st}")
    return d


def apply_advdiff(nx, ny, nu, a, v) -> np.ndarray:
    v = _f64(v)
    out = np.zeros_like(v)
    lib().or_apply_advdiff(nx, ny, nu, a, _p(v), _p(out))
    return out


def apply_advdiff_up3(nx, ny, nu, a, v) -> np.ndarray:
    """nu (v_xx + v_yy) + a (v_x + v_y) on periodic [-1,1]^2, upwind gradient."""
    v = _f64(v)
    out = np.zeros_like(v)
    lib().or_apply_advdiff_up3(nx, ny, nu, a, _p(v), _p(out))
    return out


def burgers_up3_f(nx, ny, nu, a, u) -> np.ndarray:
    """nu (u_xx + u_yy) + (a/2) ((u^2)_x + (u^2)_y) on periodic [-1,1]^2."""
    u = _f64(u)
    out = np.zeros_like(u)
    lib().or_burgers_up3_f(nx, ny, nu, a, _p(u), _p(out))
    return out


def burgers_up3_J(nx, ny, nu, a, u, v) -> np.ndarray:
    u = _f64(u)
    v = _f64(v)
    out = np.zeros_like(v)
    lib().or_burgers_up3_J(nx, ny, nu, a, _p(u), _p(v), _p(out))
    return out


def burgers_f(nx, ny, nu, u) -> np.ndarray:
    u = _f64(u)
    out = np.zeros_like(u)
    lib().or_burgers_f(nx, ny, nu, _p(u), _p(out))
    return out


def burgers_J(nx, ny, nu, u, v) -> np.ndarray:
    u, v = _f64(u), _f64(v)
    out = np.zeros_like(u)
    lib().or_burgers_J(nx, ny, nu, _p(u), _p(v), _p(out))
    return out


def power_iteration(kind, nx, ny, nu, a, u, v0, max_iters=10, parallel=False):
    v0 = _f64(v0)
    u = _f64(u) if u is not None else None
    rho = np.zeros(1)
    it = C.c_int(0)
    st = lib(parallel).or_power_iteration(kind, nx, ny, nu, a, _p(u), _p(v0), max_iters, _p(rho), C.byref(it))
    return float(rho[0]), int(it.value), st


def leja_phi(kind, nx, ny, nu, a, u, l, w, c, gamma, h, rtol, atol, xi):
    w = _f64(w)
    xi = _f64(xi)
    u = _f64(u) if u is not None else None
    out = np.zeros_like(w)
    it = C.c_int(0)
    st = lib().or_leja_phi(kind, nx, ny, nu, a, _p(u), l, _p(w), c, gamma, h, rtol, atol, _p(xi), len(xi),
                           _p(out), C.byref(it))
    return out, int(it.value), st


# ---------------------------------------------------------------------------
# Divided differences above binary128 (mpmath).  The Newton coefficients of
# phi_l(h (c + gamma xi)) at the Leja points, by the same plain recursion
# d_j <- (d_j - d_k)/(xi_j - xi_k) (Sec. 2.1, Eq. 2), carried out with
# `dps` decimal digits.  Where the spectrum is far from the real focal
# interval (advection-dominated grids) the Newton basis grows like 4^m, and
# binary128's absolute rounding floor (about 1e-34 of the largest value)
# times that growth stops the series from converging; the recursion itself
# is unchanged, only its working precision is raised.
# ---------------------------------------------------------------------------


def _phi_mp(mp, l, z):
    """phi_l(z) at the working precision: the power series sum z^k/(k+l)!
    for |z| < 1, else the recursion phi_{l+1} = (phi_l - 1/l!)/z from exp."""
    if abs(z) < 1:
        term = mp.mpf(1) / mp.factorial(l)
        total = term
        tiny = mp.mpf(10) ** (-mp.dps - 5)
        k = 1
        while True:
            term = term * z / (k + l)
            total += term
            if abs(term) <= tiny * abs(total):
                break
            k += 1
        return total
    phi = mp.exp(z)
    inv_fact = mp.mpf(1)
    for k in range(l):
        phi = (phi - inv_fact) / z
        inv_fact = inv_fact / (k + 1)
    return phi


def dd_digits(K: int) -> int:
    """Working digits for K coefficients: the basis may grow by up to 4 per
    iteration (log10 4 = 0.6 digits), plus 40 digits of headroom."""
    return 40 + int(0.7 * K)


def _divdiff_rows(d, x):
    """In place: d_j <- (d_j - d_k)/(x_j - x_k) for k < j, row by row."""
    for j in range(1, len(d)):
        dj, xj = d[j], x[j]
        for k in range(j):
            dj = (dj - d[k]) / (xj - x[k])
        d[j] = dj
    return d


def divdiff_values_mp(x, f, dps: int = 60) -> np.ndarray:
    """Divided differences of the values f (doubles, taken exactly) at the
    nodes x with dps digits, rounded to double."""
    import mpmath

    with mpmath.workdps(dps):
        mp = mpmath.mp
        xs = [mp.mpf(float(v)) for v in _f64(x)]
        d = [mp.mpf(float(v)) for v in _f64(f)]
        return np.array([float(v) for v in _divdiff_rows(d, xs)])


def leja_coeffs_mp(l: int, h: float, c: float, gamma: float, xi, dps: int | None = None) -> np.ndarray:
    """d_j = f[xi_0..xi_j], f(xi) = phi_l(h (c + gamma xi)), with dps digits
    (default dd_digits(len(xi))), rounded to double at the end."""
    import mpmath

    xi = _f64(xi)
    K = len(xi)
    with mpmath.workdps(dps or dd_digits(K)):
        mp = mpmath.mp
        H, Cc, G = mp.mpf(float(h)), mp.mpf(float(c)), mp.mpf(float(gamma))
        x = [mp.mpf(float(v)) for v in xi]
        d = [_phi_mp(mp, l, H * (Cc + G * xj)) for xj in x]
        return np.array([float(v) for v in _divdiff_rows(d, x)])


def leja_phi_mp(kind, nx, ny, nu, a, u, l, w, c, gamma, h, rtol, atol, xi, dps=None, k0=128, want_growth=False,
                regroup=False):
    """leja_phi with the Newton coefficients from leja_coeffs_mp.  Row j of
    the recursion needs only rows < j, so the coefficients are formed for
    the first k0 points and the table is doubled (up to len(xi)) while the
    loop runs out of coefficients; a run that stops inside a shorter table
    is the run with the full one.  Returns (out, iters, status), plus with
    want_growth the basis growth max_m ||y_m|| / ||y_0||.  regroup: the
    diffusion-advection operator evaluated per neighbour (another rounding
    order of the same operator, see rounding_sensitivity)."""
    w = _f64(w)
    xi = _f64(xi)
    u = _f64(u) if u is not None else None
    out = np.zeros_like(w)
    it = C.c_int(0)
    growth = np.zeros(1)
    K = min(k0, len(xi))
    while True:
        d = leja_coeffs_mp(l, h, c, gamma, xi[:K], dps)
        st = lib().or_leja_phi_given(kind, nx, ny, nu, a, _p(u), _p(w), c, gamma, rtol, atol, _p(xi), _p(d), K,
                                     _p(out), C.byref(it), _p(growth), 1 if regroup else 0)
        if st != E_NOCONV or K >= len(xi):
            if want_growth:
                return out, int(it.value), st, float(growth[0])
            return out, int(it.value), st
        K = min(2 * K, len(xi))


def rounding_sensitivity(nx, ny, nu, a, l, w, c, gamma, h, rtol, atol, xi, ref=None):
    """How far the diffusion-advection Leja result moves when the operator
    is evaluated in another order: the relative L2 difference of the runs
    with the stencil grouped per difference quotient (the oracle's own form)
    and per neighbour.  Both are exact evaluations of the same operator up
    to rounding, so no implementation of the method can be expected to agree
    with the oracle much more closely than this on the given problem.
    ref: the first run's result, if already computed."""
    if ref is None:
        ref, _, _ = leja_phi_mp(ADVDIFF, nx, ny, nu, a, None, l, w, c, gamma, h, rtol, atol, xi)
    alt, _, st = leja_phi_mp(ADVDIFF, nx, ny, nu, a, None, l, w, c, gamma, h, rtol, atol, xi, regroup=True)
    if st != OK:
        return float("inf")
    return float(np.linalg.norm(alt - ref) / np.linalg.norm(ref))


def leja_phi_vertical(kind, nx, ny, nu, a, u, l, alphas, w, c, gamma, h, rtol, atol, xi):
    """phi_l(alpha_j h Op) w for every alpha_j from one Newton basis; returns
    (outputs [nc, n], iters, status)."""
    w = _f64(w)
    xi = _f64(xi)
    al = _f64(alphas)
    u = _f64(u) if u is not None else None
    out = np.zeros((len(al), w.size))
    it = C.c_int(0)
    st = lib().or_leja_phi_vertical(kind, nx, ny, nu, a, _p(u), l, len(al), _p(al), _p(w), c, gamma, h, rtol, atol,
                                    _p(xi), len(xi), out.ctypes.data_as(_dp), C.byref(it))
    return out, int(it.value), st


def ros_eu(kind, nx, ny, nu, a, u, c, gamma, h, rtol, atol, xi, source=None, parallel=False):
    """Rosenbrock-Euler step; source: optional time-independent S added to f;
    parallel: the OpenMP build (CPU-baseline timing only)."""
    u = _f64(u)
    xi = _f64(xi)
    S = _f64(source) if source is not None else None
    out = np.zeros_like(u)
    it = C.c_int(0)
    st = lib(parallel).or_ros_eu_src(kind, nx, ny, nu, a, _p(u), _p(S) if S is not None else None, c, gamma, h, rtol, atol,
                             _p(xi), len(xi), _p(out), C.byref(it))
    return out, int(it.value), st


def exprb32(kind, nx, ny, nu, a, u, c, gamma, h, rtol, atol, xi, source=None):
    u = _f64(u)
    xi = _f64(xi)
    S = _f64(source) if source is not None else None
    lo = np.zeros_like(u)
    hi = np.zeros_like(u)
    err = np.zeros(1)
    it = C.c_int(0)
    st = lib().or_exprb32_src(kind, nx, ny, nu, a, _p(u), _p(S) if S is not None else None, c, gamma, h, rtol,
                              atol, _p(xi), len(xi), _p(lo), _p(hi), _p(err), C.byref(it))
    return lo, hi, float(err[0]), int(it.value), st


def epirk4s3a(kind, nx, ny, nu, a, u, c, gamma, h, rtol, atol, xi, source=None):
    """EPIRK4s3A step: returns (u3 embedded third order, u4 fourth order,
    err = ||u4 - u3||, Leja iterations of the vertical phi_1 loop and the
    phi_3, phi_4 loops, status)."""
    u = _f64(u)
    xi = _f64(xi)
    S = _f64(source) if source is not None else None
    lo = np.zeros_like(u)
    hi = np.zeros_like(u)
    err = np.zeros(1)
    it = C.c_int(0)
    st = lib().or_epirk4s3a_src(kind, nx, ny, nu, a, _p(u), _p(S) if S is not None else None, c, gamma, h, rtol,
                                atol, _p(xi), len(xi), _p(lo), _p(hi), _p(err), C.byref(it))
    return lo, hi, float(err[0]), int(it.value), st


def spectral_interval(rho: float):
    """c and gamma from a spectral-radius estimate: lambda = -1.05 rho,
    c = lambda/2, gamma = -lambda/4 (Sec. 2.2, Listing 7)."""
    lam = -1.05 * rho
    return lam / 2.0, -lam / 4.0


def controller(h, err, tol):
    return lib().or_controller(h, err, tol)


def integrate_exprb32(kind, nx, ny, nu, a, u0, v0, t_final, h0, tol, leja_tol, xi, max_attempts=1000,
                      want_log=False):
    """Adaptive EXPRB32 run; returns (u, steps, rejected, leja_iters, h_next, t, status), plus with
    want_log an array of attempts (t, step tried, error estimate, accepted)."""
    u = _f64(u0).copy()
    v0 = _f64(v0)
    xi = _f64(xi)
    steps, rej = C.c_int(0), C.c_int(0)
    its = C.c_longlong(0)
    h, t = np.zeros(1), np.zeros(1)
    log = np.full((max_attempts, 4), np.nan)
    st = lib().or_integrate_exprb32_log(kind, nx, ny, nu, a, _p(u), _p(v0), t_final, h0, tol, leja_tol, _p(xi),
                                        len(xi), max_attempts, C.byref(steps), C.byref(rej), C.byref(its), _p(h),
                                        _p(t), log.ctypes.data_as(_dp), max_attempts)
    res = (u, steps.value, rej.value, its.value, float(h[0]), float(t[0]), st)
    if want_log:
        return res + (log[:steps.value + rej.value].copy(),)
    return res


# ---------------------------------------------------------------------------
# The unfused form: Jacobian action by central finite differences of f
# (Sec. 2.3), f the kind's own (rhs=None) or a Python function of one float64
# array returning f(u) (Sec. 2's user right-hand side).
# ---------------------------------------------------------------------------

EPS0_FD = 2.0 ** -18  # default relative difference step, about the cube root of the unit roundoff


def _rhs_cb(rhs, n):
    if rhs is None:
        return _RHS()

    def cb(inp, out, _user):
        x = np.ctypeslib.as_array(inp, shape=(n,))
        y = np.ctypeslib.as_array(out, shape=(n,))
        y[:] = rhs(x.copy())

    return _RHS(cb)


def fd_jv(kind, nx, ny, nu, a, u, v, eps0=EPS0_FD, rhs=None):
    """J(u) v = [f(u + e v) - f(u - e v)] / (2 e), e = eps0 (1 + ||u||) / ||v||."""
    v = _f64(v)
    u = _f64(u) if u is not None else None
    out = np.zeros_like(v)
    cb = _rhs_cb(rhs, v.size)
    st = lib().or_fd_jv(kind, nx, ny, nu, a, cb, None, eps0, _p(u), _p(v), _p(out))
    if st != OK:
        raise RuntimeError(f"or_fd_jv status {st}")
    return out


def power_iteration_fd(kind, nx, ny, nu, a, u, v0, max_iters=10, eps0=EPS0_FD, rhs=None):
    v0 = _f64(v0)
    u = _f64(u) if u is not None else None
    rho = np.zeros(1)
    it = C.c_int(0)
    cb = _rhs_cb(rhs, v0.size)
    st = lib().or_power_iteration_fd(kind, nx, ny, nu, a, cb, None, eps0, _p(u), _p(v0), max_iters, _p(rho),
                                     C.byref(it))
    return float(rho[0]), int(it.value), st


def leja_phi_fd(kind, nx, ny, nu, a, u, l, w, c, gamma, h, rtol, atol, xi, eps0=EPS0_FD, rhs=None):
    w = _f64(w)
    xi = _f64(xi)
    u = _f64(u) if u is not None else None
    out = np.zeros_like(w)
    it = C.c_int(0)
    cb = _rhs_cb(rhs, w.size)
    st = lib().or_leja_phi_fd(kind, nx, ny, nu, a, cb, None, eps0, _p(u), l, _p(w), c, gamma, h, rtol, atol,
                              _p(xi), len(xi), _p(out), C.byref(it))
    return out, int(it.value), st


def ros_eu_fd(kind, nx, ny, nu, a, u, c, gamma, h, rtol, atol, xi, eps0=EPS0_FD, rhs=None):
    u = _f64(u)
    xi = _f64(xi)
    out = np.zeros_like(u)
    it = C.c_int(0)
    cb = _rhs_cb(rhs, u.size)
    st = lib().or_ros_eu_fd(kind, nx, ny, nu, a, cb, None, eps0, _p(u), c, gamma, h, rtol, atol, _p(xi), len(xi),
                            _p(out), C.byref(it))
    return out, int(it.value), st


def exprb32_fd(kind, nx, ny, nu, a, u, c, gamma, h, rtol, atol, xi, eps0=EPS0_FD, rhs=None):
    u = _f64(u)
    xi = _f64(xi)
    lo = np.zeros_like(u)
    hi = np.zeros_like(u)
    err = np.zeros(1)
    it = C.c_int(0)
    cb = _rhs_cb(rhs, u.size)
    st = lib().or_exprb32_fd(kind, nx, ny, nu, a, cb, None, eps0, _p(u), c, gamma, h, rtol, atol, _p(xi), len(xi),
                             _p(lo), _p(hi), _p(err), C.byref(it))
    return lo, hi, float(err[0]), int(it.value), st
