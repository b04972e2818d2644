"""Pins of the oracle's upwind discretisation (the paper's Sec. 3 problems on
periodic [-1,1)^2: second-order central Laplacian, third-order upwind
gradient) and of the Leja loop and integrators on it.

References: the order of accuracy on smooth functions (closed-form
derivatives), the Fourier symbol written out from the stencil, the exact
Fourier solution of the linear problem, the exactness of central
differences of a quadratic map, the quadratic remainder, and the dense
augmented-matrix exponential on a small grid.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
import synth
from fourier import phi_apply_symbol, rel_l2, symbol_up3

TOL = 1e-10


def _xy(n):
    return synth.grid_pm1(n, n)


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_upwind_gradient_is_third_order(sign):
    # D applied to sin(pi x) + cos(pi y): the error against the exact
    # derivative shrinks by ~2^3 per halving of the spacing
    errs = []
    for n in (32, 64, 128):
        X, Y = _xy(n)
        u = (np.sin(np.pi * X) + np.cos(np.pi * Y)).reshape(-1)
        exact = (np.pi * np.cos(np.pi * X) - np.pi * np.sin(np.pi * Y)).reshape(-1)
        g = oracle.apply_advdiff_up3(n, n, 0.0, sign, u) * sign
        errs.append(np.max(np.abs(g - exact)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 7.0 < r1 < 9.0 and 7.0 < r2 < 9.0, (errs, r1, r2)


def test_laplacian_is_second_order():
    errs = []
    for n in (32, 64, 128):
        X, Y = _xy(n)
        u = (np.sin(np.pi * X) * np.cos(2 * np.pi * Y)).reshape(-1)
        exact = (-5 * np.pi**2 * np.sin(np.pi * X) * np.cos(2 * np.pi * Y)).reshape(-1)
        errs.append(np.max(np.abs(oracle.apply_advdiff_up3(n, n, 1.0, 0.0, u) - exact)))
    assert 3.8 < errs[0] / errs[1] < 4.2 and 3.8 < errs[1] / errs[2] < 4.2


@pytest.mark.parametrize("a", [10.0, -3.0])
def test_upwind_operator_symbol(a):
    # the operator is diagonal in Fourier space with the symbol written out
    # from the stencil; the upwind part is dissipative (Re <= 0)
    nx, ny, nu = 48, 40, 1.0
    v = synth.random_field(nx * ny, seed=3)
    lam = symbol_up3(nx, ny, nu, a)
    ref = np.real(np.fft.ifft2(lam * np.fft.fft2(v.reshape(ny, nx)))).reshape(-1)
    assert rel_l2(oracle.apply_advdiff_up3(nx, ny, nu, a, v), ref) <= 1e-13
    assert np.all(lam.real <= 1e-9 * np.abs(lam).max())


@pytest.mark.parametrize("l", [0, 1, 3])
def test_leja_phi_upwind_matches_fourier(l):
    # the paper's Problem I coefficients (diffusion 1, advection 10) on 64^2
    n, nu, a = 64, 1.0, 10.0
    u0 = synth.problem1_ic(n, n)
    lam = symbol_up3(n, n, nu, a)
    c, g = oracle.spectral_interval(float(np.abs(lam).max()))
    h = 50 * synth.cfl_step_pm1(n, n, nu, a)
    xi = oracle.leja_points(1000)
    out, iters, st = oracle.leja_phi(oracle.ADVDIFF_UP3, n, n, nu, a, None, l, u0, c, g, h, TOL, TOL, xi)
    assert st == oracle.OK
    assert rel_l2(out, phi_apply_symbol(l, lam, h, u0, n, n)) <= 100 * TOL
    # and Rosenbrock-Euler is the exact exponential for the linear problem
    ue, _, st = oracle.ros_eu(oracle.ADVDIFF_UP3, n, n, nu, a, u0, c, g, h, TOL, TOL, xi)
    assert st == oracle.OK and rel_l2(ue, phi_apply_symbol(0, lam, h, u0, n, n)) <= 100 * TOL


def test_burgers_upwind_jacobian_is_the_derivative():
    # f is quadratic in u, so the central difference of f along v is J(u) v
    # exactly up to rounding; and f(u + p) - f(u) - J(u) p = (a/2) D(p^2)
    n, nu, a = 24, 1.0, 10.0
    u = synth.problem3_ic(n, n, seed=2)
    v = synth.random_field(n * n, seed=4)
    eps = 1e-3
    fd = (oracle.burgers_up3_f(n, n, nu, a, u + eps * v) - oracle.burgers_up3_f(n, n, nu, a, u - eps * v)) / (2 * eps)
    Jv = oracle.burgers_up3_J(n, n, nu, a, u, v)
    assert rel_l2(fd, Jv) <= 1e-9
    p = 0.1 * v
    rem = oracle.burgers_up3_f(n, n, nu, a, u + p) - oracle.burgers_up3_f(n, n, nu, a, u) - \
        oracle.burgers_up3_J(n, n, nu, a, u, p)
    quad = oracle.apply_advdiff_up3(n, n, 0.0, a / 2, p * p)
    assert rel_l2(rem, quad) <= 1e-9
    # the Laplacian and the flux difference are in conservation form: f has zero mean
    assert abs(oracle.burgers_up3_f(n, n, nu, a, u).mean()) <= 1e-10 * np.abs(u).max() * a * n


def test_leja_phi_burgers_upwind_dense():
    # 16^2 with a = 4 keeps the Jacobian's spectrum diffusion-dominated
    # (real Leja points need that regime)
    n, nu, a = 16, 1.0, 4.0
    u = synth.problem3_ic(n, n, seed=5)
    w = synth.random_field(n * n, seed=6)
    J = np.zeros((n * n, n * n))
    e = np.zeros(n * n)
    for k in range(n * n):
        e[:] = 0.0
        e[k] = 1.0
        J[:, k] = oracle.burgers_up3_J(n, n, nu, a, u, e)
    rho = float(np.max(np.abs(np.linalg.eigvals(J))))
    c, g = oracle.spectral_interval(rho)
    h = 20 * synth.cfl_step_pm1(n, n, nu, a * np.abs(u).max())
    xi = oracle.leja_points(1000)
    B = np.zeros((n * n + 1, n * n + 1))
    B[:-1, :-1] = h * J
    B[:-1, -1] = w
    ref = scipy.linalg.expm(B)[:-1, -1]  # phi_1(hJ) w (augmented-matrix identity)
    out, it, st = oracle.leja_phi(oracle.BURGERS_UP3, n, n, nu, a, u, 1, w, c, g, h, 1e-12, 1e-12, xi)
    assert st == oracle.OK
    assert rel_l2(out, ref) <= 1e-9
