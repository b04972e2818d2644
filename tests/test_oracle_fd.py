"""Pins of the oracle's unfused form: the Jacobian action by finite
differences of the right-hand side (Sec. 2.3) and a caller's right-hand side
(Sec. 2).

Reading (the paper names finite differences without a formula): the central
quotient J(u)v = [f(u + e v) - f(u - e v)] / (2 e), e = eps0 (1 + ||u||) / ||v||.

References: the exact truncation term of the central quotient of a cubic
(which fixes both the quotient and the step rule), second-order convergence
on a non-polynomial f, exactness on quadratics against the analytic
linearisation (itself pinned by Fourier and dense checks), the exact affine
solution by Fourier, and the dense augmented-matrix exponential.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
import synth
from fourier import phi_apply_symbol, rel_l2, symbol

TOL = 1e-10


def rms(x):
    return float(np.sqrt(np.mean(x * x)))


def lap(n, v):
    """Central Laplacian on the periodic unit square (spacing 1/n), n x n."""
    V = v.reshape(n, n)
    L = (np.roll(V, 1, 0) + np.roll(V, -1, 0) + np.roll(V, 1, 1) + np.roll(V, -1, 1) - 4 * V) * n * n
    return L.reshape(-1)


@pytest.mark.parametrize("with_u", [True, False])
def test_fd_quotient_and_step_rule_on_a_cubic(with_u):
    # f(u) = u^3 point-wise: the central quotient is 3 u^2 v + e^2 v^3 exactly,
    # so the residual after removing 3 u^2 v fixes e = eps0 (1 + ||u||) / ||v||
    n = 12
    u = synth.random_field(n * n, seed=1) if with_u else None
    v = 3.0 * synth.random_field(n * n, seed=2)
    eps0 = 1e-2
    jv = oracle.fd_jv(0, n, n, 0.0, 0.0, u, v, eps0=eps0, rhs=lambda x: x**3)
    u0 = u if with_u else np.zeros(n * n)
    e = eps0 * (1.0 + rms(u0)) / rms(v)
    assert np.allclose(jv - 3 * u0**2 * v, e * e * v**3, rtol=1e-6, atol=1e-12)


def test_fd_is_second_order_on_a_smooth_f():
    # f(u) = nu Lap u + sin u: J(u)v = nu Lap v + cos(u) v; halving eps0
    # divides the error by ~4 (a one-sided quotient would give ~2)
    n, nu = 16, 0.01
    u = synth.gaussians_ic(n, n, seed=3)
    v = synth.random_field(n * n, seed=4)
    exact = nu * lap(n, v) + np.cos(u) * v
    errs = [rel_l2(oracle.fd_jv(0, n, n, 0, 0, u, v, eps0=e0, rhs=lambda x: nu * lap(n, x) + np.sin(x)), exact)
            for e0 in (4e-2, 2e-2, 1e-2)]
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4, errs


@pytest.mark.parametrize("kind", [oracle.BURGERS, oracle.BURGERS_UP3, oracle.ADVDIFF, oracle.ADVDIFF_UP3])
def test_fd_exact_on_quadratic_kinds(kind):
    # every problem kind's f is at most quadratic, so the central quotient is
    # the analytic linearisation up to rounding (amplified by 1/e)
    n, nu, a = 24, 0.05, 1.5
    u = synth.problem3_ic(n, n, seed=5)
    v = synth.random_field(n * n, seed=6)
    if kind == oracle.BURGERS:
        ref = oracle.burgers_J(n, n, nu, u, v)
    elif kind == oracle.BURGERS_UP3:
        ref = oracle.burgers_up3_J(n, n, nu, a, u, v)
    elif kind == oracle.ADVDIFF:
        ref = oracle.apply_advdiff(n, n, nu, a, v)
    else:
        ref = oracle.apply_advdiff_up3(n, n, nu, a, v)
    assert rel_l2(oracle.fd_jv(kind, n, n, nu, a, u, v, eps0=1e-2), ref) <= 1e-12
    assert rel_l2(oracle.fd_jv(kind, n, n, nu, a, u, v), ref) <= 1e-9  # default step: rounding / e


def test_fd_zero_vector_and_zero_input():
    n = 8
    u = synth.random_field(n * n, seed=7)
    assert np.all(oracle.fd_jv(oracle.BURGERS, n, n, 0.1, 0, u, np.zeros(n * n)) == 0.0)
    xi = oracle.leja_points(100)
    out, it, st = oracle.leja_phi_fd(oracle.BURGERS, n, n, 0.1, 0, u, 1, np.zeros(n * n), -10.0, 5.0, 0.1,
                                     TOL, TOL, xi)
    assert st == oracle.OK and it == 1 and np.all(out == 0.0)


def test_leja_phi_fd_smooth_f_matches_dense_expm():
    # non-polynomial f = nu Lap u - sin u on a small grid (J symmetric and
    # negative definite for 0 <= u <= 1): phi_1(h J(u)) w through the
    # augmented-matrix exponential of the analytic Jacobian; the FD form
    # carries the O(e^2) truncation and the rounding / e of the quotient
    n, nu = 10, 0.02
    N = n * n
    u = synth.gaussians_ic(n, n, seed=8)
    w = synth.random_field(N, seed=9)
    E = np.eye(N)
    J = np.stack([nu * lap(n, E[:, k]) for k in range(N)], axis=1) - np.diag(np.cos(u))
    rho = float(np.max(np.abs(np.linalg.eigvals(J))))
    c, g = oracle.spectral_interval(rho)
    h = 4.0 / rho * 10
    B = np.zeros((N + 1, N + 1))
    B[:N, :N] = h * J
    B[:N, N] = w
    ref = scipy.linalg.expm(B)[:N, N]  # phi_1(hJ) w
    xi = oracle.leja_points(1000)
    out, it, st = oracle.leja_phi_fd(0, n, n, 0, 0, u, 1, w, c, g, h, 1e-12, 1e-12, xi,
                                     rhs=lambda x: nu * lap(n, x) - np.sin(x))
    assert st == oracle.OK
    assert rel_l2(out, ref) <= 1e-8


def test_ros_eu_fd_affine_problem_is_exact():
    # f(u) = A u + S from a caller's function: the Rosenbrock-Euler step is
    # the exact solution u + h phi_1(hA)(A u + S), computed here by Fourier
    n, nu, a = 64, 0.01, 1.0  # diffusion-dominated: the spectrum hugs the real interval
    u = synth.gaussians_ic(n, n, seed=1)
    S = synth.source_field(n, n)
    lam = symbol(n, n, nu, a)
    c, g = oracle.spectral_interval(float(np.abs(lam).max()))
    h = 50 * synth.cfl_step(n, n, nu, a)
    xi = oracle.leja_points(1000)

    def f(x):
        return oracle.apply_advdiff(n, n, nu, a, x) + S

    out, it, st = oracle.ros_eu_fd(0, n, n, nu, a, u, c, g, h, TOL, TOL, xi, rhs=f)
    assert st == oracle.OK
    ref = u + h * phi_apply_symbol(1, lam, h, f(u), n, n)
    assert rel_l2(out, ref) <= 1e-8


@pytest.mark.parametrize("kind", [oracle.BURGERS, oracle.BURGERS_UP3])
def test_exprb32_and_power_fd_match_analytic_on_burgers(kind):
    # quadratic f: with a large step the quotient is exact, so every stage of
    # the unfused form reproduces the analytic-Jacobian integrator
    if kind == oracle.BURGERS:
        n, nu, a = 32, 0.01, 0.0
        u = synth.burgers_ic(n, n, seed=2)
        h = 20 * synth.cfl_step(n, n, nu, 1.0)
    else:  # the paper's Problem III coefficients
        n, nu, a = 32, 1.0, 10.0
        u = synth.problem3_ic(n, n, seed=2)
        h = 30 * synth.cfl_step_pm1(n, n, nu, a * np.abs(u).max())
    v0 = synth.power_start(n * n, 5)
    rho, pit, st = oracle.power_iteration(kind, n, n, nu, a, u, v0, 10)
    rho_fd, pit_fd, st_fd = oracle.power_iteration_fd(kind, n, n, nu, a, u, v0, 10, eps0=1e-2)
    assert st == st_fd == oracle.OK and pit == pit_fd and abs(rho - rho_fd) <= 1e-12 * rho
    c, g = oracle.spectral_interval(rho)
    xi = oracle.leja_points(1000)
    lo, hi, err, it, st = oracle.exprb32(kind, n, n, nu, a, u, c, g, h, TOL, TOL, xi)
    lo2, hi2, err2, it2, st2 = oracle.exprb32_fd(kind, n, n, nu, a, u, c, g, h, TOL, TOL, xi, eps0=1e-2)
    assert st == st2 == oracle.OK and abs(it - it2) <= 1
    assert rel_l2(lo2, lo) <= 1e-12 and rel_l2(hi2, hi) <= 1e-12
    assert abs(err2 - err) <= 1e-6 * err
