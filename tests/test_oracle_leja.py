"""Pins of the oracle's Leja interpolation, power iteration and integrators.

References used: the exact Fourier solution of the periodic linear problem
(numpy FFT), the dense matrix exponential (scipy.linalg.expm) on grids of 16^2
or less with the augmented-matrix identity for phi_l, invariants that the
exact operator functions satisfy (linearity, semigroup, mean conservation),
and the integrators' convergence orders.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
import synth
from fourier import phi_apply, rel_l2, spectral_radius

TOL = 1e-10


def _cfg1(seed=1, n=64, nu=1e-2, a=1.0):
    u0 = synth.gaussians_ic(n, n, seed=seed)
    h = 50 * synth.cfl_step(n, n, nu, a)
    rho = spectral_radius(n, n, nu, a)
    c, gamma = oracle.spectral_interval(rho)
    return u0, h, c, gamma


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("l", [0, 1, 3])
def test_leja_phi_matches_fourier(seed, l):
    n, nu, a = 64, 1e-2, 1.0
    u0, h, c, gamma = _cfg1(seed)
    xi = oracle.leja_points(400)
    out, iters, st = oracle.leja_phi(oracle.ADVDIFF, n, n, nu, a, None, l, u0, c, gamma, h, TOL, TOL, xi)
    assert st == oracle.OK
    ref = phi_apply(l, n, n, nu, a, h, u0)
    err = rel_l2(out, ref)
    assert err <= 100 * TOL, err
    assert 20 <= iters <= 200


def _dense(apply, n_pts):
    M = np.zeros((n_pts, n_pts))
    e = np.zeros(n_pts)
    for k in range(n_pts):
        e[:] = 0.0
        e[k] = 1.0
        M[:, k] = apply(e)
    return M


def _phi_dense(M, v, l):
    # Saad (1992) / Sidje (EXPOKIT): for the augmented matrix
    # [[M, v, 0], [0, 0, I_{l-1}], [0, 0, 0]], the top block of
    # exp(.) e_{n+l} is phi_l(M) v.
    n = M.shape[0]
    if l == 0:
        return scipy.linalg.expm(M) @ v
    B = np.zeros((n + l, n + l))
    B[:n, :n] = M
    B[:n, n] = v
    for k in range(l - 1):
        B[n + k, n + k + 1] = 1.0
    E = scipy.linalg.expm(B)
    return E[:n, n + l - 1]


@pytest.mark.parametrize("l", [0, 1, 3])
def test_leja_phi_matches_dense_expm_advdiff(l):
    nx, ny, nu, a = 12, 10, 2e-2, 0.2  # diffusion-dominated: real focal interval
    v = synth.random_field(nx * ny, seed=4)
    h = 40 * synth.cfl_step(nx, ny, nu, a)
    A = _dense(lambda e: oracle.apply_advdiff(nx, ny, nu, a, e), nx * ny)
    rho = np.max(np.abs(np.linalg.eigvals(A)))
    c, gamma = oracle.spectral_interval(rho)
    xi = oracle.leja_points(400)
    out, iters, st = oracle.leja_phi(oracle.ADVDIFF, nx, ny, nu, a, None, l, v, c, gamma, h, TOL, TOL, xi)
    assert st == oracle.OK
    ref = _phi_dense(h * A, v, l)
    assert rel_l2(out, ref) <= 100 * TOL


@pytest.mark.parametrize("l", [1, 3])
def test_leja_phi_matches_dense_expm_burgers_jacobian(l):
    n, nu = 12, 5e-3
    u = synth.burgers_ic(n, n, seed=2)
    v = synth.random_field(n * n, seed=9)
    h = 30 * synth.cfl_step(n, n, nu, np.max(np.abs(u)))
    J = _dense(lambda e: oracle.burgers_J(n, n, nu, u, e), n * n)
    rho = np.max(np.abs(np.linalg.eigvals(J)))
    c, gamma = oracle.spectral_interval(rho)
    xi = oracle.leja_points(400)
    out, iters, st = oracle.leja_phi(oracle.BURGERS, n, n, nu, 0.0, u, l, v, c, gamma, h, TOL, TOL, xi)
    assert st == oracle.OK
    ref = _phi_dense(h * J, v, l)
    assert rel_l2(out, ref) <= 100 * TOL


def test_linearity_semigroup_mean_and_constants():
    # diffusion-dominated, so that the real focal interval also covers 2h
    n, nu, a = 32, 1e-2, 0.25
    u0, h, c, gamma = _cfg1(1, n=n, nu=nu, a=a)
    w = synth.random_field(n * n, seed=8)
    xi = oracle.leja_points(400)

    def E(v, hh=h, l=0):
        out, _, st = oracle.leja_phi(oracle.ADVDIFF, n, n, nu, a, None, l, v, c, gamma, hh, TOL, TOL, xi)
        assert st == oracle.OK
        return out

    # linearity
    al, be = 0.7, -1.9
    lhs = E(al * u0 + be * w)
    rhs = al * E(u0) + be * E(w)
    # exact up to the interpolation error of each of the three applications
    scale = abs(al) * np.linalg.norm(u0) + abs(be) * np.linalg.norm(w)
    assert np.linalg.norm(lhs - rhs) <= 100 * TOL * scale
    # semigroup: exp(2hA) v = exp(hA) exp(hA) v
    two = E(u0, hh=2 * h)
    twice = E(E(u0))
    assert rel_l2(two, twice) <= 100 * TOL
    # mean conservation: 1^T A = 0 and z = 0 is the first node, so
    # mean(phi_l(hA) v) = mean(v)/l! regardless of the iteration count
    for l in (0, 1, 3):
        out = E(w + 0.3, l=l)
        assert abs(out.mean() - (w + 0.3).mean() / math.factorial(l)) <= 1e-14 * np.abs(w).max()
    # constants map to constant / l!
    for l in (0, 2):
        out = E(np.full(n * n, 2.5), l=l)
        assert np.max(np.abs(out - 2.5 / math.factorial(l))) <= 1e-14


def test_power_iteration_lower_bound():
    n, nu, a = 64, 1e-2, 1.0
    v0 = synth.power_start(n * n, seed=5)
    rho, it, st = oracle.power_iteration(oracle.ADVDIFF, n, n, nu, a, None, v0, 10)
    exact = spectral_radius(n, n, nu, a)
    assert st == oracle.OK and 2 <= it <= 10
    assert 0.8 * exact <= rho <= exact * (1 + 1e-12)


def test_status_codes():
    n, nu, a = 16, 1e-2, 1.0
    u0, h, c, gamma = _cfg1(1, n=n)
    xi = oracle.leja_points(5)
    out, iters, st = oracle.leja_phi(oracle.ADVDIFF, n, n, nu, a, None, 0, u0, c, gamma, h, TOL, TOL, xi)
    assert st == oracle.E_NOCONV and iters == 4
    bad = u0.copy()
    bad[7] = np.nan
    out, iters, st = oracle.leja_phi(oracle.ADVDIFF, n, n, nu, a, None, 0, bad, c, gamma, h, TOL, TOL,
                                     oracle.leja_points(100))
    assert st == oracle.E_NONFINITE and iters == 1


def test_ros_eu_linear_is_exp():
    n, nu, a = 64, 1e-2, 1.0
    u0, h, c, gamma = _cfg1(2, n=n)
    xi = oracle.leja_points(400)
    out, iters, st = oracle.ros_eu(oracle.ADVDIFF, n, n, nu, a, u0, c, gamma, h, TOL, TOL, xi)
    assert st == oracle.OK
    assert rel_l2(out, phi_apply(0, n, n, nu, a, h, u0)) <= 100 * TOL


def test_exprb32_linear_has_zero_remainder():
    n, nu, a = 64, 1e-2, 1.0
    u0, h, c, gamma = _cfg1(2, n=n)
    xi = oracle.leja_points(400)
    lo, hi, err, iters, st = oracle.exprb32(oracle.ADVDIFF, n, n, nu, a, u0, c, gamma, h, TOL, TOL, xi)
    assert st == oracle.OK
    assert err == 0.0 and np.array_equal(lo, hi)


@pytest.mark.parametrize("l", [0, 1, 2])
def test_vertical_interpolation_matches_fourier(l):
    # phi_l(alpha_j h A) w for three step fractions from one Newton basis
    # against the exact Fourier solution of each
    n, nu, a = 64, 1e-2, 0.7
    u0, h, c, gamma = _cfg1(4, n=n, a=a)
    xi = oracle.leja_points(400)
    alphas = [1.0 / 3.0, 2.0 / 3.0, 1.0]
    outs, iters, st = oracle.leja_phi_vertical(oracle.ADVDIFF, n, n, nu, a, None, l, alphas, u0, c, gamma, h, TOL,
                                               TOL, xi)
    assert st == oracle.OK
    singles = []
    for j, al in enumerate(alphas):
        ref = phi_apply(l, n, n, nu, a, al * h, u0)
        assert rel_l2(outs[j], ref) <= 100 * TOL, (j, rel_l2(outs[j], ref))
        one, it1, st1 = oracle.leja_phi(oracle.ADVDIFF, n, n, nu, a, None, l, u0, c, gamma, al * h, TOL, TOL, xi)
        assert st1 == oracle.OK
        singles.append(it1)
    # the shared loop runs until the slowest polynomial has converged
    assert iters >= max(singles)
    assert singles[0] < singles[-1]  # smaller steps need fewer terms


def test_vertical_interpolation_burgers_jacobian_dense():
    # phi_1(alpha h J(u)) w against the dense augmented-matrix exponential
    n, nu = 10, 2e-2
    u = synth.burgers_ic(n, n, seed=3)
    w = synth.random_field(n * n, seed=4)
    h = 20 * synth.cfl_step(n, n, nu, np.abs(u).max())
    J = _dense(lambda e: oracle.burgers_J(n, n, nu, u, e), n * n)
    rho = np.max(np.abs(np.linalg.eigvals(J)))
    c, gamma = oracle.spectral_interval(rho)
    xi = oracle.leja_points(400)
    alphas = [0.5, 1.0]
    outs, iters, st = oracle.leja_phi_vertical(oracle.BURGERS, n, n, nu, 0.0, u, 1, alphas, w, c, gamma, h, 1e-12,
                                               1e-12, xi)
    assert st == oracle.OK
    for j, al in enumerate(alphas):
        ref = _phi_dense(al * h * J, w, 1)
        assert rel_l2(outs[j], ref) <= 1e-9


def _exact_with_source(n, nu, a, h, u0, S):
    # u' = A u + S over one step h, mode by mode: exp(h lam) u^ + h phi_1(h lam) S^
    from fourier import phi_complex, symbol

    lam = symbol(n, n, nu, a)
    U = np.fft.fft2(u0.reshape(n, n))
    Sh = np.fft.fft2(S.reshape(n, n))
    return np.real(np.fft.ifft2(np.exp(h * lam) * U + h * phi_complex(1, h * lam) * Sh)).reshape(-1)


@pytest.mark.parametrize("seed", [1, 2])
def test_ros_eu_with_source_is_exact_for_linear_problem(seed):
    # Problem II of Sec. 3 (Eq. 4): with f(u) = A u + S the Rosenbrock-Euler step is
    # the exact solution of the linear ODE with a constant source
    n, nu, a = 64, 1e-2, 1.0
    u0, h, c, gamma = _cfg1(seed, n=n)
    S = synth.source_field(n, n, seed=20 + seed)
    xi = oracle.leja_points(400)
    out, iters, st = oracle.ros_eu(oracle.ADVDIFF, n, n, nu, a, u0, c, gamma, h, TOL, TOL, xi, source=S)
    assert st == oracle.OK
    ref = _exact_with_source(n, nu, a, h, u0, S)
    assert rel_l2(out, ref) <= 100 * TOL
    # without the source the step differs by h phi_1(hA) S, which is not small
    plain, _, _ = oracle.ros_eu(oracle.ADVDIFF, n, n, nu, a, u0, c, gamma, h, TOL, TOL, xi)
    assert rel_l2(plain, ref) > 1e-2


def test_source_mean_growth_and_exprb32_remainder():
    # 1^T A = 0, so the mean grows by exactly h mean(S) per step; and the
    # EXPRB32 remainder stays 0 for an affine right-hand side
    n, nu, a = 48, 1e-2, 0.7
    u0, h, c, gamma = _cfg1(3, n=n, a=a)
    S = synth.source_field(n, n, seed=31)
    xi = oracle.leja_points(400)
    out, _, st = oracle.ros_eu(oracle.ADVDIFF, n, n, nu, a, u0, c, gamma, h, TOL, TOL, xi, source=S)
    assert st == oracle.OK
    assert abs((out.mean() - u0.mean()) - h * S.mean()) <= 1e-12 * (abs(h * S.mean()) + abs(u0.mean()))
    lo, hi, err, it, st = oracle.exprb32(oracle.ADVDIFF, n, n, nu, a, u0, c, gamma, h, TOL, TOL, xi, source=S)
    # F(k) = (A k + S) - A k is S up to the rounding of the two sums, so R
    # and the error estimate vanish to round-off only
    assert st == oracle.OK and err <= 1e-15 * np.linalg.norm(u0) and rel_l2(hi, lo) <= 1e-15
    assert np.array_equal(lo, out)


def _burgers_run(step, u0, n, nu, T, nsteps, xi, tol=1e-13):
    h = T / nsteps
    u = u0.copy()
    v0 = synth.power_start(n * n, seed=5)
    for _ in range(nsteps):
        rho, _, _ = oracle.power_iteration(oracle.BURGERS, n, n, nu, 0.0, u, v0, 10)
        c, gamma = oracle.spectral_interval(rho)
        if step == "ros_eu":
            u, it, st = oracle.ros_eu(oracle.BURGERS, n, n, nu, 0.0, u, c, gamma, h, tol, tol, xi)
        else:
            _, u, err, it, st = oracle.exprb32(oracle.BURGERS, n, n, nu, 0.0, u, c, gamma, h, tol, tol, xi)
        assert st == oracle.OK
    return u


@pytest.mark.slow
def test_integrator_convergence_orders():
    # Global error at a fixed end time against a fine EXPRB32 reference:
    # Ros-Eu is second order, EXPRB32 third order.
    n, nu = 24, 5e-3
    u0 = synth.burgers_ic(n, n, seed=1)
    T = 0.04
    xi = oracle.leja_points(600)
    ref = _burgers_run("exprb32", u0, n, nu, T, 64, xi)
    slopes = {}
    for step in ("ros_eu", "exprb32"):
        errs = [np.linalg.norm(_burgers_run(step, u0, n, nu, T, m, xi) - ref) for m in (2, 4, 8)]
        slopes[step] = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(1.7 <= s <= 2.6 for s in slopes["ros_eu"]), slopes
    assert all(2.6 <= s <= 3.8 for s in slopes["exprb32"]), slopes
