"""Pins of the oracle's high-precision divided differences (mpmath).

Where the spectrum lies far from the real focal interval (advection-dominated
grids, 4 nu n / a of order 1) the Newton basis grows geometrically, and the
binary128 recursion's absolute rounding floor (about 1e-34 of the largest
value), multiplied by that growth, stops the series from converging.  The
oracle then forms the same divided differences by the same recursion with
more digits (oracle.leja_coeffs_mp).  These tests pin that path to what the
mathematics fixes: phi_l's closed form at high precision, exactness on
cubics, the first two coefficients in closed form, the interpolation
property of the Newton form, and -- for the whole Leja loop on grids where
binary128 fails -- the exact Fourier solution of the discrete operator.
"""
import math

import numpy as np
import pytest

import oracle
import synth

mpmath = pytest.importorskip("mpmath")


def test_phi_mp_matches_closed_form():
    # phi_l(z) = (e^z - sum_{k<l} z^k / k!) / z^l, written out at 400 digits
    for l in range(0, 5):
        for z in (-300.0, -57.3, -1.0, -0.3, 0.7, 3.0, 1e-5):
            with mpmath.workdps(400):
                zz = mpmath.mpf(z)
                ref = (mpmath.exp(zz) - sum(zz**k / mpmath.factorial(k) for k in range(l))) / zz**l
            with mpmath.workdps(120):
                got = oracle._phi_mp(mpmath.mp, l, mpmath.mpf(z))
                assert abs(got - ref) <= mpmath.mpf(10) ** -100 * abs(ref), (l, z)


def test_divdiff_mp_exact_on_cubics():
    # for p(x) = 3 x^3 - x + 5 the divided differences at any distinct nodes
    # end with the leading coefficient 3 and are zero beyond degree 3; the
    # nodes k/8 (in a scrambled order) make every value exact in double
    x = np.random.default_rng(1).permutation(np.arange(-20, 21)) / 8.0
    f = 3 * x**3 - x + 5
    d = oracle.divdiff_values_mp(x, f, dps=80)
    assert d[3] == 3.0
    assert np.max(np.abs(d[4:])) <= 1e-60
    # d_0 = p(x_0), d_1 = (p(x_1) - p(x_0)) / (x_1 - x_0)
    p = lambda t: 3 * t**3 - t + 5
    assert d[0] == p(x[0])
    assert d[1] == pytest.approx((p(x[1]) - p(x[0])) / (x[1] - x[0]), rel=1e-15)


@pytest.mark.parametrize("l,hg", [(0, 26.0), (1, 60.0), (3, 100.0)])
def test_leja_coeffs_mp_first_two_closed_form(l, hg):
    # z = h (c + gamma xi) with c = -2 gamma: xi_0 = 2 -> z = 0, xi_1 = -2 -> z = -4 h gamma
    h, gamma = 1.0, hg
    c = -2.0 * gamma
    xi = oracle.leja_points(60)
    d = oracle.leja_coeffs_mp(l, h, c, gamma, xi)
    assert d[0] == 1.0 / math.factorial(l)
    with mpmath.workdps(60):
        z = mpmath.mpf(-4 * h * gamma)
        phi = (mpmath.exp(z) - sum(z**k / mpmath.factorial(k) for k in range(l))) / z**l
        d1 = (phi - mpmath.mpf(1) / mpmath.factorial(l)) / -4
    assert d[1] == pytest.approx(float(d1), rel=1e-15)


def test_leja_coeffs_mp_agree_with_binary128_above_its_floor():
    xi = oracle.leja_points(200)
    for l, hg in ((0, 26.0), (1, 80.0), (3, 150.0)):
        c = -2.0 * hg
        dm = oracle.leja_coeffs_mp(l, 1.0, c, hg, xi)
        dq = oracle.leja_coeffs(l, 1.0, c, hg, xi)
        # binary128's rounding floor is absolute (~1e-34 of the largest value)
        assert np.max(np.abs(dm - dq)) <= 1e-32 * np.max(np.abs(dm))
        # above the floor the two agree to double rounding
        big = np.abs(dm) > 1e-20 * np.max(np.abs(dm))
        assert np.max(np.abs(dm[big] - dq[big]) / np.abs(dm[big])) <= 1e-13


def test_newton_form_interpolates_phi():
    # the Newton form sum_j d_j prod_{k<j} (x - xi_k) reproduces
    # phi_l(h (c + gamma x)) off the nodes, far below binary128's floor
    l, h, gamma = 1, 1.0, 40.0
    c = -2.0 * gamma
    K = 160
    xi = oracle.leja_points(K)
    dps = oracle.dd_digits(K)
    d = oracle.leja_coeffs_mp(l, h, c, gamma, xi)  # rounded to double: 1e-16 relative each
    rng = np.random.default_rng(3)
    with mpmath.workdps(dps):
        for x in rng.uniform(-2, 2, 12):
            xm = mpmath.mpf(float(x))
            z = h * (c + gamma * xm)
            ref = (mpmath.exp(z) - 1) / z
            acc, prod = mpmath.mpf(0), mpmath.mpf(1)
            scale = mpmath.mpf(0)
            for j in range(K):
                term = mpmath.mpf(float(d[j])) * prod
                acc += term
                scale = max(scale, abs(term))
                prod *= xm - mpmath.mpf(float(xi[j]))
            # the error is the rounding of each d_j to double, times the
            # largest term of the sum
            assert abs(acc - ref) <= 1e-15 * scale + mpmath.mpf(10) ** -40, x


def _advdiff_exact_case(n, nu, a, seed):
    import fourier

    u0 = synth.gaussians_ic(n, n, seed=seed)
    h = 50 * synth.cfl_step(n, n, nu, a)
    c, g = oracle.spectral_interval(fourier.spectral_radius(n, n, nu, a))
    return u0, h, c, g, fourier.phi_apply(0, n, n, nu, a, h, u0)


@pytest.mark.parametrize("k", [46, 197, 226, 253])
def test_leja_loop_with_mp_coefficients_is_exact_where_binary128_fails(k):
    # instances of the 256-instance batched workload (seed 7) with
    # 4 nu n / a < 2: the binary128 oracle runs into its floor (non-finite
    # or not converged), the mp coefficients converge to the exact solution
    d = synth.batch_instances(256, seed=7)[k]
    n, nu, a = d["n"], d["nu"], d["a"]
    assert 4 * nu * n / a < 2
    u0 = synth.gaussians_ic(n, n, seed=d["seed"])
    u0, h, c, g, exact = _advdiff_exact_case(n, nu, a, d["seed"])
    xi = oracle.leja_points(1000)
    _, _, st_q = oracle.leja_phi(oracle.ADVDIFF, n, n, nu, a, None, 0, u0, c, g, h, 1e-10, 1e-10, xi)
    assert st_q != 0
    out, it, st = oracle.leja_phi_mp(oracle.ADVDIFF, n, n, nu, a, None, 0, u0, c, g, h, 1e-10, 1e-10, xi)
    assert st == 0 and it < 200
    assert np.linalg.norm(out - exact) <= 100 * 1e-10 * np.linalg.norm(exact)
    # z = 0 is a node and 1^T A = 0: the mean is conserved to round-off
    assert abs(out.mean() - u0.mean()) <= 1e-13 * np.abs(u0).max()


@pytest.mark.parametrize("seed", [2, 4, 5])
def test_config1_power_bound_mp_is_exact(seed):
    # 64^2, nu = 1e-2, a = 1 (4 nu n / a = 2.6) with the 10-pass power bound:
    # binary128 and mp coefficients differ by a few 1e-10 here; the mp run is
    # within the Leja tolerance of the exact solution
    import fourier

    n, nu, a = 64, 1e-2, 1.0
    u0 = synth.gaussians_ic(n, n, seed=seed)
    h = 50 * synth.cfl_step(n, n, nu, a)
    rho, _, st = oracle.power_iteration(oracle.ADVDIFF, n, n, nu, a, None, synth.power_start(n * n, seed=5), 10)
    c, g = oracle.spectral_interval(rho)
    exact = fourier.phi_apply(0, n, n, nu, a, h, u0)
    out, it, st = oracle.leja_phi_mp(oracle.ADVDIFF, n, n, nu, a, None, 0, u0, c, g, h, 1e-10, 1e-10,
                                     oracle.leja_points(1000))
    assert st == 0
    assert np.linalg.norm(out - exact) <= 100 * 1e-10 * np.linalg.norm(exact)


@pytest.mark.parametrize("k,hard", [(0, False), (31, True)])
def test_rounding_sensitivity_of_regrouped_stencil(k, hard):
    # the per-neighbour grouping is the same operator: both runs stay within
    # the Leja tolerance of the exact solution; on a diffusion-dominated
    # instance they agree to round-off, on an advection-dominated one
    # (4 nu n / a = 1.87) the growing Newton basis amplifies the different
    # rounding far above it
    d = synth.batch_instances(256, seed=7)[k]
    n, nu, a = d["n"], d["nu"], d["a"]
    u0, h, c, g, exact = _advdiff_exact_case(n, nu, a, d["seed"])
    xi = oracle.leja_points(1000)
    out, it, st = oracle.leja_phi_mp(oracle.ADVDIFF, n, n, nu, a, None, 0, u0, c, g, h, 1e-10, 1e-10, xi)
    alt, it2, st2 = oracle.leja_phi_mp(oracle.ADVDIFF, n, n, nu, a, None, 0, u0, c, g, h, 1e-10, 1e-10, xi,
                                       regroup=True)
    assert st == 0 and st2 == 0 and abs(it - it2) <= 1
    for x in (out, alt):
        assert np.linalg.norm(x - exact) <= 100 * 1e-10 * np.linalg.norm(exact)
    delta = oracle.rounding_sensitivity(n, n, nu, a, 0, u0, c, g, h, 1e-10, 1e-10, xi, ref=out)
    assert delta == pytest.approx(np.linalg.norm(alt - out) / np.linalg.norm(out), rel=1e-12)
    if hard:
        assert delta > 1e-11
    else:
        assert delta < 1e-14
