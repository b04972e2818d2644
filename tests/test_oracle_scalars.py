"""Pins of the oracle's scalar parts: Leja points, phi_l, divided differences.

Each check compares the oracle with something the mathematics fixes
independently of the oracle's own code: closed forms, brute-force maximisers,
high-precision evaluation of a closed form (mpmath), exactness on polynomials
and the interpolation property of the Newton form.
"""
import math

import numpy as np
import pytest

import oracle

mpmath = pytest.importorskip("mpmath")


# ---------------------------------------------------------------- Leja points
def test_leja_first_points_closed_form():
    # Sec. 2.1: xi_0 has maximal modulus (+2 by the sign reading), then -2,
    # then the maximiser of |x^2 - 4| (0), then of |x (x^2 - 4)|: +-2/sqrt(3),
    # the tie going to the larger point.
    xi = oracle.leja_points_compute(4)
    assert xi[0] == 2.0 and xi[1] == -2.0 and xi[2] == 0.0
    assert abs(xi[3] - 2.0 / math.sqrt(3.0)) <= 4.5e-16  # two ulps


def test_leja_brute_force_maximiser():
    xi = oracle.leja_points(120)
    grid = np.linspace(-2.0, 2.0, 400001)
    for j in list(range(3, 40)) + [60, 90, 119]:
        logs_grid = np.sum(np.log(np.abs(grid[:, None] - xi[None, :j]) + 1e-300), axis=1)
        val = np.sum(np.log(np.abs(xi[j] - xi[:j])))
        # the greedy point is at least as good as every grid point (up to rounding)
        assert val >= logs_grid.max() - 1e-10, j
        # and it is the grid's best region: the grid point closest to xi[j]
        # is within a cell of the grid's argmax, or the two values tie
        k = int(np.argmax(logs_grid))
        assert abs(grid[k] - xi[j]) < 1e-3 or abs(logs_grid[k] - val) < 1e-6, j


def test_leja_capacity_and_range():
    # [-2, 2] has logarithmic capacity 1, so prod_k |xi_j - xi_k|^(1/j) -> 1.
    xi = oracle.leja_points(1000)
    assert np.all(np.abs(xi) <= 2.0)
    assert len(np.unique(xi)) == 1000
    g = [np.prod(np.abs(xi[j] - xi[:j])) ** (1.0 / j) for j in (100, 500, 999)]
    assert 1.0 <= g[2] <= g[1] <= g[0] <= 1.05
    assert g[2] < 1.01


def test_leja_golden_table_is_the_oracle():
    fresh = oracle.leja_points_compute(150)
    tab = oracle.leja_points(1000)[:150]
    assert np.array_equal(fresh, tab)


# ---------------------------------------------------------------- phi_l
def _phi_mp(l, z):
    # phi_l(z) = (e^z - sum_{k<l} z^k / k!) / z^l, phi_l(0) = 1/l!  (closed form
    # of the recursion in Sec. 1), evaluated with 60 significant digits.
    mpmath.mp.dps = 60
    z = mpmath.mpf(z)
    if z == 0:
        return mpmath.mpf(1) / mpmath.factorial(l)
    s = mpmath.exp(z)
    for k in range(l):
        s -= z**k / mpmath.factorial(k)
    return s / z**l


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("z", [0.0, 1e-9, -1e-4, 0.3, -0.99, 1.0, -1.0, 2.5, -7.0, -40.0, -400.0])
def test_phi_against_closed_form(l, z):
    ref = float(_phi_mp(l, z))
    got = oracle.phi(l, z)
    assert abs(got - ref) <= 2e-16 * abs(ref) + 1e-300


def test_phi_textbook_values():
    assert oracle.phi(1, 1.0) == pytest.approx(math.e - 1.0, rel=1e-15)
    assert oracle.phi(2, 1.0) == pytest.approx(math.e - 2.0, rel=1e-15)
    assert oracle.phi(1, -1.0) == pytest.approx(-math.expm1(-1.0), rel=1e-15)
    for l in range(6):
        assert oracle.phi(l, 0.0) == 1.0 / math.factorial(l)


# ---------------------------------------------------------------- divided differences
def test_divdiff_polynomial_exactness():
    rng = np.random.default_rng(3)
    x = rng.uniform(-2, 2, size=12)
    coef = [0.7, -1.3, 2.0, 0.25]  # 0.7 - 1.3 x + 2 x^2 + 0.25 x^3
    f = np.polyval(coef[::-1], x)
    d = oracle.divdiff_values(x, f)
    assert d[0] == pytest.approx(f[0], rel=1e-15)
    assert d[3] == pytest.approx(0.25, rel=1e-13)
    assert np.all(np.abs(d[4:]) <= 1e-12)


def test_divdiff_exp_equispaced_closed_form():
    # exp[x0, x0+delta, ..., x0+k delta] = e^x0 (e^delta - 1)^k / (k! delta^k).
    # Nodes are exact binary numbers; the values e^x are rounded to double, and
    # that rounding propagates with the weights 1/prod_{i != j}|x_j - x_i| of
    # the explicit divided-difference formula, which bounds the error allowed.
    x0, delta = -1.75, 0.125
    n = 25
    x = x0 + delta * np.arange(n + 1)
    f = np.exp(x)
    d = oracle.divdiff_values(x, f)
    mpmath.mp.dps = 50
    for k in range(n + 1):
        ref = mpmath.exp(x0) * (mpmath.exp(delta) - 1) ** k / (mpmath.factorial(k) * mpmath.mpf(delta) ** k)
        cond = sum(abs(f[j]) / np.prod([abs(x[j] - x[i]) for i in range(k + 1) if i != j]) for j in range(k + 1))
        assert abs(d[k] - float(ref)) <= 2.3e-16 * cond + 1e-15 * abs(float(ref)), k


@pytest.mark.parametrize("l", [0, 1, 3])
def test_leja_coeffs_first_two_closed_form(l):
    # xi_0 = 2 and c + 2 gamma = 0 give d_0 = phi_l(0) = 1/l!;
    # xi_1 = -2 gives d_1 = (phi_l(h lambda) - 1/l!) / (-4), lambda = c - 2 gamma.
    rho, h = 1.0e3, 0.05
    lam = -1.05 * rho
    c, gamma = lam / 2.0, -lam / 4.0
    xi = oracle.leja_points(10)
    d = oracle.leja_coeffs(l, h, c, gamma, xi)
    assert d[0] == pytest.approx(1.0 / math.factorial(l), rel=1e-15)
    ref = (_phi_mp(l, h * lam) - mpmath.mpf(1) / mpmath.factorial(l)) / (-4)
    assert d[1] == pytest.approx(float(ref), rel=1e-14)


@pytest.mark.parametrize("l,hg", [(0, 0.5), (1, 8.0), (1, 26.0), (3, 26.0), (0, 60.0)])
def test_leja_coeffs_interpolate(l, hg):
    # The Newton form sum_j d_j prod_{k<j} (x - xi_k) reproduces f(x) =
    # phi_l(h (c + gamma x)) on [-2, 2] once enough points are used.  A wrong
    # coefficient anywhere breaks this at points that are not nodes.
    K = 400
    xi = oracle.leja_points(K)
    h = 1.0
    gamma = hg
    c = -2.0 * gamma
    d = oracle.leja_coeffs(l, h, c, gamma, xi)
    rng = np.random.default_rng(11)
    for x in rng.uniform(-2, 2, size=25):
        w, s = 1.0, 0.0
        for j in range(K):
            s += d[j] * w
            w *= x - xi[j]
        ref = float(_phi_mp(l, h * (c + gamma * x)))
        assert abs(s - ref) <= 1e-13 * max(1.0, abs(ref)), (x, s, ref)
