"""Pins of the oracle's EPIRK4s3A step (a fourth-order integrator of the
paper's Table 2, with the coefficients that the stiff order conditions fix
for the stage nodes 1/2 and 2/3).

* The coefficients: (b2, b3) = (32, -27/2) and (e2, e3) = (-144, 81) are the
  solutions of sum_i b_i c_i^2 = 2, sum_i b_i c_i^3 = 0 and
  sum_i e_i c_i^2 = 0, sum_i e_i c_i^3 = 6 (exact rational arithmetic).
* Global convergence order on Burgers: 4 for u_high, 3 for the embedded
  u_low (a wrong sign or a dropped stage breaks either).
* A linear problem: the remainders vanish, so u_low = u_high = the
  Rosenbrock-Euler step = exp(hA)u (exact Fourier solution), err = 0; with
  a source S as well (F(k) = A k + S - A k = S cancels in R).
"""
import math
from fractions import Fraction as Fr

import numpy as np

import oracle
import synth


def test_coefficients_solve_the_stiff_order_conditions():
    c2, c3 = Fr(1, 2), Fr(2, 3)
    b2, b3, e2, e3 = Fr(32), Fr(-27, 2), Fr(-144), Fr(81)
    assert b2 * c2**2 + b3 * c3**2 == 2 and b2 * c2**3 + b3 * c3**3 == 0
    assert e2 * c2**2 + e3 * c3**2 == 0 and e2 * c2**3 + e3 * c3**3 == 6


def _burgers_run(which, u0, n, nu, T, nsteps, xi, tol=1e-13):
    h = T / nsteps
    u = u0.copy()
    v0 = synth.power_start(n * n, seed=5)
    for _ in range(nsteps):
        rho, _, _ = oracle.power_iteration(oracle.BURGERS, n, n, nu, 0.0, u, v0, 10)
        c, g = oracle.spectral_interval(rho)
        lo, hi, err, it, st = oracle.epirk4s3a(oracle.BURGERS, n, n, nu, 0.0, u, c, g, h, tol, tol, xi)
        assert st == oracle.OK
        u = hi if which == "u_high" else lo
    return u


def test_convergence_orders():
    n, nu = 24, 5e-3
    u0 = synth.burgers_ic(n, n, seed=1)
    T = 0.04
    xi = oracle.leja_points(600)
    ref = _burgers_run("u_high", u0, n, nu, T, 64, xi)
    slopes = {}
    for which in ("u_high", "u_low"):
        errs = [np.linalg.norm(_burgers_run(which, u0, n, nu, T, m, xi) - ref) for m in (2, 4, 8)]
        slopes[which] = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(3.7 <= s <= 4.6 for s in slopes["u_high"]), slopes
    assert all(2.7 <= s <= 3.5 for s in slopes["u_low"]), slopes


def test_linear_problem_is_exact():
    import fourier

    n, nu, a = 32, 1e-2, 0.1  # diffusion-dominated (4 nu n / a = 12.8)
    u0 = synth.gaussians_ic(n, n, seed=2)
    h = 40 * synth.cfl_step(n, n, nu, a)
    c, g = oracle.spectral_interval(fourier.spectral_radius(n, n, nu, a))
    xi = oracle.leja_points(1000)
    lo, hi, err, it, st = oracle.epirk4s3a(oracle.ADVDIFF, n, n, nu, a, u0, c, g, h, 1e-12, 1e-12, xi)
    assert st == oracle.OK and err == 0.0 and np.array_equal(lo, hi)
    ros, _, _ = oracle.ros_eu(oracle.ADVDIFF, n, n, nu, a, u0, c, g, h, 1e-12, 1e-12, xi)
    exact = fourier.phi_apply(0, n, n, nu, a, h, u0)
    assert np.linalg.norm(hi - exact) <= 100 * 1e-12 * np.linalg.norm(exact)
    assert np.linalg.norm(hi - ros) <= 100 * 1e-12 * np.linalg.norm(exact)
    # with a time-independent source: the exact affine solution
    S = synth.source_field(n, n, seed=21)
    lo, hi, err, it, st = oracle.epirk4s3a(oracle.ADVDIFF, n, n, nu, a, u0, c, g, h, 1e-12, 1e-12, xi, source=S)
    ros, _, _ = oracle.ros_eu(oracle.ADVDIFF, n, n, nu, a, u0, c, g, h, 1e-12, 1e-12, xi, source=S)
    assert st == oracle.OK and err <= 1e-14 * np.linalg.norm(u0)
    assert np.linalg.norm(hi - ros) <= 100 * 1e-12 * np.linalg.norm(ros)
