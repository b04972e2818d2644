"""Pins of the oracle's step control and adaptive EXPRB32 driver.

The paper notes that the embedded error estimate may drive the step size
(Sec. 2.2) without giving a controller; the reading is the classical one for
a third-order pair, h_new = h min(2, max(0.2, 0.9 (tol/err)^(1/3))), with a
step accepted when err <= tol.  The checks below are fixed by that reading
and by the mathematics of the integrator, not by re-running the oracle's own
formula:

* a planted error err = tol (0.9/f)^3 must give exactly the factor f inside
  (0.2, 2), and the clipped factors outside;
* on a linear problem EXPRB32's remainder R = h (F(a) - F(u)) vanishes
  identically, so every error estimate is 0, every step is accepted and the
  step doubles: the number of steps to T is the closed form
  ceil(log2(T/h0 + 1)), the last step is clipped to end at T, and the final
  state is exp(T A) u0 (the exact Fourier solution, within the Leja
  tolerance per step);
* on Burgers the attempt log obeys what any accept/reject driver must:
  time advances by exactly the accepted steps, a rejected attempt is retried
  from the same time with a smaller step, every accepted step has
  err <= tol, the run contains rejections, and the final state agrees with a
  100 times tighter run to within a small multiple of the tolerance.
"""
import math

import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("f", [0.2001, 0.25, 0.5, 0.9, 1.0, 1.3, 1.77, 1.999])
def test_controller_planted_error(f):
    h, tol = 3.7e-4, 1e-6
    err = tol * (0.9 / f) ** 3
    assert oracle.controller(h, err, tol) == pytest.approx(h * f, rel=1e-14)


def test_controller_clipping():
    h, tol = 1.0, 1e-8
    assert oracle.controller(h, 0.0, tol) == 2.0  # err = 0: the largest growth
    assert oracle.controller(h, tol * 1e-6, tol) == 2.0
    assert oracle.controller(h, tol * 1e6, tol) == pytest.approx(0.2, rel=1e-15)
    # the factor is monotone in err and continuous at both clips
    e = tol * np.logspace(-3, 3, 301)
    fs = np.array([oracle.controller(h, x, tol) for x in e])
    assert np.all(np.diff(fs) <= 0)
    assert np.max(np.abs(np.diff(fs))) < 0.06


def test_integrate_linear_problem_doubles_every_step():
    import fourier

    n, nu, a = 32, 1e-2, 0.5
    u0 = synth.gaussians_ic(n, n, seed=3)
    v0 = synth.power_start(n * n, seed=5)
    h0 = 2 * synth.cfl_step(n, n, nu, a)
    T = 20 * h0
    xi = oracle.leja_points(1000)
    u, steps, rej, its, h_next, t, st, log = oracle.integrate_exprb32(
        oracle.ADVDIFF, n, n, nu, a, u0, v0, T, h0, 1e-6, 1e-12, xi, want_log=True)
    assert st == 0
    k = math.ceil(math.log2(T / h0 + 1))
    assert rej == 0 and steps == k
    assert np.all(log[:, 2] == 0.0) and np.all(log[:, 3] == 1.0)
    # tried steps h0, 2 h0, 4 h0, ... and the last one clipped to reach T
    assert np.allclose(log[:-1, 1], h0 * 2.0 ** np.arange(k - 1), rtol=1e-14)
    assert log[-1, 1] == pytest.approx(T - h0 * (2 ** (k - 1) - 1), rel=1e-12)
    assert t == pytest.approx(T, rel=1e-14)
    assert h_next == pytest.approx(2 * log[-1, 1], rel=1e-14)
    exact = fourier.phi_apply(0, n, n, nu, a, T, u0)
    assert np.linalg.norm(u - exact) <= 100 * k * 1e-12 * np.linalg.norm(exact)


def test_integrate_burgers_attempt_log_and_accuracy():
    n, nu = 32, 2e-2
    u0 = synth.burgers_ic(n, n, seed=1)
    v0 = synth.power_start(n * n, seed=5)
    h0 = 50 * synth.cfl_step(n, n, nu, np.abs(u0).max())
    T, tol = 10 * h0, 1e-5
    xi = oracle.leja_points(1000)
    u, steps, rej, its, h_next, t, st, log = oracle.integrate_exprb32(
        oracle.BURGERS, n, n, nu, 0.0, u0, v0, T, h0, tol, 1e-12, xi, want_log=True)
    assert st == 0 and rej >= 1 and steps >= 2
    assert len(log) == steps + rej
    acc = log[:, 3] == 1.0
    assert np.all(log[acc, 2] <= tol) and np.all(log[~acc, 2] > tol)
    # time advances by exactly the accepted steps
    tt = 0.0
    for i in range(len(log)):
        assert log[i, 0] == tt
        if acc[i]:
            tt += log[i, 1]
        elif i + 1 < len(log):
            # a rejection is retried from the same time with a smaller step
            assert log[i + 1, 0] == log[i, 0] and log[i + 1, 1] < log[i, 1]
    assert t == tt and t == pytest.approx(T, rel=1e-14)
    # the controlled run against a run at a 100x tighter tolerance
    ref = oracle.integrate_exprb32(oracle.BURGERS, n, n, nu, 0.0, u0, v0, T, h0, tol * 1e-2, 1e-12, xi,
                                   max_attempts=5000)
    assert ref[6] == 0
    e = np.linalg.norm(u - ref[0]) / np.sqrt(u.size)
    assert e <= 10 * tol, e
