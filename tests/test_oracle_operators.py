"""Pins of the oracle's stencil operators against discrete Fourier closed forms.

On the periodic grid, a single mode exp(i(tx*i + ty*j)) is an eigenvector of
the central-difference operators; its eigenvalue (the symbol) is written out
here from the definition of the differences, not from the oracle's code.
"""
import numpy as np
import pytest

import oracle
import synth


def _mode(nx, ny, kx, ky, phase=0.3):
    tx, ty = 2 * np.pi * kx / nx, 2 * np.pi * ky / ny
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    arg = tx * i + ty * j + phase
    return tx, ty, np.cos(arg).reshape(-1), np.sin(arg).reshape(-1)


@pytest.mark.parametrize("nx,ny,kx,ky", [(16, 16, 1, 2), (32, 24, 5, 11), (7, 9, 3, 4), (64, 64, 32, 32)])
def test_advdiff_symbol(nx, ny, kx, ky):
    nu, a = 0.013, 0.7
    dx, dy = 1.0 / nx, 1.0 / ny
    tx, ty, cosm, sinm = _mode(nx, ny, kx, ky)
    lam_re = nu * (2 * np.cos(tx) - 2) / dx**2 + nu * (2 * np.cos(ty) - 2) / dy**2
    lam_im = a * (np.sin(tx) / dx + np.sin(ty) / dy)
    # A cos(arg) = Re(lambda e^{i arg}) = lam_re cos - lam_im sin
    got = oracle.apply_advdiff(nx, ny, nu, a, cosm)
    ref = lam_re * cosm - lam_im * sinm
    scale = abs(lam_re) + abs(lam_im) + 1.0
    assert np.max(np.abs(got - ref)) <= 1e-13 * scale


@pytest.mark.parametrize("nx,ny", [(16, 16), (24, 20)])
def test_burgers_f_single_mode(nx, ny):
    nu = 5e-3
    dx, dy = 1.0 / nx, 1.0 / ny
    tx, ty, cosm, sinm = _mode(nx, ny, 2, 3)
    u = sinm
    lap = ((2 * np.cos(tx) - 2) / dx**2 + (2 * np.cos(ty) - 2) / dy**2) * u
    du = (np.sin(tx) / dx + np.sin(ty) / dy) * cosm  # (D_x + D_y) sin(arg)
    ref = nu * lap - u * du
    got = oracle.burgers_f(nx, ny, nu, u)
    assert np.max(np.abs(got - ref)) <= 1e-12 * (1 + np.max(np.abs(ref)))


def test_burgers_J_two_modes_and_quadratic_remainder():
    nx, ny, nu = 20, 16, 7e-3
    dx, dy = 1.0 / nx, 1.0 / ny
    tx1, ty1, c1, s1 = _mode(nx, ny, 1, 2, 0.1)
    tx2, ty2, c2, s2 = _mode(nx, ny, 3, 1, 0.7)
    u, v = s1, 0.5 * c2
    lap_v = ((2 * np.cos(tx2) - 2) / dx**2 + (2 * np.cos(ty2) - 2) / dy**2) * v
    du = (np.sin(tx1) / dx + np.sin(ty1) / dy) * c1
    dv = -0.5 * (np.sin(tx2) / dx + np.sin(ty2) / dy) * s2
    ref = nu * lap_v - v * du - u * dv
    got = oracle.burgers_J(nx, ny, nu, u, v)
    assert np.max(np.abs(got - ref)) <= 1e-12 * (1 + np.max(np.abs(ref)))
    # f is quadratic: f(u + p) - f(u) - J(u) p = -p (D p), exactly in exact arithmetic
    rng = np.random.default_rng(5)
    uu = synth.burgers_ic(nx, ny, seed=3)
    p = 1e-2 * rng.standard_normal(nx * ny)
    P = p.reshape(ny, nx)
    Dp = ((np.roll(P, -1, 1) - np.roll(P, 1, 1)) / (2 * dx) + (np.roll(P, -1, 0) - np.roll(P, 1, 0)) / (2 * dy)).reshape(-1)
    rem = oracle.burgers_f(nx, ny, nu, uu + p) - oracle.burgers_f(nx, ny, nu, uu) - oracle.burgers_J(nx, ny, nu, uu, p)
    assert np.max(np.abs(rem - (-p * Dp))) <= 1e-11 * np.max(np.abs(oracle.burgers_f(nx, ny, nu, uu)))
