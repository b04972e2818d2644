"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds only workload recipes: initial conditions, start vectors,
batch instance parameters and the explicit CFL step that defines h.  It holds
none of the method's arithmetic (no Leja points, no divided differences, no
stencil application), so both the CUDA path and the CPU oracle can draw their
inputs from it without sharing any of the computation they are compared on.

Grid convention (used by every consumer): x_i = i/nx, y_j = j/ny on the
periodic unit square [0,1)^2, storage index j*nx + i (x fastest), float64.

Random numbers come from numpy's PCG64 (``numpy.random.default_rng(seed)``).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "grid",
    "gaussians_ic",
    "burgers_ic",
    "power_start",
    "cfl_step",
    "batch_instances",
    "random_field",
]


def grid(nx: int, ny: int):
    """Return the (X, Y) coordinate arrays of shape (ny, nx)."""
    x = np.arange(nx, dtype=np.float64) / nx
    y = np.arange(ny, dtype=np.float64) / ny
    X, Y = np.meshgrid(x, y, indexing="xy")
    return X, Y


def _periodic_sq_dist(X, Y, cx, cy):
    """Squared minimum-image distance on the periodic unit square."""
    dx = np.abs(X - cx)
    dy = np.abs(Y - cy)
    dx = np.minimum(dx, 1.0 - dx)
    dy = np.minimum(dy, 1.0 - dy)
    return dx * dx + dy * dy


def gaussians_ic(nx: int, ny: int | None = None, seed: int = 1, count: int = 3) -> np.ndarray:
    """Sum of ``count`` periodic Gaussians, the advection-diffusion initial state.

    u0 = sum_k exp(-|x - c_k|^2_per / w_k^2), c_k ~ U[0,1)^2, w_k ~ U[0.05, 0.1].
    Returns a C-contiguous float64 vector of length nx*ny.
    """
    ny = nx if ny is None else ny
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(count, 2))
    widths = rng.uniform(0.05, 0.1, size=count)
    X, Y = grid(nx, ny)
    u = np.zeros((ny, nx), dtype=np.float64)
    for k in range(count):
        u += np.exp(-_periodic_sq_dist(X, Y, centres[k, 0], centres[k, 1]) / widths[k] ** 2)
    return np.ascontiguousarray(u.reshape(-1))


def burgers_ic(nx: int, ny: int | None = None, seed: int = 1) -> np.ndarray:
    """Sinusoid plus Gaussian, the viscous Burgers initial state (|u0| <= 1).

    u0 = 0.5 sin(2 pi (x + p1)) sin(2 pi (y + p2)) + 0.5 exp(-|x - c|^2_per / w^2),
    p1, p2 ~ U[0,1), c ~ U[0,1)^2, w ~ U[0.05, 0.1].
    """
    ny = nx if ny is None else ny
    rng = np.random.default_rng(seed)
    p1, p2 = rng.uniform(0.0, 1.0, size=2)
    cx, cy = rng.uniform(0.0, 1.0, size=2)
    w = rng.uniform(0.05, 0.1)
    X, Y = grid(nx, ny)
    u = 0.5 * np.sin(2 * np.pi * (X + p1)) * np.sin(2 * np.pi * (Y + p2))
    u += 0.5 * np.exp(-_periodic_sq_dist(X, Y, cx, cy) / w**2)
    return np.ascontiguousarray(u.reshape(-1))


def source_field(nx: int, ny: int | None = None, seed: int = 21) -> np.ndarray:
    """Time-independent source S of the diffusion-advection problem with
    sources: two periodic Gaussians of unit height.

    S = sum_{k<2} exp(-|x - c_k|^2_per / s_k), c_k ~ U[0,1)^2,
    s_k ~ U[0.01, 0.0125] (the squared widths 0.04 and 0.05 of the paper's
    two source Gaussians on [-1,1]^2, rescaled to the unit square).
    """
    ny = nx if ny is None else ny
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(2, 2))
    s2 = rng.uniform(0.01, 0.0125, size=2)
    X, Y = grid(nx, ny)
    S = np.zeros((ny, nx), dtype=np.float64)
    for k in range(2):
        S += np.exp(-_periodic_sq_dist(X, Y, centres[k, 0], centres[k, 1]) / s2[k])
    return np.ascontiguousarray(S.reshape(-1))


def grid_pm1(nx: int, ny: int):
    """Cell coordinates of the periodic [-1,1)^2 grid, x_i = -1 + 2 i / nx."""
    x = -1.0 + 2.0 * np.arange(nx) / nx
    y = -1.0 + 2.0 * np.arange(ny) / ny
    return np.meshgrid(x, y, indexing="xy")


def problem1_ic(nx: int, ny: int | None = None, seed: int | None = None) -> np.ndarray:
    """Initial state of the paper's diffusion-advection problems on [-1,1)^2:
    1 + exp(-((x - x0)^2 + (y - y0)^2) / 0.01) with (x0, y0) = (-0.5, -0.5);
    a seed moves the centre by U[-0.1, 0.1]^2 (test variants)."""
    ny = nx if ny is None else ny
    x0, y0 = -0.5, -0.5
    if seed is not None:
        rng = np.random.default_rng(seed)
        x0, y0 = np.array([x0, y0]) + rng.uniform(-0.1, 0.1, size=2)
    X, Y = grid_pm1(nx, ny)
    return np.ascontiguousarray((1.0 + np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / 0.01)).reshape(-1))


def problem2_source(nx: int, ny: int | None = None) -> np.ndarray:
    """Source of the paper's diffusion-advection problem with sources on
    [-1,1)^2: exp(-((x+0.4)^2 + (y-0.6)^2)/0.05) + exp(-((x-0.25)^2 + (y+0.1)^2)/0.04)."""
    ny = nx if ny is None else ny
    X, Y = grid_pm1(nx, ny)
    S = np.exp(-((X + 0.4) ** 2 + (Y - 0.6) ** 2) / 0.05) + np.exp(-((X - 0.25) ** 2 + (Y + 0.1) ** 2) / 0.04)
    return np.ascontiguousarray(S.reshape(-1))


def problem3_ic(nx: int, ny: int | None = None, seed: int | None = None) -> np.ndarray:
    """Initial state of the paper's Burgers problem on [-1,1)^2:
    2 + 0.01 (sin 2 pi x + sin 2 pi y + sin(8 pi x + 0.3) + sin(8 pi y + 0.3));
    a seed adds U[0, 1) phases to the four sines (test variants)."""
    ny = nx if ny is None else ny
    ph = np.zeros(4) if seed is None else np.random.default_rng(seed).uniform(0.0, 1.0, size=4)
    X, Y = grid_pm1(nx, ny)
    u = 2.0 + 0.01 * (np.sin(2 * np.pi * X + ph[0]) + np.sin(2 * np.pi * Y + ph[1]) +
                      np.sin(8 * np.pi * X + 0.3 + ph[2]) + np.sin(8 * np.pi * Y + 0.3 + ph[3]))
    return np.ascontiguousarray(u.reshape(-1))


def cfl_step_pm1(nx: int, ny: int, nu: float, adv: float) -> float:
    """Explicit step limit on [-1,1)^2 (spacing 2/n), read as for cfl_step:
    min(dx^2 / (4 nu), dx / (2 |adv|))."""
    dx = 2.0 / max(nx, ny)
    lim = dx * dx / (4.0 * nu) if nu > 0 else np.inf
    if adv != 0.0:
        lim = min(lim, dx / (2.0 * abs(adv)))
    return float(lim)


def power_start(n_points: int, seed: int = 12345) -> np.ndarray:
    """Start vector of the power iteration: standard normal entries.

    A constant vector would lie in the null space of the periodic operator,
    so the start vector is random.
    """
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n_points)


def random_field(n_points: int, seed: int) -> np.ndarray:
    """A generic seeded test vector (standard normal)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n_points)


def cfl_step(nx: int, ny: int, nu: float, adv: float) -> float:
    """Explicit CFL step used to set h = k * dt_CFL in the workloads.

    dt_CFL = min(dx^2 / (4 nu), dx / (2 |adv|)) with dx = min(1/nx, 1/ny):
    the forward-Euler limit of the 5-point diffusion stencil and the limit of
    2D central advection.  For Burgers, |adv| is max |u0|.
    """
    dx = min(1.0 / nx, 1.0 / ny)
    cands = []
    if nu > 0:
        cands.append(dx * dx / (4.0 * nu))
    if adv != 0:
        cands.append(dx / (2.0 * abs(adv)))
    if not cands:
        raise ValueError("cfl_step needs nu > 0 or adv != 0")
    return min(cands)


def batch_instances(count: int = 256, seed: int = 7, sizes=(128, 256, 512, 1024)):
    """Parameters of the batched advection-diffusion workload.

    n ~ U{sizes}, nu log-uniform in [1e-3, 1e-1], a ~ U[0, 2], and an
    initial-state seed per instance.  Returns a list of dicts.
    """
    rng = np.random.default_rng(seed)
    n = rng.choice(np.asarray(sizes), size=count)
    nu = 10.0 ** rng.uniform(-3.0, -1.0, size=count)
    a = rng.uniform(0.0, 2.0, size=count)
    ic_seed = rng.integers(1, 2**31 - 1, size=count)
    return [
        {"n": int(n[i]), "nu": float(nu[i]), "a": float(a[i]), "seed": int(ic_seed[i])}
        for i in range(count)
    ]
