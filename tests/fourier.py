"""Exact reference solutions for the periodic advection-diffusion operator.

The central-difference operator A on the periodic nx x ny grid is
block-circulant, so numpy's FFT diagonalises it.  Its symbol at the discrete
frequencies tx = 2 pi kx/nx, ty = 2 pi ky/ny is

    lambda = nu (2 cos tx - 2)/dx^2 + nu (2 cos ty - 2)/dy^2
             + i a (sin tx / dx + sin ty / dy),

written here from the definition of the differences.  phi_l(hA) v is then
IFFT(phi_l(h lambda) FFT(v)) exactly (up to rounding), for any l.
"""
import math

import numpy as np


def symbol(nx, ny, nu, a):
    tx = 2 * np.pi * np.fft.fftfreq(nx)
    ty = 2 * np.pi * np.fft.fftfreq(ny)
    TX, TY = np.meshgrid(tx, ty, indexing="xy")
    dx, dy = 1.0 / nx, 1.0 / ny
    re = nu * (2 * np.cos(TX) - 2) / dx**2 + nu * (2 * np.cos(TY) - 2) / dy**2
    im = a * (np.sin(TX) / dx + np.sin(TY) / dy)
    return re + 1j * im


def symbol_up3(nx, ny, nu, a):
    """Symbol of the paper's discretisation on periodic [-1,1)^2 (spacing
    2/n): central Laplacian plus a times the third-order upwind gradient,
    whose one-axis stencil for a > 0 is (-v_{i+2} + 6 v_{i+1} - 3 v_i - 2 v_{i-1}) / 6
    (mirrored for a < 0)."""
    tx = 2 * np.pi * np.fft.fftfreq(nx)
    ty = 2 * np.pi * np.fft.fftfreq(ny)
    TX, TY = np.meshgrid(tx, ty, indexing="xy")
    dx, dy = 2.0 / nx, 2.0 / ny

    def sigma(t):
        if a >= 0:
            return (-np.exp(2j * t) + 6 * np.exp(1j * t) - 3 - 2 * np.exp(-1j * t)) / 6.0
        return (2 * np.exp(1j * t) + 3 - 6 * np.exp(-1j * t) + np.exp(-2j * t)) / 6.0

    lap = nu * (2 * np.cos(TX) - 2) / dx**2 + nu * (2 * np.cos(TY) - 2) / dy**2
    return lap + a * (sigma(TX) / dx + sigma(TY) / dy)


def phi_apply_symbol(l, lam, h, v, nx, ny):
    V = np.fft.fft2(np.asarray(v, dtype=np.float64).reshape(ny, nx))
    return np.real(np.fft.ifft2(phi_complex(l, h * lam) * V)).reshape(-1)


def phi_complex(l, z):
    """phi_l(z) elementwise for complex arrays: power series for |z| < 1,
    the recursion phi_{k+1} = (phi_k - 1/k!)/z from exp otherwise."""
    z = np.asarray(z, dtype=np.complex128)
    out = np.empty_like(z)
    small = np.abs(z) < 1.0
    zs = z[small]
    term = np.full_like(zs, 1.0 / math.factorial(l))
    s = term.copy()
    for k in range(1, 40):
        term = term * zs / (k + l)
        s = s + term
    out[small] = s
    zb = z[~small]
    ph = np.exp(zb)
    for k in range(l):
        ph = (ph - 1.0 / math.factorial(k)) / zb
    out[~small] = ph
    return out


def phi_apply(l, nx, ny, nu, a, h, v):
    lam = symbol(nx, ny, nu, a)
    V = np.fft.fft2(np.asarray(v, dtype=np.float64).reshape(ny, nx))
    return np.real(np.fft.ifft2(phi_complex(l, h * lam) * V)).reshape(-1)


def spectral_radius(nx, ny, nu, a):
    return float(np.max(np.abs(symbol(nx, ny, nu, a))))


def rel_l2(x, ref):
    return float(np.linalg.norm(np.asarray(x) - np.asarray(ref)) / np.linalg.norm(ref))
