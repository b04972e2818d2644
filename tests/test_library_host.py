"""CPU checks of the CUDA library: it loads, it exports every symbol that
include/lexgb.h declares, and its host-side numerics (Leja points, Newton
coefficients) agree with the oracle.  No GPU work is launched here."""
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lx():
    import paper_2310_08344_gb300 as m

    m.lib()
    return m


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?!typedef\b)(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             text, flags=re.M):
            if m.group(1) not in ("if", "while", "for", "return", "sizeof"):
                names.append(m.group(1))
    return names


def test_exports_every_declared_symbol(lx):
    names = declared_functions()
    assert "phi_l_apply" in names and "leja_setup" in names and "expint_step" in names
    assert "leja_setup_rhs" in names and "lx_rhs_builtin" in names
    L = lx.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_leja_points_match_oracle(lx):
    xi = lx.lx_leja_points(1000)
    ref = oracle.leja_points(1000)
    assert np.max(np.abs(xi - ref)) <= 1e-12


@pytest.mark.parametrize("l,hg", [(0, 0.5), (1, 8.0), (1, 26.0), (3, 26.0), (0, 60.0), (1, 100.0), (3, 1e-3),
                                  (2, 250.0)])
def test_leja_coeffs_match_oracle(lx, l, hg):
    # FP64 Opitz/Taylor against the binary128 recursion.  The coefficients are
    # compared relative to their largest magnitude: the Newton terms d_j y_j
    # with ||y_j|| = O(1) (capacity 1) make that the error that matters.
    h, gamma = 1.0, hg
    c = -2.0 * gamma
    K = lx.lx_leja_coeff_count(h, c, gamma, 1000)
    xi = oracle.leja_points(K)
    d = lx.lx_leja_coeffs(l, h, c, gamma, xi)
    do = oracle.leja_coeffs(l, h, c, gamma, xi)
    assert np.max(np.abs(d - do)) <= 1e-12 * np.max(np.abs(do))
    assert abs(d[0] - do[0]) <= 4e-16 * abs(do[0])


def test_coeff_count_bound(lx):
    # beyond the count the coefficients are below the 1e-40 bound: the
    # binary128 oracle shows only its rounding floor (~1e-35) there
    for hg in (5.0, 26.0, 80.0):
        c = -2.0 * hg
        K = lx.lx_leja_coeff_count(1.0, c, hg, 1000)
        assert 32 < K < 1000
        xi = oracle.leja_points(min(1000, K + 40))
        do = oracle.leja_coeffs(1, 1.0, c, hg, xi)
        assert np.max(np.abs(do[K:])) <= 1e-33


def test_invalid_arguments(lx):
    from paper_2310_08344_gb300 import LexgbError

    with pytest.raises(LexgbError):
        lx.lx_leja_points(0)
    with pytest.raises(LexgbError):
        lx.lx_leja_coeffs(1, 1.0, -1.0, 0.0, np.array([2.0, -2.0]))


def test_classical_controller_matches_oracle(lx):
    rng = np.random.default_rng(2)
    for _ in range(500):
        h = 10 ** rng.uniform(-6, 0)
        tol = 10 ** rng.uniform(-10, -2)
        err = tol * 10 ** rng.uniform(-4, 4) if rng.uniform() > 0.05 else 0.0
        a = lx.lx_controller_classical(h, err, tol)
        b = oracle.controller(h, err, tol)
        assert abs(a - b) <= 2e-15 * b  # cbrt vs pow(., 1/3): an ulp or two
        assert 0.2 * h * (1 - 1e-15) <= a <= 2.0 * h * (1 + 1e-15)


def test_spectral_interval_is_listing7(lx):
    # lambda = -1.05 rho; the focal interval [c - 2 gamma, c + 2 gamma] is
    # [lambda, 0] (the Leja point xi_0 = 2 maps to z = 0)
    from paper_2310_08344_gb300 import LexgbError

    for rho in (1e-3, 1.0, 316285.6445, 1.7e8):
        c, g = lx.spectral_interval(rho)
        assert c + 2 * g == 0.0
        assert abs((c - 2 * g) - (-1.05 * rho)) <= 2e-16 * 1.05 * rho
        assert g > 0 and c < 0
        assert (c, g) == oracle.spectral_interval(rho)
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(LexgbError):
            lx.spectral_interval(bad)
