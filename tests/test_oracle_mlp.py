"""Pin of the MLP oracle: its analytic gradient against central finite
differences of its loss (exact float64 network), and BF16 rounding."""
import numpy as np

from oracle import mlp


def _data(B=37, seed=3):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, 5)) * [2.0, 1.0, 0.3, 1.5, 0.7] + [1.0, 3.0, 0.5, -0.5, 0.2]
    T = rng.standard_normal((B, 2)) * [0.3, 0.8] + [0.1, 3.5]
    norm = np.array([1.0, 3.0, 0.5, -0.5, 0.2, 2.0, 1.0, 0.3, 1.5, 0.7, 0.1, 3.5, 0.3, 0.8])
    return X, T, norm


def test_gradient_matches_finite_differences():
    X, T, norm = _data()
    p = mlp.init_params(1)
    p[mlp.N_PARAMS - 2:] = [0.05, -0.1]
    loss, g = mlp.loss_and_grad(p, norm, X, T, emulate=False)
    rng = np.random.default_rng(0)
    idx = rng.choice(mlp.N_PARAMS, size=60, replace=False)
    idx = np.concatenate([idx, [0, 4 * 64, 320, 320 + 64 + 5, mlp.N_PARAMS - 1, mlp.N_PARAMS - 3]])
    for i in idx:
        e = np.zeros_like(p)
        h = 1e-6 * max(1.0, abs(p[i]))
        e[i] = h
        lp, _ = mlp.loss_and_grad(p + e, norm, X, T, emulate=False)
        lm, _ = mlp.loss_and_grad(p - e, norm, X, T, emulate=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_bf16_rounding():
    # bfloat16: 8 significant bits, round to nearest, ties to even
    x = np.array([1.0, 1.0 + 2.0**-8, 1.0 + 2.0**-9, 1.0 + 2.0**-7 + 2.0**-8, -3.14159, 0.0, 1.0 + 2.0**-8 + 2.0**-12])
    want = np.array([1.0, 1.0, 1.0, 1.0 + 2.0**-6, -3.140625, 0.0, 1.0 + 2.0**-7])
    assert np.array_equal(mlp.bf16(x), want)
