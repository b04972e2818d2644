"""CPU oracle of the controller MLP (5 -> 64 -> 64 -> 64 -> 2, ReLU).

TEST INFRASTRUCTURE ONLY.  Plain numpy in float64.  With ``emulate=True`` the
quantities the GPU keeps in BF16 (weights, normalised inputs, hidden
activations, output and hidden-layer gradients) are rounded to BF16
(round-to-nearest-even) so that the GPU's BF16-in / FP32-accumulate result can
be compared within BF16 tolerance; with ``emulate=False`` it is the exact
network, pinned by central finite differences in the tests.

Parameter vector layout: W1[5][64], b1[64], W2[64][64], b2[64], W3[64][64],
b3[64], W4[64][2], b4[2]  (W[i][j] connects input i to output j).
Normalisation vector: mean_x[5], std_x[5], mean_y[2], std_y[2].
Loss: sum over rows and outputs of (y_n - t_n)^2 / (2 B) on normalised outputs.
"""
import numpy as np

SIZES = [(5, 64), (64, 64), (64, 64), (64, 2)]
N_PARAMS = sum(i * o + o for i, o in SIZES)


def bf16(x):
    x32 = np.asarray(x, dtype=np.float32)
    b = x32.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, k = [], 0
    for i, o in SIZES:
        W = p[k:k + i * o].reshape(i, o)
        k += i * o
        b = p[k:k + o]
        k += o
        out.append((W, b))
    return out


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in SIZES:
        parts.append(rng.standard_normal(i * o) * np.sqrt(2.0 / i))
        parts.append(np.zeros(o))
    return np.concatenate(parts)


def forward(p, norm, X, emulate=True):
    r = bf16 if emulate else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unpack(p)
    mx, sx, my, sy = norm[0:5], norm[5:10], norm[10:12], norm[12:14]
    Xn = r((np.asarray(X, dtype=np.float64) - mx) / sx)
    acts = [Xn]
    H = Xn
    for li, (W, b) in enumerate(layers):
        Z = H @ r(W) + b
        if li < 3:
            H = r(np.maximum(Z, 0.0))
            acts.append(H)
        else:
            H = Z
    Yn = H
    return Yn, acts, (my, sy)


def predict(p, norm, X, emulate=True):
    Yn, _, (my, sy) = forward(p, norm, X, emulate)
    return Yn * sy + my


def loss_and_grad(p, norm, X, T, emulate=True):
    r = bf16 if emulate else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unpack(p)
    Yn, acts, (my, sy) = forward(p, norm, X, emulate)
    B = X.shape[0]
    Tn = (np.asarray(T, dtype=np.float64) - my) / sy
    E = Yn - Tn
    loss = float(np.sum(E * E) / (2.0 * B))
    dZ = r(E / B)
    grads = [None] * 4
    for li in range(3, -1, -1):
        W, _ = layers[li]
        Hin = acts[li]
        grads[li] = (Hin.T @ dZ, dZ.sum(axis=0))
        if li > 0:
            dH = dZ @ r(W).T
            dZ = r(dH * (acts[li] > 0))
    flat = []
    for dW, db in grads:
        flat.append(dW.reshape(-1))
        flat.append(db)
    return loss, np.concatenate(flat)
