"""Learned step-size controller: training data, training, evaluation.

The network (see include/lexgb.h, mlp_*) maps the features of an attempted
EXPRB32 step -- log(rho h), log(h / dt_CFL), iters / 100, log10(err / tol),
||u|| -- to log(h_next / h) and log(iters predicted).  Labels come from the
method itself: at a state u with current step h, the nine steps
h_j = h 2^(j/2), j = -4..4, are candidates, and the label is the candidate
with the most simulated time per Leja iteration (largest h_j / iters_j)
among those whose error estimate stays below 0.8 tol.  To save work the
candidates are attempted from h upward until one fails the bound (larger
steps only have larger errors), or from h downward until one passes it;
the smaller, unattempted candidates are passed over because the Leja count
grows sublinearly in h, so h / iters grows with h -- `exhaustive=True`
attempts all nine instead, which is how that shortcut is checked.  Every
step of the computation (power bounds, EXPRB32 steps, the network's forward
and backward passes, Adam) runs in the CUDA library; this module only
orchestrates the calls and keeps the samples.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import binding as B

FEATURES = ("log(rho h)", "log(h/dt_CFL)", "iters/100", "log10(err/tol)", "||u||")
# the trained network shipped with the package (train_controller.py writes it)
MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "controller_burgers.npz")
CANDIDATES = tuple(range(-4, 5))  # h_j = h 2^(j/2)
TARGET = 0.8  # the label's error bound, as a fraction of tol


def _norm_u(u):
    return float(u.norm().item() / math.sqrt(u.numel()))


def label_state(ctx, u, v0, h, tol, leja_tol, lo, his, exhaustive=False):
    """Attempt the candidate steps at state u.  Returns (rho, attempts, best)
    with attempts[j] = (h_j, err_j, iters_j) for the attempted candidates
    (a dict keyed by j) and best the j of the label, or None when no
    attempted candidate meets the bound."""
    st, rho, _ = B.power_bound(ctx, u, v0, 10)
    if st != 0:
        return None, {}, None
    c, g = B.spectral_interval(rho)
    target = TARGET * tol
    att = {}

    def attempt(j):
        hj = h * 2.0 ** (j / 2.0)
        st_, err, it = B.expint_step(ctx, u, lo, his[j], c, g, hj, leja_tol, leja_tol)
        att[j] = (hj, err if st_ == 0 else float("inf"), it)
        return att[j][1] <= target

    if exhaustive:
        for j in CANDIDATES:
            attempt(j)
    elif attempt(0):
        for j in CANDIDATES[CANDIDATES.index(0) + 1:]:
            if not attempt(j):
                break
    else:
        for j in reversed(CANDIDATES[:CANDIDATES.index(0)]):
            if attempt(j):
                break
    ok = [j for j in att if att[j][1] <= target]
    best = max(ok, key=lambda j: att[j][0] / max(att[j][2], 1)) if ok else None
    return rho, att, best


def generate_samples(n, nu, u0_list, v0, tol, leja_tol, steps_per_traj, dt_cfl, rng, stream=None, h_scale=None,
                     precision=None, exhaustive=False):
    """Samples (X [S,5], Y [S,2]) along trajectories of viscous Burgers
    started from each state of u0_list (torch CUDA float64 vectors)."""
    import torch

    prec = B.FP64 if precision is None else precision
    ctx = B.leja_setup(n, n, nu, 0.0, B.BURGERS, prec, B.EXPRB32, 1000, stream)
    lo = torch.empty_like(u0_list[0])
    his = {j: torch.empty_like(u0_list[0]) for j in CANDIDATES}
    X, Y = [], []
    for u0 in u0_list:
        u = u0.clone()
        # current steps from ~dt_CFL (a cautious start) to 100 dt_CFL
        h = dt_cfl * 50.0 * (2.0 ** rng.uniform(-6.0, 1.0) if h_scale is None else h_scale)
        for _ in range(steps_per_traj):
            rho, att, best = label_state(ctx, u, v0, h, tol, leja_tol, lo, his, exhaustive)
            if rho is None or 0 not in att:
                break
            h0, err0, it0 = att[0]
            x = [math.log(rho * h0), math.log(h0 / dt_cfl), it0 / 100.0, math.log10(max(err0, 1e-300) / tol),
                 _norm_u(u)]
            if best is None:
                # even a quarter of h fails: label the smallest candidate
                best = min(att)
            hb, eb, ib = att[best]
            if all(math.isfinite(v) for v in x):
                X.append(x)
                Y.append([math.log(hb / h0), math.log(max(ib, 1))])
            if eb <= tol:
                u.copy_(his[best])
            h = hb * 2.0 ** rng.uniform(-1.0, 1.0)
            if rng.uniform() < 0.2:  # now and then a cautious step again
                h = dt_cfl * 50.0 * 2.0 ** rng.uniform(-6.0, 0.0)
    ctx.close()
    return np.asarray(X, dtype=np.float32), np.asarray(Y, dtype=np.float32)


def normalisation(X, Y):
    sx = X.std(0)
    sy = Y.std(0)
    sx[sx < 1e-6] = 1.0
    sy[sy < 1e-6] = 1.0
    return np.concatenate([X.mean(0), sx, Y.mean(0), sy]).astype(np.float32)


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in [(5, 64), (64, 64), (64, 64), (64, 2)]:
        parts.append(rng.standard_normal(i * o) * math.sqrt(2.0 / i))
        parts.append(np.zeros(o))
    return np.concatenate(parts).astype(np.float32)


def train(X, Y, epochs=30, batch=1024, lr=2e-3, seed=0, stream=None):
    """Train on the GPU (mini-batch Adam).  Returns (model, losses)."""
    import torch

    norm = normalisation(X, Y)
    model = B.mlp_setup(batch, init_params(seed), norm, stream)
    rng = np.random.default_rng(seed)
    xd = torch.from_numpy(X).cuda()
    yd = torch.from_numpy(Y).cuda()
    S = X.shape[0]
    losses = []
    for _ in range(epochs):
        perm = torch.from_numpy(rng.permutation(S)).cuda()
        xs, ys = xd[perm].contiguous(), yd[perm].contiguous()
        for k in range(0, S - batch + 1 if S >= batch else 1, batch):
            bsz = min(batch, S - k)
            st, loss, _ = B.mlp_train_step(model, xs[k:k + bsz], ys[k:k + bsz], bsz, adam=True, lr=lr)
            if st != 0:
                raise B.LexgbError(st, "mlp_train_step")
            losses.append(loss)
    return model, norm, losses


def save_model(path, model, norm, meta):
    """Write the network's FP32 master weights, its normalisation vector and
    a JSON description of how it was trained."""
    w = B.mlp_get_weights(model)
    blob = np.frombuffer(json.dumps(meta, sort_keys=True).encode(), dtype=np.uint8)
    np.savez(path, w=w, norm=np.asarray(norm, dtype=np.float32), meta=blob)


def load_model(path=MODEL_PATH, batch_max=64, stream=None):
    """(model, meta) from a file written by save_model."""
    with np.load(path) as d:
        w, norm = d["w"].copy(), d["norm"].copy()
        meta = json.loads(bytes(d["meta"]).decode())
    if w.size != B.mlp_param_count() or norm.size != 14:
        raise ValueError(f"{path}: not a controller network of this library")
    return B.mlp_setup(batch_max, w, norm, stream), meta
