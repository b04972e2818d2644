"""Learned step-size controller: training data, training, evaluation.

The network (see include/lexgb.h, mlp_*) maps the features of an attempted
EXPRB32 step -- log(rho h), log(h / dt_CFL), iters / 100, log10(err / tol),
||u|| -- to log(h_next / h) and log(iters predicted).  Labels come from the
method itself: at a state u with current step h, the thirteen steps
h_j = h 2^(j/2), j = -4..8 (a quarter to sixteen times h), are each
attempted in increasing order until one exceeds the target below; the
label step h* is where
the measured error crosses 0.8 tol (log-log interpolation between the two
neighbouring attempts; the largest attempt if all stay below, the smallest if
none does).  That is the largest step the error test accepts with a margin,
hence the one with the most simulated time per Leja iteration, since the
iteration count grows sublinearly in h.  Every step of the computation (power bounds, EXPRB32
steps, the network's forward and backward passes, Adam) runs in the CUDA
library; this module only orchestrates the calls and keeps the samples.
"""
from __future__ import annotations

import math

import numpy as np

from . import binding as B

FEATURES = ("log(rho h)", "log(h/dt_CFL)", "iters/100", "log10(err/tol)", "||u||")


def _norm_u(u):
    return float(u.norm().item() / math.sqrt(u.numel()))


def generate_samples(n, nu, u0_list, v0, tol, leja_tol, steps_per_traj, dt_cfl, rng, stream=None, h_scale=None):
    """Samples (X [S,5], Y [S,2]) along trajectories of viscous Burgers
    started from each state of u0_list (torch CUDA float64 vectors)."""
    import torch

    ctx = B.leja_setup(n, n, nu, 0.0, B.BURGERS, B.FP64, B.EXPRB32, 1000, stream)
    js = list(range(-4, 9))
    j0 = js.index(0)
    lo = torch.empty_like(u0_list[0])
    his = [torch.empty_like(u0_list[0]) for _ in js]
    X, Y = [], []
    for u0 in u0_list:
        u = u0.clone()
        # current steps from ~dt_CFL (a cautious start) to 100 dt_CFL
        h = dt_cfl * 50.0 * (2.0 ** rng.uniform(-6.0, 1.0) if h_scale is None else h_scale)
        for _ in range(steps_per_traj):
            st, rho, _ = B.power_bound(ctx, u, v0, 10)
            if st != 0:
                break
            c, g = B.spectral_interval(rho)
            target = 0.8 * tol
            res = []
            for k, j in enumerate(js):
                hj = h * 2.0 ** (j / 2.0)
                st, err, it = B.expint_step(ctx, u, lo, his[k], c, g, hj, leja_tol, leja_tol)
                e = err if st == 0 else float("inf")
                res.append((hj, e, it))
                if j >= 0 and not (e <= target):
                    break  # past the target: larger steps only cost more Leja iterations
            h0, err0, it0 = res[j0]
            best = 0
            hb, ib = res[0][0], res[0][2]
            for k in range(len(res)):
                if res[k][1] <= target:
                    best = k
            if res[best][1] <= target:
                hb, ib = res[best][0], res[best][2]
                if best < len(res) - 1 and math.isfinite(res[best + 1][1]) and res[best + 1][1] > target and \
                        res[best][1] > 0:
                    e0, e1 = math.log(res[best][1]), math.log(res[best + 1][1])
                    f = (math.log(target) - e0) / (e1 - e0)
                    hb = math.exp(math.log(res[best][0]) + f * (math.log(res[best + 1][0]) - math.log(res[best][0])))
                    ib = res[best][2] + f * (res[best + 1][2] - res[best][2])
            x = [math.log(rho * h0), math.log(h0 / dt_cfl), it0 / 100.0,
                 math.log10(max(err0, 1e-300) / tol), _norm_u(u)]
            if all(math.isfinite(v) for v in x):
                X.append(x)
                Y.append([math.log(hb / h0), math.log(max(ib, 1))])
            if res[best][1] <= tol:
                u.copy_(his[best])
            h = res[best][0] * 2.0 ** rng.uniform(-1.0, 1.0)
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
