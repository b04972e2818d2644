"""Train the learned step-size controller and write its weights.

    python -m paper_2310_08344_gb300.train_controller [--samples N] [--out PATH]

Training data are labelled states of viscous Burgers trajectories
(u_t = nu (u_xx + u_yy) - u (u_x + u_y), periodic unit square) integrated
by the library's EXPRB32 step at 256^2 and 512^2, started from the two
seeded initial-state families of the workloads: sums of three periodic
Gaussians, and a sinusoid plus a Gaussian (amplitude <= 1).  Each state is
labelled as in learned.py (candidates h 2^(j/2), j = -4..4; the label
maximises h / iters subject to err <= 0.8 tol, tol = 1e-4, Leja tolerance
1e-10).  Features are scale-free (rho h, h / dt_CFL, err / tol), so a
network trained on these grids serves finer ones -- provided the training
states cover the finer grids' regime: at 2048^2 and nu = 5e-3 a step of
k dt_CFL has the same rho h as at 256^2 but a far smaller error, so the
error bound stops binding and the Leja cost (which grows faster than h at
large rho h) decides.  The coarse grids reach that regime with larger
diffusion coefficients (nu scaled with the square of the grid ratio makes
rho h per unit of physical time that of the finer grid), so the groups
take nu = 5e-3 and larger values on each grid.  The network is
then trained on the GPU by the library's BF16 tensor-core kernels (Adam,
mini-batches of 1024) and written with learned.save_model, together with a
description of the run.  Seeds: trajectories from 11 (the training seed),
network initialisation 0.
"""
from __future__ import annotations

import argparse
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

from . import binding as B  # noqa: E402
from . import learned  # noqa: E402

TOL, LEJA_TOL = 1e-4, 1e-10
# (grid, diffusion coefficient): the workload's 5e-3 and values that put the
# coarse grids into the regime of 1024^2 and 2048^2 at 5e-3
GROUPS = ((256, 5e-3), (256, 8e-2), (256, 0.32), (512, 5e-3), (512, 8e-2))
STEPS_PER_TRAJECTORY = 40


def collect(samples: int, seed: int = 11, log=print):
    import torch

    rng = np.random.default_rng(seed)
    per_group = math.ceil(samples / (len(GROUPS) * 2))
    X, Y, groups = [], [], []
    for n, nu in GROUPS:
        v0 = torch.from_numpy(synth.power_start(n * n, seed=5)).cuda()
        for family in ("gaussians", "sinusoid+gaussian"):
            got, k, t0 = 0, 0, time.perf_counter()
            while got < per_group:
                s = int(rng.integers(1, 2**31 - 1))
                u0 = synth.gaussians_ic(n, n, seed=s) if family == "gaussians" else synth.burgers_ic(n, n, seed=s)
                u0 = torch.from_numpy(u0).cuda()
                dt = synth.cfl_step(n, n, nu, float(u0.abs().max().item()))
                x, y = learned.generate_samples(n, nu, [u0], v0, TOL, LEJA_TOL, STEPS_PER_TRAJECTORY, dt, rng)
                if len(x):
                    X.append(x)
                    Y.append(y)
                    got += len(x)
                k += 1
            groups.append({"grid": n, "nu": nu, "family": family, "trajectories": k, "samples": got,
                           "seconds": round(time.perf_counter() - t0, 1)})
            log(f"  {n}^2 nu={nu} {family}: {got} samples from {k} trajectories in {groups[-1]['seconds']} s")
    return np.concatenate(X), np.concatenate(Y), groups


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--samples", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--out", default=learned.MODEL_PATH)
    args = ap.parse_args(argv)
    B.lib()
    t0 = time.perf_counter()
    X, Y, groups = collect(args.samples)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    model, norm, losses = learned.train(X, Y, epochs=args.epochs, batch=1024, lr=2e-3, seed=0)
    t_train = time.perf_counter() - t0
    meta = {"samples": int(X.shape[0]), "groups": groups, "tol": TOL, "leja_tol": LEJA_TOL,
            "candidates": "h 2^(j/2), j = -4..4", "label": "max h/iters subject to err <= 0.8 tol",
            "epochs": args.epochs, "batch": 1024, "lr": 2e-3, "loss_first": float(losses[0]),
            "loss_last": float(np.mean(losses[-20:])), "generate_s": round(t_gen, 1), "train_s": round(t_train, 1),
            "label_factor_mean": float(np.exp(Y[:, 0]).mean()), "features": list(learned.FEATURES)}
    learned.save_model(args.out, model, norm, meta)
    print(f"{X.shape[0]} samples ({t_gen:.0f} s), {args.epochs} epochs ({t_train:.0f} s), "
          f"loss {losses[0]:.4f} -> {meta['loss_last']:.4f}; wrote {args.out}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
