"""Oracle runs for many independent problems in a pool of worker processes.

The workers are started with the "spawn" method, so none of them inherits
the parent's CUDA context (a forked child of a process that has used CUDA
can hang).  Each worker rebuilds its inputs from the seeded recipes in
synth/ and returns only the oracle's result.
"""
import multiprocessing
import os


def _batch_instance(args):
    import numpy as np

    import fourier
    import oracle
    import synth

    n, nu, a, seed, l, tol, mult = args
    u0 = synth.gaussians_ic(n, n, seed=seed)
    c, g = oracle.spectral_interval(fourier.spectral_radius(n, n, nu, a))
    h = mult * synth.cfl_step(n, n, nu, a)
    xi = oracle.leja_points(1000)
    out, it, st = oracle.leja_phi_mp(oracle.ADVDIFF, n, n, nu, a, None, l, u0, c, g, h, tol, tol, xi)
    delta = oracle.rounding_sensitivity(n, n, nu, a, l, u0, c, g, h, tol, tol, xi, ref=out)
    exact = fourier.phi_apply(l, n, n, nu, a, h, u0)
    e_exact = float(np.linalg.norm(out - exact) / np.linalg.norm(exact))
    return np.asarray(out), it, st, delta, e_exact


def batch_oracle(instances, l=0, tol=1e-10, mult=50, procs=None):
    """phi_l(h A) u0 by the oracle (mp divided differences) for every
    instance dict of synth.batch_instances, h = mult * dt_CFL and the
    symbol's spectral radius.  Returns, per instance, (out, iters, status,
    delta, e_exact): delta the oracle's rounding sensitivity
    (oracle.rounding_sensitivity), e_exact its relative L2 distance from the
    exact Fourier solution."""
    items = [(d["n"], d["nu"], d["a"], d["seed"], l, tol, mult) for d in instances]
    procs = procs or max(1, min(16, os.cpu_count() or 1))
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(procs) as pool:
        return pool.map(_batch_instance, items, chunksize=1)
