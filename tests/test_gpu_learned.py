"""What the learned step-size controller gains over the classical one.

Training samples come from the method itself (Burgers trajectories,
thirteen candidate steps per state from a quarter to sixteen times the
current one, label = the largest step whose error estimate stays below
0.8 tol).  The network is trained
on the GPU with the library's tensor-core kernels.  Then an unseen initial
state is integrated to the same end time with both controllers, once from a
well-chosen and once from a cautious first step; the embedded error test
accepts or rejects every step in all runs.  Reported: Leja
iterations (the paper's cost proxy), attempts, rejections and the error of
the final state against a tight-tolerance reference."""
import math
import time

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_08344_gb300 as m

    return m


def test_learned_controller_gain(lx):
    from paper_2310_08344_gb300 import learned

    n, nu, tol, leja_tol = 96, 2e-2, 1e-4, 1e-10
    rng = np.random.default_rng(11)
    v0 = torch.from_numpy(synth.power_start(n * n, seed=5)).cuda()
    ics = [torch.from_numpy(synth.burgers_ic(n, n, seed=100 + k)).cuda() for k in range(24)]
    dt = synth.cfl_step(n, n, nu, 1.0)
    t0 = time.perf_counter()
    X, Y = learned.generate_samples(n, nu, ics, v0, tol, leja_tol, 40, dt, rng)
    t_gen = time.perf_counter() - t0
    assert X.shape[0] >= 800 and np.all(np.isfinite(X)) and np.all(np.isfinite(Y))
    model, norm, losses = learned.train(X, Y, epochs=300, batch=256, lr=2e-3, seed=0)
    assert losses[-1] < losses[0]

    u0 = synth.burgers_ic(n, n, seed=12)
    T = 1500 * dt  # tens of controlled steps
    ctx = lx.leja_setup(n, n, nu, 0.0, lx.BURGERS, lx.FP64, lx.EXPRB32)
    ref = torch.from_numpy(u0).cuda()
    st, info_ref = lx.lx_integrate(ctx, ref, v0, T, 1e-9, leja_tol, 100000, 0.0, 3 * dt, 10)
    assert st == 0 and abs(info_ref["t"] - T) <= 1e-12 * T
    print(f"\nsamples {X.shape[0]} (generated in {t_gen:.1f} s), final loss {losses[-1]:.4f}")
    # two first steps: a well-chosen one (25 dt_CFL) and a cautious one (dt_CFL)
    for h0 in (25 * dt, dt):
        runs = {}
        for name in ("classical", "learned"):
            u = torch.from_numpy(u0).cuda()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            if name == "classical":
                st, info = lx.lx_integrate(ctx, u, v0, T, tol, leja_tol, 100000, 0.0, h0, 10)
            else:
                st, info = lx.lx_integrate_learned(ctx, u, v0, T, tol, leja_tol, model, dt, 100000, 0.0, h0, 10)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t1
            assert st == 0 and abs(info["t"] - T) <= 1e-12 * T
            err = float((u - ref).norm().item() / ref.norm().item())
            runs[name] = dict(info, wall=wall, err=err)
        c, l = runs["classical"], runs["learned"]
        gain_iters = c["leja_iters"] / l["leja_iters"]
        gain_wall = c["wall"] / l["wall"]
        print(f"first step {h0 / dt:.0f} dt_CFL:")
        for k, v in runs.items():
            print(f"  {k:9s}: steps {v['steps']:4d} rejected {v['rejected']:3d} leja_iters {v['leja_iters']:6d} "
                  f"wall {v['wall']*1e3:8.1f} ms  rel err vs reference {v['err']:.2e}")
        print(f"  gain (classical / learned): Leja iterations {gain_iters:.3f}, wall time {gain_wall:.3f}")
        # the same accuracy class: the learned run's error stays within a few times the classical one
        assert l["err"] <= max(3.0 * c["err"], 10 * tol)
        assert c["steps"] >= 20
        # and it does not cost much more than the classical controller
        assert gain_iters >= 0.8
