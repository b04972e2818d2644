"""GPU parity of the batched form: every instance against the oracle.

Instances of uneven sizes advance together in one launch per iteration; each
must give the oracle's result for its own problem (relative L2 <= 1e-10,
iterations +-1) and the oracle's status.  Advection-dominated instances
(4 nu n / a < 2, where the Newton basis grows geometrically) are judged by
the oracle with divided differences above binary128 precision
(oracle.leja_phi_mp), as is the full 256-instance batched workload."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def lx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_08344_gb300 as m

    return m


def _instances(sizes, seed):
    # diffusion-dominated draws (4 nu n / a >= 5), where the oracle's
    # binary128 coefficients resolve the converged series
    rng = np.random.default_rng(seed)
    out = []
    for n in sizes:
        nu = 10 ** rng.uniform(-2.5, -1.5)
        nmax = max(n)
        a = min(rng.uniform(0.0, 1.0), 4 * nu * nmax / 5.0)
        out.append((n[0], n[1], nu, a, int(rng.integers(1, 1000))))
    return out


def _symbol_radius(nx, ny, nu, a):
    import fourier

    return fourier.spectral_radius(nx, ny, nu, a)


@pytest.mark.parametrize("sizes", [
    [(64, 64), (128, 128), (192, 64), (64, 256), (128, 32), (256, 256), (64, 64), (128, 96)],   # wide kernel
    [(64, 64), (96, 80), (33, 45), (128, 128), (1, 7), (70, 70)],                               # generic kernel
])
def test_batch_matches_oracle(lx, sizes):
    inst = _instances(sizes, seed=len(sizes))
    inst.append((128, 128, 1e-3, 2.0, 5))  # advection-dominated (4 nu n / a = 0.26)
    xi = oracle.leja_points(1000)
    b = lx.batch_setup([(nx, ny, nu, a) for (nx, ny, nu, a, _) in inst])
    ws, outs, cs, gs, hs, refs = [], [], [], [], [], []
    for (nx, ny, nu, a, s) in inst:
        u0 = synth.gaussians_ic(nx, ny, seed=s)
        h = 50 * synth.cfl_step(nx, ny, nu, a) if nx > 1 else 1e-3
        c, g = oracle.spectral_interval(max(_symbol_radius(nx, ny, nu, a), 1.0))
        ws.append(torch.from_numpy(u0).cuda())
        outs.append(torch.empty(nx * ny, dtype=torch.float64, device="cuda"))
        cs.append(c)
        gs.append(g)
        hs.append(h)
        ref = oracle.leja_phi_mp(oracle.ADVDIFF, nx, ny, nu, a, None, 0, u0, c, g, h, TOL, TOL, xi)
        delta = oracle.rounding_sensitivity(nx, ny, nu, a, 0, u0, c, g, h, TOL, TOL, xi, ref=ref[0])
        import fourier

        exact = fourier.phi_apply(0, nx, ny, nu, a, h, u0)
        e_ex_o = float(np.linalg.norm(ref[0] - exact) / np.linalg.norm(exact))
        refs.append(ref + (delta, e_ex_o, exact))
    for rep in range(2):  # the second call reuses the cached coefficients
        st, its, sts = lx.batch_step(b, 0, ws, outs, cs, gs, hs, TOL, TOL)
        for k, (ref, it_o, st_o, delta, e_ex_o, exact) in enumerate(refs):
            check_instance("FP64", outs[k].cpu().numpy(), its[k], sts[k], ref, it_o, st_o, delta, e_ex_o, exact,
                           (rep, k))


# Float-float carries a 2^-48 unit roundoff against FP64's 2^-53.
DF64_ROUNDING = 32.0


def check_instance(prec, got, it, st, ref, it_o, st_o, delta, e_exact_o, exact, where):
    """The bar for one instance.  Where the problem amplifies rounding
    (delta, the oracle's own change under a regrouped stencil, above
    1e-11), agreement is held to a small multiple of delta -- no evaluation
    order of the method can do better; float-float, with its larger unit
    roundoff, may then also need more iterations before the stopping test
    sees the series converge."""
    assert st_o == 0 and st == 0, (where, st, st_o)
    u = DF64_ROUNDING if prec == "DF64" else 1.0
    bar = max(TOL, 4.0 * u * delta)
    e = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert e <= bar, (where, e, bar, delta)
    if u * delta <= 1e-11:
        assert abs(it - it_o) <= 1, (where, it, it_o)
    else:
        # the stopping test may see the series converge later (never
        # earlier), and the result stays as close to the exact Fourier
        # solution as the oracle's plus the rounding allowance
        assert it >= it_o - 1, (where, it, it_o)
        e_ex = float(np.linalg.norm(got - exact) / np.linalg.norm(exact))
        assert e_ex <= e_exact_o + 1.01 * bar, (where, e_ex, e_exact_o, bar)
    return e


@pytest.fixture(scope="module")
def config4_oracle():
    # the full batched workload: 256 instances, n in {128, ..., 1024}, nu
    # log-uniform in [1e-3, 1e-1], a uniform in [0, 2] (seed 7), exp(hA)u0
    # at h = 50 dt_CFL, each by the oracle with mp divided differences
    # (about a tenth of the instances are advection-dominated)
    import oracle_pool

    inst = synth.batch_instances(256, seed=7)
    return inst, oracle_pool.batch_oracle(inst, l=0, tol=TOL, mult=50)


@pytest.mark.parametrize("prec", ["FP64", "DF64"])
def test_full_config4_batch_matches_oracle(lx, config4_oracle, prec):
    import fourier

    inst, refs = config4_oracle
    probs = [(d["n"], d["n"], d["nu"], d["a"]) for d in inst]
    b = lx.batch_setup(probs, precision=getattr(lx, prec))
    ws, outs, cs, gs, hs = [], [], [], [], []
    for d in inst:
        n = d["n"]
        ws.append(torch.from_numpy(synth.gaussians_ic(n, n, seed=d["seed"])).cuda())
        outs.append(torch.empty(n * n, dtype=torch.float64, device="cuda"))
        c, g = lx.spectral_interval(_symbol_radius(n, n, d["nu"], d["a"]))
        cs.append(c)
        gs.append(g)
        hs.append(50 * synth.cfl_step(n, n, d["nu"], d["a"]))
    st, its, sts = lx.batch_step(b, 0, ws, outs, cs, gs, hs, TOL, TOL)
    worst, hard, loose = 0.0, 0, 0
    for k, (ref, it_o, st_o, delta, e_ex_o) in enumerate(refs):
        d = inst[k]
        exact = fourier.phi_apply(0, d["n"], d["n"], d["nu"], d["a"], hs[k], ws[k].cpu().numpy())
        e = check_instance(prec, outs[k].cpu().numpy(), its[k], sts[k], ref, it_o, st_o, delta, e_ex_o, exact,
                           (k, d))
        worst = max(worst, e)
        hard += 4 * d["nu"] * d["n"] < 2 * d["a"]
        loose += delta > 1e-11
    assert st == 0
    print(f"config-4 batch {prec}: 256 instances ({hard} with 4 nu n / a < 2, {loose} with rounding "
          f"sensitivity above 1e-11), worst rel_l2 vs oracle {worst:.2e}")
    b.close()


def test_batch_float_float_matches_oracle(lx):
    # float-float batch: every nx a multiple of 128, uneven sizes and
    # coefficients, each instance against the oracle
    sizes = [(128, 128), (256, 64), (128, 200), (384, 128), (128, 37), (256, 256)]
    inst = _instances(sizes, seed=11)
    xi = oracle.leja_points(1000)
    b = lx.batch_setup([(nx, ny, nu, a) for (nx, ny, nu, a, _) in inst], precision=lx.DF64)
    ws, outs, cs, gs, hs, u0s = [], [], [], [], [], []
    for (nx, ny, nu, a, s) in inst:
        u0 = synth.gaussians_ic(nx, ny, seed=s) * 10.0 ** (s % 7 - 3)  # magnitudes 1e-3 .. 1e3 per instance
        h = 50 * synth.cfl_step(nx, ny, nu, a)
        c, g = oracle.spectral_interval(max(_symbol_radius(nx, ny, nu, a), 1.0))
        ws.append(torch.from_numpy(u0).cuda())
        outs.append(torch.empty(nx * ny, dtype=torch.float64, device="cuda"))
        cs.append(c)
        gs.append(g)
        hs.append(h)
        u0s.append(u0)
    # two tolerances, so that instances stop after odd and even counts (the
    # float-float batch takes two Leja iterations per pass)
    parities = set()
    for tol in (TOL, 3e-9):
        refs = [oracle.leja_phi(oracle.ADVDIFF, nx, ny, nu, a, None, 1, u0, c, g, h, tol, 0.0, xi)
                for (nx, ny, nu, a, _), u0, c, g, h in zip(inst, u0s, cs, gs, hs)]
        for rep in range(2):
            st, its, sts = lx.batch_step(b, 1, ws, outs, cs, gs, hs, tol, 0.0)
            for k, (ref, it_o, st_o) in enumerate(refs):
                assert st_o == 0 and sts[k] == 0, (k, sts[k])
                assert abs(its[k] - it_o) <= 1, (k, its[k], it_o)
                got = outs[k].cpu().numpy()
                bar = TOL if its[k] == it_o else 100 * tol
                assert np.linalg.norm(got - ref) <= bar * np.linalg.norm(ref), k
                parities.add(its[k] % 2)
    assert parities == {0, 1}
    from paper_2310_08344_gb300 import LexgbError

    with pytest.raises(LexgbError):
        lx.batch_setup([(96, 96, 1e-2, 0.5)], precision=lx.DF64)  # nx % 128 != 0


def test_batch_host_loop_matches_graph(lx, monkeypatch):
    # the host-driven loop (for profilers) launches the same kernel as the
    # graph's while loop: identical results and iteration counts
    sizes = [(128, 128), (256, 64), (128, 37)]
    inst = _instances(sizes, seed=13)
    ws, cs, gs, hs = [], [], [], []
    for (nx, ny, nu, a, s) in inst:
        ws.append(torch.from_numpy(synth.gaussians_ic(nx, ny, seed=s)).cuda())
        hs.append(50 * synth.cfl_step(nx, ny, nu, a))
        c, g = oracle.spectral_interval(max(_symbol_radius(nx, ny, nu, a), 1.0))
        cs.append(c)
        gs.append(g)
    res = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("LEXGB_STREAM_LOOP", mode)
        for prec in (lx.FP64, lx.DF64):
            b = lx.batch_setup([(nx, ny, nu, a) for (nx, ny, nu, a, _) in inst], precision=prec)
            outs = [torch.empty(nx * ny, dtype=torch.float64, device="cuda") for (nx, ny, _, _, _) in inst]
            st, its, sts = lx.batch_step(b, 1, ws, outs, cs, gs, hs, TOL, 0.0)
            assert st == 0
            res[(mode, prec)] = (list(its), [o.cpu().numpy() for o in outs])
    for prec in (lx.FP64, lx.DF64):
        a_its, a_out = res[("0", prec)]
        b_its, b_out = res[("1", prec)]
        assert a_its == b_its
        for x, y in zip(a_out, b_out):
            assert np.array_equal(x, y)
