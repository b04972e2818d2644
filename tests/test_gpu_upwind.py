"""GPU parity on the paper's own discretisation (periodic [-1,1)^2, central
Laplacian, third-order upwind gradient): the diffusion-advection problems
with and without a source (the paper's Problems I and II) and the flux-form
Burgers problem (Problem III), against the oracle on the same inputs.
Bar: relative L2 <= 1e-10 and the same Leja iteration count +-1 (FP64 and
float-float); the mixed form is held to 1e-5 and reported.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10
NU, A = 1.0, 10.0  # the paper's Problems I-III: diffusion 1, advection / flux coefficient 10


@pytest.fixture(scope="module")
def lx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_08344_gb300 as m

    return m


@pytest.fixture(scope="module")
def xi_oracle():
    return oracle.leja_points(1000)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _interval(kind, nx, ny, a, u):
    rho, _, _ = oracle.power_iteration(kind, nx, ny, NU, a, u, synth.power_start(nx * ny, 5), 10)
    return oracle.spectral_interval(rho)


@pytest.mark.parametrize("prec", ["FP64", "MIXED", "DF64"])
@pytest.mark.parametrize("nx,ny", [(64, 64), (96, 50), (128, 128)])
@pytest.mark.parametrize("a", [A, -4.0])
def test_phi_advdiff_up3(lx, xi_oracle, prec, nx, ny, a):
    u0 = synth.problem1_ic(nx, ny, seed=3)
    h = 50 * synth.cfl_step_pm1(nx, ny, NU, a)
    c, g = _interval(oracle.ADVDIFF_UP3, nx, ny, a, None)
    ctx = lx.leja_setup(nx, ny, NU, a, lx.ADVDIFF_UP3, getattr(lx, prec))
    out = torch.empty(nx * ny, dtype=torch.float64, device="cuda")
    for l in (0, 1):
        st, it = lx.phi_l_apply(ctx, l, None, dev(u0), out, c, g, h, TOL, TOL)
        ref, it_o, st_o = oracle.leja_phi(oracle.ADVDIFF_UP3, nx, ny, NU, a, None, l, u0, c, g, h, TOL, TOL, xi_oracle)
        assert st == 0 and st_o == 0
        e = rel(out.cpu().numpy(), ref)
        if prec == "MIXED":
            print(f"mixed up3 {nx}x{ny} l={l}: rel_l2 vs FP64 oracle {e:.3e}")
            assert e <= 1e-5 and abs(it - it_o) <= 3
        else:
            assert e <= TOL and abs(it - it_o) <= 1


@pytest.mark.parametrize("prec,nx,ny", [("FP64", 64, 64), ("FP64", 80, 48), ("MIXED", 64, 64), ("MIXED", 80, 48),
                                        ("DF64", 128, 128), ("DF64", 256, 72)])
def test_phi_burgers_up3(lx, xi_oracle, prec, nx, ny):
    u = synth.problem3_ic(nx, ny, seed=4)
    w = synth.random_field(nx * ny, seed=5)
    h = 30 * synth.cfl_step_pm1(nx, ny, NU, A * np.abs(u).max())
    c, g = _interval(oracle.BURGERS_UP3, nx, ny, A, u)
    ctx = lx.leja_setup(nx, ny, NU, A, lx.BURGERS_UP3, getattr(lx, prec))
    out = torch.empty(nx * ny, dtype=torch.float64, device="cuda")
    st, it = lx.phi_l_apply(ctx, 1, dev(u), dev(w), out, c, g, h, TOL, TOL)
    ref, it_o, st_o = oracle.leja_phi(oracle.BURGERS_UP3, nx, ny, NU, A, u, 1, w, c, g, h, TOL, TOL, xi_oracle)
    assert st == 0 and st_o == 0
    bar = 1e-5 if prec == "MIXED" else TOL
    assert rel(out.cpu().numpy(), ref) <= bar and abs(it - it_o) <= (3 if prec == "MIXED" else 1)


@pytest.mark.parametrize("kind", [2, 3])
@pytest.mark.parametrize("prec", ["FP64", "DF64"])
@pytest.mark.parametrize("nx,ny,a", [(128, 64, A), (256, 100, A), (256, 100, -4.0)])
def test_power_bound_up3(lx, kind, prec, nx, ny, a):
    # (the float-float Burgers passes run the pipelined product-form kernel:
    # two column strips and a ragged row range on the larger grid)
    u = synth.problem3_ic(nx, ny, seed=6) * np.sign(a) if kind == 3 else None
    v0 = synth.power_start(nx * ny, 5)
    ctx = lx.leja_setup(nx, ny, NU, a, kind, getattr(lx, prec))
    st, rho, it = lx.power_bound(ctx, dev(u) if u is not None else None, dev(v0), 10)
    rho_o, it_o, st_o = oracle.power_iteration(kind, nx, ny, NU, a, u, v0, 10)
    assert st == 0 and st_o == 0 and it == it_o
    assert abs(rho - rho_o) <= 1e-12 * rho_o


@pytest.mark.parametrize("kind,integ,prec,source", [(2, 0, "FP64", False), (2, 0, "FP64", True), (2, 0, "DF64", True),
                                                    (2, 1, "DF64", False), (3, 0, "FP64", False),
                                                    (3, 1, "FP64", False), (3, 1, "FP64", True), (3, 1, "DF64", False),
                                                    (3, 0, "DF64", True)])
def test_expint_step_up3(lx, xi_oracle, kind, integ, prec, source):
    # Problem I (Ros-Eu), Problem II (with the paper's source), Problem III
    # (EXPRB32, with and without a source)
    n = 128 if prec == "DF64" else 64
    if kind == 2:
        u = synth.problem1_ic(n, n)
        h = 50 * synth.cfl_step_pm1(n, n, NU, A)
    else:
        u = synth.problem3_ic(n, n)
        h = 30 * synth.cfl_step_pm1(n, n, NU, A * np.abs(u).max())
    S = synth.problem2_source(n, n) if source else None
    c, g = _interval(kind, n, n, A, u if kind == 3 else None)
    ctx = lx.leja_setup(n, n, NU, A, kind, getattr(lx, prec), integ)
    if source:
        Sd = dev(S)
        assert lx.lx_ctx_set_source(ctx, Sd) == 0
    lo = torch.empty(n * n, dtype=torch.float64, device="cuda")
    hi = torch.empty(n * n, dtype=torch.float64, device="cuda")
    st, err, it = lx.expint_step(ctx, dev(u), lo, hi, c, g, h, TOL, TOL)
    if integ == 0:
        ref, it_o, st_o = oracle.ros_eu(kind, n, n, NU, A, u, c, g, h, TOL, TOL, xi_oracle, source=S)
        assert st == 0 and st_o == 0 and abs(it - it_o) <= 1
        assert rel(hi.cpu().numpy(), ref) <= TOL
    else:
        rlo, rhi, rerr, it_o, st_o = oracle.exprb32(kind, n, n, NU, A, u, c, g, h, TOL, TOL, xi_oracle, source=S)
        assert st == 0 and st_o == 0 and abs(it - it_o) <= 2
        assert rel(lo.cpu().numpy(), rlo) <= TOL and rel(hi.cpu().numpy(), rhi) <= TOL
        if kind == 2:
            assert err <= 1e-14 and rerr <= 1e-14
        else:
            assert abs(err - rerr) <= 1e-6 * rerr


def test_up3_forms_not_offered(lx):
    from paper_2310_08344_gb300 import LexgbError

    with pytest.raises(LexgbError):
        lx.leja_setup(96, 96, NU, A, lx.BURGERS_UP3, lx.DF64)  # float-float Burgers needs nx % 128 == 0


@pytest.mark.parametrize("kind,prec,nx,ny", [(2, "FP64", 64, 64), (2, "FP64", 96, 50), (2, "MIXED", 64, 64),
                                             (2, "DF64", 96, 50), (2, "DF64", 128, 64), (3, "FP64", 80, 48),
                                             (3, "DF64", 128, 64), (3, "MIXED", 64, 64)])
@pytest.mark.parametrize("alphas", [[1.0], [0.25, 0.5, 0.75, 1.0], [0.5, 1.0, 0.3]])
def test_phi_vertical_up3(lx, xi_oracle, kind, prec, nx, ny, alphas):
    # several phi_1(alpha_j h Op) w from one Newton basis on the paper's
    # discretisation, against the oracle's vertical loop (same stop rule)
    if kind == 2:
        u = None
        w = synth.problem1_ic(nx, ny, seed=11)
        h = 50 * synth.cfl_step_pm1(nx, ny, NU, A)
    else:
        u = synth.problem3_ic(nx, ny, seed=12)
        w = synth.random_field(nx * ny, seed=13)
        h = 30 * synth.cfl_step_pm1(nx, ny, NU, A * np.abs(u).max())
    c, g = _interval(kind, nx, ny, A, u)
    ctx = lx.leja_setup(nx, ny, NU, A, kind, getattr(lx, prec))
    outs = [torch.empty(nx * ny, dtype=torch.float64, device="cuda") for _ in alphas]
    st, it = lx.phi_l_apply_vertical(ctx, 1, alphas, dev(u) if u is not None else None, dev(w), outs, c, g, h,
                                     TOL, TOL)
    ref, it_o, st_o = oracle.leja_phi_vertical(kind, nx, ny, NU, A, u, 1, alphas, w, c, g, h, TOL, TOL, xi_oracle)
    assert st == 0 and st_o == 0
    bar, dit = (1e-5, 3) if prec == "MIXED" else (TOL, 1)
    assert abs(it - it_o) <= dit
    for j in range(len(alphas)):
        assert rel(outs[j].cpu().numpy(), ref[j]) <= bar


@pytest.mark.parametrize("name,strip_h", [("leja_iter_df_pipe_up3_b3", 0), ("leja_iter_df_pipe_up3_b3", 8),
                                          ("leja_iter_df_pipe_up3_b2", 32), ("leja_iter_df_up3", 8),
                                          ("leja_iter_df_pipe2_up3_b3", 0), ("leja_iter_df_pipe2_up3_b3", 8),
                                          ("leja_iter_df_pipe2_up3_b3", 32), ("leja_iter_df_pipe2_up3_b2", 0),
                                          ("leja_iter_df_pipe2_up3_b4", 0), ("leja_iter_df_pipe2x_up3_b3", 0),
                                          ("leja_iter_df_pipe2x_up3_b3", 8), ("leja_iter_df_pipe2x_up3_b3", 40),
                                          ("leja_iter_df_pipe2x_up3_b3_s5", 0)])
@pytest.mark.parametrize("a", [A, -4.0])
def test_df64_up3_candidates(lx, xi_oracle, name, strip_h, a):
    # every float-float candidate of the upwind operator on a grid with two
    # column strips and a ragged row range, both upwind sides
    nx, ny = 256, 100
    u0 = synth.problem1_ic(nx, ny, seed=7)
    h = 40 * synth.cfl_step_pm1(nx, ny, NU, a)
    c, g = _interval(oracle.ADVDIFF_UP3, nx, ny, a, None)
    ctx = lx.leja_setup(nx, ny, NU, a, lx.ADVDIFF_UP3, lx.DF64)
    assert lx.lx_ctx_select_kernel(ctx, name, strip_h) == 0
    out = torch.empty(nx * ny, dtype=torch.float64, device="cuda")
    st, it = lx.phi_l_apply(ctx, 1, None, dev(u0), out, c, g, h, TOL, TOL)
    ref, it_o, st_o = oracle.leja_phi(oracle.ADVDIFF_UP3, nx, ny, NU, a, None, 1, u0, c, g, h, TOL, TOL, xi_oracle)
    assert st == 0 and st_o == 0 and abs(it - it_o) <= 1
    assert rel(out.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("name,strip_h", [("leja_iter_df_pipe_burgers_up3_b2", 0), ("leja_iter_df_pipe_burgers_up3_b2", 8),
                                          ("leja_iter_df_pipe_burgers_up3_b1", 32),
                                          ("leja_iter_df_pipe_burgers_up3z_b3", 0),
                                          ("leja_iter_df_pipe_burgers_up3z_b3", 8),
                                          ("leja_iter_df_pipe_burgers_up3z_b3", 128),
                                          ("leja_iter_df_pipe_burgers_up3z_b2", 0),
                                          ("leja_iter_df_pipe_burgers_up3z_b2", 32)])
@pytest.mark.parametrize("a", [A, -4.0])
def test_df64_burgers_up3_candidates(lx, xi_oracle, name, strip_h, a):
    nx, ny = 256, 100
    u = synth.problem3_ic(nx, ny, seed=9) * np.sign(a)  # keep a u > 0 (the upwind side follows sign(a))
    w = synth.random_field(nx * ny, seed=10)
    h = 30 * synth.cfl_step_pm1(nx, ny, NU, abs(a) * np.abs(u).max())
    c, g = _interval(oracle.BURGERS_UP3, nx, ny, a, u)
    ctx = lx.leja_setup(nx, ny, NU, a, lx.BURGERS_UP3, lx.DF64)
    assert lx.lx_ctx_select_kernel(ctx, name, strip_h) == 0
    out = torch.empty(nx * ny, dtype=torch.float64, device="cuda")
    st, it = lx.phi_l_apply(ctx, 3, dev(u), dev(w), out, c, g, h, TOL, TOL)
    ref, it_o, st_o = oracle.leja_phi(oracle.BURGERS_UP3, nx, ny, NU, a, u, 3, w, c, g, h, TOL, TOL, xi_oracle)
    assert st == 0 and st_o == 0 and abs(it - it_o) <= 1
    assert rel(out.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("name", ["leja_iter_df_pipe_burgers_up3z_b3", "leja_iter_df_pipe_burgers_up3z_b2"])
@pytest.mark.parametrize("strip_h", [0, 8])
@pytest.mark.parametrize("a", [A, -4.0])
def test_df64_burgers_up3_square_form(lx, xi_oracle, name, strip_h, a):
    # square grid: the product form's six-term stencil (pair sums of y and z
    # along x and y, two of them carried from the row before) in the Leja
    # loop after its first launch, and in the power passes after the first;
    # both upwind sides
    nx = ny = 256
    u = synth.problem3_ic(nx, ny, seed=9) * np.sign(a)
    w = synth.random_field(nx * ny, seed=10)
    h = 30 * synth.cfl_step_pm1(nx, ny, NU, abs(a) * np.abs(u).max())
    v0 = synth.power_start(nx * ny, seed=5)
    rho, passes, st = oracle.power_iteration(oracle.BURGERS_UP3, nx, ny, NU, a, u, v0, 10)
    assert st == 0
    c, g = oracle.spectral_interval(rho)
    ctx = lx.leja_setup(nx, ny, NU, a, lx.BURGERS_UP3, lx.DF64)
    assert lx.lx_ctx_select_kernel(ctx, name, strip_h) == 0
    st, rho_g, passes_g = lx.power_bound(ctx, dev(u), dev(v0), 10)
    assert st == 0 and passes_g == passes and abs(rho_g - rho) <= 1e-12 * rho
    out = torch.empty(nx * ny, dtype=torch.float64, device="cuda")
    st, it = lx.phi_l_apply(ctx, 1, dev(u), dev(w), out, c, g, h, TOL, TOL)
    ref, it_o, st_o = oracle.leja_phi(oracle.BURGERS_UP3, nx, ny, NU, a, u, 1, w, c, g, h, TOL, TOL, xi_oracle)
    assert st == 0 and st_o == 0 and abs(it - it_o) <= 1
    assert rel(out.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("name", ["leja_iter_df_pipe2x_up3_b3", "leja_iter_df_pipe2x_up3_b3_s5"])
@pytest.mark.parametrize("n", [256, 384])
@pytest.mark.parametrize("strip_h", [0, 8, 40])
@pytest.mark.parametrize("tol", [1e-10, 1e-7])
@pytest.mark.parametrize("a", [A, -4.0])
def test_df64_up3_lean_square(lx, xi_oracle, name, n, strip_h, tol, a):
    # the issue-lean two-step kernel on square grids: pair sums of the x and
    # y neighbours with the (-s) pair carried along the walk, the three halo
    # columns 16 output rows at a time (segments of 8 and 40 rows cut chunks
    # short), both upwind sides, stops after odd and even counts
    u0 = synth.problem1_ic(n, n, seed=17)
    h = 40 * synth.cfl_step_pm1(n, n, NU, a)
    c, g = _interval(oracle.ADVDIFF_UP3, n, n, a, None)
    ctx = lx.leja_setup(n, n, NU, a, lx.ADVDIFF_UP3, lx.DF64)
    assert lx.lx_ctx_select_kernel(ctx, name, strip_h) == 0
    out = torch.empty(n * n, dtype=torch.float64, device="cuda")
    for l in (0, 1):
        st, it = lx.phi_l_apply(ctx, l, None, dev(u0), out, c, g, h, tol, tol)
        ref, it_o, st_o = oracle.leja_phi(oracle.ADVDIFF_UP3, n, n, NU, a, None, l, u0, c, g, h, tol, tol, xi_oracle)
        assert st == 0 and st_o == 0 and abs(it - it_o) <= 1
        bar = 1e-10 if it == it_o else 100 * tol
        assert rel(out.cpu().numpy(), ref) <= bar


@pytest.mark.parametrize("name", ["leja_iter_df_pipe2_up3_b3", "leja_iter_df_pipe_up3_b3",
                                  "leja_iter_df_pipe2x_up3_b3"])
@pytest.mark.parametrize("tol", [1e-10, 3e-9, 1e-7, 1e-5])
@pytest.mark.parametrize("a", [A, -4.0])
def test_df64_up3_two_step_stop_parities(lx, xi_oracle, name, tol, a):
    # the two-step kernel tests the stop after each of its two iterations;
    # several tolerances give odd and even counts, and an odd stop must
    # return p_{m+1} (the output pass removes the extra term)
    nx, ny = 128, 72
    u0 = synth.problem1_ic(nx, ny, seed=17)
    h = 40 * synth.cfl_step_pm1(nx, ny, NU, a)
    c, g = _interval(oracle.ADVDIFF_UP3, nx, ny, a, None)
    ctx = lx.leja_setup(nx, ny, NU, a, lx.ADVDIFF_UP3, lx.DF64)
    assert lx.lx_ctx_select_kernel(ctx, name, 0) == 0
    out = torch.empty(nx * ny, dtype=torch.float64, device="cuda")
    for l in (0, 1):
        st, it = lx.phi_l_apply(ctx, l, None, dev(u0), out, c, g, h, tol, tol)
        ref, it_o, st_o = oracle.leja_phi(oracle.ADVDIFF_UP3, nx, ny, NU, a, None, l, u0, c, g, h, tol, tol,
                                          xi_oracle)
        assert st == 0 and st_o == 0 and abs(it - it_o) <= 1
        bar = 1e-10 if it == it_o else 100 * tol
        assert rel(out.cpu().numpy(), ref) <= bar


def test_full_size_problem1_exact(lx):
    # Problem I at 4096^2 with the paper's tolerance and step (100 dt_CFL),
    # default kernel (two Leja iterations per pass): exp(hA)u against the
    # exact Fourier solution of the discrete operator
    from fourier import phi_apply_symbol, symbol_up3

    n = 4096
    u0 = synth.problem1_ic(n, n)
    lam = symbol_up3(n, n, NU, A)
    c, g = oracle.spectral_interval(float(np.abs(lam).max()))
    h = 100 * synth.cfl_step_pm1(n, n, NU, A)
    ctx = lx.leja_setup(n, n, NU, A, lx.ADVDIFF_UP3, lx.DF64)
    out = torch.empty(n * n, dtype=torch.float64, device="cuda")
    st, it = lx.phi_l_apply(ctx, 0, None, dev(u0), out, c, g, h, 1e-12, 1e-12)
    assert st == 0
    e = rel(out.cpu().numpy(), phi_apply_symbol(0, lam, h, u0, n, n))
    print(f"Problem I 4096^2: {lx.lx_ctx_kernel_name(ctx)}, iters {it}, rel_l2 vs exact {e:.3e}")
    assert e <= 1e-9


def test_full_size_problem3_properties(lx):
    # Problem III at 4096^2, one EXPRB32 step of 100 dt_CFL at tol 1e-12:
    # the flux form conserves the mean exactly (1^T J = 0 and sum R = 0), and
    # the float-float and FP64 paths (independent kernels) agree
    n = 4096
    u0 = synth.problem3_ic(n, n)
    v0 = synth.power_start(n * n, seed=5)
    h = 100 * synth.cfl_step_pm1(n, n, NU, A * np.abs(u0).max())
    res = {}
    for prec in ("DF64", "FP64"):
        ctx = lx.leja_setup(n, n, NU, A, lx.BURGERS_UP3, getattr(lx, prec), lx.EXPRB32)
        ud = dev(u0)
        st, rho, _ = lx.power_bound(ctx, ud, dev(v0), 10)
        assert st == 0
        c, g = lx.spectral_interval(rho)
        lo, hi = torch.empty_like(ud), torch.empty_like(ud)
        st, err, it = lx.expint_step(ctx, ud, lo, hi, c, g, h, 1e-12, 1e-12)
        assert st == 0
        res[prec] = (lo.cpu().numpy(), hi.cpu().numpy(), err, it)
        del ctx
    lo, hi, err, it = res["DF64"]
    assert abs(hi.mean() - u0.mean()) <= 1e-12 * np.abs(u0).max()
    assert abs(lo.mean() - u0.mean()) <= 1e-12 * np.abs(u0).max()
    assert rel(hi, res["FP64"][1]) <= 1e-10 and rel(lo, res["FP64"][0]) <= 1e-10
    assert abs(it - res["FP64"][3]) <= 2 and abs(err - res["FP64"][2]) <= 1e-6 * res["FP64"][2] + 1e-15
    print(f"Problem III 4096^2: iters {it}, err {err:.3e}, df64 vs FP64 {rel(hi, res['FP64'][1]):.2e}")


@pytest.mark.parametrize("scale", [1.0, 1e100, 1e-100])
@pytest.mark.parametrize("source", [False, True])
def test_df64_ros_eu_up3_rhs_forms(lx, xi_oracle, scale, source):
    # the float-float right-hand side of the upwind Rosenbrock-Euler step
    # (values beyond the float-float range take the FP64 formula; the loop
    # input is scaled by a power of two) against the oracle, on grids with a
    # ragged row count and two column strips
    nx, ny = 256, 72
    u = synth.problem1_ic(nx, ny, seed=19) * scale
    S = synth.problem2_source(nx, ny) * scale if source else None
    h = 50 * synth.cfl_step_pm1(nx, ny, NU, A)
    c, g = _interval(2, nx, ny, A, None)
    ctx = lx.leja_setup(nx, ny, NU, A, lx.ADVDIFF_UP3, lx.DF64, lx.ROS_EU)
    if source:
        Sd = dev(S)
        assert lx.lx_ctx_set_source(ctx, Sd) == 0
    hi = torch.empty(nx * ny, dtype=torch.float64, device="cuda")
    st, err, it = lx.expint_step(ctx, dev(u), None, hi, c, g, h, TOL, TOL * scale)
    ref, it_o, st_o = oracle.ros_eu(2, nx, ny, NU, A, u, c, g, h, TOL, TOL * scale, xi_oracle, source=S)
    assert st == 0 and st_o == 0 and abs(it - it_o) <= 1
    assert rel(hi.cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("integ", [0, 1])
@pytest.mark.parametrize("source", [False, True])
def test_df64_burgers_up3_rhs_ranges(lx, xi_oracle, integ, source):
    # the float-float right-hand side and EXPRB32 remainder of the upwind
    # Burgers step on a state with sign changes, exact zeros and values below
    # the float-float range (their neighbourhoods take the FP64 formula),
    # against the oracle on a grid with a ragged row count (the float-float
    # Burgers form needs nx % 128 == 0)
    nx, ny = 256, 72
    u = synth.problem3_ic(nx, ny, seed=23) - 2.0
    u[::97] = 0.0
    u[5::131] = 1e-25
    u[11::173] = -3e-17
    S = synth.problem2_source(nx, ny) if source else None
    h = 30 * synth.cfl_step_pm1(nx, ny, NU, A * np.abs(u).max())
    c, g = _interval(3, nx, ny, A, u)
    ctx = lx.leja_setup(nx, ny, NU, A, lx.BURGERS_UP3, lx.DF64, integ)
    if source:
        Sd = dev(S)
        assert lx.lx_ctx_set_source(ctx, Sd) == 0
    lo = torch.empty(nx * ny, dtype=torch.float64, device="cuda")
    hi = torch.empty(nx * ny, dtype=torch.float64, device="cuda")
    st, err, it = lx.expint_step(ctx, dev(u), lo, hi, c, g, h, TOL, TOL)
    if integ == 0:
        ref, it_o, st_o = oracle.ros_eu(3, nx, ny, NU, A, u, c, g, h, TOL, TOL, xi_oracle, source=S)
        assert st == 0 and st_o == 0 and abs(it - it_o) <= 1
        assert rel(hi.cpu().numpy(), ref) <= TOL
    else:
        rlo, rhi, rerr, it_o, st_o = oracle.exprb32(3, nx, ny, NU, A, u, c, g, h, TOL, TOL, xi_oracle, source=S)
        assert st == 0 and st_o == 0 and abs(it - it_o) <= 2
        assert rel(lo.cpu().numpy(), rlo) <= TOL and rel(hi.cpu().numpy(), rhi) <= TOL
        assert abs(err - rerr) <= 1e-6 * rerr
