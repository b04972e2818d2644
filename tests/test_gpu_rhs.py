"""GPU parity of the unfused form: a caller's right-hand side (Sec. 2) with
the Jacobian action by central finite differences (Sec. 2.3), against the
oracle's finite-difference form on the same inputs and difference step.

Bars.  With eps0 = 1e-2 the central quotient of the at most quadratic
problem right-hand sides is exact up to rounding amplified by
2^-53 / eps0 ~ 1e-14, so the FP64 bar of the fused path holds: relative L2
<= 1e-10, iterations +-1.  At the default eps0 = 2^-18 the quotient
amplifies the rounding of f by 1/e: the engine's f and the oracle's f round
differently (summation order of the stencil), and the two sides differ by
about C 2^-53 / eps0 with C the ratio of the stencil terms' magnitudes to
the result (measured on the CPU between two implementations of the same f:
up to 1.6e-10 on 64^2).  That bar is 100 * 2^-53 / eps0 = 2.9e-9.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10
EPS0_DEFAULT = 2.0 ** -18
BAR_DEFAULT = 100 * 2.0 ** -53 / EPS0_DEFAULT

# (kind, nx, ny, nu, a): the central problems on the unit square and the
# paper's upwind problems on [-1,1)^2 (Problems I and III coefficients)
PROBLEMS = [(0, 64, 64, 1e-2, 1.0), (1, 64, 48, 5e-3, 0.0), (2, 64, 64, 1.0, 10.0), (3, 64, 64, 1.0, 10.0),
            (2, 96, 50, 1.0, -4.0)]


@pytest.fixture(scope="module")
def lx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_08344_gb300 as m

    return m


@pytest.fixture(scope="module")
def xi():
    return oracle.leja_points(1000)


def bp(prob):
    """(kind, nx, ny, nu, a) -> the binding's problem tuple (nx, ny, nu, a, kind)."""
    kind, nx, ny, nu, a = prob
    return (nx, ny, nu, a, kind)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _state(kind, nx, ny, nu, a):
    if kind in (0, 2):
        u = synth.gaussians_ic(nx, ny, seed=1) if kind == 0 else synth.problem1_ic(nx, ny, seed=1)
        return u, None
    u = synth.burgers_ic(nx, ny, seed=2) if kind == 1 else synth.problem3_ic(nx, ny, seed=2)
    return u, u


def _step(kind, nx, ny, nu, a, u):
    if kind == 0:
        return 50 * synth.cfl_step(nx, ny, nu, a)
    if kind == 1:
        return 50 * synth.cfl_step(nx, ny, nu, np.abs(u).max())
    if kind == 2:
        return 50 * synth.cfl_step_pm1(nx, ny, nu, abs(a))
    return 30 * synth.cfl_step_pm1(nx, ny, nu, abs(a) * np.abs(u).max())


def _oracle_f(kind, nx, ny, nu, a, x):
    if kind == 0:
        return oracle.apply_advdiff(nx, ny, nu, a, x)
    if kind == 1:
        return oracle.burgers_f(nx, ny, nu, x)
    if kind == 2:
        return oracle.apply_advdiff_up3(nx, ny, nu, a, x)
    return oracle.burgers_up3_f(nx, ny, nu, a, x)


@pytest.mark.parametrize("prob", PROBLEMS + [(3, 80, 40, 1.0, -3.0)])
def test_rhs_builtin_matches_oracle(lx, prob):
    kind, nx, ny, nu, a = prob
    x = synth.problem3_ic(nx, ny, seed=3) + 0.1 * synth.random_field(nx * ny, seed=4)
    out = torch.empty(nx * ny, dtype=torch.float64, device="cuda")
    assert lx.lx_rhs_builtin(bp(prob), dev(x), out) == 0
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), _oracle_f(kind, nx, ny, nu, a, x)) <= 1e-13


@pytest.mark.parametrize("prob", PROBLEMS)
@pytest.mark.parametrize("eps0", [1e-2, EPS0_DEFAULT])
def test_phi_rhs_builtin(lx, xi, prob, eps0):
    kind, nx, ny, nu, a = prob
    n = nx * ny
    u, lin = _state(kind, nx, ny, nu, a)
    rho, _, _ = oracle.power_iteration(kind, nx, ny, nu, a, lin, synth.power_start(n, 5), 10)
    c, g = oracle.spectral_interval(rho)
    h = _step(kind, nx, ny, nu, a, u)
    w = h * _oracle_f(kind, nx, ny, nu, a, u)
    ctx = lx.leja_setup_rhs(n, problem=bp(prob), eps0=eps0)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    bar = TOL if eps0 == 1e-2 else BAR_DEFAULT
    for l in (0, 1, 3):
        st, it = lx.phi_l_apply_rhs(ctx, l, dev(u), dev(w), out, c, g, h, TOL, TOL)
        ref, it_o, st_o = oracle.leja_phi_fd(kind, nx, ny, nu, a, u, l, w, c, g, h, TOL, TOL, xi, eps0=eps0)
        assert st == 0 and st_o == 0
        assert abs(it - it_o) <= 1
        assert rel(out.cpu().numpy(), ref) <= bar


def test_phi_rhs_torch_callback_nonpolynomial(lx, xi):
    # a right-hand side the engine knows nothing about, written with torch
    # operations: f(u) = nu Lap u - sin u (J symmetric negative definite for
    # 0 <= u <= 1); the oracle runs the same f written with numpy
    nx = ny = 64
    nu = 1e-2
    n = nx * ny

    def f_torch(x, out):
        X = x.view(ny, nx)
        L = (torch.roll(X, 1, 1) + torch.roll(X, -1, 1) - 2 * X) * (nx * nx) + \
            (torch.roll(X, 1, 0) + torch.roll(X, -1, 0) - 2 * X) * (ny * ny)
        out.copy_((nu * L - torch.sin(X)).view(-1))

    def f_np(x):
        X = x.reshape(ny, nx)
        L = (np.roll(X, 1, 1) + np.roll(X, -1, 1) - 2 * X) * (nx * nx) + \
            (np.roll(X, 1, 0) + np.roll(X, -1, 0) - 2 * X) * (ny * ny)
        return (nu * L - np.sin(X)).reshape(-1)

    u = synth.gaussians_ic(nx, ny, seed=5)
    w = synth.random_field(n, seed=6)
    rho, _, st_o = oracle.power_iteration_fd(0, nx, ny, 0, 0, u, synth.power_start(n, 5), 10, rhs=f_np)
    assert st_o == 0
    ctx = lx.leja_setup_rhs(n, f=f_torch)
    st, rho_g, pit = lx.power_bound_rhs(ctx, dev(u), dev(synth.power_start(n, 5)), 10)
    assert st == 0 and abs(rho_g - rho) <= 1e-6 * rho
    c, g = oracle.spectral_interval(rho)
    h = 50 * synth.cfl_step(nx, ny, nu, 1.0)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    st, it = lx.phi_l_apply_rhs(ctx, 1, dev(u), dev(w), out, c, g, h, TOL, TOL)
    ref, it_o, st_o = oracle.leja_phi_fd(0, nx, ny, 0, 0, u, 1, w, c, g, h, TOL, TOL, xi, rhs=f_np)
    assert st == 0 and st_o == 0 and abs(it - it_o) <= 1
    assert rel(out.cpu().numpy(), ref) <= BAR_DEFAULT
    stats = lx.lx_rhs_ctx_stats(ctx)
    assert stats["leja_iterations"] == it and stats["rhs_calls"] >= 2 * it


@pytest.mark.parametrize("prob", [PROBLEMS[1], PROBLEMS[3]])
@pytest.mark.parametrize("with_u", [True, False])
def test_power_bound_rhs(lx, prob, with_u):
    kind, nx, ny, nu, a = prob
    n = nx * ny
    u, _ = _state(kind, nx, ny, nu, a)
    uu = u if with_u else None
    v0 = synth.power_start(n, 7)
    ctx = lx.leja_setup_rhs(n, problem=bp(prob), eps0=1e-2)
    st, rho, it = lx.power_bound_rhs(ctx, dev(uu) if with_u else None, dev(v0), 10)
    rho_o, it_o, st_o = oracle.power_iteration_fd(kind, nx, ny, nu, a, uu, v0, 10, eps0=1e-2)
    assert st == 0 and st_o == 0 and it == it_o
    assert abs(rho - rho_o) <= 1e-12 * rho_o


@pytest.mark.parametrize("prob", PROBLEMS)
@pytest.mark.parametrize("integ", [0, 1])
def test_expint_step_rhs(lx, xi, prob, integ):
    kind, nx, ny, nu, a = prob
    n = nx * ny
    u, lin = _state(kind, nx, ny, nu, a)
    rho, _, _ = oracle.power_iteration(kind, nx, ny, nu, a, u, synth.power_start(n, 5), 10)
    c, g = oracle.spectral_interval(rho)
    h = _step(kind, nx, ny, nu, a, u)
    ctx = lx.leja_setup_rhs(n, problem=bp(prob), eps0=1e-2, integrator=integ)
    lo = torch.empty(n, dtype=torch.float64, device="cuda")
    hi = torch.empty(n, dtype=torch.float64, device="cuda")
    st, err, it = lx.expint_step_rhs(ctx, dev(u), lo, hi, c, g, h, TOL, TOL)
    if integ == 0:
        ref, it_o, st_o = oracle.ros_eu_fd(kind, nx, ny, nu, a, u, c, g, h, TOL, TOL, xi, eps0=1e-2)
        assert st == 0 and st_o == 0 and abs(it - it_o) <= 1 and err == 0.0
        assert rel(hi.cpu().numpy(), ref) <= TOL
    else:
        rlo, rhi, rerr, it_o, st_o = oracle.exprb32_fd(kind, nx, ny, nu, a, u, c, g, h, TOL, TOL, xi, eps0=1e-2)
        assert st == 0 and st_o == 0 and abs(it - it_o) <= 2
        assert rel(lo.cpu().numpy(), rlo) <= TOL and rel(hi.cpu().numpy(), rhi) <= TOL
        # the remainder is a difference of nearly equal terms: its norm is
        # compared against the rounding floor of those terms
        floor = 1e-9 * h * np.linalg.norm(_oracle_f(kind, nx, ny, nu, a, u)) / np.sqrt(n)
        assert abs(err - rerr) <= 1e-6 * rerr + floor


def test_expint_step_rhs_with_source(lx, xi):
    # Problem II through a caller's function: f(u) = A u + S with the paper's
    # discretisation; the engine's f plus the source, written with torch
    nx = ny = 64
    nu, a = 1.0, 10.0
    n = nx * ny
    prob = (nx, ny, nu, a, 2)
    S = synth.problem2_source(nx, ny)
    Sd = dev(S)

    def f_torch(x, out):
        assert lx.lx_rhs_builtin(prob, x, out, torch.cuda.current_stream()) == 0
        out.add_(Sd)

    u = synth.problem1_ic(nx, ny, seed=1)
    rho, _, _ = oracle.power_iteration(2, nx, ny, nu, a, None, synth.power_start(n, 5), 10)
    c, g = oracle.spectral_interval(rho)
    h = 50 * synth.cfl_step_pm1(nx, ny, nu, a)
    ctx = lx.leja_setup_rhs(n, f=f_torch, eps0=1e-2)
    hi = torch.empty(n, dtype=torch.float64, device="cuda")
    st, err, it = lx.expint_step_rhs(ctx, dev(u), None, hi, c, g, h, TOL, TOL)
    ref, it_o, st_o = oracle.ros_eu_fd(2, nx, ny, nu, a, u, c, g, h, TOL, TOL, xi, eps0=1e-2,
                                       rhs=lambda x: oracle.apply_advdiff_up3(nx, ny, nu, a, x) + S)
    assert st == 0 and st_o == 0 and abs(it - it_o) <= 1
    assert rel(hi.cpu().numpy(), ref) <= TOL
    # and the fused path with the source gives the same step (the central
    # quotient of an affine f is the operator itself)
    ref2, _, _ = oracle.ros_eu(2, nx, ny, nu, a, u, c, g, h, TOL, TOL, xi, source=S)
    assert rel(hi.cpu().numpy(), ref2) <= 1e-9


def test_rhs_zero_input_and_callback_error(lx):
    n = 32 * 32
    ctx = lx.leja_setup_rhs(n, problem=(32, 32, 1e-2, 1.0, 0))
    out = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
    zero = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, it = lx.phi_l_apply_rhs(ctx, 1, None, zero, out, -50.0, 25.0, 0.1, TOL, TOL)
    assert st == 0 and it == 1 and float(out.abs().max()) == 0.0

    calls = {"k": 0}

    def f_bad(x, out):
        calls["k"] += 1
        if calls["k"] == 3:
            raise RuntimeError("planted failure of the caller's right-hand side")
        out.copy_(-x)

    bad = lx.leja_setup_rhs(n, f=f_bad)
    w = dev(synth.random_field(n, seed=3))
    st, _ = lx.phi_l_apply_rhs(bad, 1, None, w, out, -1.0, 0.5, 1.0, TOL, TOL)
    assert st == lx.E_CALLBACK
    # the context stays usable: f = -x is linear, phi_1(-h) w = (1 - e^-h)/h w
    st, it = lx.phi_l_apply_rhs(bad, 1, None, w, out, -1.0, 0.5, 1.0, 1e-13, 1e-13)
    assert st == 0
    ref = (1.0 - np.exp(-1.0)) * w.cpu().numpy()
    assert rel(out.cpu().numpy(), ref) <= 1e-10


def test_rhs_setup_rejects(lx):
    from paper_2310_08344_gb300 import LexgbError

    with pytest.raises(LexgbError):
        lx.leja_setup_rhs(0, problem=(8, 8, 1.0, 0.0, 0))
    with pytest.raises(LexgbError):
        lx.leja_setup_rhs(64, problem=(8, 8, 1.0, 0.0, 0), eps0=-1.0)
    with pytest.raises(LexgbError):
        lx.leja_setup_rhs(64, problem=(8, 8, 1.0, 0.0, 0), integrator=5)


def test_rhs_statuses_match_oracle(lx, xi):
    # a non-finite right-hand side and a too-small point table give the
    # statuses of the oracle's loop (LX_E_NONFINITE, LX_E_NOCONV)
    nx = ny = 32
    n = nx * ny
    w = synth.random_field(n, seed=21)

    def f_nan(x, out):
        out.copy_(-x)
        out[5] = float("nan")

    ctx = lx.leja_setup_rhs(n, f=f_nan)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    st, it = lx.phi_l_apply_rhs(ctx, 1, None, dev(w), out, -1.0, 0.5, 1.0, TOL, TOL)

    def f_nan_np(x):
        y = -x.copy()
        y[5] = np.nan
        return y

    _, it_o, st_o = oracle.leja_phi_fd(0, nx, ny, 0, 0, None, 1, w, -1.0, 0.5, 1.0, TOL, TOL, xi, rhs=f_nan_np)
    assert st == st_o == lx.binding.E_NONFINITE and it == it_o == 1
    # a stiff linear f with a 16-point table: the engine's coefficient count
    # bounds the loop first, and both sides report no convergence
    small = lx.leja_setup_rhs(n, problem=(nx, ny, 1.0, 0.0, 0), max_leja=16)
    rho = 8.0 * nx * nx
    c, g = oracle.spectral_interval(rho)
    st, it = lx.phi_l_apply_rhs(small, 0, None, dev(w), out, c, g, 50.0 / rho, 1e-14, 1e-14)
    _, it_o, st_o = oracle.leja_phi_fd(0, nx, ny, 1.0, 0.0, None, 0, w, c, g, 50.0 / rho, 1e-14, 1e-14,
                                       oracle.leja_points(16))
    assert st == lx.binding.E_NOCONV and st_o == oracle.E_NOCONV
