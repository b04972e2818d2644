"""The allocation-free entry point phi_l_apply_noalloc against phi_l_apply
and against the CPU oracle.

phi_l_apply_noalloc serves callers that cannot allocate device memory where
they call (an application-owned memory pool that holds the whole device, or
a loop that cannot afford an allocation's device synchronisation): its
scratch is a fixed array inside the library.  Here it is called through the
C ABI twice in a row -- the second call sees the scratch the first one left
behind -- and each result is compared with the context-based entry point on
the same inputs and with the oracle, to the FP64 parity tolerance used by
the other GPU tests.  The cases cover the two-point-per-lane kernel (nx a
multiple of 64, aligned vectors), the one-point kernel (nx = 200) and the
no-convergence exit of the host-driven loop.  This file is collected last so
that a stop at its first failure happens after every other test has run.
"""
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


def _case(nx, ny, seed, nu=1e-2, a=0.5):
    u0 = synth.gaussians_ic(nx, ny, seed=seed) + 0.05 * synth.random_field(nx * ny, seed + 100)
    h = 50 * synth.cfl_step(nx, ny, nu, a)
    # spectral radius of the central-difference operator: the symbol's maximum
    tx = 2 * np.pi * np.fft.fftfreq(nx)[None, :]
    ty = 2 * np.pi * np.fft.fftfreq(ny)[:, None]
    lam = nu * (2 * np.cos(tx) - 2) * nx**2 + nu * (2 * np.cos(ty) - 2) * ny**2 + 1j * a * (
        np.sin(tx) * nx + np.sin(ty) * ny)
    c, g = oracle.spectral_interval(float(np.abs(lam).max()))
    return u0, h, c, g, nu, a


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("nx,ny,seed,l", [(192, 160, 3, 1), (512, 512, 4, 0), (200, 130, 5, 3)])
def test_noalloc_matches_context_path_and_oracle_twice(lx, nx, ny, seed, l):
    stream = torch.cuda.current_stream()
    u0, h, c, g, nu, a = _case(nx, ny, seed)
    w = torch.from_numpy(u0).cuda()
    ctx = lx.leja_setup(nx, ny, nu, a, lx.ADVDIFF, lx.FP64, lx.ROS_EU, 1000, stream)
    ref = torch.empty_like(w)
    st, it_ref = lx.phi_l_apply(ctx, l, None, w, ref, c, g, h, TOL, TOL)
    assert st == 0
    ref_np = ref.cpu().numpy()
    orc, it_o, st_o = oracle.leja_phi(oracle.ADVDIFF, nx, ny, nu, a, None, l, u0, c, g, h, TOL, TOL,
                                      oracle.leja_points(1000))
    assert st_o == 0
    for call in range(2):
        out = torch.full_like(w, float("nan"))
        st, it = lx.phi_l_apply_noalloc(nx, ny, nu, a, l, w, out, c, g, h, TOL, TOL, stream)
        assert st == 0, (call, st)
        assert it == it_ref, (call, it, it_ref)
        assert abs(it - it_o) <= 1, (call, it, it_o)
        got = out.cpu().numpy()
        assert _rel(got, ref_np) <= TOL, call
        assert _rel(got, orc) <= TOL, call
    ctx.close()


def test_noalloc_no_convergence_matches_context_path(lx):
    # rtol = atol = 0: no iteration passes the test, both entry points run to
    # the end of their coefficient table and report LX_E_NOCONV with the same
    # iteration count and the same partial sum
    stream = torch.cuda.current_stream()
    nx, ny = 128, 96
    u0, h, c, g, nu, a = _case(nx, ny, 6)
    w = torch.from_numpy(u0).cuda()
    ctx = lx.leja_setup(nx, ny, nu, a, lx.ADVDIFF, lx.FP64, lx.ROS_EU, 1000, stream)
    ref = torch.empty_like(w)
    st_ref, it_ref = lx.phi_l_apply(ctx, 0, None, w, ref, c, g, h, 0.0, 0.0)
    assert st_ref == 4
    assert it_ref == lx.lx_leja_coeff_count(h, c, g, 1000) - 1
    for call in range(2):
        out = torch.full_like(w, float("nan"))
        st, it = lx.phi_l_apply_noalloc(nx, ny, nu, a, 0, w, out, c, g, h, 0.0, 0.0, stream)
        assert st == 4 and it == it_ref, (call, st, it, it_ref)
        assert _rel(out.cpu().numpy(), ref.cpu().numpy()) <= TOL
    ctx.close()


def test_noalloc_rejects_oversize_and_unsupported(lx):
    w = torch.zeros(513 * 512, dtype=torch.float64, device="cuda")
    out = torch.empty_like(w)
    st, _ = lx.phi_l_apply_noalloc(513, 512, 1e-2, 0.5, 0, w, out, -1.0, 0.5, 1e-3, TOL, TOL)
    assert st == 1  # LX_E_INVAL: beyond LX_NOALLOC_MAX_POINTS
    assert "LX_NOALLOC_MAX_POINTS" in lx.lib().lx_last_cuda_error().decode()
