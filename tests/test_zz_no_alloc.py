"""The allocation-free entry point phi_l_apply_noalloc against phi_l_apply.

phi_l_apply_noalloc serves callers that cannot allocate device memory where
they call (during CUDA stream capture, under an application-owned memory
pool, in loops that cannot afford an allocation's synchronisation): its
scratch is a fixed array inside the library.  Here it is called through the
C ABI twice in a row -- the second call sees the scratch the first one left
behind -- and each result is compared with the context-based entry point on
the same inputs, to the FP64 parity tolerance used by the other GPU tests.
This file is collected last so that a stop at its first failure happens
after every other test has run.
"""
import numpy as np
import pytest

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
    rho = float(np.abs(lam).max())
    lam_min = -1.05 * rho
    return u0, h, lam_min / 2.0, -lam_min / 4.0, nu, a


def test_noalloc_matches_context_path_twice(lx):
    stream = torch.cuda.current_stream()
    for (nx, ny, seed, l) in [(192, 160, 3, 1), (512, 512, 4, 0)]:
        u0, h, c, g, nu, a = _case(nx, ny, seed)
        w = torch.from_numpy(u0).cuda()
        ctx = lx.leja_setup(nx, ny, nu, a, lx.ADVDIFF, lx.FP64, lx.ROS_EU, 1000, stream)
        ref = torch.empty_like(w)
        st, it_ref = lx.phi_l_apply(ctx, l, None, w, ref, c, g, h, TOL, TOL)
        assert st == 0
        ref_np = ref.cpu().numpy()
        for call in range(2):
            out = torch.full_like(w, float("nan"))
            st, it = lx.phi_l_apply_noalloc(nx, ny, nu, a, l, w, out, c, g, h, TOL, TOL, stream)
            assert st == 0, (call, st)
            assert it == it_ref, (call, it, it_ref)
            got = out.cpu().numpy()
            assert np.linalg.norm(got - ref_np) <= TOL * np.linalg.norm(ref_np), call
        ctx.close()


def test_noalloc_rejects_oversize_and_unsupported(lx):
    w = torch.zeros(513 * 512, dtype=torch.float64, device="cuda")
    out = torch.empty_like(w)
    st, _ = lx.phi_l_apply_noalloc(513, 512, 1e-2, 0.5, 0, w, out, -1.0, 0.5, 1e-3, TOL, TOL)
    assert st == 1  # LX_E_INVAL: beyond LX_NOALLOC_MAX_POINTS
    assert "LX_NOALLOC_MAX_POINTS" in lx.lib().lx_last_cuda_error().decode()
