"""GPU parity of the controller MLP's tensor-core kernels against the oracle.

Forward outputs within 1e-3 of the BF16-emulating oracle (relative to the
output scale), gradients within 2e-2 relative L2 (BF16 operands, FP32
accumulation on the GPU against float64 accumulation in the oracle), and a
short training run that lowers the loss."""
import numpy as np
import pytest

from oracle import mlp as omlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_08344_gb300 as m

    return m


def _problem(B, seed):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((B, 5)) * [2.0, 1.0, 0.3, 1.5, 0.7] + [1.0, 3.0, 0.5, -0.5, 0.2]).astype(np.float32)
    T = (rng.standard_normal((B, 2)) * [0.3, 0.8] + [0.1, 3.5]).astype(np.float32)
    norm = np.array([1.0, 3.0, 0.5, -0.5, 0.2, 2.0, 1.0, 0.3, 1.5, 0.7, 0.1, 3.5, 0.3, 0.8], dtype=np.float32)
    p = omlp.init_params(seed).astype(np.float32)
    p[omlp.N_PARAMS - 2:] = [0.05, -0.1]
    return X, T, norm, p


@pytest.mark.parametrize("B", [1, 37, 300, 1024])
def test_forward_matches_oracle(lx, B):
    X, T, norm, p = _problem(B, 5)
    m = lx.mlp_setup(1024, p, norm)
    xd = torch.from_numpy(X).cuda()
    yd = torch.full((B, 2), 12345.0, dtype=torch.float32, device="cuda")
    assert lx.mlp_forward(m, xd, yd, B) == 0
    ref = omlp.predict(p.astype(np.float64), norm.astype(np.float64), X.astype(np.float64), emulate=True)
    got = yd.cpu().numpy()
    bad = np.where(~np.isfinite(got).all(axis=1) | (got == 12345.0).any(axis=1))[0]
    assert bad.size == 0, ("rows not written or not finite", bad[:20], got[bad[:4]])
    scale = np.abs(ref).max(axis=0) + 1e-3
    assert np.max(np.abs(got - ref) / scale) <= 1e-2
    assert np.max(np.abs(got - ref)) <= 1e-3 * np.abs(ref).max() + 5e-3
    if B <= 64:
        yh = lx.mlp_forward_host(m, X)
        assert np.array_equal(yh, got)


@pytest.mark.parametrize("B", [64, 300, 1024])
def test_gradient_matches_oracle(lx, B):
    X, T, norm, p = _problem(B, 7)
    m = lx.mlp_setup(1024, p, norm)
    st, loss, g = lx.mlp_train_step(m, torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), B, adam=False,
                                    want_grad=True)
    assert st == 0
    lo, go = omlp.loss_and_grad(p.astype(np.float64), norm.astype(np.float64), X.astype(np.float64),
                                T.astype(np.float64), emulate=True)
    assert abs(loss - lo) <= 1e-3 * lo
    assert np.linalg.norm(g - go) <= 2e-2 * np.linalg.norm(go)
    # per layer as well, so that no block of the gradient hides behind another
    k = 0
    for i, o in omlp.SIZES:
        for size in (i * o, o):
            blk = slice(k, k + size)
            assert np.linalg.norm(g[blk] - go[blk]) <= 3e-2 * np.linalg.norm(go[blk]) + 1e-6, (k, size)
            k += size
    # the weights did not move without the Adam flag
    assert np.array_equal(lx.mlp_get_weights(m), p)


def test_training_lowers_loss(lx):
    rng = np.random.default_rng(0)
    B = 1024
    X = rng.uniform(-1, 1, size=(8 * B, 5)).astype(np.float32)
    T = np.stack([np.sin(2 * X[:, 0]) + 0.5 * X[:, 1] * X[:, 2], np.abs(X[:, 3]) - X[:, 4] ** 2], axis=1)
    T = T.astype(np.float32)
    norm = np.concatenate([X.mean(0), X.std(0), T.mean(0), T.std(0)]).astype(np.float32)
    p = omlp.init_params(2).astype(np.float32)
    m = lx.mlp_setup(B, p, norm)
    xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    losses = []
    for it in range(400):
        k = it % 8
        st, loss, _ = lx.mlp_train_step(m, xd[k * B:(k + 1) * B], td[k * B:(k + 1) * B], B, adam=True, lr=3e-3)
        assert st == 0
        losses.append(loss)
    assert np.mean(losses[-16:]) <= 0.1 * np.mean(losses[:8])
