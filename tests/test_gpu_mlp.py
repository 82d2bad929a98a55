"""The warm-start MLP's CUDA kernels (forward, backward, Adam) against the
numpy FP64 reference (oracle/mlp_ref.py) with the same bf16-rounded weights."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

WIDTHS = [4, 256, 256, 256, 768]


def _setup(torch, B, seed=0):
    from paper_0705_0497_gb300 import api
    m = api.MLP(WIDTHS, seed=seed)
    rng = np.random.default_rng(seed + 1)
    X = rng.uniform(-1, 1, (B, WIDTHS[0])).astype(np.float32)
    T = (0.5 * np.sin(3.0 * X @ rng.standard_normal((WIDTHS[0], WIDTHS[-1])))).astype(np.float32)
    return m, X, T, torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()


@pytest.mark.parametrize("B", [1, 37, 300])
def test_forward_matches_reference(torch_cuda, B):
    import oracle.mlp_ref as R
    m, X, T, Xd, Td = _setup(torch_cuda, B)
    p = m.params()
    Y = m.forward(Xd).cpu().numpy()
    Yr = R.forward(WIDTHS, p, X, bf16=True)[-1]
    assert np.max(np.abs(Y - Yr)) <= 1e-5 * max(1.0, np.max(np.abs(Yr))), np.max(np.abs(Y - Yr))


@pytest.mark.parametrize("B", [37, 300])
def test_gradients_match_reference(torch_cuda, B):
    import oracle.mlp_ref as R
    m, X, T, Xd, Td = _setup(torch_cuda, B, seed=4)
    p = m.params()
    g, loss = m.gradients(Xd, Td)
    g = g.cpu().numpy()
    lr, gr = R.loss_and_grad(WIDTHS, p, X, T, bf16=True)
    assert abs(float(loss.item()) - lr) <= 1e-5 * lr
    lay, _ = R.layout(WIDTHS)
    for (ow, ob, a, b) in lay:
        for lo, hi in ((ow, ow + a * b), (ob, ob + b)):
            err = np.max(np.abs(g[lo:hi] - gr[lo:hi]))
            assert err <= 1e-4 * np.max(np.abs(gr[lo:hi])) + 1e-12, (lo, err, np.max(np.abs(gr[lo:hi])))
    g2, _ = m.gradients(Xd, Td)
    assert np.array_equal(g, g2.cpu().numpy())      # deterministic


def test_params_round_trip_and_training_lowers_the_loss(torch_cuda):
    m, X, T, Xd, Td = _setup(torch_cuda, 256, seed=7)
    p = m.params()
    m.set_params(p)
    assert np.array_equal(m.params(), p)
    l0 = float(m.gradients(Xd, Td)[1].item())
    for _ in range(400):
        loss = m.train_step(Xd, Td, 1e-3)
    l1 = float(loss.item())
    assert l1 < 0.1 * l0, (l0, l1)
