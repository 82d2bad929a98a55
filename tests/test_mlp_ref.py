"""Pins of the CPU reference of the warm-start MLP (oracle/mlp_ref.py): the
analytic gradient against central finite differences of the loss (FP64),
and the bf16 rounding against hand-worked ties and torch's own conversion."""
import numpy as np


def _ref():
    import oracle.mlp_ref as R
    return R


def test_gradient_matches_finite_differences():
    R = _ref()
    rng = np.random.default_rng(3)
    widths = [3, 7, 5, 4]
    _, n = R.layout(widths)
    p = rng.standard_normal(n) * 0.5
    X = rng.standard_normal((6, 3))
    T = rng.standard_normal((6, 4))
    loss, g = R.loss_and_grad(widths, p, X, T)
    h = 1e-6
    fd = np.zeros(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd[i] = (R.loss_and_grad(widths, p + e, X, T)[0] - R.loss_and_grad(widths, p - e, X, T)[0]) / (2 * h)
    assert np.max(np.abs(g - fd)) <= 1e-8 * max(1.0, np.max(np.abs(fd))), np.max(np.abs(g - fd))
    # forward: the last layer is linear, the hidden ones tanh
    H = R.forward(widths, p, X)
    assert np.all(np.abs(H[1]) < 1) and np.all(np.abs(H[2]) < 1)
    assert abs(loss - np.mean((H[-1] - T) ** 2)) < 1e-15


def test_bf16_rounding():
    R = _ref()
    import torch
    # ties go to the even neighbour (8 significant bits)
    assert R.bf16_round(1.0 + 2.0 ** -8) == 1.0
    assert R.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert R.bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    x = np.random.default_rng(5).standard_normal(100000).astype(np.float32) * 10.0
    t = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(R.bf16_round(x), t)
