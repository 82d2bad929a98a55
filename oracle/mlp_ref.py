"""CPU reference of the warm-start MLP (test infrastructure, like the rest of
`oracle/`): plain numpy in FP64, no blocking or fusion.

Layers l = 1..L: Z_l = H_{l-1} W_l + b_l with H_0 = X; H_l = tanh(Z_l) for
l < L, the output Y = Z_L.  Loss = mean over all outputs of (Y - T)^2.
Parameters in one flat vector: for each layer W_l [in][out] row-major, then
b_l [out].  The library computes with bf16 weights: pass bf16=True to round
the weights as the library does (round to nearest even to 8 significant
bits), the biases stay as given.

Pinned in tests/test_mlp_ref.py by central finite differences of the loss
and by a one-layer case with a closed-form gradient.
"""
import numpy as np


def layout(widths):
    """[(offset of W, offset of b, in, out)] per layer, and the total size."""
    out, off = [], 0
    for a, b in zip(widths[:-1], widths[1:]):
        out.append((off, off + a * b, a, b))
        off += a * b + b
    return out, off


def bf16_round(x):
    """Round float values to bfloat16 (nearest, ties to even), as float64."""
    x32 = np.asarray(x, np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(widths, params, bf16=False):
    lay, n = layout(widths)
    assert params.size == n
    Ws, bs = [], []
    for (ow, ob, a, b) in lay:
        W = np.asarray(params[ow:ow + a * b], np.float64).reshape(a, b)
        Ws.append(bf16_round(W) if bf16 else W)
        bs.append(np.asarray(params[ob:ob + b], np.float64))
    return Ws, bs


def forward(widths, params, X, bf16=False):
    Ws, bs = unpack(widths, params, bf16)
    H = [np.asarray(X, np.float64)]
    for l, (W, b) in enumerate(zip(Ws, bs)):
        Z = H[-1] @ W + b
        H.append(np.tanh(Z) if l < len(Ws) - 1 else Z)
    return H


def loss_and_grad(widths, params, X, T, bf16=False):
    """Loss and its gradient with respect to the flat parameters (FP64; with
    bf16=True the gradient is taken at the rounded weights)."""
    Ws, bs = unpack(widths, params, bf16)
    H = forward(widths, params, X, bf16)
    Y = H[-1]
    T = np.asarray(T, np.float64)
    n = Y.size
    loss = float(np.sum((Y - T) ** 2) / n)
    dZ = 2.0 * (Y - T) / n
    lay, size = layout(widths)
    g = np.zeros(size)
    for l in range(len(Ws) - 1, -1, -1):
        ow, ob, a, b = lay[l]
        g[ow:ow + a * b] = (H[l].T @ dZ).ravel()
        g[ob:ob + b] = dZ.sum(axis=0)
        if l > 0:
            dZ = (dZ @ Ws[l].T) * (1.0 - H[l] ** 2)
    return loss, g
