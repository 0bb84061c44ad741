"""CPU oracle of the per-column warm-start MLP (TEST INFRASTRUCTURE ONLY).

Plain numpy statement of the network 16 -> 128 -> 128 -> 128 -> 32 (ReLU), its mean-squared loss
on the first 22 outputs and the gradient by the chain rule, in FP64.  With `bf16=True` every
tensor-core operand is first rounded to BF16 (round to nearest even): the inputs X, the weights,
the hidden activations H1..H3 as they enter the next layer, and the back-propagated dY and dZ as
they enter the dW and dH products; biases, bias gradients and accumulation stay wide.  That is
the arithmetic the GPU kernels specify (BF16 operands, FP32 accumulation), so the two agree up
to accumulation order.  With `bf16=False` it is the exact FP64 network (pinned by central
differences in tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np

IN, HID, OUT, OUT_USED = 16, 128, 32, 22
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (HID, HID)), ("b3", (HID,)), ("W4", (OUT, HID)), ("b4", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(p):
    out, off = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(p[off:off + n], dtype=np.float64).reshape(shp)
        off += n
    return out


def flatten(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def bf16_bits_to_float(bits):
    return (np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def float_to_bf16_bits(x):
    return (np.ascontiguousarray(bf16_round(x).astype(np.float32)).view(np.uint32) >> 16).astype(np.uint16)


def forward(params, X, bf16=True):
    """Returns (Y, cache) for X [n, 16] (float64 values)."""
    P = unflatten(params)
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    x = r(X)
    H1 = r(np.maximum(x @ r(P["W1"]).T + P["b1"], 0.0))
    H2 = r(np.maximum(H1 @ r(P["W2"]).T + P["b2"], 0.0))
    H3 = r(np.maximum(H2 @ r(P["W3"]).T + P["b3"], 0.0))
    Y = H3 @ r(P["W4"]).T + P["b4"]
    return Y, (x, H1, H2, H3, P)


def loss_and_gradient(params, X, T, bf16=True):
    """Loss (1/n) sum_rows sum_{j<22} (Y - T)^2 and its gradient (flat, parameter layout)."""
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    Y, (x, H1, H2, H3, P) = forward(params, X, bf16)
    n = X.shape[0]
    D = np.zeros_like(Y)
    D[:, :OUT_USED] = Y[:, :OUT_USED] - T[:, :OUT_USED]
    loss = float(np.sum(D * D) / n)
    dY = 2.0 / n * D
    g = {"b4": dY.sum(0), "W4": r(dY).T @ H3}
    dH3 = r(dY) @ r(P["W4"])
    dZ3 = dH3 * (H3 > 0)
    g["b3"], g["W3"] = dZ3.sum(0), r(dZ3).T @ H2
    dH2 = r(dZ3) @ r(P["W3"])
    dZ2 = dH2 * (H2 > 0)
    g["b2"], g["W2"] = dZ2.sum(0), r(dZ2).T @ H1
    dH1 = r(dZ2) @ r(P["W2"])
    dZ1 = dH1 * (H1 > 0)
    g["b1"], g["W1"] = dZ1.sum(0), r(dZ1).T @ x
    return loss, flatten(g)


def adam(params, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (returns new params, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
