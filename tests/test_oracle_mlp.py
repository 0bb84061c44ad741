"""Pins of the CPU MLP oracle (no GPU): central differences of the exact FP64 network, the BF16
rounding rule against torch's own BF16 conversion, and a closed-form single-layer case."""
import numpy as np
import pytest

from oracle import mlp


def small_params(rng, scale=0.3):
    return rng.normal(scale=scale, size=mlp.NPARAM)


def test_gradient_matches_central_differences_fp64():
    rng = np.random.default_rng(0)
    p = small_params(rng)
    X = rng.normal(size=(6, mlp.IN))
    T = rng.normal(size=(6, mlp.OUT))
    _, g = mlp.loss_and_gradient(p, X, T, bf16=False)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    for i in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_gradient(pp, X, T, bf16=False)[0] - mlp.loss_and_gradient(pm, X, T, bf16=False)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-8)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(size=1000) * 10.0 ** rng.integers(-6, 6, 1000),
                        [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)
    bits = mlp.float_to_bf16_bits(x)
    assert np.array_equal(mlp.bf16_bits_to_float(bits), ref)


def test_single_layer_closed_form():
    """With W2 = W3 = I-like positive maps and zero biases the network reduces to a linear map on
    positive inputs: Y = W4 W3 W2 W1 x for x, W >= 0 (ReLU inactive)."""
    rng = np.random.default_rng(2)
    P = {name: np.zeros(shp) for name, shp in mlp.SHAPES}
    P["W1"] = rng.uniform(0, 1, (mlp.HID, mlp.IN))
    P["W2"] = np.eye(mlp.HID)
    P["W3"] = np.eye(mlp.HID)
    P["W4"] = rng.uniform(0, 1, (mlp.OUT, mlp.HID))
    X = rng.uniform(0, 1, (5, mlp.IN))
    Y, _ = mlp.forward(mlp.flatten(P), X, bf16=False)
    np.testing.assert_allclose(Y, X @ P["W1"].T @ P["W4"].T, rtol=1e-12)
