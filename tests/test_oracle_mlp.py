"""Pins for the FP64 perceptron reference: analytic gradients against
central finite differences, and BF16 rounding against known values."""
import numpy as np

from oracle import mlp


def test_bf16_rounding_known_values():
    x = np.array([1.0, 1.00390625, 1.005859375, 3.14159265, -2.5, 65504.0], dtype=np.float32)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: rounds to even (1.0);
    # 1 + 1.5 * 2^-8 rounds up to 1 + 2^-7
    want = [1.0, 1.0, 1.0078125, 3.140625, -2.5, 65536.0]
    assert list(mlp.bf16_round(x)) == want


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    din, hid, B = 5, 7, 6
    n = din * hid + hid + hid * hid + hid + hid + 1
    p = rng.normal(0, 0.5, n)
    x = rng.normal(0, 1, (B, din))
    t = rng.normal(0, 1, B)
    g = mlp.gradients(p, x, t, din, hid, round_weights=False)
    eps = 1e-6
    num = np.zeros(n)
    for i in range(n):
        d = np.zeros(n)
        d[i] = eps
        num[i] = (mlp.loss(p + d, x, t, din, hid, False) - mlp.loss(p - d, x, t, din, hid, False)) / (2 * eps)
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-7)


def test_forward_shapes_and_relu():
    din, hid = 3, 4
    n = din * hid + hid + hid * hid + hid + hid + 1
    p = np.zeros(n)
    p[-1] = 2.5  # b3
    y, _ = mlp.forward(p, np.ones((2, din)), din, hid)
    assert list(y) == [2.5, 2.5]
