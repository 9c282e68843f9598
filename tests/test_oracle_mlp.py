"""Pins of the oracle MLP (learned warm start): finite differences, GELU special values, golden forward."""
import math
import os
import sys

import numpy as np

from oracle import mlp

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
import make_golden  # noqa: E402


def test_gelu_special_values():
    assert mlp.gelu(np.array(0.0)) == 0.0
    # gelu(x) - gelu(-x) = x (since Phi(x) + Phi(-x) = 1)
    x = np.linspace(-4, 4, 17)
    np.testing.assert_allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-15)
    # Phi(1) = 0.8413447460685429 (standard normal CDF)
    assert abs(mlp.gelu(np.array(1.0)) - 0.8413447460685429) < 1e-15
    # derivative by central differences
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), atol=1e-8)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    D, H, r, B = 8, 12, 5, 7
    params = {"W1": rng.standard_normal((H, D)) * 0.5, "b1": rng.standard_normal(H) * 0.1,
              "W2": rng.standard_normal((H, H)) * 0.3, "b2": rng.standard_normal(H) * 0.1,
              "W3": rng.standard_normal((r, H)) * 0.3, "b3": rng.standard_normal(r) * 0.1}
    X = rng.standard_normal((B, D))
    C = rng.standard_normal((B, r))
    _, g = mlp.loss_and_grads(params, X, C)
    h = 1e-6
    for k in params:
        flat = params[k].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 10)):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = mlp.loss_and_grads(params, X, C)
            flat[idx] = old - h
            lm, _ = mlp.loss_and_grads(params, X, C)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-9, (k, idx, fd, an)


def test_forward_hand_computed_network():
    """A 2 -> 2 -> 2 -> 2 network whose pre-activations land on 1, -1, 1 and 2, so that every hidden value is a
    tabulated standard normal CDF value (gelu(t) = t Phi(t); Phi(1) = 0.8413447460685429, Phi(2) =
    0.9772498680518208, Abramowitz and Stegun Table 26.1).  The output is written out by hand; it changes if
    GELU is applied to the output layer, if any bias is dropped, or if any weight matrix is transposed."""
    P1, P2 = 0.8413447460685429, 0.9772498680518208
    h1 = np.array([P1, -(1.0 - P1)])            # gelu(1), gelu(-1) = -Phi(-1)
    params = {
        "W1": np.array([[1.0, 2.0], [0.5, 1.0]]), "b1": np.array([0.0, -1.5]),
        # a2 = W2 h1 + b2 = (1, 2): b2 chosen from the tabulated values
        "W2": np.array([[1.0, 1.0], [2.0, 1.0]]),
        "b2": np.array([1.0 - (h1[0] + h1[1]), 2.0 - (2 * h1[0] + h1[1])]),
        "W3": np.array([[2.0, -1.0], [0.0, 1.0]]), "b3": np.array([0.5, -1.0]),
    }
    X = np.array([[0.5, 0.25]])                # a1 = W1 x + b1 = (1, -1)
    Y, (_, a1, h1_o, a2, h2) = mlp.forward(params, X)
    np.testing.assert_allclose(a1[0], [1.0, -1.0], atol=1e-15)
    np.testing.assert_allclose(h1_o[0], h1, atol=1e-15)
    np.testing.assert_allclose(a2[0], [1.0, 2.0], atol=1e-15)
    np.testing.assert_allclose(h2[0], [P1, 2.0 * P2], atol=1e-15)
    # y = W3 (gelu(1), gelu(2)) + b3 = (2 Phi(1) - 2 Phi(2) + 0.5, 2 Phi(2) - 1)
    np.testing.assert_allclose(Y[0], [2 * P1 - 2 * P2 + 0.5, 2 * P2 - 1.0], rtol=0, atol=1e-15)
    assert abs(Y[0, 0] - 0.2281897560334442) < 1e-15


def test_forward_matches_golden():
    ref = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "mlp_forward_8_16_16_4.txt"))
    Y, _ = mlp.forward(make_golden._weights(), make_golden._inputs())
    np.testing.assert_allclose(Y, ref, rtol=1e-14, atol=1e-15)


def test_adam_reduces_loss():
    rng = np.random.default_rng(1)
    D, H, r, B = 4, 16, 3, 64
    params = {"W1": rng.standard_normal((H, D)) * 0.5, "b1": np.zeros(H),
              "W2": rng.standard_normal((H, H)) * 0.25, "b2": np.zeros(H),
              "W3": rng.standard_normal((r, H)) * 0.25, "b3": np.zeros(r)}
    X = rng.standard_normal((B, D))
    C = np.stack([np.sin(X[:, 0]), X[:, 1] * X[:, 2], np.cos(X[:, 3])], axis=1)
    l0, _ = mlp.loss_and_grads(params, X, C)
    st = {}
    for _ in range(300):
        _, g = mlp.loss_and_grads(params, X, C)
        mlp.adam_step(params, g, st, lr=1e-2)
    l1, _ = mlp.loss_and_grads(params, X, C)
    assert l1 < 0.2 * l0
