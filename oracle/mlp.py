"""Oracle MLP for the learned warm start (FP64, numpy).  Test infrastructure only.

The network maps standardised material parameters x = (log sigma_s, sigma_a)
to reduced-basis coefficients c (the Galerkin coefficients of eq. greedy-rom
on the final greedy basis):
    h1 = gelu(W1 x + b1), h2 = gelu(W2 h1 + b2), y = W3 h2 + b3
with the exact GELU gelu(t) = t * Phi(t) = 0.5 t (1 + erf(t / sqrt 2))
(Hendrycks and Gimpel 2016).  Loss: mean over the batch of
0.5 * ||y - c||^2 / r.  Backward pass by the chain rule; Adam (Kingma and Ba
2015) with bias correction.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def gelu(t):
    return 0.5 * t * (1.0 + erf(t / math.sqrt(2.0)))


def gelu_grad(t):
    return 0.5 * (1.0 + erf(t / math.sqrt(2.0))) + t * np.exp(-0.5 * t * t) / math.sqrt(2.0 * math.pi)


def forward(params, X):
    """Returns (Y, cache).  params: dict W1 [H,D], b1 [H], W2 [H,H], b2 [H], W3 [r,H], b3 [r]."""
    a1 = X @ params["W1"].T + params["b1"]
    h1 = gelu(a1)
    a2 = h1 @ params["W2"].T + params["b2"]
    h2 = gelu(a2)
    Y = h2 @ params["W3"].T + params["b3"]
    return Y, (X, a1, h1, a2, h2)


def loss_and_grads(params, X, C):
    """Loss = mean_b 0.5 * ||Y_b - C_b||^2 / r and its gradients."""
    Y, (X, a1, h1, a2, h2) = forward(params, X)
    B, r = Y.shape
    diff = Y - C
    loss = 0.5 * float(np.sum(diff * diff)) / (B * r)
    dY = diff / (B * r)
    g = {}
    g["W3"] = dY.T @ h2
    g["b3"] = dY.sum(axis=0)
    dh2 = dY @ params["W3"]
    da2 = dh2 * gelu_grad(a2)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ params["W2"]
    da1 = dh1 * gelu_grad(a1)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(axis=0)
    return loss, g


def adam_step(params, grads, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state holds m, v and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] * grads[k]
        mhat = m / (1 - beta1 ** t)
        vhat = v / (1 - beta2 ** t)
        params[k] -= lr * mhat / (np.sqrt(vhat) + eps)
