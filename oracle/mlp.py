"""CPU reference of the learned surrogate (TEST INFRASTRUCTURE ONLY).

A plain MLP, written from its definition: features [sin phi, cos phi],
hidden layers h = GELU(x W^T + b) (tanh form of GELU), logits z = h W^T + b,
q = softmax(z), loss = mean over the batch of KL(p || q), and its backward
pass by the chain rule.  Matrix products use numpy in float64.

With ``bf16=True`` the values the GPU stores in bfloat16 (features, weights,
pre-activations, activations, output and hidden gradients) are rounded to
bfloat16 at the same points, so the GPU kernels can be compared against it
tightly; with ``bf16=False`` it is the exact FP64 model (pinned by finite
differences in tests/test_oracle_pins.py).
"""
from __future__ import annotations

import numpy as np
import torch

C_GELU = np.sqrt(2.0 / np.pi)


def bf16(x):
    return torch.tensor(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(C_GELU * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    u = C_GELU * (z + 0.044715 * z ** 3)
    t = np.tanh(u)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * C_GELU * (1.0 + 3 * 0.044715 * z * z)


def features(phases):
    phases = np.asarray(phases, dtype=np.float64)
    return np.concatenate([np.sin(phases), np.cos(phases)], axis=1)


def softmax(z):
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def forward(params, phases, bf=True):
    """params: list of (W [out][in], b [out]).  Returns logits and the cache."""
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    x = r(features(phases))
    cache = {"x": [x], "z": []}
    for W, b in params[:-1]:
        z = r(x @ r(W).T + b)
        x = r(gelu(z))
        cache["z"].append(z)
        cache["x"].append(x)
    W, b = params[-1]
    logits = x @ r(W).T + b
    return logits, cache


def loss_and_grads(params, phases, target, bf=True):
    """Mean KL(target || softmax(logits)) and its gradients (dW, db) per layer."""
    r = bf16 if bf else (lambda a: np.asarray(a, dtype=np.float64))
    logits, cache = forward(params, phases, bf)
    B = logits.shape[0]
    q = softmax(logits)
    p = np.asarray(target, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        kl = np.where(p > 0, p * (np.log(p) - np.log(q)), 0.0).sum(axis=1)
    g = r((q - p) / B)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, b = params[l]
        xin = cache["x"][l]
        grads[l] = (g.T @ xin, g.sum(axis=0))
        if l > 0:
            g = r((g @ r(W)) * gelu_grad(cache["z"][l - 1]))
    return kl.mean(), kl, grads
