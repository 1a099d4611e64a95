"""FP64 reference of the learned surrogate of the data term (test infrastructure).

The surrogate predicts, for every pixel and label, the log of the label's
kernel sum T_i(x) = log sum_j k_rho k_sigma [exp(-TSM/beta)] (Sec. 3.1,
Eq. color and Eq. post_text without the 1/m_i and the kernel normalisers);
the log-likelihood then follows exactly as
    L_i(x) = T_i(x) - log m_i - log(2 pi rho_i(x)^2) - 1.5 log(2 pi sigma_c2).

Network (weights used in bf16, masters in fp32, arithmetic here in fp64):
    x_n = (x - mu_x) / sd_x                      x: [R, G, B, x/W, y/H, a_1..a_16]
    h1 = silu(W1 x_n + b1)      W1: 64 x 21
    h2 = silu(W2 h1 + b2)       W2: 64 x 64
    h3 = silu(W3 h2 + b3)       W3: 64 x 64
    z  = W4 h3 + b4             W4: n x 64       z approximates (T - mu_t) / sd_t
Loss: mean over the batch and labels of (z - t)^2 / 2.
Optimiser: Adam with bias correction.

Pinned by tests/test_oracle_mlp.py: the analytic gradient against central
finite differences of the loss, silu against its definition via
scipy.special.expit, and Adam against a hand-computed first step.
"""
from __future__ import annotations

import numpy as np

N_IN = 21
HID = 64
LAYERS = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")


def shapes(n_labels: int) -> dict:
    return {"W1": (HID, N_IN), "b1": (HID,), "W2": (HID, HID), "b2": (HID,),
            "W3": (HID, HID), "b3": (HID,), "W4": (n_labels, HID), "b4": (n_labels,)}


def sigmoid(u):
    with np.errstate(over="ignore"):
        return 1.0 / (1.0 + np.exp(-u))


def silu(u):
    return u * sigmoid(u)


def silu_grad(u):
    s = sigmoid(u)
    return s * (1.0 + u * (1.0 - s))


def forward(params: dict, X: np.ndarray):
    """X: (B, 21) standardised features. Returns z (B, n) and the cache."""
    X = np.asarray(X, np.float64)
    u1 = X @ params["W1"].T + params["b1"]
    h1 = silu(u1)
    u2 = h1 @ params["W2"].T + params["b2"]
    h2 = silu(u2)
    u3 = h2 @ params["W3"].T + params["b3"]
    h3 = silu(u3)
    z = h3 @ params["W4"].T + params["b4"]
    return z, (X, u1, h1, u2, h2, u3, h3)


def loss(params: dict, X: np.ndarray, T: np.ndarray) -> float:
    z, _ = forward(params, X)
    return float(0.5 * np.mean((z - T) ** 2))


def backward(params: dict, cache, dz: np.ndarray) -> dict:
    """Gradients of sum(dz * z) with respect to every parameter."""
    X, u1, h1, u2, h2, u3, h3 = cache
    g = {}
    g["W4"] = dz.T @ h3
    g["b4"] = dz.sum(0)
    d3 = (dz @ params["W4"]) * silu_grad(u3)
    g["W3"] = d3.T @ h2
    g["b3"] = d3.sum(0)
    d2 = (d3 @ params["W3"]) * silu_grad(u2)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(0)
    d1 = (d2 @ params["W2"]) * silu_grad(u1)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(0)
    return g


def loss_and_grad(params: dict, X: np.ndarray, T: np.ndarray):
    """Mean squared-error loss and its gradient (analytic backward)."""
    z, cache = forward(params, X)
    B, n = z.shape
    dz = (z - T) / (B * n)
    return float(0.5 * np.mean((z - T) ** 2)), backward(params, cache, dz)


def adam_step(params: dict, grads: dict, state: dict, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place; state holds 'm', 'v' dicts and the step 't'."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state["m"].setdefault(k, np.zeros_like(params[k]))
        v = state["v"].setdefault(k, np.zeros_like(params[k]))
        m[:] = b1 * m + (1 - b1) * grads[k]
        v[:] = b2 * v + (1 - b2) * grads[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even), as float64."""
    f = np.ascontiguousarray(np.asarray(a, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def features(image, lead16, W, H, pix):
    """Raw 21-feature rows of the listed pixels (before standardisation)."""
    pix = np.asarray(pix, np.int64)
    img = np.asarray(image, np.float64).reshape(-1, 3)
    f = np.zeros((len(pix), N_IN))
    f[:, 0:3] = img[pix]
    f[:, 3] = (pix % W) / W
    f[:, 4] = (pix // W) / H
    f[:, 5:21] = np.asarray(lead16, np.float64)[pix][:, :16]
    return f
