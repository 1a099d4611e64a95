"""FP64 reference of the learned surrogate of the data term (test infrastructure).

The surrogate predicts, for every pixel and label, the log of the label's
kernel sum T_i(x) = log sum_j k_rho k_sigma [exp(-TSM/beta)] (Sec. 3.1,
Eq. color and Eq. post_text without the 1/m_i and the kernel normalisers);
the log-likelihood then follows exactly as
    L_i(x) = T_i(x) - log m_i - log(2 pi rho_i(x)^2) - 1.5 log(2 pi sigma_c2).

Network (weights used in bf16, masters in fp32, arithmetic here in fp64):
    x_n = (x - mu_x) / sd_x                      x: features(), n_in of them
    h1 = silu(W1 x_n + b1)      W1: 64 x n_in
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


def shapes(n_labels: int, n_in: int = N_IN) -> dict:
    return {"W1": (HID, n_in), "b1": (HID,), "W2": (HID, HID), "b2": (HID,),
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


def deltas(params: dict, cache, dz: np.ndarray):
    """Derivatives of sum(dz * z) with respect to the pre-activations of the
    output and hidden layers: (dz, d3, d2, d1)."""
    X, u1, h1, u2, h2, u3, h3 = cache
    d3 = (dz @ params["W4"]) * silu_grad(u3)
    d2 = (d3 @ params["W3"]) * silu_grad(u2)
    d1 = (d2 @ params["W2"]) * silu_grad(u1)
    return dz, d3, d2, d1


def backward(params: dict, cache, dz: np.ndarray) -> dict:
    """Gradients of sum(dz * z) with respect to every parameter."""
    X, u1, h1, u2, h2, u3, h3 = cache
    dz, d3, d2, d1 = deltas(params, cache, dz)
    g = {}
    g["W4"] = dz.T @ h3
    g["b4"] = dz.sum(0)
    g["W3"] = d3.T @ h2
    g["b3"] = d3.sum(0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(0)
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


def n_inputs(feature_set: int, n_labels: int) -> int:
    """Inputs of feature set 0 (basic) or 1 (extended)."""
    return N_IN if feature_set == 0 else N_IN + n_labels + 24


def features(image, lead16, W, H, pix, feature_set=0, dist2=None, d_min=1.0):
    """Raw feature rows of the listed pixels (before standardisation).

    Set 0: [R, G, B, x/W, y/H, a_1..a_16] (a = the leading codes). Set 1 adds
    log max(d_i, d_min) for every label i (d_i = the exact distance to label
    i's nearest scribble; dist2 is (n_labels, P) squared distances) and
    sin, cos of 2^f pi x/W and of 2^f pi y/H for f = 0..5.
    """
    pix = np.asarray(pix, np.int64)
    img = np.asarray(image, np.float64).reshape(-1, 3)
    x = (pix % W).astype(np.float64)
    y = (pix // W).astype(np.float64)
    cols = [img[pix], (x / W)[:, None], (y / H)[:, None],
            np.asarray(lead16, np.float64)[pix][:, :16]]
    if feature_set == 1:
        d = np.sqrt(np.asarray(dist2, np.float64)[:, pix]).T
        cols.append(np.log(np.maximum(d, d_min)))
        for f in range(6):
            ax = np.pi * 2.0 ** f * x / W
            ay = np.pi * 2.0 ** f * y / H
            cols += [np.sin(ax)[:, None], np.cos(ax)[:, None], np.sin(ay)[:, None],
                     np.cos(ay)[:, None]]
    return np.concatenate(cols, axis=1)


def surrogate_L(params: dict, stats, feats, m_counts, rho, sigma_c2, rho_variance=0, h=None,
                kappa_beta=1.0):
    """Log-likelihoods (cnt, n) the surrogate answers with, in FP64.

    T = sd_t z + mu_t from the network on the standardised features (stats =
    mu_x, sd_x, mu_t, sd_t concatenated); then
    L_i = T_i - log m_i - log(2 pi s2_i) - 1.5 log(2 pi sigma_c2) with
    s2 = rho^2 (rho as the location kernel's standard deviation) or rho (as
    its variance), Sec. 3.1 Eq. color's normalisers; when the Hamming
    distances h (cnt, n) to the labels' majority co-supports are given (the
    factorised mode), plus the texture log-posterior of Eq. post_text with
    beta_i = kappa_beta rho_i. Returns (L, z).
    """
    feats = np.asarray(feats, np.float64)
    stats = np.asarray(stats, np.float64)
    nin, n = feats.shape[1], len(m_counts)
    mu_x, sd_x = stats[:nin], stats[nin:2 * nin]
    mu_t, sd_t = stats[2 * nin:2 * nin + n], stats[2 * nin + n:2 * nin + 2 * n]
    z, _ = forward(params, (feats - mu_x) / sd_x)
    rho = np.asarray(rho, np.float64)
    s2 = rho if rho_variance else rho * rho
    L = (z * sd_t + mu_t - np.log(np.asarray(m_counts, np.float64)) - np.log(2 * np.pi * s2)
         - 1.5 * np.log(2 * np.pi * sigma_c2))
    if h is not None:
        u = -np.asarray(h, np.float64) / (kappa_beta * rho)
        um = u.max(axis=1, keepdims=True)
        L = L + u - (um + np.log(np.exp(u - um).sum(axis=1, keepdims=True)))
    return L, z
