"""FP64 reference of the convex multilabel segmentation (Sec. 4) on the data
term -L (test infrastructure only; no code shared with the CUDA path).

Energy (Eq. energy1) relaxed as in Sec. 4.1 and minimised by the primal-dual
iteration of Sec. 4.2 (Eq. algo): dual ascent in xi (projected onto
|xi(x)| <= lambda g(x) / 2) and mu (projected onto mu <= 0), primal descent
in m (projected onto [0, 1]) and u (projected onto the simplex by
Michelot's algorithm), over-relaxation of u and m; the result is binarised
by argmax (Sec. 4.2).

Discretisation (the paper gives none): forward differences with a zero
difference across the last row / column for the gradient, its negative
adjoint for the divergence. Edge weight g(x) = exp(-|grad I(x)| / gamma) /
(2 gamma), |grad I| the Euclidean norm of the forward differences of the
three channels of 255 I (8-bit scale), gamma = 5. Step sizes by diagonal
preconditioning (Pock and Chambolle, alpha = 1): 1/2 for xi and mu, 1/5 for
u, 1/|Omega| for m. Start: u = 1/n, m = 1, xi = 0, mu = 0.

Parity: pinned in ``tests/test_oracle_segment.py`` (Michelot against a
sort-based projection, lambda = 0 reduces to the pointwise argmin, a
constant data term keeps the uniform start, two-label symmetry).
"""
from __future__ import annotations

import numpy as np


def grad(u):
    """Forward differences along x (axis -1) and y (axis -2), zero across the
    last column / row."""
    gx = np.zeros_like(u)
    gy = np.zeros_like(u)
    gx[..., :, :-1] = u[..., :, 1:] - u[..., :, :-1]
    gy[..., :-1, :] = u[..., 1:, :] - u[..., :-1, :]
    return gx, gy


def div(px, py):
    """Negative adjoint of ``grad``."""
    d = np.zeros_like(px)
    d[..., :, 0] += px[..., :, 0]
    d[..., :, 1:-1] += px[..., :, 1:-1] - px[..., :, :-2]
    d[..., :, -1] -= px[..., :, -2] if px.shape[-1] > 1 else 0.0
    d[..., 0, :] += py[..., 0, :]
    d[..., 1:-1, :] += py[..., 1:-1, :] - py[..., :-2, :]
    d[..., -1, :] -= py[..., -2, :] if py.shape[-2] > 1 else 0.0
    return d


def edge_weight(image, gamma=5.0):
    """g(x) = exp(-|grad I(x)| / gamma) / (2 gamma) on the 8-bit scale."""
    I = 255.0 * np.asarray(image, np.float64).transpose(2, 0, 1)  # (3, H, W)
    gx, gy = grad(I)
    mag = np.sqrt((gx * gx + gy * gy).sum(axis=0))
    return np.exp(-mag / gamma) / (2.0 * gamma)


def project_simplex_michelot(y):
    """Michelot's algorithm: projection of each column of y (n, ...) onto
    {u >= 0, sum u = 1}. Repeatedly project onto the hyperplane restricted to
    the active indices and drop those that came out negative."""
    y = np.asarray(y, np.float64)
    n = y.shape[0]
    flat = y.reshape(n, -1)
    active = np.ones_like(flat, dtype=bool)
    u = flat.copy()
    for _ in range(n):
        cnt = active.sum(axis=0)
        shift = (np.where(active, flat, 0.0).sum(axis=0) - 1.0) / cnt
        u = np.where(active, flat - shift, 0.0)
        neg = active & (u < 0.0)
        if not neg.any():
            break
        active &= ~neg
    return u.reshape(y.shape)


def segment(f, image, lam, nu=0.0, gamma=5.0, iterations=300):
    """Primal-dual iteration of Eq. (algo) on the data term f (n, H, W).
    Returns (u (n, H, W), labels (H, W) int32)."""
    f = np.asarray(f, np.float64)
    n, H, W = f.shape
    g = edge_weight(image, gamma)
    bound = lam * g / 2.0
    t_xi, t_mu, t_u, t_m = 0.5, 0.5, 0.2, 1.0 / (H * W)
    u = np.full_like(f, 1.0 / n)
    ub = u.copy()
    m = np.ones(n)
    mb = m.copy()
    px = np.zeros_like(f)
    py = np.zeros_like(f)
    mu = np.zeros_like(f)
    for _ in range(iterations):
        gx, gy = grad(ub)
        px += t_xi * gx
        py += t_xi * gy
        scale = np.maximum(1.0, np.sqrt(px * px + py * py) / np.maximum(bound, 1e-300))
        px /= scale
        py /= scale
        mu = np.minimum(0.0, mu + t_mu * (mb[:, None, None] - ub))
        m_new = np.clip(m - t_m * (nu + mu.sum(axis=(1, 2))), 0.0, 1.0)
        u_new = project_simplex_michelot(u - t_u * (-div(px, py) + f - mu))
        ub = 2.0 * u_new - u
        mb = 2.0 * m_new - m
        u, m = u_new, m_new
    return u, np.argmax(u, axis=0).astype(np.int32)


def dice(labels, truth, n):
    """Eq. (dice): mean over labels of 2 |A_i & B_i| / (|A_i| + |B_i|)."""
    s = 0.0
    for i in range(n):
        a, b = labels == i, truth == i
        den = a.sum() + b.sum()
        s += 2.0 * (a & b).sum() / den if den else 1.0
    return s / n
