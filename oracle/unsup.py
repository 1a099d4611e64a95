"""Reference of the unsupervised mode (Sec. 3.2, "Unsupervised Segmentation")
(test infrastructure only; no code shared with the CUDA path).

The paper's steps, in its order: k-means on the colour pixels gives colour
classes; k-medians on the approximated co-supports iota(O s_x) (Eq. map_tsm)
gives texture classes; the initial segments are all (colour class, texture
class) pairs, represented by the two classes' centroids; each pixel gets a
colour and a texture likelihood as in Eq. post_text; the MDL prior (the
solver's nu, ``oracle/segment.py``) then removes segments.

Readings where the paper is silent:
- centres start at caller-given pixels (the random draw is an input); a
  fixed number of rounds, each an assignment followed by an update, then a
  last assignment to the final centres; a class without members keeps its
  centre;
- k-means: squared Euclidean distance on RGB; a centroid is the mean of its
  members' values rounded to multiples of 2^-24, formed from exact integer
  sums: float32(S / (cnt 2^24)) with S = sum of rint(2^24 v);
- k-medians: l1 distance on iota; a centre is the elementwise median of its
  members (the mean of the two middle values for an even count);
- the assignments are decided in FP32 (the kernel's precision) with the
  distances accumulated in a fixed order, colour ((d0^2 + d1^2) + d2^2),
  texture over codes j = 0 .. k-1 in turn; ties go to the lower class;
- colour likelihood softmax_a(-|I(x) - mu_a|^2 / (2 sigma_c2)) (the
  Gaussian colour kernel of Eq. color); texture likelihood
  softmax_b(-||c_b - iota(O s_x)||_1 / beta) (Eq. post_text with one beta:
  there are no scribble locations); segment i = a n_t + b has
  f_i = -log P_colour(a) - log P_texture(b). Normalising over the n
  segments instead of over each factor's classes adds log n to every f_i.

Parity: pinned in ``tests/test_oracle_unsup.py`` (scipy's k-means and
nearest-centroid routine, numpy's median and scipy's city-block distances,
objective monotonicity, the median's l1 optimality, closed forms of the
data term).
"""
from __future__ import annotations

import numpy as np

import oracle

SCALE = float(2 ** 24)


def assign_colour(X, C):
    """Nearest colour centre, FP32 distances ((d0^2 + d1^2) + d2^2), lowest
    class on ties. X (N, 3) float32, C (n_c, 3) float32 -> (N,) int32."""
    X = np.asarray(X, np.float32)
    C = np.asarray(C, np.float32)
    d = np.empty((C.shape[0], X.shape[0]), np.float32)
    for a in range(C.shape[0]):
        t0 = X[:, 0] - C[a, 0]
        t1 = X[:, 1] - C[a, 1]
        t2 = X[:, 2] - C[a, 2]
        d[a] = (t0 * t0 + t1 * t1) + t2 * t2
    return np.argmin(d, axis=0).astype(np.int32)


def colour_means(X, lab, C):
    """Centroids from exact integer sums of the values rounded to 2^-24;
    classes without members keep their centre."""
    Q = np.rint(np.asarray(X, np.float32).astype(np.float64) * SCALE).astype(np.int64)
    out = np.asarray(C, np.float32).copy()
    for a in range(out.shape[0]):
        sel = lab == a
        cnt = int(sel.sum())
        if cnt:
            S = Q[sel].sum(axis=0)
            out[a] = (S.astype(np.float64) / (float(cnt) * SCALE)).astype(np.float32)
    return out


def kmeans_fp32(X, init, iterations):
    """k-means on the rows of X (N, 3) from the centres X[init]; returns
    (centres (n_c, 3) float32, assignment (N,) int32 to those centres)."""
    X = np.asarray(X, np.float32)
    C = X[np.asarray(init, np.int64)].copy()
    for _ in range(iterations):
        C = colour_means(X, assign_colour(X, C), C)
    return C, assign_colour(X, C)


def assign_texture(V, C):
    """Nearest texture centre in l1, FP32 sums over j = 0 .. k-1 in turn,
    lowest class on ties. V (k, N) float32 (code-major), C (n_t, k) float32."""
    V = np.asarray(V, np.float32)
    C = np.asarray(C, np.float32)
    d = np.zeros((C.shape[0], V.shape[1]), np.float32)
    for b in range(C.shape[0]):
        acc = np.zeros(V.shape[1], np.float32)
        for j in range(V.shape[0]):
            acc = acc + np.abs(C[b, j] - V[j])
        d[b] = acc
    return np.argmin(d, axis=0).astype(np.int32)


def median_fp32(vals):
    """Elementwise median over the rows of (m, k) float32 values: the middle
    value for odd m, (lo + hi) * 0.5 in FP32 for even m."""
    v = np.sort(np.asarray(vals, np.float32), axis=0)
    m = v.shape[0]
    if m % 2:
        return v[m // 2].copy()
    return ((v[m // 2 - 1] + v[m // 2]) * np.float32(0.5)).astype(np.float32)


def kmedians_fp32(V, init, iterations):
    """k-medians on the columns of V (k, N) from the centres V[:, init];
    returns (centres (n_t, k) float32, assignment (N,) int32)."""
    V = np.asarray(V, np.float32)
    C = V[:, np.asarray(init, np.int64)].T.copy()
    for _ in range(iterations):
        lab = assign_texture(V, C)
        for b in range(C.shape[0]):
            sel = lab == b
            if sel.any():
                C[b] = median_fp32(V[:, sel].T)
    return C, assign_texture(V, C)


def _log_softmax(t):
    tmax = t.max(axis=0)
    return t - (tmax + np.log(np.exp(t - tmax).sum(axis=0)))


def data_term_from_centres(image, iota_km, colour_c, texture_c, sigma_c2, beta):
    """f (n_c n_t, H, W) float64 from the centres: segment a n_t + b gets
    -log softmax_a(-|I - mu_a|^2 / (2 sigma_c2)) - log softmax_b(-l1 / beta)."""
    image = np.asarray(image, np.float32)
    H, W = image.shape[:2]
    X = image.reshape(-1, 3).astype(np.float64)
    mu = np.asarray(colour_c, np.float64)
    lc = _log_softmax(-((X[None, :, :] - mu[:, None, :]) ** 2).sum(axis=2) / (2.0 * sigma_c2))
    c = np.asarray(texture_c, np.float64)
    io = np.asarray(iota_km, np.float64)  # (k, P)
    l1 = np.abs(c[:, :, None] - io[None, :, :]).sum(axis=1)  # (n_t, P)
    lt = _log_softmax(-l1 / beta)
    n_c, n_t = mu.shape[0], c.shape[0]
    f = -(lc[:, None, :] + lt[None, :, :]).reshape(n_c * n_t, H, W)
    return f


def data_term(image, omega, mask, p, iota_sigma, sigma_c2, beta, n_colour, n_texture,
              colour_init, texture_init, kmeans_iterations=10, kmedians_iterations=10):
    """The unsupervised data term of Sec. 3.2 on an image: FP64 codes of
    every pixel (the C oracle), iota, k-means on the colours, k-medians on
    iota rounded to FP32 (the decision precision), f from the centres.
    Returns a dict: f (n, H, W) float64, colour_centres, colour_assign,
    texture_centres, texture_assign, iota (k, P) float64."""
    image = np.asarray(image, np.float32)
    H, W = image.shape[:2]
    assert len(colour_init) == n_colour and len(texture_init) == n_texture
    a, _ = oracle.codes(image, omega, mask, p, 0.0)
    io = oracle.iota(a, iota_sigma).T.copy()  # (k, P)
    cc, ca = kmeans_fp32(image.reshape(-1, 3), colour_init, kmeans_iterations)
    tc, ta = kmedians_fp32(io.astype(np.float32), texture_init, kmedians_iterations)
    f = data_term_from_centres(image, io, cc, tc, sigma_c2, beta)
    return {"f": f, "colour_centres": cc, "colour_assign": ca.reshape(H, W),
            "texture_centres": tc, "texture_assign": ta.reshape(H, W), "iota": io}
