"""Reference of the unsupervised mode (Sec. 3.2, "Unsupervised Segmentation")
(test infrastructure only; no code shared with the CUDA path).

The paper's steps, in its order: k-means on the colour pixels gives colour
classes; k-medians on the approximated co-supports iota(O s_x) (Eq. map_tsm)
gives texture classes; the initial segments are all (colour class, texture
class) pairs, represented by the two classes' centroids; each pixel gets a
colour and a texture likelihood as in Eq. post_text; the MDL prior (the
solver's nu, ``oracle/segment.py``) then removes segments.

Everything here is FP64: distances, decisions and centres. It follows the
definitions, not any kernel's arithmetic (no fixed point, no FP32 decision
order).

Readings where the paper is silent:
- centres start at caller-given points (the random draw is an input); a
  fixed number of rounds, each an assignment followed by an update, then a
  last assignment to the final centres; a class without members keeps its
  centre; ties go to the lower class;
- k-means: squared Euclidean distance on RGB; a centroid is the mean of its
  members;
- k-medians: l1 distance on iota; a centre is the elementwise median of its
  members (the mean of the two middle values for an even count, the
  k-medians centre of Eq. approx_cosupp);
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


def colour_dist2(X, C):
    """Squared Euclidean distances (n_c, N) between the rows of X (N, 3) and
    the centres C (n_c, 3), in float64."""
    X = np.asarray(X, np.float64)
    C = np.asarray(C, np.float64)
    return ((X[None, :, :] - C[:, None, :]) ** 2).sum(axis=2)


def assign_colour(X, C):
    """Nearest colour centre, lowest class on ties -> (N,) int32."""
    return np.argmin(colour_dist2(X, C), axis=0).astype(np.int32)


def colour_means(X, lab, C):
    """k-means update: each class's centre is the mean of its members;
    classes without members keep their centre. float64 (n_c, 3)."""
    X = np.asarray(X, np.float64)
    out = np.asarray(C, np.float64).copy()
    for a in range(out.shape[0]):
        sel = lab == a
        if sel.any():
            out[a] = X[sel].mean(axis=0)
    return out


def kmeans(X, init, iterations):
    """k-means on the rows of X (N, 3) from the centres X[init]; returns
    (centres (n_c, 3) float64, assignment (N,) int32 to those centres)."""
    X = np.asarray(X, np.float64)
    C = X[np.asarray(init, np.int64)].copy()
    for _ in range(iterations):
        C = colour_means(X, assign_colour(X, C), C)
    return C, assign_colour(X, C)


def texture_l1(V, C):
    """l1 distances (n_t, N) between the columns of V (k, N) (code-major)
    and the centres C (n_t, k), in float64."""
    V = np.asarray(V, np.float64)
    C = np.asarray(C, np.float64)
    return np.stack([np.abs(C[b][:, None] - V).sum(axis=0) for b in range(C.shape[0])])


def assign_texture(V, C):
    """Nearest texture centre in l1, lowest class on ties -> (N,) int32."""
    return np.argmin(texture_l1(V, C), axis=0).astype(np.int32)


def texture_medians(V, lab, C):
    """k-medians update: each class's centre is the elementwise median of its
    members (Eq. approx_cosupp); classes without members keep their centre."""
    V = np.asarray(V, np.float64)
    out = np.asarray(C, np.float64).copy()
    for b in range(out.shape[0]):
        sel = lab == b
        if sel.any():
            out[b] = oracle.median_rows(V[:, sel].T)
    return out


def kmedians(V, init, iterations):
    """k-medians on the columns of V (k, N) from the centres V[:, init];
    returns (centres (n_t, k) float64, assignment (N,) int32)."""
    V = np.asarray(V, np.float64)
    C = V[:, np.asarray(init, np.int64)].T.copy()
    for _ in range(iterations):
        C = texture_medians(V, assign_texture(V, C), C)
    return C, assign_texture(V, C)


def margins(D):
    """Decision margin of each point: the second smallest minus the smallest
    distance over the classes (rows of D); +inf with one class."""
    if D.shape[0] < 2:
        return np.full(D.shape[1], np.inf)
    srt = np.sort(D, axis=0)
    return srt[1] - srt[0]


def _log_softmax(t):
    tmax = t.max(axis=0)
    return t - (tmax + np.log(np.exp(t - tmax).sum(axis=0)))


def data_term_from_centres(image, iota_km, colour_c, texture_c, sigma_c2, beta):
    """f (n_c n_t, H, W) float64 from the centres: segment a n_t + b gets
    -log softmax_a(-|I - mu_a|^2 / (2 sigma_c2)) - log softmax_b(-l1 / beta)."""
    image = np.asarray(image, np.float32)
    H, W = image.shape[:2]
    X = image.reshape(-1, 3)
    mu = np.asarray(colour_c, np.float64)
    lc = _log_softmax(-colour_dist2(X, mu) / (2.0 * sigma_c2))
    lt = _log_softmax(-texture_l1(iota_km, texture_c) / beta)
    n_c, n_t = mu.shape[0], np.asarray(texture_c).shape[0]
    return -(lc[:, None, :] + lt[None, :, :]).reshape(n_c * n_t, H, W)


def iota_all(image, omega, mask, p, iota_sigma):
    """iota(O s_x) of every pixel from the FP64 codes, code-major (k, P)."""
    a, _ = oracle.codes(image, omega, mask, p, 0.0)
    return oracle.iota(a, iota_sigma).T.copy()


def data_term(image, omega, mask, p, iota_sigma, sigma_c2, beta, n_colour, n_texture,
              colour_init, texture_init, kmeans_iterations=10, kmedians_iterations=10):
    """The unsupervised data term of Sec. 3.2 on an image: FP64 codes of
    every pixel (the C oracle), iota, k-means on the colours, k-medians on
    iota, f from the centres, all in float64.
    Returns a dict: f (n, H, W), colour_centres, colour_assign,
    texture_centres, texture_assign, iota (k, P)."""
    image = np.asarray(image, np.float32)
    H, W = image.shape[:2]
    assert len(colour_init) == n_colour and len(texture_init) == n_texture
    io = iota_all(image, omega, mask, p, iota_sigma)
    cc, ca = kmeans(image.reshape(-1, 3), colour_init, kmeans_iterations)
    tc, ta = kmedians(io, texture_init, kmedians_iterations)
    f = data_term_from_centres(image, io, cc, tc, sigma_c2, beta)
    return {"f": f, "colour_centres": cc, "colour_assign": ca.reshape(H, W),
            "texture_centres": tc, "texture_assign": ta.reshape(H, W), "iota": io}
