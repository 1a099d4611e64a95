"""CPU FP64 oracle for the co-sparse data term (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA path
and never imports the product package.

``oracle.c`` evaluates the paper's definitions literally in double precision
(Sec. 2, Eq. 1, Eq. tsm_clean, Eq. tex-rep, Sec. 3.1 Eq. color / post_text /
joined, Eq. energy1); the smooth co-support texture (Eq. map_tsm,
approx_cosupp and post_text on iota, ``iota`` / ``median_rows`` /
``smooth_reps`` / ``smooth_log_posterior``) is numpy on the C oracle's FP64
codes and Parzen sum (mode 2); ``segment.py`` is the FP64 primal-dual
multilabel segmentation of Sec. 4 on the data term; ``unsup.py`` is the
unsupervised mode of Sec. 3.2 (k-means on colour, k-medians on iota, the
two-factor data term); ``mlp.py`` holds the surrogate network's FP64 forward,
analytic backward and Adam step. This module compiles ``oracle.c`` with gcc
(no FMA contraction) and wraps it with ctypes.

Parity status of each function is recorded next to it; every function here is
pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_pins.py``,
``tests/test_oracle_mlp.py``, ``tests/test_oracle_segment.py`` and
``tests/test_oracle_unsup.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (OpenMP if available)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-shared", "-fPIC"]
    tmp = _SO + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", src, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [src, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i, d = ctypes.c_int, ctypes.c_double
            lib.oracle_codes.argtypes = [P, i, i, P, i, P, i, d, P, i, P, P, i]
            lib.oracle_patches.argtypes = [P, i, i, P, i, P, i, P, i]
            lib.oracle_tsm.argtypes = [P, P, i]
            lib.oracle_majority.argtypes = [P, i, i, P, P]
            lib.oracle_dist2.argtypes = [i, i, i, P, P, P, i, P]
            lib.oracle_likelihood.argtypes = [P, i, i, P, P, i, i, P, P, d, d, d, d, i, i, P, i,
                                              P, P, P, P]
            for f in ("oracle_codes", "oracle_patches", "oracle_tsm", "oracle_majority",
                      "oracle_dist2", "oracle_likelihood"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def n_words(k: int) -> int:
    return (k + 31) // 32


def patches(image, mask, p, pix=None, order=0):
    """Normalised masked gray patches s_x (Sec. 2, Sec. 3.1), FP64, one row per
    pixel. order 0: mask, centre, normalise; order 1: centre, mask, centre
    again, normalise."""
    image = _c(image, np.float32)
    mask = _c(mask, np.float32)
    H, W = image.shape[:2]
    pix = None if pix is None else _c(pix, np.int32)
    cnt = H * W if pix is None else len(pix)
    out = np.zeros((cnt, p * p), np.float64)
    rc = _load().oracle_patches(_p(image), H, W, _p(mask), p, _p(pix), cnt, _p(out), int(order))
    if rc:
        raise ValueError("oracle_patches: invalid arguments")
    return out


def codes(image, omega, mask, p, tau, pix=None, want_codes=True, order=0):
    """Codes a = O s (Sec. 2) and co-support bitmasks (Eq. 1 with |a_j| <= tau)
    of the patches of ``patches(..., order)``.

    Returns (codes (cnt, k) float64 or None, bitmask (cnt, ceil(k/32)) uint32).
    """
    image = _c(image, np.float32)
    omega = _c(omega, np.float32)
    mask = _c(mask, np.float32)
    H, W = image.shape[:2]
    k = omega.shape[0]
    assert omega.shape[1] == p * p and mask.shape[0] == p * p
    pix = None if pix is None else _c(pix, np.int32)
    cnt = H * W if pix is None else len(pix)
    cod = np.zeros((cnt, k), np.float64) if want_codes else None
    bm = np.zeros((cnt, n_words(k)), np.uint32)
    rc = _load().oracle_codes(_p(image), H, W, _p(omega), k, _p(mask), p, float(tau), _p(pix),
                              cnt, _p(cod), _p(bm), int(order))
    if rc:
        raise ValueError("oracle_codes: invalid arguments")
    return cod, bm


def tsm(a_bits, b_bits, k) -> int:
    """Eq. (tsm_clean) on two packed co-support bitmasks."""
    a = _c(a_bits, np.uint32)
    b = _c(b_bits, np.uint32)
    return int(_load().oracle_tsm(_p(a), _p(b), k))


def majority(bits_smp, k, label_off):
    """Eq. (tex-rep): majority co-support of each label, (n_labels, Wk) uint32."""
    bits_smp = _c(bits_smp, np.uint32)
    label_off = _c(label_off, np.int32)
    nl = len(label_off) - 1
    rep = np.zeros((nl, n_words(k)), np.uint32)
    if _load().oracle_majority(_p(bits_smp), k, nl, _p(label_off), _p(rep)):
        raise ValueError("oracle_majority: a label has no samples")
    return rep


def dist2(H, W, label_off, sample_pix, pix=None):
    """Squared distance to the nearest scribble of each label (Sec. 3.1), int64
    (n_labels, cnt), brute force over the samples."""
    label_off = _c(label_off, np.int32)
    sample_pix = _c(sample_pix, np.int32)
    nl = len(label_off) - 1
    pix = None if pix is None else _c(pix, np.int32)
    cnt = H * W if pix is None else len(pix)
    out = np.zeros((nl, cnt), np.int64)
    if _load().oracle_dist2(H, W, nl, _p(label_off), _p(sample_pix), _p(pix), cnt, _p(out)):
        raise ValueError("oracle_dist2: a label has no samples")
    return out


def likelihood(image, bits_px, bits_smp, k, label_off, sample_pix, sigma_c2=1.3, alpha=1.3,
               d_min=1.0, kappa_beta=1.0, mode=0, pix=None, want_dist2=False, rho_variance=0):
    """Log-likelihoods L (n_labels, cnt), data term -L and label posteriors.
    rho_variance = 1 reads rho as the location kernel's variance (Sec. 3.1),
    0 as its standard deviation.

    Returns dict with 'L', 'neglog', 'post' (float64) and optionally 'dist2'.
    """
    image = _c(image, np.float32)
    H, W = image.shape[:2]
    bits_px = _c(bits_px, np.uint32)
    bits_smp = _c(bits_smp, np.uint32)
    label_off = _c(label_off, np.int32)
    sample_pix = _c(sample_pix, np.int32)
    nl = len(label_off) - 1
    pix = None if pix is None else _c(pix, np.int32)
    cnt = H * W if pix is None else len(pix)
    assert bits_px.shape == (cnt, n_words(k)), (bits_px.shape, cnt)
    assert bits_smp.shape == (int(label_off[-1]), n_words(k))
    L = np.zeros((nl, cnt), np.float64)
    neg = np.zeros_like(L)
    post = np.zeros_like(L)
    d2 = np.zeros((nl, cnt), np.int64) if want_dist2 else None
    rc = _load().oracle_likelihood(_p(image), H, W, _p(bits_px), _p(bits_smp), k, nl,
                                   _p(label_off), _p(sample_pix), float(sigma_c2), float(alpha),
                                   float(d_min), float(kappa_beta), int(mode),
                                   int(rho_variance), _p(pix), cnt,
                                   _p(L), _p(neg), _p(post), _p(d2))
    if rc:
        raise ValueError("oracle_likelihood: invalid arguments")
    out = {"L": L, "neglog": neg, "post": post}
    if want_dist2:
        out["dist2"] = d2
    return out


def iota(a, sigma):
    """Eq. (map_tsm): smooth co-support indicator exp(-a_j^2 / sigma), elementwise."""
    a = np.asarray(a, np.float64)
    return np.exp(-(a * a) / float(sigma))


def median_rows(values):
    """Elementwise median over the rows of a (m, k) array (Eq. approx_cosupp):
    the middle value of each column for odd m, the mean of the two middle
    values for even m. Written out with a sort per column."""
    v = np.sort(np.asarray(values, np.float64), axis=0)
    m = v.shape[0]
    if m < 1:
        raise ValueError("median of an empty set")
    if m % 2:
        return v[m // 2].copy()
    return 0.5 * (v[m // 2 - 1] + v[m // 2])


def smooth_reps(iota_smp, label_off):
    """Eq. (approx_cosupp) / Sec. 3.1: each label's textural representative
    c_i, the elementwise median of its samples' smooth co-supports;
    (n_labels, k) float64."""
    label_off = np.asarray(label_off)
    return np.stack([median_rows(iota_smp[label_off[i]:label_off[i + 1]])
                     for i in range(len(label_off) - 1)])


def smooth_log_posterior(iota_px, reps, beta):
    """Eq. (post_text): log of the texture posterior of each label,
    log softmax_i(-||c_i - iota(O s_x)||_1 / beta_i(x)); iota_px (cnt, k),
    reps (n, k), beta (n, cnt) -> (n, cnt) float64."""
    l1 = np.abs(reps[:, None, :] - iota_px[None, :, :]).sum(axis=2)  # (n, cnt)
    t = -l1 / beta
    tmax = t.max(axis=0)
    return t - (tmax + np.log(np.exp(t - tmax).sum(axis=0)))


def data_term(problem, pix=None, mode=None, want_dist2=False):
    """Whole oracle pipeline on a synthetic problem: codes and co-supports at
    the listed pixels and at every scribble sample, then the likelihoods."""
    prm = problem.params
    p = prm.p
    mode = prm.mode if mode is None else mode
    k = problem.omega.shape[0]
    smooth = mode == 2
    order = int(getattr(prm, "patch_order", 0))
    a_px, bits_px = codes(problem.image, problem.omega, problem.mask, p, prm.tau, pix=pix,
                          want_codes=smooth, order=order)
    a_smp, bits_smp = codes(problem.image, problem.omega, problem.mask, p, prm.tau,
                            pix=problem.sample_pix, want_codes=smooth, order=order)
    out = likelihood(problem.image, bits_px, bits_smp, k, problem.label_off, problem.sample_pix,
                     prm.sigma_c2, prm.alpha, prm.d_min, prm.kappa_beta, mode, pix=pix,
                     want_dist2=want_dist2 or smooth,
                     rho_variance=int(getattr(prm, "rho_variance", 0)))
    if smooth:
        # Sec. 3.1 with Eq. (map_tsm), (approx_cosupp), (post_text): the Parzen
        # sum times the softmax texture posterior on smooth co-supports,
        # beta_i(x) = kappa_beta rho_i(x), rho_i(x) = alpha max(|x - x_v|, d_min)
        sigma = getattr(prm, "iota_sigma", 0.01)
        reps = smooth_reps(iota(a_smp, sigma), problem.label_off)
        rho = prm.alpha * np.maximum(np.sqrt(out["dist2"].astype(np.float64)), prm.d_min)
        L = out["L"] + smooth_log_posterior(iota(a_px, sigma), reps, prm.kappa_beta * rho)
        lmax = L.max(axis=0)
        post = np.exp(L - (lmax + np.log(np.exp(L - lmax).sum(axis=0))))
        out.update({"L": L, "neglog": -L, "post": post, "reps": reps})
        if not want_dist2:
            del out["dist2"]
    out["bits_px"] = bits_px
    out["bits_smp"] = bits_smp
    return out
