"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test states which passage it follows and which plausible mistake it
catches. Sources of truth used here: closed forms derived by hand
(tests/golden/), scipy library routines (Euclidean distance transform,
Gaussian log-densities, Hamming distance, logsumexp, softmax), and exact
invariances of the definitions.
"""
import math
import os

import numpy as np
import pytest
from scipy import ndimage, special, stats
from scipy.spatial import distance

import oracle
from paper_1312_4746_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    rows = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                parts = line.split()
                rows[parts[0]] = np.array([float(v) for v in parts[1:]])
    return rows


def _ramp_image(H, W, c=0.01, channel=0):
    img = np.zeros((H, W, 3), np.float32)
    img[:, :, channel] = (c * np.arange(W, dtype=np.float64))[None, :]
    return img


# ---------------------------------------------------------------- patches (Sec. 2, Sec. 3.1)


def test_patch_ramp_closed_form():
    """Sec. 2 zero-mean/unit-norm patch of a horizontal ramp, interior and at
    the clamped left edge (golden closed form). Catches a transposed window,
    a wrong clamp, a missing centring or normalisation."""
    g = _gold("patch_ramp_p5.txt")
    img = _ramp_image(9, 12)
    mask = np.ones(25, np.float32)
    s = oracle.patches(img, mask, 5, pix=np.array([4 * 12 + 6, 4 * 12 + 0], np.int32))
    np.testing.assert_allclose(s[0].reshape(5, 5), np.tile(g["interior"], (5, 1)), atol=1e-7)
    np.testing.assert_allclose(s[1].reshape(5, 5), np.tile(g["left_edge"], (5, 1)), atol=1e-7)


def test_patch_vertical_ramp_is_transpose():
    """A vertical ramp gives the transposed closed form (window order dy*p+dx)."""
    g = _gold("patch_ramp_p5.txt")
    img = np.zeros((12, 9, 3), np.float32)
    img[:, :, 1] = (0.02 * np.arange(12))[:, None]
    s = oracle.patches(img, np.ones(25, np.float32), 5, pix=np.array([6 * 9 + 4], np.int32))
    np.testing.assert_allclose(s[0].reshape(5, 5), np.tile(g["interior"], (5, 1)).T, atol=1e-7)


@pytest.mark.parametrize("ch,wt", [(1, 0.587), (2, 0.114)])
def test_gray_weights_closed_form(ch, wt):
    """Gray = 0.299 R + 0.587 G + 0.114 B: with R a horizontal ramp and channel
    ``ch`` a vertical ramp of the same slope, the interior patch is
    (0.299 (dx-2) + w (dy-2)) / norm with norm^2 = 5 * 10 * (0.299^2 + w^2).
    Catches wrong or swapped channel weights."""
    H = W = 11
    img = np.zeros((H, W, 3), np.float32)
    img[:, :, 0] = (0.01 * np.arange(W))[None, :]
    img[:, :, ch] = (0.01 * np.arange(H))[:, None]
    s = oracle.patches(img, np.ones(25, np.float32), 5, pix=np.array([5 * W + 5], np.int32))
    dy, dx = np.mgrid[0:5, 0:5]
    expect = 0.299 * (dx - 2) + wt * (dy - 2)
    expect = expect / math.sqrt(50.0 * (0.299**2 + wt**2))
    np.testing.assert_allclose(s[0].reshape(5, 5), expect, atol=2e-6)


def test_mask_applied_before_centring():
    """Sec. 3.1 applies the Gaussian mask before the normalisation, so a
    constant image gives s = (w - mean w) / ||w - mean w||, not zero."""
    p = 7
    w = synth.make_mask(p).astype(np.float64)
    img = np.full((15, 15, 3), 0.5, np.float32)
    s = oracle.patches(img, w.astype(np.float32), p, pix=np.array([7 * 15 + 7], np.int32))[0]
    c = w - w.mean()
    np.testing.assert_allclose(s, c / np.linalg.norm(c), atol=1e-12)


def test_patch_invariants_random():
    """Sec. 2: every patch has zero mean and unit l2 norm."""
    pr = synth.make_problem(20, 24, 2, 10, p=5, seed=3)
    s = oracle.patches(pr.image, pr.mask, 5)
    np.testing.assert_allclose(s.sum(1), 0.0, atol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-12)


def test_gain_invariance_exact():
    """Bias-gain model (Sec. 2): doubling the image is exact in floating point
    and must leave codes bit-identical."""
    pr = synth.make_problem(16, 20, 2, 10, p=5, seed=4)
    a1, b1 = oracle.codes(pr.image * 0.5, pr.omega, pr.mask, 5, 0.1)
    a2, b2 = oracle.codes(pr.image, pr.omega, pr.mask, 5, 0.1)
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)


def test_centre_first_constant_image_is_flat():
    """patch_order 1 centres the gray values before the mask: a constant
    image gives g - mean g = 0 exactly, so s = 0 (where order 0 gives the
    centred mask), and every code is in the co-support."""
    p = 7
    w = synth.make_mask(p)
    img = np.full((15, 15, 3), 0.5, np.float32)
    pix = np.array([7 * 15 + 7], np.int32)
    assert np.all(oracle.patches(img, w, p, pix=pix, order=1) == 0.0)
    assert np.abs(oracle.patches(img, w, p, pix=pix, order=0)).max() > 0.1


def test_centre_first_ramp_closed_form():
    """Horizontal gray ramp g = c dx + b, symmetric mask w(dy, dx): order 1
    gives v = w (c (dx - r)), whose mean is zero by the mask's symmetry, so
    s = w (dx - r) / ||w (dx - r)||, independent of the bias b."""
    p, r = 5, 2
    w = synth.make_mask(p).astype(np.float64).reshape(p, p)
    H, W = 9, 11
    xs = np.arange(W, dtype=np.float64)
    img = np.repeat((0.05 * xs + 0.3)[None, :, None], H, axis=0).repeat(3, axis=2)
    img = img.astype(np.float32)
    q = 4 * W + 5
    s = oracle.patches(img, w.reshape(-1).astype(np.float32), p, pix=np.array([q], np.int32),
                       order=1)[0].reshape(p, p)
    # the gray value of channel-equal pixels is the value itself (weights sum to 1)
    dx = np.arange(p, dtype=np.float64)[None, :] - r
    e = w * dx
    np.testing.assert_allclose(s, e / np.linalg.norm(e), atol=2e-7)
    s2 = oracle.patches(img + np.float32(0.25), w.reshape(-1).astype(np.float32), p,
                        pix=np.array([q], np.int32), order=1)[0].reshape(p, p)
    np.testing.assert_allclose(s2, s, atol=2e-7)
    s0 = oracle.patches(img, w.reshape(-1).astype(np.float32), p, pix=np.array([q], np.int32),
                        order=0)[0].reshape(p, p)
    assert np.abs(s0 - s).max() > 1e-2  # the literal order differs here


def test_orders_agree_for_a_uniform_mask():
    """With a constant mask, w (g - mean g) already has zero mean and equals
    w g - mean(w g): both orders give the same patch and codes."""
    pr = synth.make_problem(16, 18, 2, 8, p=5, seed=19)
    w = np.full(25, 0.7, np.float32)
    a0, b0 = oracle.codes(pr.image, pr.omega, w, 5, 0.1, order=0)
    a1, b1 = oracle.codes(pr.image, pr.omega, w, 5, 0.1, order=1)
    np.testing.assert_allclose(a1, a0, rtol=0, atol=1e-12)
    s1 = oracle.patches(pr.image, pr.mask, 5, order=1)
    np.testing.assert_allclose(s1.sum(1), 0.0, atol=1e-12)
    np.testing.assert_allclose(np.linalg.norm(s1, axis=1), 1.0, atol=1e-12)


def test_flat_window_all_cosupport():
    """An all-zero window has sum c^2 == 0, so s = 0, a = 0 and every j is in
    the co-support (Eq. 1)."""
    img = np.zeros((9, 9, 3), np.float32)
    om = synth.make_omega(40, 25, 1)
    a, b = oracle.codes(img, om, np.ones(25, np.float32), 5, 0.1)
    assert np.all(a == 0.0)
    assert np.all(b[:, 0] == 0xFFFFFFFF) and np.all(b[:, 1] == 0xFF)


# ---------------------------------------------------------------- codes and co-support (Sec. 2, Eq. 1)


def test_codes_select_rows():
    """a = O s (Sec. 2): rows that are unit vectors e_t pick s_t; a row that
    depends on dy only is orthogonal to a horizontal-ramp patch (a_j = 0, in
    the co-support); the all-ones row gives sum(s) = 0. Catches O^T s or a
    row/column mix-up."""
    n, p = 25, 5
    rows = [np.eye(n)[t] for t in (0, 3, 7, 12, 24)]
    rows.append(np.repeat(np.array([1.0, -2.0, 0.5, 3.0, 1.0]), 5) / 4.0)  # f(dy)
    rows.append(np.ones(n) / 5.0)
    om = np.array(rows, np.float32)
    img = _ramp_image(9, 12)
    a, b = oracle.codes(img, om, np.ones(n, np.float32), p, 0.1,
                        pix=np.array([4 * 12 + 6], np.int32))
    s = (np.arange(5) - 2) / math.sqrt(50.0)
    expect = [s[t % 5] for t in (0, 3, 7, 12, 24)] + [0.0, 0.0]
    np.testing.assert_allclose(a[0], expect, atol=1e-7)
    bits = [(b[0, 0] >> j) & 1 for j in range(7)]
    assert bits == [int(abs(v) <= 0.1) for v in expect]


def test_cosupport_threshold_inclusive():
    """The co-support test |a_j| <= tau is inclusive at the threshold."""
    pr = synth.make_problem(12, 12, 2, 5, p=5, seed=5)
    a, _ = oracle.codes(pr.image, pr.omega, pr.mask, 5, 0.1, pix=np.array([50], np.int32))
    j = 7
    tau = abs(a[0, j])
    _, b_eq = oracle.codes(pr.image, pr.omega, pr.mask, 5, tau, pix=np.array([50], np.int32))
    _, b_lo = oracle.codes(pr.image, pr.omega, pr.mask, 5, np.nextafter(tau, 0.0),
                           pix=np.array([50], np.int32))
    assert (b_eq[0, 0] >> j) & 1 == 1
    assert (b_lo[0, 0] >> j) & 1 == 0


def test_bitmask_matches_codes():
    """Packing: bit j of word j >> 5 is set iff |a_j| <= tau; pad bits are 0."""
    pr = synth.make_problem(10, 14, 2, 5, p=7, k=98, seed=6)
    a, b = oracle.codes(pr.image, pr.omega, pr.mask, 7, 0.1)
    unpacked = np.unpackbits(b.view(np.uint8), axis=1, bitorder="little")
    assert np.array_equal(unpacked[:, :98].astype(bool), np.abs(a) <= 0.1)
    assert not unpacked[:, 98:].any()


# ---------------------------------------------------------------- TSM (Eq. tsm_clean) and majority (Eq. tex-rep)


def test_tsm_is_hamming():
    """Eq. (tsm_clean) equals the Hamming distance of the indicator vectors
    (scipy), is symmetric, bounded by k and zero on equal inputs."""
    rng = np.random.default_rng(7)
    k = 98
    for _ in range(20):
        a = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
        b = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
        a[3] &= 0x3
        b[3] &= 0x3
        ua = np.unpackbits(a.view(np.uint8), bitorder="little")[:k]
        ub = np.unpackbits(b.view(np.uint8), bitorder="little")[:k]
        h = oracle.tsm(a, b, k)
        assert h == round(distance.hamming(ua, ub) * k)
        assert h == oracle.tsm(b, a, k) and 0 <= h <= k and oracle.tsm(a, a, k) == 0


def test_majority_counts_and_tie():
    """Eq. (tex-rep): set iff count >= m/2. m = 2 with one vote is a tie and
    sets the bit; m = 3 with one vote does not; m = 1 copies the sample."""
    k = 40
    rng = np.random.default_rng(8)
    bits = rng.integers(0, 2**32, (6, 2), dtype=np.uint64).astype(np.uint32)
    bits[:, 1] &= 0xFF
    off = np.array([0, 1, 3, 6], np.int32)
    rep = oracle.majority(bits, k, off)
    u = np.unpackbits(bits.view(np.uint8), axis=1, bitorder="little")[:, :k].astype(int)
    for i in range(3):
        cnt = u[off[i]:off[i + 1]].sum(0)
        m = off[i + 1] - off[i]
        expect = (2 * cnt >= m)
        got = np.unpackbits(rep[i].view(np.uint8), bitorder="little")[:k].astype(bool)
        assert np.array_equal(got, expect)
    assert np.array_equal(rep[0], bits[0])
    # explicit tie: two samples disagreeing everywhere -> every bit set
    two = np.array([[0xFFFFFFFF, 0x0], [0x0, 0xFF]], np.uint32)
    r2 = oracle.majority(two, 40, np.array([0, 2], np.int32))
    assert r2[0, 0] == 0xFFFFFFFF and r2[0, 1] == 0xFF


# ---------------------------------------------------------------- nearest-scribble distance (Sec. 3.1)


def test_dist2_matches_scipy_edt():
    """Squared distance to the nearest scribble equals scipy's exact Euclidean
    distance transform, squared; it is 0 on the scribble pixels."""
    pr = synth.make_problem(40, 56, 3, 25, p=5, seed=9)
    d2 = oracle.dist2(pr.H, pr.W, pr.label_off, pr.sample_pix)
    for i in range(pr.n_labels):
        seeds = np.ones(pr.H * pr.W, bool)
        seeds[pr.sample_pix[pr.label_off[i]:pr.label_off[i + 1]]] = False
        edt = ndimage.distance_transform_edt(seeds.reshape(pr.H, pr.W))
        assert np.array_equal(d2[i], np.rint(edt.ravel() ** 2).astype(np.int64))
        assert np.all(d2[i][pr.sample_pix[pr.label_off[i]:pr.label_off[i + 1]]] == 0)


# ---------------------------------------------------------------- likelihood (Sec. 3.1 Eq. color / post_text)


def _setup(H=14, W=18, nl=2, m=6, p=5, seed=10):
    pr = synth.make_problem(H, W, nl, m, p=p, seed=seed)
    _, bpx = oracle.codes(pr.image, pr.omega, pr.mask, p, 0.1)
    _, bsm = oracle.codes(pr.image, pr.omega, pr.mask, p, 0.1, pix=pr.sample_pix)
    return pr, bpx, bsm


def _kernel_terms(pr, bpx, bsm, q, s, rho, beta, texture=True, rho_variance=False):
    """log of one summand via scipy's Gaussian log-densities (location
    covariance rho^2 I, or rho I when rho is read as the variance)."""
    W = pr.W
    y, x = divmod(q, W)
    sp = pr.sample_pix[s]
    sy, sx = divmod(int(sp), W)
    cov = (rho if rho_variance else rho * rho) * np.eye(2)
    loc = stats.multivariate_normal(mean=[0, 0], cov=cov).logpdf([x - sx, y - sy])
    Ix = pr.image.reshape(-1, 3)[q].astype(np.float64)
    Is = pr.image.reshape(-1, 3)[sp].astype(np.float64)
    col = stats.multivariate_normal(mean=[0, 0, 0], cov=1.3 * np.eye(3)).logpdf(Ix - Is)
    k = pr.omega.shape[0]
    ux = np.unpackbits(bpx[q].view(np.uint8), bitorder="little")[:k]
    us = np.unpackbits(bsm[s].view(np.uint8), bitorder="little")[:k]
    tex = -distance.hamming(ux, us) * k / beta if texture else 0.0
    return loc + col + tex


def _rho_beta(pr, q, i, alpha=1.3, d_min=1.0, kb=1.0):
    d2 = oracle.dist2(pr.H, pr.W, pr.label_off, pr.sample_pix, pix=np.array([q], np.int32))
    rho = alpha * max(math.sqrt(d2[i, 0]), d_min)
    return rho, kb * rho


def test_single_sample_closed_form():
    """m_i = 1: L_i is one Gaussian location term (width alpha*max(d, d_min))
    times one colour Gaussian times exp(-TSM/beta); for x != x_1 the location
    exponent is the constant -1/(2 alpha^2)."""
    pr, bpx, bsm = _setup(m=1)
    out = oracle.likelihood(pr.image, bpx, bsm, pr.k, pr.label_off, pr.sample_pix)
    for q in (0, 37, 100, 251):
        for i in range(pr.n_labels):
            rho, beta = _rho_beta(pr, q, i)
            s = pr.label_off[i]
            expect = _kernel_terms(pr, bpx, bsm, q, s, rho, beta)
            assert abs(out["L"][i, q] - expect) < 1e-10
            y, x = divmod(q, pr.W)
            sy, sx = divmod(int(pr.sample_pix[s]), pr.W)
            d2 = (x - sx) ** 2 + (y - sy) ** 2
            if d2 >= 1:
                assert abs(-d2 / (2 * rho * rho) + 1 / (2 * 1.3**2)) < 1e-12


def test_parzen_sum_scipy():
    """Eq. (color) with the per-sample texture factor: log of the mean over
    the label's samples of the product of kernels, via scipy logsumexp.
    Catches a dropped 1/m_i, a wrong normaliser or a wrong sign."""
    pr, bpx, bsm = _setup(m=5)
    out = oracle.likelihood(pr.image, bpx, bsm, pr.k, pr.label_off, pr.sample_pix)
    for q in (3, 88, 190):
        for i in range(pr.n_labels):
            rho, beta = _rho_beta(pr, q, i)
            terms = [_kernel_terms(pr, bpx, bsm, q, s, rho, beta)
                     for s in range(pr.label_off[i], pr.label_off[i + 1])]
            expect = special.logsumexp(terms) - math.log(len(terms))
            assert abs(out["L"][i, q] - expect) < 1e-10


def test_rho_variance_reading_scipy():
    """rho read as the location kernel's variance (Sec. 3.1 names it so):
    the Parzen sum against scipy with covariance rho I; beta = kappa_beta rho
    unchanged. A dropped switch (rho^2 kept in the exponent or in the
    normaliser) fails here."""
    pr, bpx, bsm = _setup(m=4, seed=17)
    out = oracle.likelihood(pr.image, bpx, bsm, pr.k, pr.label_off, pr.sample_pix,
                            rho_variance=1)
    for q in (2, 61, 140, 251):
        for i in range(pr.n_labels):
            rho, beta = _rho_beta(pr, q, i)
            terms = [_kernel_terms(pr, bpx, bsm, q, s, rho, beta, rho_variance=True)
                     for s in range(pr.label_off[i], pr.label_off[i + 1])]
            expect = special.logsumexp(terms) - math.log(len(terms))
            assert abs(out["L"][i, q] - expect) < 1e-10


def test_rho_readings_agree_at_unit_rho():
    """With rho = 1 at every pixel (alpha = 1 / d_min and every distance
    below d_min) the two readings are the same kernel, in every mode."""
    pr, bpx, bsm = _setup(m=3, seed=18)
    kw = dict(alpha=1e-3, d_min=1e3)
    for mode in (0, 1):
        a = oracle.likelihood(pr.image, bpx, bsm, pr.k, pr.label_off, pr.sample_pix, mode=mode,
                              **kw)
        b = oracle.likelihood(pr.image, bpx, bsm, pr.k, pr.label_off, pr.sample_pix, mode=mode,
                              rho_variance=1, **kw)
        np.testing.assert_allclose(a["L"], b["L"], rtol=0, atol=1e-12)
    c = oracle.likelihood(pr.image, bpx, bsm, pr.k, pr.label_off, pr.sample_pix, rho_variance=1)
    d = oracle.likelihood(pr.image, bpx, bsm, pr.k, pr.label_off, pr.sample_pix)
    assert np.abs(c["L"] - d["L"]).max() > 1e-3  # and differ elsewhere


def test_duplicate_samples_weight_the_parzen_sum():
    """A scribble pixel listed twice counts twice: L is the log of the
    list's mean, so doubling every sample of a label changes nothing, and
    doubling one sample weights its term by 2 (scipy logsumexp with
    weights); the per-sample texture kernel and the distances see the list
    as given."""
    pr, bpx, bsm = _setup(m=4, seed=20)
    off = pr.label_off
    base = oracle.likelihood(pr.image, bpx, bsm, pr.k, off, pr.sample_pix)
    # every sample of every label twice
    rep = np.concatenate([np.repeat(pr.sample_pix[off[i]:off[i + 1]], 2)
                          for i in range(pr.n_labels)]).astype(np.int32)
    off2 = (2 * off).astype(np.int32)
    _, bsm2 = oracle.codes(pr.image, pr.omega, pr.mask, 5, 0.1, pix=rep)
    two = oracle.likelihood(pr.image, bpx, bsm2, pr.k, off2, rep)
    np.testing.assert_allclose(two["L"], base["L"], rtol=0, atol=1e-12)
    # the first sample of label 0 twice
    s0 = int(off[0])
    one = np.insert(pr.sample_pix, s0, pr.sample_pix[s0]).astype(np.int32)
    off1 = off.copy().astype(np.int32)
    off1[1:] += 1
    _, bsm1 = oracle.codes(pr.image, pr.omega, pr.mask, 5, 0.1, pix=one)
    out = oracle.likelihood(pr.image, bpx, bsm1, pr.k, off1, one)
    for q in (5, 90):
        rho, beta = _rho_beta(pr, q, 0)
        terms = [_kernel_terms(pr, bpx, bsm, q, s, rho, beta) for s in range(off[0], off[1])]
        w = np.ones(len(terms))
        w[0] = 2.0
        expect = special.logsumexp(terms, b=w) - math.log(w.sum())
        assert abs(out["L"][0, q] - expect) < 1e-10


def test_constant_image_is_plain_kde():
    """A constant image makes every patch identical (TSM = 0) and every
    colour difference zero, so L_i is a plain 2-D Gaussian KDE of the scribble
    locations (bandwidth rho_i(x)) plus the colour normaliser."""
    pr = synth.make_problem(12, 16, 2, 4, p=5, seed=11)
    pr.image[:] = 0.3
    _, bpx = oracle.codes(pr.image, pr.omega, pr.mask, 5, 0.1)
    _, bsm = oracle.codes(pr.image, pr.omega, pr.mask, 5, 0.1, pix=pr.sample_pix)
    assert (bpx == bpx[0]).all()
    out = oracle.likelihood(pr.image, bpx, bsm, pr.k, pr.label_off, pr.sample_pix)
    col0 = stats.multivariate_normal(mean=np.zeros(3), cov=1.3 * np.eye(3)).logpdf(np.zeros(3))
    for q in (0, 17, 120, 191):
        y, x = divmod(q, pr.W)
        for i in range(2):
            rho, _ = _rho_beta(pr, q, i)
            pts = [divmod(int(v), pr.W) for v in pr.sample_pix[pr.label_off[i]:pr.label_off[i + 1]]]
            kde = np.mean([stats.multivariate_normal(mean=[sx, sy], cov=rho * rho * np.eye(2)).pdf([x, y])
                           for sy, sx in pts])
            assert abs(out["L"][i, q] - (math.log(kde) + col0)) < 1e-10


def test_posterior_normalised_and_softmax():
    """Label posteriors are the softmax of L over labels and sum to 1."""
    pr, bpx, bsm = _setup(nl=3, m=4)
    out = oracle.likelihood(pr.image, bpx, bsm, pr.k, pr.label_off, pr.sample_pix)
    np.testing.assert_allclose(out["post"].sum(0), 1.0, atol=1e-14)
    np.testing.assert_allclose(out["post"], special.softmax(out["L"], axis=0), atol=1e-14)
    np.testing.assert_array_equal(out["neglog"], -out["L"])


def test_sample_permutation_invariance():
    """The Parzen sum is over a set: permuting samples within a label leaves
    L unchanged (to rounding)."""
    pr, bpx, bsm = _setup(nl=2, m=8)
    out1 = oracle.likelihood(pr.image, bpx, bsm, pr.k, pr.label_off, pr.sample_pix)
    rng = np.random.default_rng(12)
    perm = np.concatenate([pr.label_off[i] + rng.permutation(pr.label_off[i + 1] - pr.label_off[i])
                           for i in range(2)])
    out2 = oracle.likelihood(pr.image, bpx, bsm[perm], pr.k, pr.label_off, pr.sample_pix[perm])
    np.testing.assert_allclose(out1["L"], out2["L"], atol=1e-12)


def test_translation_invariance():
    """Shifting image content and scribbles by an integer offset leaves L
    unchanged at pixels whose windows (and the samples' windows) stay inside
    both images."""
    big = synth.make_problem(30, 34, 2, 6, p=5, seed=13)
    sh = 3
    img1 = big.image[: 30 - sh, : 34 - sh]
    img2 = big.image[sh:, sh:]
    H2, W2 = img2.shape[:2]
    rng = np.random.default_rng(14)
    ys = rng.integers(2 + sh, H2 - 2 - sh, 12)
    xs = rng.integers(2 + sh, W2 - 2 - sh, 12)
    smp1 = (ys + sh) * W2 + (xs + sh)  # same content in img1 coordinates
    smp2 = ys * W2 + xs
    off = np.array([0, 6, 12], np.int32)
    res = []
    for img, smp, d in ((img1, smp1, sh), (img2, smp2, 0)):
        _, bs = oracle.codes(img, big.omega, big.mask, 5, 0.1, pix=smp.astype(np.int32))
        qy, qx = np.mgrid[8:14, 8:16]
        pix = ((qy + d) * W2 + (qx + d)).ravel().astype(np.int32)
        _, bp = oracle.codes(img, big.omega, big.mask, 5, 0.1, pix=pix)
        res.append(oracle.likelihood(img, bp, bs, big.k, off, smp.astype(np.int32), pix=pix)["L"])
    np.testing.assert_allclose(res[0], res[1], atol=1e-12)


def test_factorised_reduces_to_parzen():
    """Factorised form, Eq. (joined): with identical co-supports everywhere
    (constant image) the texture posterior is uniform, so L_F = L_S - log n."""
    pr = synth.make_problem(12, 16, 3, 4, p=5, seed=15)
    pr.image[:] = 0.7
    _, bpx = oracle.codes(pr.image, pr.omega, pr.mask, 5, 0.1)
    _, bsm = oracle.codes(pr.image, pr.omega, pr.mask, 5, 0.1, pix=pr.sample_pix)
    s = oracle.likelihood(pr.image, bpx, bsm, pr.k, pr.label_off, pr.sample_pix, mode=0)
    f = oracle.likelihood(pr.image, bpx, bsm, pr.k, pr.label_off, pr.sample_pix, mode=1)
    np.testing.assert_allclose(f["L"], s["L"] - math.log(3), atol=1e-12)


def test_beta_limits():
    """Sec. 3.1: large beta makes the texture factor uninformative (per-sample
    form reduces to the colour-location Parzen sum, checked with scipy); small
    beta makes the texture posterior winner-take-all (factorised form)."""
    pr, bpx, bsm = _setup(nl=3, m=4, seed=16)
    big = oracle.likelihood(pr.image, bpx, bsm, pr.k, pr.label_off, pr.sample_pix,
                            kappa_beta=1e15, mode=0)
    for q in (5, 77):
        for i in range(3):
            rho, beta = _rho_beta(pr, q, i)
            terms = [_kernel_terms(pr, bpx, bsm, q, s, rho, beta, texture=False)
                     for s in range(pr.label_off[i], pr.label_off[i + 1])]
            assert abs(big["L"][i, q] - (special.logsumexp(terms) - math.log(4))) < 1e-9
    # factorised form, large beta: texture posterior uniform -> L_F = Parzen - log n
    f_big = oracle.likelihood(pr.image, bpx, bsm, pr.k, pr.label_off, pr.sample_pix,
                              kappa_beta=1e15, mode=1)
    np.testing.assert_allclose(f_big["L"], big["L"] - math.log(3), atol=1e-9)
    # small beta: the label with the smallest TSM/rho takes the whole texture mass
    small = oracle.likelihood(pr.image, bpx, bsm, pr.k, pr.label_off, pr.sample_pix,
                              kappa_beta=1e-6, mode=1)
    rep = oracle.majority(bsm, pr.k, pr.label_off)
    d2 = oracle.dist2(pr.H, pr.W, pr.label_off, pr.sample_pix)
    for q in range(0, pr.H * pr.W, 7):
        rho = 1.3 * np.maximum(np.sqrt(d2[:, q]), 1.0)
        h = np.array([oracle.tsm(bpx[q], rep[i], pr.k) for i in range(3)]) / rho
        order = np.argsort(h)
        if h[order[1]] - h[order[0]] < 1e-3:
            continue
        win = order[0]
        # parzen part of the winner is unchanged: its texture log-posterior is ~0
        assert abs(small["L"][win, q] - f_big["L"][win, q] - math.log(3)) < 1e-6


# ---------------------------------------------------------------- smooth texture (Sec. 2, Sec. 3.1)

def test_iota_closed_form():
    """Eq. (map_tsm): iota(0) = 1, iota(sqrt(sigma)) = 1/e, even in a, and it
    tends to the co-support indicator as sigma -> 0."""
    s = 0.01
    np.testing.assert_array_equal(oracle.iota([0.0, -0.0], s), [1.0, 1.0])
    assert abs(oracle.iota([math.sqrt(s)], s)[0] - math.exp(-1.0)) < 1e-15
    a = np.array([-0.3, -0.05, 0.02, 0.4])
    np.testing.assert_array_equal(oracle.iota(a, s), oracle.iota(-a, s))
    assert np.all(oracle.iota(a, 1e-9) < 1e-300)


def test_median_rows_hand_values():
    """Eq. (approx_cosupp): elementwise median; odd m -> the middle value,
    even m -> the mean of the two middle values, m = 1 -> the row itself;
    independent of the row order."""
    v = np.array([[0.9, 0.1], [0.1, 0.4], [0.5, 0.7]])
    np.testing.assert_array_equal(oracle.median_rows(v), [0.5, 0.4])
    np.testing.assert_array_equal(oracle.median_rows(v[:2]), [0.5, 0.25])
    np.testing.assert_array_equal(oracle.median_rows(v[1:2]), v[1])
    np.testing.assert_array_equal(oracle.median_rows(v[::-1]), [0.5, 0.4])
    w = np.array([[4.0], [1.0], [3.0], [2.0]])
    np.testing.assert_array_equal(oracle.median_rows(w), [2.5])


def test_smooth_posterior_closed_form():
    """Eq. (post_text) on a hand example: representatives (1, 0) and (0, 1),
    a pixel with iota = (1, 0): l1 distances 0 and 2, so with beta = 1 the
    log posteriors are -log(1 + e^-2) and -2 - log(1 + e^-2); they sum to 1 in
    probability; equal representatives give the uniform posterior; small beta
    is winner-take-all, large beta uniform."""
    reps = np.array([[1.0, 0.0], [0.0, 1.0]])
    px = np.array([[1.0, 0.0]])
    lp = oracle.smooth_log_posterior(px, reps, np.ones((2, 1)))
    z = math.log(1.0 + math.exp(-2.0))
    np.testing.assert_allclose(lp[:, 0], [-z, -2.0 - z], rtol=0, atol=1e-15)
    assert abs(np.exp(lp).sum() - 1.0) < 1e-15
    same = oracle.smooth_log_posterior(px, np.ones((3, 2)), np.ones((3, 1)))
    np.testing.assert_allclose(same, -math.log(3), atol=1e-15)
    win = oracle.smooth_log_posterior(px, reps, np.full((2, 1), 1e-3))
    assert win[0, 0] > -1e-12 and win[1, 0] < -1e3
    flat = oracle.smooth_log_posterior(px, reps, np.full((2, 1), 1e12))
    np.testing.assert_allclose(flat, -math.log(2), atol=1e-9)


@pytest.mark.parametrize("val", [0.0, 0.7])
def test_smooth_mode_constant_image(val):
    """Constant image: every masked patch is the same (the zero image: s = 0,
    all codes 0, iota = 1), so every pixel and sample has the same smooth
    co-support, every representative equals it and the texture posterior is
    uniform: L (mode 2) = Parzen sum - log n."""
    pr = synth.make_problem(12, 16, 3, 4, p=5, seed=15)
    pr.image[:] = val
    pr.params.mode = 2
    out = oracle.data_term(pr)
    a0, _ = oracle.codes(pr.image, pr.omega, pr.mask, 5, 0.1, pix=np.array([0], np.int32))
    np.testing.assert_array_equal(out["reps"], np.repeat(oracle.iota(a0, 0.01), 3, axis=0))
    if val == 0.0:
        np.testing.assert_array_equal(out["reps"], np.ones((3, pr.k)))
    _, bpx = oracle.codes(pr.image, pr.omega, pr.mask, 5, 0.1)
    _, bsm = oracle.codes(pr.image, pr.omega, pr.mask, 5, 0.1, pix=pr.sample_pix)
    parzen = oracle.likelihood(pr.image, bpx, bsm, pr.k, pr.label_off, pr.sample_pix, mode=2)
    np.testing.assert_allclose(out["L"], parzen["L"] - math.log(3), atol=1e-12)
    np.testing.assert_allclose(out["post"].sum(axis=0), 1.0, atol=1e-12)


def test_smooth_mode_single_sample_labels():
    """One scribble sample per label: each representative is that sample's
    smooth co-support, so at a sample's own pixel the l1 distance to its
    label's representative is 0 and that label's texture posterior is the
    largest; the Parzen part is the mode-2 C oracle's."""
    pr = synth.make_problem(20, 24, 3, 1, p=5, seed=17)
    pr.params.mode = 2
    out = oracle.data_term(pr, pix=pr.sample_pix)
    a_smp, _ = oracle.codes(pr.image, pr.omega, pr.mask, 5, 0.1, pix=pr.sample_pix)
    np.testing.assert_array_equal(out["reps"], oracle.iota(a_smp, 0.01))
    _, bpx = oracle.codes(pr.image, pr.omega, pr.mask, 5, 0.1, pix=pr.sample_pix)
    parzen = oracle.likelihood(pr.image, bpx, bpx, pr.k, pr.label_off, pr.sample_pix,
                               mode=2, pix=pr.sample_pix)
    tex = out["L"] - parzen["L"]  # log texture posterior at each sample pixel
    for q in range(3):
        assert np.argmax(tex[:, q]) == q or np.isclose(tex[q, q], tex[:, q].max())
