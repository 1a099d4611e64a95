"""Pins of the unsupervised-mode reference (oracle/unsup.py, Sec. 3.2)."""
import numpy as np
import pytest

from oracle import unsup


def _blobs(rng, n, centres, spread):
    lab = rng.integers(0, len(centres), n)
    X = np.asarray(centres, np.float64)[lab] + rng.normal(0, spread, (n, len(centres[0])))
    return X.astype(np.float32), lab


def test_kmeans_matches_scipy_kmeans2():
    """Same start and round count as scipy's Lloyd iteration (float64 means):
    the centres agree to float64 rounding, and the final assignment is
    scipy's nearest-centroid routine on those centres."""
    vq = pytest.importorskip("scipy.cluster.vq")
    rng = np.random.default_rng(10)
    X, _ = _blobs(rng, 3000, [[0.2, 0.3, 0.7], [0.8, 0.1, 0.2], [0.5, 0.9, 0.4],
                              [0.1, 0.1, 0.1]], 0.08)
    init = [5, 17, 400, 1234]
    for T in (1, 4, 12):
        C, lab = unsup.kmeans(X, init, T)
        ref, _ = vq.kmeans2(X.astype(np.float64), X[init].astype(np.float64), iter=T,
                            minit="matrix", missing="warn")
        np.testing.assert_allclose(C, ref, rtol=0, atol=1e-13)
        lab_ref, _ = vq.vq(X.astype(np.float64), C.astype(np.float64))
        np.testing.assert_array_equal(lab, lab_ref)


def test_kmeans_objective_non_increasing_and_blob_means():
    rng = np.random.default_rng(11)
    centres = [[0.1, 0.2, 0.3], [0.9, 0.8, 0.7], [0.2, 0.9, 0.1]]
    X, truth = _blobs(rng, 2400, centres, 0.02)
    init = [int(np.nonzero(truth == a)[0][0]) for a in range(3)]
    prev = np.inf
    for T in range(6):
        C, lab = unsup.kmeans(X, init, T)
        obj = float(((X.astype(np.float64) - C[lab]) ** 2).sum())
        assert obj <= prev * (1 + 1e-12)
        prev = obj
    np.testing.assert_array_equal(lab, truth)
    for a in range(3):
        np.testing.assert_allclose(C[a], X[truth == a].astype(np.float64).mean(axis=0),
                                   rtol=0, atol=1e-14)


def test_kmeans_empty_class_keeps_centre_and_ties_go_low():
    X = np.array([[0, 0, 0], [1, 1, 1], [1, 1, 0.9]], np.float32)
    C, lab = unsup.kmeans(X, [0, 0, 1], 3)  # classes 0 and 1 start equal
    np.testing.assert_array_equal(lab, [0, 2, 2])  # the tie goes to class 0
    np.testing.assert_array_equal(C[1], X[0])  # class 1 never wins a pixel
    assert float(C[2, 2]) == (1.0 + float(np.float32(0.9))) / 2


def test_mean_is_the_true_mean():
    """A centroid is the plain mean of its members (no rounding of the
    values): a hand case with a value far below the others' spacing, and
    the update of one class leaves the others alone."""
    X = np.array([[2.0 ** -25, 0.5, 1.0], [0.0, 0.25, 1.0], [0.7, 0.7, 0.7]], np.float32)
    C0 = np.array([[0.0, 0.0, 0.0], [9.0, 9.0, 9.0], [0.6, 0.6, 0.6]])
    C = unsup.colour_means(X, np.array([0, 0, 2]), C0)
    np.testing.assert_array_equal(C[0], [2.0 ** -26, 0.375, 1.0])
    np.testing.assert_array_equal(C[1], C0[1])
    np.testing.assert_array_equal(C[2], X[2].astype(np.float64))


def test_texture_medians_match_numpy_median():
    """The k-medians update against numpy's median per class (odd, even and
    single-member classes); an empty class keeps its centre."""
    rng = np.random.default_rng(12)
    k, N = 7, 31
    V = rng.uniform(0, 1, (k, N)).astype(np.float32)
    lab = np.array([0] * 10 + [1] * 11 + [3] * 1 + [0] * 9, np.int32)[:N]
    C0 = rng.uniform(0, 1, (4, k))
    C = unsup.texture_medians(V, lab, C0)
    for b in (0, 1, 3):
        np.testing.assert_array_equal(C[b], np.median(V[:, lab == b].astype(np.float64), axis=1))
    np.testing.assert_array_equal(C[2], C0[2])


def test_kmedians_assignment_and_centres():
    """Assignment = argmin of scipy's city-block distances (float64) on data
    without near ties; every centre is its members' elementwise median; the
    l1 objective does not grow over the rounds."""
    dist = pytest.importorskip("scipy.spatial.distance")
    rng = np.random.default_rng(13)
    k, N = 9, 1500
    base = rng.uniform(0, 1, (4, k))
    truth = rng.integers(0, 4, N)
    V = np.clip(base[truth] + rng.laplace(0, 0.03, (N, k)), 0, 1).astype(np.float32).T.copy()
    init = [int(np.nonzero(truth == b)[0][0]) for b in range(4)]
    prev = np.inf
    for T in (0, 1, 2, 5):
        C, lab = unsup.kmedians(V, init, T)
        D = dist.cdist(V.T.astype(np.float64), C, "cityblock")
        srt = np.sort(D, axis=1)
        clear = (srt[:, 1] - srt[:, 0]) > 1e-12
        np.testing.assert_array_equal(lab[clear], np.argmin(D, axis=1)[clear])
        obj = float(D[np.arange(N), lab].sum())
        assert obj <= prev * (1 + 1e-6)
        prev = obj
    # centres after T rounds are the medians of the members of round T's assignment
    C4, _ = unsup.kmedians(V, init, 4)
    lab4 = unsup.assign_texture(V, unsup.kmedians(V, init, 3)[0])
    for b in range(4):
        np.testing.assert_array_equal(C4[b], np.median(V[:, lab4 == b].astype(np.float64), axis=1))


def test_median_is_l1_optimal():
    rng = np.random.default_rng(14)
    v = rng.uniform(0, 1, (15, 5)).astype(np.float32)
    c = unsup.texture_medians(v.T, np.zeros(15, np.int32), np.zeros((1, 5)))[0]
    cost = np.abs(v - c).sum()
    for _ in range(50):
        d = c + rng.normal(0, 0.05, 5)
        assert np.abs(v - d).sum() >= cost - 1e-12


def test_data_term_closed_forms():
    rng = np.random.default_rng(15)
    H, W, k = 4, 5, 6
    img = rng.uniform(0, 1, (H, W, 3)).astype(np.float32)
    io = rng.uniform(0, 1, (k, H * W))
    cc = rng.uniform(0, 1, (3, 3)).astype(np.float32)
    tc = rng.uniform(0, 1, (2, k)).astype(np.float32)
    f = unsup.data_term_from_centres(img, io, cc, tc, 0.05, 0.7)
    # the product of two normalised posteriors is normalised over the 6 segments
    np.testing.assert_allclose(np.exp(-f).sum(axis=0), 1.0, atol=1e-12)
    # hand evaluation at one pixel
    x, q = img[2, 3].astype(np.float64), 2 * W + 3
    ec = np.array([np.exp(-((x - cc[a]) ** 2).sum() / 0.1) for a in range(3)])
    et = np.array([np.exp(-np.abs(tc[b] - io[:, q]).sum() / 0.7) for b in range(2)])
    want = -np.log(np.outer(ec / ec.sum(), et / et.sum())).reshape(6)
    np.testing.assert_allclose(f[:, 2, 3], want, rtol=1e-12)
    # one class on each side: f = 0; a huge beta: the texture factor is uniform
    f1 = unsup.data_term_from_centres(img, io, cc[:1], tc[:1], 0.05, 0.7)
    np.testing.assert_allclose(f1, 0.0, atol=1e-15)
    fb = unsup.data_term_from_centres(img, io, cc, tc, 0.05, 1e300)
    fc = unsup.data_term_from_centres(img, io, cc, tc[:1], 0.05, 0.7)
    np.testing.assert_allclose(fb[0::2], fc + np.log(2.0), atol=1e-12)


def test_data_term_start_pixels_prefer_their_segment():
    """With zero rounds every centre is its start pixel's value, so a start
    pixel's own (colour, texture) segment has the smallest f there."""
    import oracle
    from paper_1312_4746_gb300 import synth
    pr = synth.make_problem(24, 28, 2, 8, p=5, k=50, seed=16)
    ci, ti = [3, 300, 600], [50, 500]
    out = unsup.data_term(pr.image, pr.omega, pr.mask, 5, 0.01, 0.02, 0.5, 3, 2, ci, ti,
                          kmeans_iterations=0, kmedians_iterations=0)
    f = out["f"].reshape(6, -1)
    for a, qa in enumerate(ci):
        # the colour factor is largest for class a at its start pixel
        col = [np.exp(-f[a2 * 2:(a2 + 1) * 2, qa]).sum() for a2 in range(3)]
        assert int(np.argmax(col)) == a
    for b, qb in enumerate(ti):
        tex = [np.exp(-f[b2::2, qb]).sum() for b2 in range(2)]
        assert int(np.argmax(tex)) == b
    assert oracle.iota(np.zeros(1), 0.01)[0] == 1.0
