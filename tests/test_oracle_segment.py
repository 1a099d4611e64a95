"""Pins of the FP64 segmentation reference (oracle/segment.py, Sec. 4)."""
import math

import numpy as np
import pytest

from oracle import segment as seg


def _project_sorted(y):
    """Projection onto the simplex by sorting (a different algorithm from
    Michelot's): theta from the largest prefix whose shifted values stay
    positive, u = max(y - theta, 0)."""
    y = np.asarray(y, np.float64)
    s = np.sort(y)[::-1]
    c = np.cumsum(s) - 1.0
    j = np.arange(1, len(y) + 1)
    rho = np.nonzero(s - c / j > 0)[0][-1]
    theta = c[rho] / (rho + 1)
    return np.maximum(y - theta, 0.0)


def test_michelot_matches_sorted_projection():
    rng = np.random.default_rng(0)
    for n in (1, 2, 3, 5, 8, 17):
        y = rng.normal(0, 2, (n, 200))
        got = seg.project_simplex_michelot(y)
        want = np.stack([_project_sorted(y[:, q]) for q in range(200)], axis=1)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
        assert np.all(got >= 0) and np.allclose(got.sum(axis=0), 1.0, atol=1e-12)


def test_projection_keeps_feasible_points():
    rng = np.random.default_rng(1)
    u = rng.dirichlet(np.ones(4), 50).T
    np.testing.assert_allclose(seg.project_simplex_michelot(u), u, atol=1e-15)


def test_div_is_negative_adjoint_of_grad():
    rng = np.random.default_rng(2)
    for shape in ((3, 7, 9), (2, 1, 5), (2, 6, 1), (1, 2, 2)):
        u = rng.normal(size=shape)
        px, py = rng.normal(size=shape), rng.normal(size=shape)
        gx, gy = seg.grad(u)
        # components that grad never produces are zero in every iterate
        px[..., :, -1] = 0.0
        py[..., -1, :] = 0.0
        lhs = (gx * px + gy * py).sum()
        rhs = -(u * seg.div(px, py)).sum()
        assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_edge_weight_closed_form():
    img = np.full((6, 8, 3), 0.3, np.float32)
    np.testing.assert_allclose(seg.edge_weight(img), 1.0 / 10.0, atol=1e-15)
    img[:, 4:, 0] = 0.5  # a vertical step of 0.2 in the red channel
    g = seg.edge_weight(img)
    step = 255.0 * (np.float64(np.float32(0.5)) - np.float64(np.float32(0.3)))
    assert abs(g[2, 3] - math.exp(-step / 5.0) / 10.0) < 1e-15
    assert abs(g[2, 5] - 0.1) < 1e-15


def test_lambda_zero_is_pointwise_argmin():
    rng = np.random.default_rng(3)
    f = rng.uniform(0, 5, (3, 10, 12))
    img = rng.uniform(0, 1, (10, 12, 3)).astype(np.float32)
    u, lab = seg.segment(f, img, lam=0.0, iterations=200)
    np.testing.assert_array_equal(lab, np.argmin(f, axis=0))
    # each step moves u by 1/5 of the data term's differences towards the
    # vertex of the smallest f: pixels whose accumulated push (gap x 200
    # steps x 1/5) exceeds 2, twice the largest distance to that vertex, have
    # reached it
    gap = np.sort(f, axis=0)[1] - np.sort(f, axis=0)[0]
    done = gap * 200 * 0.2 > 2.0
    assert np.all(np.abs(u.max(axis=0)[done] - 1.0) < 1e-9) and done.mean() > 0.5


def test_constant_data_term_keeps_uniform_start():
    img = np.random.default_rng(4).uniform(0, 1, (8, 9, 3)).astype(np.float32)
    f = np.full((4, 8, 9), 2.5)
    u, _ = seg.segment(f, img, lam=3.0, iterations=50)
    np.testing.assert_allclose(u, 0.25, atol=1e-15)


def test_label_swap_symmetry():
    rng = np.random.default_rng(5)
    f = rng.uniform(0, 3, (2, 9, 11))
    img = rng.uniform(0, 1, (9, 11, 3)).astype(np.float32)
    u, _ = seg.segment(f, img, lam=2.0, iterations=80)
    v, _ = seg.segment(f[::-1], img, lam=2.0, iterations=80)
    np.testing.assert_allclose(u, v[::-1], atol=1e-12)


def test_smoothing_removes_isolated_pixel():
    """Strong boundary cost: a single pixel whose data term prefers label 1
    inside a label-0 region is absorbed (its perimeter costs more than its
    data gain), while with lambda = 0 it keeps label 1."""
    f = np.zeros((2, 9, 9))
    f[1] = 1.0
    f[0, 4, 4], f[1, 4, 4] = 1.0, 0.0
    img = np.zeros((9, 9, 3), np.float32)  # g = 1/10 everywhere
    _, lab0 = seg.segment(f, img, lam=0.0, iterations=300)
    _, lab = seg.segment(f, img, lam=20.0, iterations=300)
    assert lab0[4, 4] == 1 and np.all(lab == 0)


def test_large_lambda_gives_the_cheapest_constant_labelling():
    """With a boundary weight far above the data costs (g = 1/10 on a
    constant image) every boundary costs more than any data gain: the
    minimiser is the constant labelling by the label of least total cost."""
    for seed in range(3):
        rng = np.random.default_rng(100 + seed)
        f = rng.uniform(0, 2, (3, 6, 7))
        u, lab = seg.segment(f, np.zeros((6, 7, 3), np.float32), lam=200.0, iterations=600)
        best = int(np.argmin(f.reshape(3, -1).sum(axis=1)))
        assert np.all(lab == best)
        np.testing.assert_allclose(u[best], 1.0, atol=1e-9)


def test_large_label_cost_keeps_one_label():
    """Eq. mdl: with nu far above the data costs (and no boundary term) a
    second label never pays for itself; the solution uses the single label
    of least total cost, where nu = 0 keeps the pointwise argmin."""
    for seed in range(3):
        rng = np.random.default_rng(200 + seed)
        f = rng.uniform(0, 2, (3, 6, 7))
        img = np.zeros((6, 7, 3), np.float32)
        _, lab0 = seg.segment(f, img, lam=0.0, nu=0.0, iterations=1500)
        _, lab = seg.segment(f, img, lam=0.0, nu=1e3, iterations=1500)
        np.testing.assert_array_equal(lab0, np.argmin(f, axis=0))
        assert np.all(lab == int(np.argmin(f.reshape(3, -1).sum(axis=1))))


def test_dice_hand_example():
    a = np.array([[0, 0, 1], [1, 1, 1]])
    b = np.array([[0, 1, 1], [1, 1, 0]])
    # label 0: |A|=2, |B|=2, overlap 1 -> 0.5; label 1: |A|=4, |B|=4, overlap 3 -> 0.75
    assert abs(seg.dice(a, b, 2) - 0.625) < 1e-15
