"""Seeded synthetic inputs for the co-sparse data term.

This module only draws inputs: textured images, scribble sample lists, an
analysis operator and a Gaussian patch mask. It contains none of the data
term's arithmetic, so both the CUDA path and the CPU oracle can be fed from
it without sharing any of the method's code.

The paper evaluates on the Graz interactive benchmark (Sec. 5.1) and on the
Berkeley BSDS300 images (Sec. 5.2), and uses an operator learned from
natural image patches (Sec. 2). None of these are available here, so the
inputs below stand in for them with the same shapes:

* images: Voronoi partitions whose cells carry oriented sinusoid gratings
  (and, from the second workload on, rotated checkerboards), an RGB tint and
  Gaussian noise, clipped to [0, 1], stored H x W x 3 float32 (HWC);
* scribbles: random-walk brush strokes inside each labelled cell, giving a
  list of unique pixel indices per label (CSR: ``label_off``,
  ``sample_pix``), like the brush scribbles of the Graz benchmark (Sec. 5.1);
* operator: k x n Gaussian rows normalised to unit length (k = 2n, the
  two-times over-complete shape of Sec. 5);
* mask: the Gaussian patch weighting of Sec. 3.1 with width p / 4.

Random numbers come from numpy ``Generator(PCG64(seed))``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Params",
    "Problem",
    "make_problem",
    "make_workload",
    "make_batch",
    "WORKLOADS",
]


@dataclasses.dataclass
class Params:
    """Scalar parameters of the data term.

    Defaults: colour kernel variance 1.3 and spatial scale alpha 1.3 (Sec. 3.1),
    co-support threshold 0.1, one-pixel floor on the scribble distance and
    beta = rho (kappa_beta = 1).
    """

    p: int = 7
    tau: float = 0.1
    sigma_c2: float = 1.3
    alpha: float = 1.3
    d_min: float = 1.0
    kappa_beta: float = 1.0
    mode: int = 0  # 0 = per-sample texture kernel, 1 = factorised (Eq. joined), 2 = smooth
    iota_sigma: float = 0.01  # Eq. map_tsm's sigma (the paper's value) for the smooth texture
    rho_variance: int = 0  # 1: rho is the location kernel's variance (else its standard deviation)
    patch_order: int = 0  # 1: centre, mask, centre again, normalise (else mask, centre, normalise)


@dataclasses.dataclass
class Problem:
    image: np.ndarray  # (H, W, 3) float32, HWC, values in [0, 1]
    omega: np.ndarray  # (k, n) float32, row-major, n = p * p
    mask: np.ndarray  # (n,) float32, window order t = dy * p + dx
    label_off: np.ndarray  # (n_labels + 1,) int32
    sample_pix: np.ndarray  # (sum m_i,) int32, pixel index y * W + x
    params: Params
    regions: np.ndarray  # (H, W) int32 ground-truth cell of each pixel
    name: str = ""

    @property
    def H(self) -> int:
        return int(self.image.shape[0])

    @property
    def W(self) -> int:
        return int(self.image.shape[1])

    @property
    def k(self) -> int:
        return int(self.omega.shape[0])

    @property
    def n_labels(self) -> int:
        return int(self.label_off.shape[0] - 1)

    @property
    def n_samples(self) -> int:
        return int(self.label_off[-1])

    @property
    def pairs(self) -> int:
        return self.H * self.W * self.n_samples


def _voronoi(rng, H, W, n_regions):
    # sites uniform in the image, kept apart so that no cell is tiny
    min_d = 0.6 * math.sqrt(H * W / n_regions)
    sites = np.zeros((n_regions, 2))
    for r in range(n_regions):
        for _ in range(1000):
            cand = np.array([rng.uniform(0, W), rng.uniform(0, H)])
            if r == 0 or np.min(np.hypot(*(sites[:r] - cand).T)) >= min_d:
                break
            min_d *= 0.995
        sites[r] = cand
    regions = np.empty((H, W), np.int32)
    xs = np.arange(W, dtype=np.float64)
    for y0 in range(0, H, 256):
        ys = np.arange(y0, min(H, y0 + 256), dtype=np.float64)
        d = (xs[None, :, None] - sites[None, None, :, 0]) ** 2 + (
            ys[:, None, None] - sites[None, None, :, 1]
        ) ** 2
        regions[y0 : y0 + len(ys)] = np.argmin(d, axis=2)
    return regions


def _texture(rng, H, W, regions, n_regions, checkers, noise):
    img = np.zeros((H, W, 3), np.float64)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    for r in range(n_regions):
        sel = regions == r
        if not sel.any():
            # keep the draw sequence independent of emptiness
            rng.uniform(3, 12), rng.uniform(0, math.pi), rng.uniform(0, 2 * math.pi)
            rng.uniform(0.2, 1.0, 3)
            continue
        period = rng.uniform(3.0, 12.0)
        theta = rng.uniform(0.0, math.pi)
        phase = rng.uniform(0.0, 2 * math.pi)
        tint = rng.uniform(0.2, 1.0, 3)
        u = math.cos(theta) * xx[sel] + math.sin(theta) * yy[sel]
        if checkers and (r % 2 == 1):
            v = -math.sin(theta) * xx[sel] + math.cos(theta) * yy[sel]
            c = (np.floor(u / period + phase / (2 * math.pi)) + np.floor(v / period)) % 2
            val = 0.15 + 0.7 * c
        else:
            val = 0.5 + 0.5 * np.sin(2 * math.pi * u / period + phase)
        img[sel] = val[:, None] * tint[None, :]
    img += rng.normal(0.0, noise, img.shape)
    return np.clip(img, 0.0, 1.0).astype(np.float32)


_BRUSHES = {
    1: np.array([[0, 0]]),
    2: np.array([[0, 0], [0, 1], [1, 0], [1, 1]]),
    3: np.array([[0, 0], [-1, 0], [1, 0], [0, -1], [0, 1], [-1, -1], [-1, 1], [1, -1], [1, 1]]),
}


def _scribbles(rng, regions, label, want):
    """Unique pixel indices of one label, drawn as random-walk brush strokes."""
    H, W = regions.shape
    inside = regions == label
    cand = np.flatnonzero(inside)
    want = min(want, len(cand))
    got: dict[int, None] = {}
    strokes = 0
    while len(got) < want and strokes < 200000:
        strokes += 1
        start = cand[rng.integers(len(cand))]
        y0, x0 = divmod(int(start), W)
        length = int(rng.integers(15, 61))
        brush = _BRUSHES[int(rng.integers(1, 4))]
        heading = rng.uniform(0, 2 * math.pi) + np.cumsum(rng.normal(0.0, 0.3, length))
        px = x0 + np.concatenate([[0.0], np.cumsum(np.cos(heading[:-1]))])
        py = y0 + np.concatenate([[0.0], np.cumsum(np.sin(heading[:-1]))])
        ix = np.rint(px).astype(np.int64)
        iy = np.rint(py).astype(np.int64)
        ok = (ix >= 0) & (ix < W) & (iy >= 0) & (iy < H)
        ok[ok] &= inside[iy[ok], ix[ok]]
        stop = np.argmin(ok) if not ok.all() else length  # stroke ends where it leaves the cell
        ix, iy = ix[:stop], iy[:stop]
        bx = (ix[:, None] + brush[None, :, 1]).ravel()
        by = (iy[:, None] + brush[None, :, 0]).ravel()
        ok = (bx >= 0) & (bx < W) & (by >= 0) & (by < H)
        bx, by = bx[ok], by[ok]
        ok = inside[by, bx]
        for pix in (by[ok] * W + bx[ok]).tolist():
            if pix not in got:
                got[pix] = None
                if len(got) == want:
                    break
    pix = np.fromiter(got.keys(), dtype=np.int64, count=len(got))
    pix.sort()
    return pix[rng.permutation(len(pix))].astype(np.int32)


def make_omega(k: int, n: int, seed: int) -> np.ndarray:
    """k x n operator with N(0, 1) rows normalised to unit l2 norm."""
    rng = np.random.Generator(np.random.PCG64(seed))
    om = rng.normal(0.0, 1.0, (k, n))
    om /= np.linalg.norm(om, axis=1, keepdims=True)
    return om.astype(np.float32)


def make_mask(p: int) -> np.ndarray:
    """Gaussian weights over a p x p window, width p / 4, centre weight 1."""
    r = (p - 1) // 2
    sw = p / 4.0
    dy, dx = np.mgrid[0:p, 0:p].astype(np.float64)
    w = np.exp(-((dy - r) ** 2 + (dx - r) ** 2) / (2.0 * sw * sw))
    return w.ravel().astype(np.float32)


def make_problem(
    H: int,
    W: int,
    n_labels: int,
    m_per_label,
    p: int,
    k: int | None = None,
    n_regions: int | None = None,
    seed: int = 0,
    checkers: bool = True,
    noise: float = 0.05,
    cap_frac: float = 0.5,
    params: Params | None = None,
    name: str = "",
) -> Problem:
    """One synthetic image with scribbles.

    ``m_per_label`` is an int or a sequence (one count per label); each count
    is capped at ``cap_frac`` of its cell's area so that small cells can hold
    their strokes.
    """
    n = p * p
    k = 2 * n if k is None else k
    n_regions = n_labels if n_regions is None else n_regions
    assert n_regions >= n_labels
    rng = np.random.Generator(np.random.PCG64(seed))
    regions = _voronoi(rng, H, W, n_regions)
    image = _texture(rng, H, W, regions, n_regions, checkers, noise)
    if np.isscalar(m_per_label):
        m_per_label = [int(m_per_label)] * n_labels
    pix = []
    for i in range(n_labels):
        area = int((regions == i).sum())
        want = max(1, min(int(m_per_label[i]), int(cap_frac * area)))
        s = _scribbles(rng, regions, i, want)
        assert len(s) >= 1, "every label needs at least one scribble sample"
        pix.append(s)
    off = np.zeros(n_labels + 1, np.int32)
    off[1:] = np.cumsum([len(s) for s in pix])
    prm = dataclasses.replace(params) if params is not None else Params()
    prm.p = p
    return Problem(
        image=image,
        omega=make_omega(k, n, seed + 1),
        mask=make_mask(p),
        label_off=off,
        sample_pix=np.concatenate(pix).astype(np.int32),
        params=prm,
        regions=regions,
        name=name,
    )


# The five workloads: image size, labels, samples, patch side, operator rows.
WORKLOADS = {
    1: dict(H=64, W=96, n_labels=3, m_per_label=300, p=5, k=50, n_regions=3, checkers=False,
            name="96x64 RGB, 3 labels x 300 samples, 5x5 patches, Omega 50x25"),
    2: dict(H=321, W=481, n_labels=5, m_per_label=2000, p=7, k=98, n_regions=6, checkers=True,
            name="481x321 RGB, 5 labels x 2000 samples, 7x7 patches, Omega 98x49"),
    4: dict(H=1024, W=1024, n_labels=10, m_per_label=20000, p=7, k=98, n_regions=10, checkers=True,
            name="1024x1024 RGB, 10 labels x 20000 samples, 7x7 patches, Omega 98x49"),
    5: dict(H=4096, W=4096, n_labels=16, m_per_label=6250, p=9, k=162, n_regions=16, checkers=True,
            name="4096x4096 RGB, 16 labels x 6250 samples, 9x9 patches, Omega 162x81"),
}


def make_workload(idx: int, seed: int | None = None) -> Problem:
    """Workload ``idx`` (1, 2, 4 or 5) with seed 1000 + idx unless given."""
    cfg = dict(WORKLOADS[idx])
    return make_problem(seed=1000 + idx if seed is None else seed, **cfg)


def make_batch(n_images: int = 64, first: int = 0, p: int = 7, k: int = 98) -> list[Problem]:
    """Batch workload: uneven sizes 240..640 x 160..480, 2..10 labels,
    500..5000 samples per label (capped at half the cell); image b uses seed
    100000 + b."""
    out = []
    for b in range(first, first + n_images):
        rng = np.random.Generator(np.random.PCG64(100000 + b))
        W = int(rng.integers(240, 641))
        H = int(rng.integers(160, 481))
        nl = int(rng.integers(2, 11))
        m = [int(v) for v in rng.integers(500, 5001, nl)]
        out.append(
            make_problem(H, W, nl, m, p, k, n_regions=nl + 1, seed=200000 + b, checkers=True,
                         name=f"batch image {b}: {W}x{H}, {nl} labels")
        )
    return out
