"""Tensor-core (tcgen05) forms of the pixel x sample sum vs the FP64 oracle.

The texture dot products are exact integers on the tensor cores (FP8 or BF16
operands with values 0 and +-1); the colour term runs through hi/lo BF16
splits (relative error about 2^-17 per factor); the location term, relative
to each pixel tile's centre, through exact pieces of the sample offsets and
three-piece splits of the pixel-side factors (relative error below 2^-24).
Bars: max probability error <= 1e-2 and argmax agreement >= 99.9% (required
of the reduced-precision forms), and max relative error on L <= 1e-4 here.
"""
import numpy as np
import pytest

import oracle
from paper_1312_4746_gb300 import synth

pytestmark = pytest.mark.gpu

L_TOL = 1e-4
P_TOL = 1e-2


@pytest.fixture(scope="module")
def env(cuda_lib):
    import torch

    import paper_1312_4746_gb300 as cs

    ctx = cs.Context(0)
    yield cs, ctx, torch
    ctx.close()


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _run(env, pr, precision, mode):
    cs, ctx, torch = env
    prm = cs.Params.from_synth(pr.params, precision=precision, mode=mode)
    img = _dev(torch, pr.image)
    c = ctx.codes(img, _dev(torch, pr.omega), _dev(torch, pr.mask), prm)
    out = ctx.likelihood(img, c["bitmask"], pr.k, pr.label_off, _dev(torch, pr.sample_pix), prm)
    ctx.sync()
    nl = pr.n_labels
    return (-out["neglog"].cpu().numpy().reshape(nl, -1).astype(np.float64),
            out["post"].cpu().numpy().reshape(nl, -1).astype(np.float64))


def _check(L, post, ref):
    rel = float(np.max(np.abs(L - ref["L"]) / np.maximum(np.abs(ref["L"]), 1.0)))
    perr = float(np.max(np.abs(post - ref["post"])))
    srt = np.sort(ref["post"], axis=0)
    tie = (srt[-1] - srt[-2]) < 1e-12 if srt.shape[0] > 1 else np.zeros(srt.shape[1], bool)
    agree = np.mean((np.argmax(post, 0) == np.argmax(ref["post"], 0)) | tie)
    assert perr <= P_TOL and agree >= 0.999, (perr, agree)
    assert rel <= L_TOL, rel
    np.testing.assert_allclose(post.sum(0), 1.0, atol=1e-5)
    return rel, perr


@pytest.mark.parametrize("precision", [1, 2])  # BF16, FP8 texture operands
@pytest.mark.parametrize("mode", [0, 1])
def test_workload1_tc(env, precision, mode):
    pr = synth.make_workload(1)
    L, post = _run(env, pr, precision, mode)
    ref = oracle.data_term(pr, mode=mode)
    _check(L, post, ref)


@pytest.mark.parametrize("H,W,nl,m,p,k,seed,precision", [
    (37, 53, 2, 17, 5, 17, 1, 2),     # k < 32, ragged tiles, one sample tile per label
    (61, 45, 3, 129, 7, 98, 2, 2),    # 129 samples: a full tile and a 1-sample tile
    (33, 70, 4, 300, 9, 162, 3, 2),   # k = 162: 6 FP8 slabs
    (130, 129, 5, 300, 7, 256, 6, 2), # k = 256: 8 FP8 slabs
    (61, 45, 3, 200, 7, 98, 7, 1),    # BF16: 7 slabs
    (40, 41, 2, 90, 5, 128, 8, 1),    # BF16 at its largest k
    (1, 7, 1, 3, 3, 40, 4, 2),        # one-row image
])
def test_ragged_tc(env, H, W, nl, m, p, k, seed, precision):
    pr = synth.make_problem(H, W, nl, m, p=p, k=k, seed=seed, cap_frac=0.9)
    for mode in (0, 1):
        L, post = _run(env, pr, precision, mode)
        ref = oracle.data_term(pr, mode=mode)
        _check(L, post, ref)


@pytest.mark.parametrize("H,W,nl,m,seed", [
    (24, 6000, 2, 150, 41),   # wide: sample offsets from a pixel tile up to ~6000 px
    (3000, 20, 3, 120, 42),   # tall
])
def test_far_samples_tc(env, H, W, nl, m, seed):
    """Pixels and samples thousands of pixels apart: the location pieces stay
    exact and L stays within the bar at sampled pixels of both ends."""
    pr = synth.make_problem(H, W, nl, m, p=5, k=50, seed=seed, cap_frac=0.9)
    L, post = _run(env, pr, 2, 0)
    rng = np.random.default_rng(seed)
    P = H * W
    pix = np.unique(np.concatenate([rng.integers(0, P, 500), [0, W - 1, P - W, P - 1]])).astype(np.int32)
    ref = oracle.data_term(pr, pix=pix)
    _check(L[:, pix], post[:, pix], ref)


def test_tc_matches_plain(env):
    """The tensor-core and CUDA-core forms agree closely on a larger image."""
    pr = synth.make_problem(96, 120, 4, 700, p=7, k=98, seed=21)
    L0, p0 = _run(env, pr, 0, 0)
    for prec in (1, 2):
        L1, p1 = _run(env, pr, prec, 0)
        assert np.max(np.abs(L1 - L0) / np.maximum(np.abs(L0), 1.0)) < 1e-4
        assert np.max(np.abs(p1 - p0)) < 1e-3


def test_tc_unsupported_k(env):
    cs, ctx, torch = env
    pr = synth.make_problem(12, 12, 2, 4, p=7, k=160, seed=9)
    prm = cs.Params.from_synth(pr.params, precision=cs.BF16)
    img = _dev(torch, pr.image)
    c = ctx.codes(img, _dev(torch, pr.omega), _dev(torch, pr.mask), prm)
    with pytest.raises(cs.CsError) as ei:
        ctx.likelihood(img, c["bitmask"], pr.k, pr.label_off, _dev(torch, pr.sample_pix), prm)
    assert ei.value.status == cs.CS_ERR_UNSUPPORTED


def test_workload2_tc_sampled(env):
    pr = synth.make_workload(2)
    L, post = _run(env, pr, 2, 0)
    rng = np.random.default_rng(15)
    P = pr.H * pr.W
    pix = np.unique(rng.integers(0, P, 3000)).astype(np.int32)
    ref = oracle.data_term(pr, pix=pix)
    _check(L[:, pix], post[:, pix], ref)


@pytest.mark.parametrize("mode,kw", [
    (0, {"kappa_beta": 0.02}),  # texture exponents of hundreds: most rows below 2^-80
    (1, {"sigma_c2": 2e-4}),    # colour exponents of hundreds in the Parzen sum
])
def test_fp64_recompute_of_underflowing_rows(env, mode, kw):
    """Rows whose FP32 sum of 2^e (e <= 0) falls below the floor are recomputed
    in double precision on the GPU; the result then matches the FP64 oracle
    to float rounding, and the rest of the image stays within the form's bar."""
    import dataclasses

    cs, ctx, torch = env
    pr = synth.make_problem(40, 52, 3, 60, p=5, k=50, seed=21, cap_frac=0.9)
    pr = dataclasses.replace(pr, params=dataclasses.replace(pr.params, **kw))
    for precision in (2, 1):
        L, post = _run(env, pr, precision, mode)
        n_ref = ctx.refined_count()
        assert n_ref > 0, "expected rows below the FP32 floor"
        ref = oracle.data_term(pr, mode=mode)
        rel = np.abs(L - ref["L"]) / np.maximum(np.abs(ref["L"]), 1.0)
        assert float(np.max(rel)) <= L_TOL, float(np.max(rel))
        # every listed pixel has at least one label row recomputed in double
        # (FP32 exponentials): those rows agree to about float rounding
        assert int((rel <= 1e-6).sum()) >= n_ref
        np.testing.assert_allclose(post.sum(0), 1.0, atol=1e-5)


def _run_tol(env, pr, precision, mode, l_tol):
    cs, ctx, torch = env
    prm = cs.Params.from_synth(pr.params, precision=precision, mode=mode, l_tol=l_tol)
    img = _dev(torch, pr.image)
    c = ctx.codes(img, _dev(torch, pr.omega), _dev(torch, pr.mask), prm)
    out = ctx.likelihood(img, c["bitmask"], pr.k, pr.label_off, _dev(torch, pr.sample_pix), prm)
    n = ctx.refined_count()
    nl = pr.n_labels
    return -out["neglog"].cpu().numpy().reshape(nl, -1).astype(np.float64), n


@pytest.mark.parametrize("mode", [0, 1])
def test_row_bound_tolerance(env, mode):
    """The a-priori row bound: with l_tol = 1e-5 every row either meets the
    plain form's 1e-5 bar or is recomputed in FP64; the bar holds at every
    tolerance; tighter tolerances recompute more pixels; l_tol = 0 recomputes
    nothing at the default parameters."""
    pr = synth.make_workload(1)
    ref = oracle.data_term(pr, mode=mode)
    P = pr.H * pr.W
    counts = {}
    for tol in (0.0, 1e-3, 1e-4, 1e-5):
        L, n = _run_tol(env, pr, 2, mode, tol)
        counts[tol] = n
        rel = float(np.max(np.abs(L - ref["L"]) / np.maximum(np.abs(ref["L"]), 1.0)))
        assert rel <= (max(tol, 1e-5) if tol > 0 else L_TOL), (tol, rel)
    assert counts[0.0] == 0
    assert counts[1e-3] <= counts[1e-4] <= counts[1e-5]
    print(f"mode {mode}: pixels recomputed in FP64 at l_tol 1e-3 / 1e-4 / 1e-5: "
          f"{counts[1e-3]} / {counts[1e-4]} / {counts[1e-5]} of {P}")
