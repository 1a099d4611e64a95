"""Smooth co-sparse texture (mode 2: Eq. map_tsm, approx_cosupp, post_text on
iota) through cs_data_term vs the FP64 oracle.

The GPU forms its codes in FP32 (the oracle in FP64): a code error e moves
iota by at most e sqrt(2 / sigma) exp(-1/2) (about 8.6 e at sigma = 0.01),
each l1 distance by at most 2 k times that and L by at most twice the l1
error over beta. Bars (those of the reduced-precision forms): max relative
error on L <= 1e-2, max probability error <= 1e-2, argmax agreement >= 99.9%;
the Parzen part is the plain or tensor-core sum of the other modes.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1312_4746_gb300 import synth

pytestmark = pytest.mark.gpu

L_BAR = 1e-2
P_BAR = 1e-2


@pytest.fixture(scope="module")
def env(cuda_lib):
    import torch

    import paper_1312_4746_gb300 as cs

    ctx = cs.Context(0)
    yield cs, ctx, torch
    ctx.close()


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _run(env, pr, precision):
    cs, ctx, torch = env
    prm = cs.Params.from_synth(pr.params, precision=precision, mode=cs.MODE_SMOOTH)
    out = ctx.data_term(_dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask),
                        pr.label_off, _dev(torch, pr.sample_pix), prm)
    ctx.sync()
    nl = pr.n_labels
    return (-out["neglog"].cpu().numpy().reshape(nl, -1).astype(np.float64),
            out["post"].cpu().numpy().reshape(nl, -1).astype(np.float64))


def _check(L, post, ref):
    rel = float(np.max(np.abs(L - ref["L"]) / np.maximum(np.abs(ref["L"]), 1.0)))
    perr = float(np.max(np.abs(post - ref["post"])))
    srt = np.sort(ref["post"], axis=0)
    tie = (srt[-1] - srt[-2]) < 1e-12
    agree = float(np.mean((np.argmax(post, 0) == np.argmax(ref["post"], 0)) | tie))
    assert rel <= L_BAR and perr <= P_BAR and agree >= 0.999, (rel, perr, agree)
    np.testing.assert_allclose(post.sum(0), 1.0, atol=1e-5)
    return rel, perr, agree


@pytest.mark.parametrize("precision", [0, 2])  # plain FP32 / FP8 tensor-core Parzen sum
def test_smooth_workload1(env, precision):
    pr = synth.make_workload(1)
    pr.params.mode = 2
    L, post = _run(env, pr, precision)
    ref = oracle.data_term(pr)
    rel, perr, agree = _check(L, post, ref)
    print(f"smooth, workload 1, precision {precision}: max rel err L {rel:.2e}, "
          f"max prob err {perr:.2e}, argmax agreement {agree:.4f}")


def test_smooth_workload2_sampled(env):
    pr = synth.make_workload(2)
    pr.params.mode = 2
    L, post = _run(env, pr, 2)
    rng = np.random.default_rng(23)
    pix = np.unique(rng.integers(0, pr.H * pr.W, 2500)).astype(np.int32)
    ref = oracle.data_term(pr, pix=pix)
    rel, perr, agree = _check(L[:, pix], post[:, pix], ref)
    print(f"smooth, workload 2 (sampled): max rel err L {rel:.2e}, max prob err {perr:.2e}, "
          f"argmax agreement {agree:.4f}")


@pytest.mark.parametrize("H,W,nl,m,p,k,seed", [
    (37, 53, 2, 2, 5, 17, 51),      # two samples per label: median = mean of the two
    (40, 33, 3, [1, 5, 40], 7, 98, 52),  # one, odd and even counts
    (24, 30, 2, 30, 9, 162, 53),    # 9x9 patches
])
def test_smooth_ragged(env, H, W, nl, m, p, k, seed):
    pr = synth.make_problem(H, W, nl, m, p=p, k=k, seed=seed, cap_frac=0.9)
    pr.params.mode = 2
    L, post = _run(env, pr, 2)
    _check(L, post, oracle.data_term(pr))


def test_smooth_zero_image_uniform_texture(env):
    """All-zero image: every patch flat, every code 0, iota = 1 everywhere,
    so the texture posterior is uniform and L = Parzen - log n (the Parzen sum
    of the factorised form is L_F + log n on this image, where its majority
    texture posterior is uniform too)."""
    cs, ctx, torch = env
    pr = synth.make_problem(20, 24, 3, 8, p=7, k=98, seed=54)
    pr.image[:] = 0.0
    pr.params.mode = 2
    L2, _ = _run(env, pr, 2)
    pr.params.mode = 1
    prm = cs.Params.from_synth(pr.params, precision=2)
    out = ctx.data_term(_dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask),
                        pr.label_off, _dev(torch, pr.sample_pix), prm)
    ctx.sync()
    L1 = -out["neglog"].cpu().numpy().reshape(3, -1).astype(np.float64)
    np.testing.assert_allclose(L2, L1, rtol=0, atol=1e-4)
    pr.params.mode = 2
    np.testing.assert_allclose(L2, oracle.data_term(pr)["L"], rtol=1e-5, atol=1e-4)


def test_smooth_only_through_data_term(env):
    """The smooth mode needs the operator: the likelihood-only entry refuses it."""
    cs, ctx, torch = env
    pr = synth.make_problem(16, 16, 2, 4, p=5, k=50, seed=55)
    prm = cs.Params.from_synth(pr.params)
    img = _dev(torch, pr.image)
    c = ctx.codes(img, _dev(torch, pr.omega), _dev(torch, pr.mask), prm)
    prm.mode = cs.MODE_SMOOTH
    with pytest.raises(cs.CsError) as ei:
        ctx.likelihood(img, c["bitmask"], pr.k, pr.label_off, _dev(torch, pr.sample_pix), prm)
    assert ei.value.status == cs.CS_ERR_UNSUPPORTED
    prm.iota_sigma = 0.0
    with pytest.raises(cs.CsError) as ei:
        ctx.data_term(img, _dev(torch, pr.omega), _dev(torch, pr.mask), pr.label_off,
                      _dev(torch, pr.sample_pix), prm)
    assert ei.value.status == cs.CS_ERR_INVALID_ARG
