"""Smooth co-sparse texture (mode 2: Eq. map_tsm, approx_cosupp, post_text on
iota) through cs_data_term vs the FP64 oracle.

The GPU forms its codes in FP32 (the oracle in FP64). The bar on L is
derived per pixel from the case's measured code error e (the largest
|a_FP32 - a_FP64| over the compared pixels and the samples, with cs_codes in
the FP32 form, the same arithmetic as the smooth kernels): iota moves by at
most d = e sqrt(2 / sigma) exp(-1/2) + 8u (8.58 e at sigma = 0.01; 8u for the
FP32 square, scale and exponential; u = 2^-24), each representative c_i (a
median) by at most d + u, each l1 distance by at most k (2 d + u) +
(k + 2) u l1_i, so the texture log-posterior by at most twice the largest
l1 error over beta_i(x), plus 16 u (max_i |t_i| + n + 2) for its FP32
log-softmax (t_i = -l1_i / beta_i). The Parzen colour-location part keeps
the bar of its form: 1e-5 relative for the plain FP32 sum, l_tol (set to
1e-4 here) for the tensor-core sum. Bars: |L - L_o| <= that sum, per pixel;
|p - p_o| <= 2.01 times it + 1e-6; argmax agreement >= 99.9%.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1312_4746_gb300 import synth

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
L_TOL_TC = 1e-4  # l_tol of the tensor-core Parzen sum in these tests


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
    prm.l_tol = L_TOL_TC
    out = ctx.data_term(_dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask),
                        pr.label_off, _dev(torch, pr.sample_pix), prm)
    ctx.sync()
    nl = pr.n_labels
    return (-out["neglog"].cpu().numpy().reshape(nl, -1).astype(np.float64),
            out["post"].cpu().numpy().reshape(nl, -1).astype(np.float64))


def _code_error(env, pr, pix):
    """Largest |a_FP32 - a_FP64| at the compared pixels and at the samples."""
    cs, ctx, torch = env
    prm = cs.Params.from_synth(pr.params, codes_form=1)
    c = ctx.codes(_dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask), prm,
                  want_codes=True)
    ctx.sync()
    a32 = c["codes"].cpu().numpy()
    where = np.unique(np.concatenate([np.arange(pr.H * pr.W) if pix is None else pix,
                                      pr.sample_pix])).astype(np.int32)
    a64, _ = oracle.codes(pr.image, pr.omega, pr.mask, pr.params.p, 0.0, pix=where)
    return float(np.max(np.abs(a32[where].astype(np.float64) - a64)))


def _bars(env, pr, ref, precision, pix=None):
    """Per-pixel bars on |L - L_o| (see the module docstring)."""
    prm = pr.params
    k = pr.k
    e = _code_error(env, pr, pix)
    sigma = prm.iota_sigma
    d = e * math.sqrt(2.0 / sigma) * math.exp(-0.5) + 8 * U
    a_px, _ = oracle.codes(pr.image, pr.omega, pr.mask, prm.p, prm.tau, pix=pix)
    io = oracle.iota(a_px, sigma)  # (cnt, k)
    l1 = np.abs(ref["reps"][:, None, :] - io[None, :, :]).sum(axis=2)  # (n, cnt)
    beta = prm.kappa_beta * prm.alpha * np.maximum(np.sqrt(ref["dist2"].astype(np.float64)),
                                                   prm.d_min)
    dt = (k * (2 * d + U) + (k + 2) * U * l1) / beta
    t = l1 / beta
    # the Parzen part's own |L| (the smooth L minus the texture log-posterior)
    lp = ref["L"] - oracle.smooth_log_posterior(io, ref["reps"], beta)
    parzen = (1e-5 if precision == 0 else L_TOL_TC) * np.maximum(np.abs(lp), 1.0)
    tex = 2 * dt.max(axis=0) + 16 * U * (t.max(axis=0) + pr.n_labels + 2)
    return parzen + tex[None, :], e


def _check(L, post, ref, bar):
    err = np.abs(L - ref["L"])
    assert np.all(err <= bar), float(np.max(err / bar))
    perr = np.abs(post - ref["post"])
    assert np.all(perr <= 2.01 * bar.max(axis=0)[None, :] + 1e-6), float(np.max(perr))
    srt = np.sort(ref["post"], axis=0)
    tie = (srt[-1] - srt[-2]) < 1e-12
    agree = float(np.mean((np.argmax(post, 0) == np.argmax(ref["post"], 0)) | tie))
    assert agree >= 0.999, agree
    np.testing.assert_allclose(post.sum(0), 1.0, atol=1e-5)
    rel = float(np.max(err / np.maximum(np.abs(ref["L"]), 1.0)))
    rbar = float(np.min(bar / np.maximum(np.abs(ref["L"]), 1.0)))
    return rel, rbar, float(np.max(perr)), agree


@pytest.mark.parametrize("precision", [0, 2])  # plain FP32 / FP8 tensor-core Parzen sum
def test_smooth_workload1(env, precision):
    pr = synth.make_workload(1)
    pr.params.mode = 2
    L, post = _run(env, pr, precision)
    ref = oracle.data_term(pr, want_dist2=True)
    bar, e = _bars(env, pr, ref, precision)
    rel, rbar, perr, agree = _check(L, post, ref, bar)
    print(f"smooth, workload 1, precision {precision}: max rel err L {rel:.2e} (smallest "
          f"relative bar {rbar:.2e}, code error {e:.2e}), max prob err {perr:.2e}, "
          f"argmax agreement {agree:.4f}")


def test_smooth_workload2_sampled(env):
    pr = synth.make_workload(2)
    pr.params.mode = 2
    L, post = _run(env, pr, 2)
    rng = np.random.default_rng(23)
    pix = np.unique(rng.integers(0, pr.H * pr.W, 2500)).astype(np.int32)
    ref = oracle.data_term(pr, pix=pix, want_dist2=True)
    bar, e = _bars(env, pr, ref, 2, pix=pix)
    rel, rbar, perr, agree = _check(L[:, pix], post[:, pix], ref, bar)
    print(f"smooth, workload 2 (sampled): max rel err L {rel:.2e} (smallest relative bar "
          f"{rbar:.2e}, code error {e:.2e}), max prob err {perr:.2e}, argmax agreement "
          f"{agree:.4f}")


@pytest.mark.parametrize("H,W,nl,m,p,k,seed", [
    (37, 53, 2, 2, 5, 17, 51),      # two samples per label: median = mean of the two
    (40, 33, 3, [1, 5, 40], 7, 98, 52),  # one, odd and even counts
    (24, 30, 2, 30, 9, 162, 53),    # 9x9 patches
])
def test_smooth_ragged(env, H, W, nl, m, p, k, seed):
    pr = synth.make_problem(H, W, nl, m, p=p, k=k, seed=seed, cap_frac=0.9)
    pr.params.mode = 2
    L, post = _run(env, pr, 2)
    ref = oracle.data_term(pr, want_dist2=True)
    _check(L, post, ref, _bars(env, pr, ref, 2)[0])


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
