"""rho read as the location kernel's variance (cs_params.rho_variance = 1,
Sec. 3.1) in every likelihood form vs the FP64 oracle with the same reading.

Bars as for the default reading: plain FP32 L within 1e-5 relative; the
tensor-core forms L within 1e-4 relative, probabilities within 1e-2 and
argmax agreement >= 99.9%; the smooth texture mode as in its own tests.
"""
import numpy as np
import pytest

import oracle
from paper_1312_4746_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(cuda_lib):
    import torch

    import paper_1312_4746_gb300 as cs

    ctx = cs.Context(0)
    yield cs, ctx, torch
    ctx.close()


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _data_term(env, pr, precision, mode):
    cs, ctx, torch = env
    prm = cs.Params.from_synth(pr.params, precision=precision, mode=mode)
    assert prm.rho_variance == pr.params.rho_variance
    out = ctx.data_term(_dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask),
                        pr.label_off, _dev(torch, pr.sample_pix), prm)
    ctx.sync()
    nl = pr.n_labels
    return (-out["neglog"].cpu().numpy().reshape(nl, -1).astype(np.float64),
            out["post"].cpu().numpy().reshape(nl, -1).astype(np.float64))


def _check(L, post, ref, l_bar):
    rel = float(np.max(np.abs(L - ref["L"]) / np.maximum(np.abs(ref["L"]), 1.0)))
    perr = float(np.max(np.abs(post - ref["post"])))
    srt = np.sort(ref["post"], axis=0)
    tie = (srt[-1] - srt[-2]) < 1e-12 if srt.shape[0] > 1 else np.zeros(srt.shape[1], bool)
    agree = float(np.mean((np.argmax(post, 0) == np.argmax(ref["post"], 0)) | tie))
    assert rel <= l_bar and perr <= 1e-2 and agree >= 0.999, (rel, perr, agree)
    return rel


@pytest.mark.parametrize("precision,bar", [(0, 1e-5), (1, 1e-4), (2, 1e-4)])
@pytest.mark.parametrize("mode", [0, 1])
def test_rho_variance_workload1(env, precision, bar, mode):
    pr = synth.make_workload(1)
    pr.params.rho_variance = 1
    pr.params.mode = mode
    L, post = _data_term(env, pr, precision, mode)
    ref = oracle.data_term(pr)
    rel = _check(L, post, ref, bar)
    # the reading changes the result (not a no-op switch)
    pr.params.rho_variance = 0
    assert np.abs(oracle.data_term(pr)["L"] - ref["L"]).max() > 1e-2
    print(f"rho as variance, precision {precision}, mode {mode}: max rel err L {rel:.2e}")


@pytest.mark.parametrize("H,W,nl,m,p,k,seed,precision", [
    (61, 45, 3, 129, 7, 98, 2, 2),   # a full sample tile and a one-sample tile
    (1, 7, 1, 3, 3, 40, 4, 0),       # one-row image, plain form
    (33, 70, 4, 300, 9, 162, 3, 2),  # k = 162
])
def test_rho_variance_ragged(env, H, W, nl, m, p, k, seed, precision):
    pr = synth.make_problem(H, W, nl, m, p=p, k=k, seed=seed)
    pr.params.rho_variance = 1
    L, post = _data_term(env, pr, precision, 0)
    _check(L, post, oracle.data_term(pr), 1e-5 if precision == 0 else 1e-4)


def test_rho_variance_smooth_mode(env):
    pr = synth.make_workload(1)
    pr.params.rho_variance = 1
    pr.params.mode = 2
    L, post = _data_term(env, pr, 2, 2)
    _check(L, post, oracle.data_term(pr), 1e-2)


def test_rho_variance_batch_matches_single(env):
    """The batch (one persistent sum over all images) takes the switch too:
    its outputs equal the single-image calls bit for bit."""
    cs, ctx, torch = env
    prs = [synth.make_problem(40 + 9 * b, 50 + 7 * b, 2 + b, 60, p=7, k=98, seed=90 + b)
           for b in range(3)]
    prm = cs.Params.from_synth(prs[0].params, precision=2, rho_variance=1)
    omega, mask = _dev(torch, prs[0].omega), _dev(torch, prs[0].mask)
    imgs = [{"img": _dev(torch, pr.image), "sample_pix": _dev(torch, pr.sample_pix),
             "label_off": pr.label_off} for pr in prs]
    outs = ctx.batch_data_term(imgs, omega, mask, prm)
    ctx.sync()
    for pr, im, o in zip(prs, imgs, outs):
        one = ctx.data_term(im["img"], omega, mask, pr.label_off, im["sample_pix"], prm)
        ctx.sync()
        np.testing.assert_array_equal(o["neglog"].cpu().numpy(), one["neglog"].cpu().numpy())


def test_switch_validation(env):
    cs, ctx, torch = env
    pr = synth.make_problem(16, 16, 2, 4, p=5, k=50, seed=95)
    args = (_dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask), pr.label_off,
            _dev(torch, pr.sample_pix))
    with pytest.raises(cs.CsError) as ei:
        ctx.data_term(*args, cs.Params.from_synth(pr.params, rho_variance=2))
    assert ei.value.status == cs.CS_ERR_INVALID_ARG
    with pytest.raises(cs.CsError) as ei:
        ctx.data_term(*args, cs.Params.from_synth(pr.params, patch_order=2))
    assert ei.value.status == cs.CS_ERR_INVALID_ARG
    with pytest.raises(cs.CsError) as ei:  # the smooth mode builds mask-first patches only
        ctx.data_term(*args, cs.Params.from_synth(pr.params, patch_order=1, mode=2))
    assert ei.value.status == cs.CS_ERR_UNSUPPORTED
