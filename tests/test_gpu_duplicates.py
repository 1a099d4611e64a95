"""Duplicated scribble samples through the C ABI vs the FP64 oracle.

Sec. 3.1 sums the kernels over the list of a label's samples (Eq. color,
Eq. post_text) and Eq. tex-rep counts them for the majority co-support, so
a pixel listed twice in a label counts twice, and a pixel may be a sample
of two labels. The cases below list pixels two and three times inside a
label, share pixels between labels, and build a three-entry label [a, b, b]
whose majority co-support is b's (2 of 3 votes) where the unique list [a, b]
would give the union of a's and b's bits (2 count >= 2): the duplicates
reach the distance seeds, the Morton sort of the sample tiles, the tile
build, the majority count and the sums. Every form (plain FP32, BF16 and FP8
tensor-core sums) in the per-sample and the factorised mode, and the
whole-pipeline call cs_data_term.

Bars: bitmasks and squared distances bit-exact; L within 1e-5 relative
(plain FP32) or 1e-4 (tensor-core forms at l_tol = 1e-4); probabilities
within 1e-4 (FP32) or 1e-2; argmax agreement >= 99.9%.
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


def _with_duplicates(pr):
    """Workload-1 scribbles rewritten with duplicates: label 0 lists one pixel
    three times and another twice; label 1 gains a pixel of label 0 and a
    repeat of its own; label 2 becomes [a, b, b] (a, b its first two pixels,
    chosen with different co-supports by the caller's check)."""
    off = pr.label_off
    lab = [pr.sample_pix[off[i]:off[i + 1]].copy() for i in range(pr.n_labels)]
    s0, s1, s2 = lab[0], lab[1], lab[2]
    lab[0] = np.concatenate([s0, [s0[0], s0[0], s0[1]]])
    lab[1] = np.concatenate([s1[:7], [s0[5]], s1[7:], [s1[3]]])
    lab[2] = np.array([s2[0], s2[1], s2[1]])
    new_off = np.zeros(pr.n_labels + 1, np.int32)
    new_off[1:] = np.cumsum([len(x) for x in lab])
    pr.label_off = new_off
    pr.sample_pix = np.concatenate(lab).astype(np.int32)
    return pr


def _check(pr, out, ref, fp32):
    nl = pr.n_labels
    assert np.array_equal(out["bitmask"].cpu().numpy().view(np.uint32), ref["bits_px"])
    assert np.array_equal(out["dist2"].cpu().numpy().reshape(nl, -1), ref["dist2"])
    L = -out["neglog"].cpu().numpy().reshape(nl, -1).astype(np.float64)
    post = out["post"].cpu().numpy().reshape(nl, -1).astype(np.float64)
    rel = float(np.max(np.abs(L - ref["L"]) / np.maximum(np.abs(ref["L"]), 1.0)))
    perr = float(np.max(np.abs(post - ref["post"])))
    srt = np.sort(ref["post"], axis=0)
    tie = (srt[-1] - srt[-2]) < 1e-12
    agree = float(np.mean((np.argmax(post, 0) == np.argmax(ref["post"], 0)) | tie))
    assert rel <= (1e-5 if fp32 else 1e-4), rel
    assert perr <= (1e-4 if fp32 else 1e-2) and agree >= 0.999, (perr, agree)
    return rel


@pytest.mark.parametrize("precision", [0, 1, 2])  # plain FP32, BF16, FP8
@pytest.mark.parametrize("mode", [0, 1])          # per-sample, factorised (majority)
def test_duplicated_samples(env, precision, mode):
    cs, ctx, torch = env
    pr = _with_duplicates(synth.make_workload(1))
    # the [a, b, b] label: its majority co-support is b's, not the union
    _, bits = oracle.codes(pr.image, pr.omega, pr.mask, pr.params.p, pr.params.tau,
                           pix=pr.sample_pix[pr.label_off[2]:pr.label_off[3]], want_codes=False)
    rep = oracle.majority(np.concatenate([np.zeros((pr.label_off[2], bits.shape[1]), np.uint32),
                                          bits]), pr.k, [0, pr.label_off[2], pr.label_off[3]])[1]
    assert np.array_equal(rep, bits[1]) and not np.array_equal(bits[0], bits[1])
    prm = cs.Params.from_synth(pr.params, precision=precision, mode=mode)
    prm.l_tol = 1e-4
    out = ctx.data_term(_dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask),
                        pr.label_off, _dev(torch, pr.sample_pix), prm, want_bitmask=True,
                        want_dist2=True)
    ctx.sync()
    ref = oracle.data_term(pr, mode=mode, want_dist2=True)
    rel = _check(pr, out, ref, precision == 0)
    # the duplicates matter: the oracle on the unique lists differs
    uniq = synth.make_workload(1)
    off = uniq.label_off
    lists = [np.unique(pr.sample_pix[pr.label_off[i]:pr.label_off[i + 1]]) for i in range(3)]
    uniq.label_off = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.int32)
    uniq.sample_pix = np.concatenate(lists).astype(np.int32)
    ref_u = oracle.data_term(uniq, mode=mode)
    assert np.max(np.abs(ref_u["L"] - ref["L"])) > 1e-3
    print(f"duplicates, precision {precision}, mode {mode}: max rel err on L {rel:.2e}")


def test_doubled_label_leaves_L(env):
    """Listing every sample of a label twice leaves its Parzen mean, hence L,
    unchanged (plain FP32 form, against the single list on the GPU too)."""
    cs, ctx, torch = env
    pr = synth.make_workload(1)
    prm = cs.Params.from_synth(pr.params, precision=0)

    def run(p):
        out = ctx.data_term(_dev(torch, p.image), _dev(torch, p.omega), _dev(torch, p.mask),
                            p.label_off, _dev(torch, p.sample_pix), prm)
        ctx.sync()
        return -out["neglog"].cpu().numpy().reshape(p.n_labels, -1).astype(np.float64)

    L1 = run(pr)
    off = pr.label_off
    s1 = pr.sample_pix[off[1]:off[2]]
    dbl = synth.make_workload(1)
    dbl.sample_pix = np.concatenate([pr.sample_pix[:off[1]], s1, s1,
                                     pr.sample_pix[off[2]:]]).astype(np.int32)
    dbl.label_off = np.array([0, off[1], off[2] + len(s1), off[3] + len(s1)], np.int32)
    L2 = run(dbl)
    np.testing.assert_allclose(L2, L1, rtol=2e-6, atol=2e-6)
    ref = oracle.data_term(dbl)
    assert float(np.max(np.abs(L2 - ref["L"]) / np.maximum(np.abs(ref["L"]), 1.0))) <= 1e-5
