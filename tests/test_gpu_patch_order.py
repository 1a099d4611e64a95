"""Patch order 1 (cs_params.patch_order: centre the gray values, mask,
centre again, normalise) vs the FP64 oracle with the same order.

The GPU computes every code of this order in double precision in the
oracle's canonical index order, so the co-support bitmasks are compared bit
for bit and the codes (rounded to FP32) to within one FP32 rounding; the
data term then sees the oracle's bitmasks, and L meets the bars of the
default order (plain FP32 1e-5 relative, tensor-core forms 1e-4).
"""
import ctypes

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


def _gpu_codes(env, pr, img=None):
    cs, ctx, torch = env
    prm = cs.Params.from_synth(pr.params, patch_order=1)
    out = ctx.codes(_dev(torch, pr.image if img is None else img), _dev(torch, pr.omega),
                    _dev(torch, pr.mask), prm, want_codes=True, want_lead16=True)
    ctx.sync()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("H,W,p,k,seed", [
    (64, 96, 5, 50, 1001),   # the 96 x 64 workload's shape
    (37, 53, 3, 17, 21),     # k < 32: one partial word
    (1, 40, 9, 162, 22),     # one-row image, 9 x 9 patches, k = 162
    (30, 1, 7, 98, 23),      # one-column image
])
def test_codes_order1_bit_exact(env, H, W, p, k, seed):
    pr = synth.make_problem(H, W, 2, 4, p=p, k=k, seed=seed, cap_frac=0.9)
    got = _gpu_codes(env, pr)
    a, bits = oracle.codes(pr.image, pr.omega, pr.mask, p, pr.params.tau, order=1)
    np.testing.assert_array_equal(got["bitmask"].view(np.uint32), bits)
    np.testing.assert_allclose(got["codes"], a, rtol=1.2e-7, atol=1e-30)
    lead = np.zeros((H * W, 16))
    lead[:, :min(k, 16)] = a[:, :min(k, 16)]
    np.testing.assert_allclose(got["lead16"], lead, rtol=1.2e-7, atol=1e-30)


def test_codes_order1_flat_and_sampled(env):
    """A constant image is flat in this order (every code 0, every bit set);
    the 481 x 321 workload at sampled pixels."""
    pr = synth.make_problem(20, 24, 2, 4, p=7, k=98, seed=24)
    img = np.full_like(pr.image, 0.4)
    got = _gpu_codes(env, pr, img=img)
    assert np.all(got["codes"] == 0.0)
    _, bits = oracle.codes(img, pr.omega, pr.mask, 7, pr.params.tau, order=1)
    np.testing.assert_array_equal(got["bitmask"].view(np.uint32), bits)
    pr = synth.make_workload(2)
    got = _gpu_codes(env, pr)
    pix = np.unique(np.random.default_rng(25).integers(0, pr.H * pr.W, 3000)).astype(np.int32)
    a, bits = oracle.codes(pr.image, pr.omega, pr.mask, pr.params.p, pr.params.tau, pix=pix,
                           order=1)
    np.testing.assert_array_equal(got["bitmask"].view(np.uint32)[pix], bits)
    np.testing.assert_allclose(got["codes"][pix], a, rtol=1.2e-7, atol=1e-30)


@pytest.mark.parametrize("precision,mode,bar", [(0, 0, 1e-5), (2, 0, 1e-4), (2, 1, 1e-4)])
def test_data_term_order1(env, precision, mode, bar):
    cs, ctx, torch = env
    pr = synth.make_workload(1)
    pr.params.patch_order = 1
    pr.params.mode = mode
    prm = cs.Params.from_synth(pr.params, precision=precision, patch_order=1)
    out = ctx.data_term(_dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask),
                        pr.label_off, _dev(torch, pr.sample_pix), prm)
    ctx.sync()
    nl = pr.n_labels
    L = -out["neglog"].cpu().numpy().reshape(nl, -1).astype(np.float64)
    ref = oracle.data_term(pr)
    rel = float(np.max(np.abs(L - ref["L"]) / np.maximum(np.abs(ref["L"]), 1.0)))
    perr = float(np.max(np.abs(out["post"].cpu().numpy().reshape(nl, -1) - ref["post"])))
    assert rel <= bar and perr <= 1e-2, (rel, perr)
    # the order changes the co-supports (not a no-op switch)
    pr.params.patch_order = 0
    assert np.abs(oracle.data_term(pr)["L"] - ref["L"]).max() > 1e-3


def test_noalloc_order1_matches_cs_codes(env):
    cs, ctx, torch = env
    pr = synth.make_problem(41, 57, 2, 4, p=7, k=98, seed=26)
    prm = cs.Params.from_synth(pr.params, patch_order=1)
    img, om, mask = _dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask)
    ref = ctx.codes(img, om, mask, prm, want_codes=True, want_lead16=True)
    ctx.sync()
    P, k = pr.H * pr.W, pr.k
    bits = torch.full((P, (k + 31) // 32), -1, dtype=torch.int32, device="cuda:0")
    codes = torch.empty((P, k), dtype=torch.float32, device="cuda:0")
    lead = torch.empty((P, 16), dtype=torch.float32, device="cuda:0")
    status = torch.full((2,), 7, dtype=torch.int32, device="cuda:0")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = cs.lib()
    rc = L.cs_codes_noalloc(cs._ptr(img), pr.H, pr.W, cs._ptr(om), k, cs._ptr(mask),
                            ctypes.byref(prm), cs._ptr(codes), cs._ptr(lead), cs._ptr(bits),
                            cs._ptr(status), stream)
    assert rc == cs.CS_OK, L.cs_last_error(None)
    torch.cuda.synchronize()
    assert status.tolist() == [0, 0]
    assert torch.equal(bits, ref["bitmask"]) and torch.equal(codes, ref["codes"])
    assert torch.equal(lead, ref["lead16"])


def test_unsup_rejects_order1(env):
    cs, ctx, torch = env
    pr = synth.make_problem(16, 16, 2, 4, p=5, k=50, seed=27)
    prm = cs.Params.from_synth(pr.params, patch_order=1)
    with pytest.raises(cs.CsError) as ei:
        ctx.unsup_data_term(_dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask),
                            prm, cs.UnsupParams.default(), [0, 1, 2, 3], [4, 5, 6, 7])
    assert ei.value.status == cs.CS_ERR_UNSUPPORTED
