"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Bar: co-support bitmasks and squared scribble distances bit-exact; FP32
log-likelihoods within max |L - L_o| / max(|L_o|, 1) <= 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_1312_4746_gb300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5


@pytest.fixture(scope="module")
def env(cuda_lib):
    import torch

    import paper_1312_4746_gb300 as cs

    ctx = cs.Context(0)
    yield cs, ctx, torch
    ctx.close()


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _run(env, pr, mode=None, want_codes=False, precision=0, codes_form=0):
    cs, ctx, torch = env
    prm = cs.Params.from_synth(pr.params, precision=precision, codes_form=codes_form)
    if mode is not None:
        prm.mode = mode
    img = _dev(torch, pr.image)
    c = ctx.codes(img, _dev(torch, pr.omega), _dev(torch, pr.mask), prm, want_codes=want_codes)
    out = ctx.likelihood(img, c["bitmask"], pr.k, pr.label_off, _dev(torch, pr.sample_pix), prm,
                         want_dist2=True)
    ctx.sync()
    nl = pr.n_labels
    return {
        "bits": c["bitmask"].cpu().numpy().view(np.uint32),
        "codes": None if c["codes"] is None else c["codes"].cpu().numpy(),
        "L": -out["neglog"].cpu().numpy().reshape(nl, -1).astype(np.float64),
        "post": out["post"].cpu().numpy().reshape(nl, -1).astype(np.float64),
        "dist2": out["dist2"].cpu().numpy().reshape(nl, -1),
    }


def _rel(L, Lo):
    return float(np.max(np.abs(L - Lo) / np.maximum(np.abs(Lo), 1.0)))


def _check_all(pr, got, ref):
    assert np.array_equal(got["bits"], ref["bits_px"]), "bitmask mismatch"
    assert np.array_equal(got["dist2"], ref["dist2"]), "dist2 mismatch"
    rel = _rel(got["L"], ref["L"])
    assert rel <= REL_TOL, rel
    assert np.max(np.abs(got["post"] - ref["post"])) < 1e-4
    np.testing.assert_allclose(got["post"].sum(0), 1.0, atol=1e-5)


@pytest.mark.parametrize("mode", [0, 1])
def test_workload1_full(env, mode):
    """96x64, 3 labels x 300 samples, 5x5 patches, Omega 50x25: every pixel."""
    pr = synth.make_workload(1)
    got = _run(env, pr, mode=mode)
    ref = oracle.data_term(pr, mode=mode, want_dist2=True)
    _check_all(pr, got, ref)


@pytest.mark.parametrize("H,W,nl,m,p,k,seed", [
    (37, 53, 2, 17, 5, 17, 1),     # k < 32, ragged image, ragged sample tile
    (61, 45, 3, 129, 7, 98, 2),    # 129 samples: one full tile plus one
    (33, 70, 4, 40, 9, 162, 3),    # 9x9 patches, k = 162 (6 words)
    (1, 7, 1, 3, 3, 40, 4),        # one-row image, windows clamp everywhere
    (5, 1, 2, 1, 5, 64, 5),        # one-column image, single sample per label
    (130, 129, 5, 300, 7, 256, 6), # k = 256 (8 words), P not a multiple of 128
    (29, 35, 2, 20, 9, 256, 13),   # 9x9 patches and k = 256: the per-tile codes kernel
])
def test_ragged_shapes(env, H, W, nl, m, p, k, seed):
    pr = synth.make_problem(H, W, nl, m, p=p, k=k, seed=seed, cap_frac=0.9)
    for mode in (0, 1):
        got = _run(env, pr, mode=mode)  # tensor-core codes (k <= 256)
        ref = oracle.data_term(pr, mode=mode, want_dist2=True)
        _check_all(pr, got, ref)
    got = _run(env, pr, codes_form=1)  # FP32 CUDA-core codes
    assert np.array_equal(got["bits"], ref["bits_px"]), "bitmask mismatch (FP32 codes)"


@pytest.mark.parametrize("codes_form,bound", [(1, 2e-5), (2, 1e-5)])
def test_codes_values(env, codes_form, bound):
    """Codes within their form's error bound of the FP64 codes (unit-norm
    operator rows): FP32 dot products, or the tensor-core GEMM over
    three-piece BF16 splits (about 2.3e-6 from splits and accumulation plus
    the FP32 patch error)."""
    pr = synth.make_problem(40, 44, 2, 10, p=7, k=98, seed=8)
    got = _run(env, pr, want_codes=True, codes_form=codes_form)
    a, bits = oracle.codes(pr.image, pr.omega, pr.mask, 7, 0.1)
    err = np.max(np.abs(got["codes"] - a))
    assert err < bound, err
    assert np.array_equal(got["bits"], bits)


def test_codes_form_selection(env):
    """k > 256: the automatic form falls back to FP32 codes; the tensor-core
    form is refused."""
    cs, ctx, torch = env
    pr = synth.make_problem(20, 21, 2, 8, p=5, k=300, seed=12)
    prm = cs.Params.from_synth(pr.params)
    img = _dev(torch, pr.image)
    c = ctx.codes(img, _dev(torch, pr.omega), _dev(torch, pr.mask), prm)
    ctx.sync()
    _, bits = oracle.codes(pr.image, pr.omega, pr.mask, 5, 0.1, want_codes=False)
    assert np.array_equal(c["bitmask"].cpu().numpy().view(np.uint32), bits)
    prm.codes_form = cs.CODES_TC
    with pytest.raises(cs.CsError) as ei:
        ctx.codes(img, _dev(torch, pr.omega), _dev(torch, pr.mask), prm)
    assert ei.value.status == cs.CS_ERR_UNSUPPORTED
    prm.codes_form = 7
    with pytest.raises(cs.CsError) as ei:
        ctx.codes(img, _dev(torch, pr.omega), _dev(torch, pr.mask), prm)
    assert ei.value.status == cs.CS_ERR_INVALID_ARG


def test_threshold_ties_exact(env):
    """tau equal to an FP64 code of some entries: those entries sit inside the
    FP32 guard band and must be decided in canonical FP64 (inclusive test)."""
    pr = synth.make_problem(24, 28, 2, 10, p=5, k=50, seed=9)
    a, _ = oracle.codes(pr.image, pr.omega, pr.mask, 5, 0.1)
    for tau in (abs(a[100, 3]), abs(a[7, 40]), np.nextafter(abs(a[55, 12]), 0)):
        pr.params.tau = float(tau)
        _, bits = oracle.codes(pr.image, pr.omega, pr.mask, 5, tau, want_codes=False)
        for cf in (1, 2):
            got = _run(env, pr, codes_form=cf)
            assert np.array_equal(got["bits"], bits), cf


def test_flat_and_constant_images(env):
    """All-zero image: every patch is flat (s = 0), all bits set. Constant
    image: identical masked patches everywhere, TSM = 0."""
    for val in (0.0, 0.4):
        pr = synth.make_problem(20, 24, 2, 8, p=7, k=98, seed=10)
        pr.image[:] = val
        ref = oracle.data_term(pr, want_dist2=True)
        for cf in (1, 2):
            got = _run(env, pr, codes_form=cf)
            _check_all(pr, got, ref)
        if val == 0.0:
            assert (got["bits"][:, :3] == np.uint32(0xFFFFFFFF)).all()


def test_cosupport_entry(env):
    cs, ctx, torch = env
    rng = np.random.default_rng(11)
    codes = rng.normal(0, 0.15, (1000, 77)).astype(np.float32)
    codes[5, 3] = np.float32(0.1)
    codes[6, 4] = np.nextafter(np.float32(0.1), np.float32(1))
    bits = ctx.cosupport(_dev(torch, codes), 0.1)
    ctx.sync()
    got = bits.cpu().numpy().view(np.uint32)
    u = np.abs(codes.astype(np.float64)) <= 0.1
    pad = np.zeros((1000, 96 - 77), bool)
    expect = np.packbits(np.concatenate([u, pad], 1), axis=1, bitorder="little").view(np.uint32)
    assert np.array_equal(got, expect)


def test_permutation_invariance(env):
    pr = synth.make_problem(50, 60, 3, 70, p=5, k=50, seed=12)
    g1 = _run(env, pr)
    rng = np.random.default_rng(13)
    perm = np.concatenate([pr.label_off[i] + rng.permutation(pr.label_off[i + 1] - pr.label_off[i])
                           for i in range(pr.n_labels)])
    pr.sample_pix = pr.sample_pix[perm]
    g2 = _run(env, pr)
    assert np.array_equal(g1["dist2"], g2["dist2"])
    assert _rel(g1["L"], g2["L"]) < 1e-6


def test_invalid_args(env):
    cs, ctx, torch = env
    pr = synth.make_problem(10, 12, 2, 4, p=5, seed=14)
    prm = cs.Params.from_synth(pr.params)
    img = _dev(torch, pr.image)
    c = ctx.codes(img, _dev(torch, pr.omega), _dev(torch, pr.mask), prm)
    bad = pr.label_off.copy()
    bad[1] = bad[0]  # empty label 0
    with pytest.raises(cs.CsError) as ei:
        ctx.likelihood(img, c["bitmask"], pr.k, bad, _dev(torch, pr.sample_pix), prm)
    assert ei.value.status == cs.CS_ERR_INVALID_ARG
    prm.p = 11
    with pytest.raises(cs.CsError) as ei:
        ctx.codes(img, _dev(torch, pr.omega), _dev(torch, pr.mask), prm)
    assert ei.value.status == cs.CS_ERR_UNSUPPORTED


def test_workload2_sampled(env):
    """481x321, 5 labels x 2000 samples, 7x7, Omega 98x49: full bitmasks and
    distances exact; L checked at 3000 sampled pixels (incl. corners)."""
    pr = synth.make_workload(2)
    got = _run(env, pr)
    rng = np.random.default_rng(15)
    P = pr.H * pr.W
    pix = np.unique(np.concatenate([rng.integers(0, P, 3000), [0, pr.W - 1, P - pr.W, P - 1]]))
    pix = pix.astype(np.int32)
    ref = oracle.data_term(pr, pix=pix, want_dist2=True)
    _, bits_all = oracle.codes(pr.image, pr.omega, pr.mask, pr.params.p, pr.params.tau,
                               want_codes=False)
    assert np.array_equal(got["bits"], bits_all)
    assert np.array_equal(got["dist2"][:, pix], ref["dist2"])
    assert _rel(got["L"][:, pix], ref["L"]) <= REL_TOL
    assert np.max(np.abs(got["post"][:, pix] - ref["post"])) < 1e-4


@pytest.mark.parametrize("precision", [0, 2])
def test_data_term_entry(env, precision):
    """cs_data_term (distance transform overlapped with the codes on a side
    stream) gives exactly what cs_codes followed by cs_likelihood gives."""
    cs, ctx, torch = env
    pr = synth.make_workload(1)
    prm = cs.Params.from_synth(pr.params, precision=precision)
    img, om, mask = _dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask)
    smp = _dev(torch, pr.sample_pix)
    one = ctx.data_term(img, om, mask, pr.label_off, smp, prm, want_bitmask=True, want_dist2=True)
    c = ctx.codes(img, om, mask, prm)
    two = ctx.likelihood(img, c["bitmask"], pr.k, pr.label_off, smp, prm, want_dist2=True)
    ctx.sync()
    assert torch.equal(one["bitmask"], c["bitmask"])
    assert torch.equal(one["dist2"], two["dist2"])
    assert torch.equal(one["neglog"], two["neglog"])
    ref = oracle.data_term(pr, want_dist2=True)
    assert np.array_equal(one["bitmask"].cpu().numpy().view(np.uint32), ref["bits_px"])
    assert np.array_equal(one["dist2"].cpu().numpy().reshape(pr.n_labels, -1), ref["dist2"])


@pytest.mark.parametrize("H,W,nl,m,seed", [
    (12, 5500, 3, [40, 1, 300], 31),   # labels x width >= 16384: envelope column pass
    (60, 90, 2, [1, 25], 32),          # short image, few columns: outward-scan column pass
    (1030, 15, 2, [3, 9], 33),         # tall and narrow: 8 envelope segments, global-memory stacks
    (200, 70, 2, [5, 30], 34),         # 2 segments, shared-memory stacks
    (400, 50, 3, [2, 17, 60], 35),     # 4 segments, shared-memory stacks
    (480, 33, 2, [1, 40], 36),         # 4 segments, global-memory stacks; segments without seeds
])
def test_distance_transform_paths(env, H, W, nl, m, seed):
    """Every column pass of the exact distance transform equals brute force."""
    cs, ctx, torch = env
    rng = np.random.default_rng(seed)
    P = H * W
    pix = [np.sort(rng.choice(P, mi, replace=False)) for mi in m]
    off = np.concatenate([[0], np.cumsum(m)]).astype(np.int32)
    smp = np.concatenate(pix).astype(np.int32)
    img = rng.uniform(0, 1, (H, W, 3)).astype(np.float32)
    k = 16
    prm = cs.Params.default(p=3)
    bits = torch.zeros((P, 1), dtype=torch.int32, device="cuda:0")
    out = ctx.likelihood(_dev(torch, img), bits, k, off, _dev(torch, smp), prm, want_dist2=True)
    ctx.sync()
    ref = oracle.dist2(H, W, off, smp)
    assert np.array_equal(out["dist2"].cpu().numpy().reshape(nl, -1), ref)
