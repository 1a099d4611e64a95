"""Unsupervised mode (Sec. 3.2) through the C ABI vs the reference
(oracle/unsup.py).

cs_kmeans and cs_kmedians decide their assignments in FP32 in the same
fixed order as the reference and form their centres exactly (integer sums;
order statistics), so on the same inputs they agree BIT FOR BIT: centres and
assignments. cs_unsup_data_term forms iota from FP32 codes where the
reference uses FP64 codes: a code error e moves iota by at most
e sqrt(2 / sigma) exp(-1/2) (8.6 e at sigma = 0.01), each l1 distance by at
most k times that and f by twice that over beta, so its colour side is
compared bit for bit and its texture side and f against the bars of the
reduced-precision forms: texture assignments equal wherever the reference's
two nearest centres are more than 1e-3 apart, max |f - f_ref| <= 1e-2 and
max |exp(-f) - exp(-f_ref)| <= 1e-2.
"""
import numpy as np
import pytest

from oracle import unsup
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


def _starts(seed, P, n):
    return np.random.default_rng(seed).choice(P, n, replace=False).astype(np.int32)


@pytest.mark.parametrize("wl,n,iters,seed", [(2, 4, 10, 71), (2, 16, 6, 72), (1, 3, 0, 73)])
def test_kmeans_bit_exact(env, wl, n, iters, seed):
    cs, ctx, torch = env
    pr = synth.make_workload(wl)
    X = pr.image.reshape(-1, 3)
    init = _starts(seed, len(X), n)
    out = ctx.kmeans(_dev(torch, X), init, iters)
    ctx.sync()
    C, lab = unsup.kmeans_fp32(X, init, iters)
    np.testing.assert_array_equal(out["centres"].cpu().numpy(), C)
    np.testing.assert_array_equal(out["assign"].cpu().numpy(), lab)


def test_kmeans_edge_cases(env):
    cs, ctx, torch = env
    X = np.array([[0, 0, 0], [1, 1, 1], [1, 1, 0.9]], np.float32)
    out = ctx.kmeans(_dev(torch, X), [0, 0, 1], 3)  # equal starts: class 1 stays empty
    ctx.sync()
    C, lab = unsup.kmeans_fp32(X, [0, 0, 1], 3)
    np.testing.assert_array_equal(out["centres"].cpu().numpy(), C)
    np.testing.assert_array_equal(out["assign"].cpu().numpy(), lab)
    one = ctx.kmeans(_dev(torch, X[:1]), [0], 2)
    ctx.sync()
    np.testing.assert_array_equal(one["centres"].cpu().numpy(), X[:1])
    # values outside [0, 1] (negative sums) round the same way
    Y = np.random.default_rng(74).normal(0, 3, (5000, 3)).astype(np.float32)
    out = ctx.kmeans(_dev(torch, Y), [1, 2, 3, 4, 5], 5)
    ctx.sync()
    C, lab = unsup.kmeans_fp32(Y, [1, 2, 3, 4, 5], 5)
    np.testing.assert_array_equal(out["centres"].cpu().numpy(), C)
    np.testing.assert_array_equal(out["assign"].cpu().numpy(), lab)


def test_kmedians_bit_exact_on_reference_iota(env):
    """k-medians on the reference's iota (FP64 codes, rounded to FP32) of the
    96 x 64 image: both sides see the same input."""
    import oracle

    cs, ctx, torch = env
    pr = synth.make_workload(1)
    a, _ = oracle.codes(pr.image, pr.omega, pr.mask, pr.params.p, 0.0)
    V = oracle.iota(a, 0.01).T.astype(np.float32).copy()  # (k, P)
    init = _starts(75, V.shape[1], 4)
    out = ctx.kmedians(_dev(torch, V), init, 10)
    ctx.sync()
    C, lab = unsup.kmedians_fp32(V, init, 10)
    np.testing.assert_array_equal(out["centres"].cpu().numpy(), C)
    np.testing.assert_array_equal(out["assign"].cpu().numpy(), lab)


@pytest.mark.parametrize("k,N,n,iters,seed,neg", [
    (98, 20000, 8, 4, 76, False),   # several member-list tiles per class, even and odd counts
    (7, 33, 5, 3, 77, True),        # negative values (signed order), tiny classes
    (3, 4, 4, 2, 78, False),        # one point per class
])
def test_kmedians_bit_exact_random(env, k, N, n, iters, seed, neg):
    cs, ctx, torch = env
    rng = np.random.default_rng(seed)
    V = rng.uniform(-1 if neg else 0, 1, (k, N)).astype(np.float32)
    V[:, N // 2] = V[:, 0]  # a duplicate point: exact ties
    init = _starts(seed + 1, N, n)
    out = ctx.kmedians(_dev(torch, V), init, iters)
    ctx.sync()
    C, lab = unsup.kmedians_fp32(V, init, iters)
    np.testing.assert_array_equal(out["centres"].cpu().numpy(), C)
    np.testing.assert_array_equal(out["assign"].cpu().numpy(), lab)


def _unsup_case(env, pr, nc, nt, seed, sigma_c2=0.02, beta=0.5, iters=(10, 10)):
    cs, ctx, torch = env
    P = pr.H * pr.W
    ci, ti = _starts(seed, P, nc), _starts(seed + 1, P, nt)
    prm = cs.Params.from_synth(pr.params)
    prm.sigma_c2 = sigma_c2
    up = cs.UnsupParams.default(n_colour=nc, n_texture=nt, kmeans_iterations=iters[0],
                                kmedians_iterations=iters[1], beta=beta)
    out = ctx.unsup_data_term(_dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask),
                              prm, up, ci, ti)
    ctx.sync()
    ref = unsup.data_term(pr.image, pr.omega, pr.mask, pr.params.p, prm.iota_sigma, sigma_c2,
                          beta, nc, nt, ci, ti, kmeans_iterations=iters[0],
                          kmedians_iterations=iters[1])
    got = {k: v.cpu().numpy() for k, v in out.items()}
    np.testing.assert_array_equal(got["colour_centres"], ref["colour_centres"])
    np.testing.assert_array_equal(got["colour_assign"], ref["colour_assign"])
    # texture side: assignments equal where the reference's decision is clear
    tc = ref["texture_centres"].astype(np.float64)
    l1 = np.abs(tc[:, :, None] - ref["iota"][None]).sum(axis=1)
    srt = np.sort(l1, axis=0)
    clear = ((srt[1] - srt[0]) > 1e-3).reshape(pr.H, pr.W) if nt > 1 else np.ones(
        (pr.H, pr.W), bool)
    ta_ok = float(np.mean(got["texture_assign"][clear] == ref["texture_assign"][clear]))
    f, fr = got["neglog"].astype(np.float64), ref["f"]
    ferr = float(np.max(np.abs(f - fr)))
    perr = float(np.max(np.abs(np.exp(-f) - np.exp(-fr))))
    assert ta_ok == 1.0 and ferr <= 1e-2 and perr <= 1e-2, (ta_ok, ferr, perr)
    np.testing.assert_allclose(np.exp(-f).sum(axis=0), 1.0, atol=1e-5)
    return ferr, perr, float(clear.mean())


def test_unsup_data_term_workload1(env):
    pr = synth.make_workload(1)
    ferr, perr, clear = _unsup_case(env, pr, 4, 4, 80)
    print(f"unsupervised 96x64, 4 x 4 segments: max |f - f_ref| {ferr:.2e}, "
          f"max prob err {perr:.2e}, clear texture decisions {clear:.4f}")


def test_unsup_data_term_full_size(env):
    """The 481 x 321 image, 16 initial segments (4 colour x 4 texture), every pixel."""
    pr = synth.make_workload(2)
    ferr, perr, clear = _unsup_case(env, pr, 4, 4, 81)
    print(f"unsupervised 481x321, 16 segments: max |f - f_ref| {ferr:.2e}, "
          f"max prob err {perr:.2e}, clear texture decisions {clear:.4f}")


@pytest.mark.parametrize("H,W,p,k,nc,nt,seed", [
    (1, 40, 3, 18, 2, 3, 82),    # one row
    (37, 23, 9, 162, 1, 5, 83),  # one colour class, 9x9 patches
    (20, 30, 7, 98, 6, 1, 84),   # one texture class
])
def test_unsup_data_term_ragged(env, H, W, p, k, nc, nt, seed):
    pr = synth.make_problem(H, W, 2, 4, p=p, k=k, seed=seed, cap_frac=0.9)
    _unsup_case(env, pr, nc, nt, seed, iters=(5, 5))


def test_unsup_segmentation_mdl_reduces_labels(env):
    """The unsupervised pipeline end to end: 16 initial segments, the
    solver's label cost nu removes segments (fewer labels in use as nu grows)."""
    cs, ctx, torch = env
    pr = synth.make_problem(120, 160, 4, 50, p=7, k=98, seed=85)
    P = pr.H * pr.W
    prm = cs.Params.from_synth(pr.params)
    prm.sigma_c2 = 0.02
    up = cs.UnsupParams.default(beta=0.5)
    out = ctx.unsup_data_term(_dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask),
                              prm, up, _starts(86, P, 4), _starts(87, P, 4))
    img = _dev(torch, pr.image)
    used = []
    for nu in (0.0, 200.0, 2000.0):
        lab = ctx.segment(out["neglog"], img, cs.SegParams.default(lam=2.0, nu=nu,
                                                                    iterations=300))["labels"]
        used.append(len(np.unique(lab.cpu().numpy())))
    print(f"labels in use for nu = 0, 200, 2000: {used}")
    assert used[0] >= used[1] >= used[2] and used[2] < used[0]


def test_unsup_invalid(env):
    cs, ctx, torch = env
    pr = synth.make_problem(16, 16, 2, 4, p=5, k=50, seed=88)
    prm = cs.Params.from_synth(pr.params)
    img, om, mk = _dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask)
    bad = [(dict(n_colour=0), [], [1, 2, 3, 4]),
           (dict(n_colour=16, n_texture=16), list(range(16)), list(range(16))),
           (dict(n_colour=2), [0, 256], [1, 2, 3, 4]),
           (dict(beta=0.0), [0, 1, 2, 3], [1, 2, 3, 4])]
    for kw, ci, ti in bad:
        up = cs.UnsupParams.default(**kw)
        with pytest.raises(cs.CsError) as ei:
            ctx.unsup_data_term(img, om, mk, prm, up, ci, ti)
        assert ei.value.status == cs.CS_ERR_INVALID_ARG, kw
    with pytest.raises(cs.CsError):
        ctx.kmeans(_dev(torch, np.zeros((4, 3), np.float32)), [0, 4], 1)
