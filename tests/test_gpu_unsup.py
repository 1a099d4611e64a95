"""Unsupervised mode (Sec. 3.2) through the C ABI vs the FP64 reference
(oracle/unsup.py).

The reference decides in float64 and forms true means and medians; the
kernels decide in FP32 (distances summed in a fixed order) and form their
centres from exact integer sums (k-means: the mean of the values rounded to
multiples of 2^-24, then rounded to FP32) or by exact order statistics
(k-medians). Every round of the GPU's own trajectory is checked against the
reference's definition:

  assignment  the GPU's class for a point is a nearest centre up to the FP32
              rounding of the distances: with D the float64 distances to the
              GPU's centres, D[gpu class] (1 - e) <= min D (1 + e), where
              e = 8u (colour, three squares and two sums) or (k + 2) u (l1
              over k codes), u = 2^-24. Where the two nearest centres are
              further apart than that, this is equality with the reference's
              decision.
  update      the GPU's next centres against the reference's update on the
              GPU's members: k-means within 2^-25 (the 2^-24 rounding of the
              values) + 2^-24 |c| (the FP32 result); k-medians within
              2^-24 |c| (the FP32 mean of the two middle values).

The independent FP64 run (reference assignments and centres from the same
starts) is compared at the end: assignments equal wherever the reference's
margin exceeds the rounding band widened by the measured centre difference.

The data term forms iota from FP32 codes where the reference uses FP64
codes. A code error e moves iota by at most e sqrt(2 / sigma) exp(-1/2)
(8.58 e at sigma = 0.01); e is measured on the case as the largest
difference between the FP32 codes (cs_codes, CS_CODES_FP32: the same
arithmetic as the iota kernel) and the FP64 codes. From it: iota within
d = 8.58 e + 8u (the FP32 square, scale and exponential), medians within
d + u |c|, each l1 distance within k d + (k + 2) u l1, the texture
log-posterior within twice that over beta; the colour and texture
log-softmax in FP32 with the fast exponential and logarithm add at most
48 u (max t_colour + max t_texture) + 16 (n_c + n_t) u + 2e-6 + 4 u |f|
(t_colour = D / (2 sigma_c2), t_texture = l1 / beta). The data term is
compared with the reference's f evaluated at the GPU's own centres (so that
a near tie decided the other way in some round cannot hide a wrong formula),
pixel by pixel against that derived bound.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import unsup
from paper_1312_4746_gb300 import synth

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
IOTA_LIP = math.sqrt(2.0 / 0.01) * math.exp(-0.5)  # max |d iota / d a| at sigma = 0.01


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


def _check_decisions(D, lab, e, slack=None):
    """lab is a nearest class of every column of D (float64 distances) up to
    a relative rounding e of each distance (plus an absolute slack)."""
    dmin = D.min(axis=0)
    dg = D[lab, np.arange(D.shape[1])]
    extra = 0.0 if slack is None else slack
    ok = dg * (1 - e) <= dmin * (1 + e) + extra
    assert ok.all(), (int((~ok).sum()), float(np.max((dg - dmin)[~ok])))
    return float(np.mean(dg == dmin))


def _kmeans_rounds(env, X, init, iters):
    """The GPU's k-means trajectory, round by round, against the reference's
    assignment and update steps; returns the GPU's last centres and
    assignment."""
    cs, ctx, torch = env
    Xd = _dev(torch, X)
    prev = None
    for T in range(iters + 1):
        out = ctx.kmeans(Xd, init, T)
        ctx.sync()
        C = out["centres"].cpu().numpy().astype(np.float64)
        lab = out["assign"].cpu().numpy()
        _check_decisions(unsup.colour_dist2(X, C), lab, 8 * U)
        if prev is not None:  # C = the update of the previous round's members
            want = unsup.colour_means(X, prev[1], prev[0])
            assert np.all(np.abs(C - want) <= 2.0 ** -25 + U * np.abs(want) + 2.0 ** -48), T
        else:
            np.testing.assert_array_equal(C, np.asarray(X, np.float64)[init])
        prev = (C, lab)
    return prev


def _compare_final(C, lab, Cr, labr, D_ref, e, kind):
    """Final GPU result against the independent FP64 run: assignments equal
    wherever the reference's margin exceeds the rounding band widened by the
    measured centre difference delta (a point's distance to a centre moves by
    at most 2 sqrt(3 D) delta + 3 delta^2 (colour) or k delta (l1) when the
    centre moves by delta per coordinate)."""
    delta = float(np.max(np.abs(C - Cr)))
    dmax = D_ref.max(axis=0)
    if kind == "colour":
        shift = 2 * np.sqrt(3 * dmax) * delta + 3 * delta ** 2
    else:
        shift = C.shape[1] * delta
    clear = unsup.margins(D_ref) > 2 * e * dmax + 2 * shift
    assert np.array_equal(lab[clear], labr[clear])
    return delta, float(clear.mean())


@pytest.mark.parametrize("wl,n,iters,seed", [(2, 4, 10, 71), (2, 16, 6, 72), (1, 3, 0, 73)])
def test_kmeans_vs_fp64(env, wl, n, iters, seed):
    pr = synth.make_workload(wl)
    X = pr.image.reshape(-1, 3)
    init = _starts(seed, len(X), n)
    C, lab = _kmeans_rounds(env, X, init, iters)
    Cr, labr = unsup.kmeans(X, init, iters)
    delta, clear = _compare_final(C, lab, Cr, labr, unsup.colour_dist2(X, Cr), 8 * U, "colour")
    print(f"k-means workload {wl}, {n} classes, {iters} rounds: max |C - C_ref| {delta:.2e}, "
          f"clear decisions {clear:.5f}, assignments equal there")
    assert delta <= 1e-6


def test_kmeans_edge_cases(env):
    X = np.array([[0, 0, 0], [1, 1, 1], [1, 1, 0.9]], np.float32)
    C, lab = _kmeans_rounds(env, X, [0, 0, 1], 3)  # equal starts: class 1 stays empty
    np.testing.assert_array_equal(lab, [0, 2, 2])
    np.testing.assert_array_equal(C[1], X[0])
    C1, _ = _kmeans_rounds(env, X[:1], [0], 2)
    np.testing.assert_array_equal(C1, X[:1])
    # values outside [0, 1] (negative sums)
    Y = np.random.default_rng(74).normal(0, 3, (5000, 3)).astype(np.float32)
    C, lab = _kmeans_rounds(env, Y, [1, 2, 3, 4, 5], 5)
    Cr, labr = unsup.kmeans(Y, [1, 2, 3, 4, 5], 5)
    _compare_final(C, lab, Cr, labr, unsup.colour_dist2(Y, Cr), 8 * U, "colour")


def _kmedians_rounds(env, V, init, iters):
    cs, ctx, torch = env
    Vd = _dev(torch, V)
    k = V.shape[0]
    prev = None
    for T in range(iters + 1):
        out = ctx.kmedians(Vd, init, T)
        ctx.sync()
        C = out["centres"].cpu().numpy().astype(np.float64)
        lab = out["assign"].cpu().numpy()
        _check_decisions(unsup.texture_l1(V, C), lab, (k + 2) * U)
        if prev is not None:
            want = unsup.texture_medians(V, prev[1], prev[0])
            assert np.all(np.abs(C - want) <= U * np.abs(want)), T
        else:
            np.testing.assert_array_equal(C, np.asarray(V, np.float64)[:, init].T)
        prev = (C, lab)
    return prev


def test_kmedians_on_reference_iota(env):
    """k-medians on the reference's iota (FP64 codes, rounded to FP32) of the
    96 x 64 image: both sides see the same input."""
    pr = synth.make_workload(1)
    a, _ = oracle.codes(pr.image, pr.omega, pr.mask, pr.params.p, 0.0)
    V = oracle.iota(a, 0.01).T.astype(np.float32).copy()  # (k, P)
    init = _starts(75, V.shape[1], 4)
    C, lab = _kmedians_rounds(env, V, init, 10)
    Cr, labr = unsup.kmedians(V, init, 10)
    delta, clear = _compare_final(C, lab, Cr, labr, unsup.texture_l1(V, Cr),
                                  (V.shape[0] + 2) * U, "l1")
    print(f"k-medians 96x64 iota: max |C - C_ref| {delta:.2e}, clear decisions {clear:.5f}")
    assert delta <= 1e-6


@pytest.mark.parametrize("k,N,n,iters,seed,neg", [
    (98, 20000, 8, 4, 76, False),   # several member-list tiles per class, even and odd counts
    (7, 33, 5, 3, 77, True),        # negative values (signed order), tiny classes
    (3, 4, 4, 2, 78, False),        # one point per class
])
def test_kmedians_random(env, k, N, n, iters, seed, neg):
    rng = np.random.default_rng(seed)
    V = rng.uniform(-1 if neg else 0, 1, (k, N)).astype(np.float32)
    V[:, N // 2] = V[:, 0]  # a duplicate point: exact ties
    init = _starts(seed + 1, N, n)
    C, lab = _kmedians_rounds(env, V, init, iters)
    Cr, labr = unsup.kmedians(V, init, iters)
    _compare_final(C, lab, Cr, labr, unsup.texture_l1(V, Cr), (k + 2) * U, "l1")


def _code_error(env, pr):
    """Largest |a_FP32 - a_FP64| over every pixel (cs_codes in the FP32 form,
    the arithmetic of the iota kernel)."""
    cs, ctx, torch = env
    prm = cs.Params.from_synth(pr.params, codes_form=1)
    c = ctx.codes(_dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask), prm,
                  want_codes=True)
    ctx.sync()
    a32 = c["codes"].cpu().numpy().astype(np.float64)
    a64, _ = oracle.codes(pr.image, pr.omega, pr.mask, pr.params.p, 0.0)
    return float(np.max(np.abs(a32 - a64)))


def _unsup_case(env, pr, nc, nt, seed, sigma_c2=0.02, beta=0.5, iters=(10, 10), rounds=False):
    cs, ctx, torch = env
    P = pr.H * pr.W
    k = pr.k
    ci, ti = _starts(seed, P, nc), _starts(seed + 1, P, nt)
    prm = cs.Params.from_synth(pr.params)
    prm.sigma_c2 = sigma_c2
    img, om, mk = _dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask)
    X = pr.image.reshape(-1, 3)
    io = unsup.iota_all(pr.image, pr.omega, pr.mask, pr.params.p, prm.iota_sigma)  # (k, P)
    d = IOTA_LIP * _code_error(env, pr) + 8 * U  # bound on |iota_GPU - iota_FP64|

    def run(ki, ti_):
        up = cs.UnsupParams.default(n_colour=nc, n_texture=nt, kmeans_iterations=ki,
                                    kmedians_iterations=ti_, beta=beta)
        out = ctx.unsup_data_term(img, om, mk, prm, up, ci, ti)
        ctx.sync()
        return {key: v.cpu().numpy() for key, v in out.items()}

    got = run(*iters)
    Cc = got["colour_centres"].astype(np.float64)
    Ct = got["texture_centres"].astype(np.float64)
    ca = got["colour_assign"].reshape(-1)
    ta = got["texture_assign"].reshape(-1)
    # final assignment steps against the reference's definition at the GPU's centres
    Dc = unsup.colour_dist2(X, Cc)
    _check_decisions(Dc, ca, 8 * U)
    Dt = unsup.texture_l1(io, Ct)
    _check_decisions(Dt, ta, (k + 2) * U, slack=2.0001 * k * d)
    if rounds:  # every update of the trajectory, from the calls with one round fewer
        for T in range(1, max(iters) + 1):
            a, b = run(min(T, iters[0]), min(T, iters[1])), run(min(T - 1, iters[0]),
                                                                min(T - 1, iters[1]))
            if T <= iters[0]:
                want = unsup.colour_means(X, b["colour_assign"].reshape(-1), b["colour_centres"])
                assert np.all(np.abs(a["colour_centres"] - want)
                              <= 2.0 ** -25 + U * np.abs(want) + 2.0 ** -48)
            if T <= iters[1]:
                want = unsup.texture_medians(io, b["texture_assign"].reshape(-1),
                                             b["texture_centres"])
                assert np.all(np.abs(a["texture_centres"] - want) <= d + U * np.abs(want))
    # the data term at the GPU's centres, against the derived bound per pixel
    fr = unsup.data_term_from_centres(pr.image, io, Cc, Ct, sigma_c2, beta).reshape(nc * nt, -1)
    f = got["neglog"].reshape(nc * nt, -1).astype(np.float64)
    tcol = Dc.max(axis=0) / (2 * sigma_c2)
    ttex = Dt.max(axis=0) / beta
    bound = (2 * (k * d + (k + 2) * U * Dt.max(axis=0)) / beta + 48 * U * (tcol + ttex)
             + 16 * (nc + nt) * U + 2e-6 + 4 * U * np.abs(fr).max(axis=0))
    ferr = np.abs(f - fr).max(axis=0)
    assert np.all(ferr <= bound), float(np.max(ferr / bound))
    perr = np.abs(np.exp(-f) - np.exp(-fr)).max(axis=0)
    assert np.all(perr <= 1.01 * bound)
    np.testing.assert_allclose(np.exp(-f).sum(axis=0), 1.0, atol=1e-5)
    # the independent FP64 run: equal colour and texture decisions where clear
    ref = unsup.data_term(pr.image, pr.omega, pr.mask, pr.params.p, prm.iota_sigma, sigma_c2,
                          beta, nc, nt, ci, ti, kmeans_iterations=iters[0],
                          kmedians_iterations=iters[1])
    dc, clear_c = _compare_final(Cc, ca, ref["colour_centres"], ref["colour_assign"].reshape(-1),
                                 unsup.colour_dist2(X, ref["colour_centres"]), 8 * U, "colour")
    dt = float(np.max(np.abs(Ct - ref["texture_centres"])))
    Dtr = unsup.texture_l1(io, ref["texture_centres"])
    band = 2 * ((k + 2) * U * Dtr.max(axis=0) + k * (d + dt))
    clear_t = unsup.margins(Dtr) > band
    assert np.array_equal(ta[clear_t], ref["texture_assign"].reshape(-1)[clear_t])
    return {"ferr": float(ferr.max()), "fbar": float(bound.min()), "perr": float(perr.max()),
            "code_err": (d - 4 * U) / IOTA_LIP, "dc": dc, "dt": dt,
            "clear_c": clear_c, "clear_t": float(clear_t.mean())}


def _report(name, r):
    print(f"{name}: max |f - f_ref| {r['ferr']:.2e} (bar >= {r['fbar']:.2e}), max prob err "
          f"{r['perr']:.2e}, max code err {r['code_err']:.2e}; vs the FP64 run: centres within "
          f"{r['dc']:.1e} (colour) / {r['dt']:.1e} (texture), clear decisions "
          f"{r['clear_c']:.4f} / {r['clear_t']:.4f}")


def test_unsup_data_term_workload1(env):
    pr = synth.make_workload(1)
    _report("unsupervised 96x64, 4 x 4 segments", _unsup_case(env, pr, 4, 4, 80, rounds=True))


def test_unsup_data_term_full_size(env):
    """The 481 x 321 image, 16 initial segments (4 colour x 4 texture), every pixel."""
    pr = synth.make_workload(2)
    _report("unsupervised 481x321, 16 segments", _unsup_case(env, pr, 4, 4, 81))


@pytest.mark.parametrize("H,W,p,k,nc,nt,seed", [
    (1, 40, 3, 18, 2, 3, 82),    # one row
    (37, 23, 9, 162, 1, 5, 83),  # one colour class, 9x9 patches
    (20, 30, 7, 98, 6, 1, 84),   # one texture class
])
def test_unsup_data_term_ragged(env, H, W, p, k, nc, nt, seed):
    pr = synth.make_problem(H, W, 2, 4, p=p, k=k, seed=seed, cap_frac=0.9)
    _unsup_case(env, pr, nc, nt, seed, iters=(5, 5), rounds=True)


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
