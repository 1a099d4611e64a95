"""Learned surrogate: the network kernels against the FP64 reference
(oracle/mlp.py), and the fitted surrogate against the exact likelihoods.

Bars (for every pixel the surrogate answers, fallback pixels included): max
posterior error <= 1e-2 and argmax agreement >= 99.9% against the exact sum;
fallback pixels equal the exact FP32 path bit for bit.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp
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


def _flat_params(p, n):
    return np.concatenate([p[k].reshape(-1) for k in mlp.LAYERS]).astype(np.float32)


def _unflat(v, n):
    out, o = {}, 0
    for k, s in mlp.shapes(n).items():
        size = int(np.prod(s))
        out[k] = v[o:o + size].reshape(s).astype(np.float64)
        o += size
    return out


@pytest.mark.parametrize("n", [3, 10, 16])
def test_forward_and_gradient_vs_oracle(env, n):
    """GPU forward outputs and the full gradient vs the FP64 analytic
    reference evaluated on the same bf16-rounded weights."""
    cs, ctx, torch = env
    rng = np.random.default_rng(n)
    p = {k: rng.normal(0, 0.5 / np.sqrt(s[-1]), s) for k, s in mlp.shapes(n).items()}
    flat = _flat_params(p, n)
    assert flat.size == cs.lib().cs_mlp_param_count(n)
    pb = _unflat(mlp.bf16_round(flat), n)  # what the kernels use
    B = 192
    X = rng.normal(0, 1, (B, mlp.N_IN)).astype(np.float32)
    T = rng.normal(0, 1, (B, n)).astype(np.float32)
    dparams = _dev(torch, flat)
    Z = ctx.mlp_forward(dparams, n, _dev(torch, X))
    g, loss = ctx.mlp_grad(dparams, n, _dev(torch, X), _dev(torch, T))
    ctx.sync()
    z_ref, _ = mlp.forward(pb, X.astype(np.float64))
    np.testing.assert_allclose(Z.cpu().numpy(), z_ref, rtol=1e-4, atol=1e-5)
    l_ref, g_ref = mlp.loss_and_grad(pb, X.astype(np.float64), T.astype(np.float64))
    assert abs(loss.item() - l_ref) <= 1e-4 * abs(l_ref)
    gg = _unflat(g.cpu().numpy(), n)
    for k in mlp.LAYERS:
        scale = np.max(np.abs(g_ref[k])) + 1e-12
        assert np.max(np.abs(gg[k] - g_ref[k])) <= 2e-4 * scale, k


def _exact(env, pr, prm):
    cs, ctx, torch = env
    img = _dev(torch, pr.image)
    c = ctx.codes(img, _dev(torch, pr.omega), _dev(torch, pr.mask), prm, want_lead16=True)
    smp = _dev(torch, pr.sample_pix)
    ex = ctx.likelihood(img, c["bitmask"], pr.k, pr.label_off, smp, prm)
    return img, c, smp, ex


@pytest.mark.parametrize("mode", [0, 1])
def test_surrogate_fit_eval(env, mode):
    """With the calibrated fallback the surrogate meets the bar on every
    pixel; the network alone (no fallback) is measured against the exact
    method: how much faster, and how far off."""
    import time

    cs, ctx, torch = env
    pr = synth.make_problem(256, 256, 4, 1500, p=7, k=98, n_regions=4, seed=31)
    prm = cs.Params.from_synth(pr.params, mode=mode)
    img, c, smp, ex = _exact(env, pr, prm)
    ctx.surrogate_fit(img, c["bitmask"], c["lead16"], pr.k, pr.label_off, smp, prm,
                      frac=0.05, steps=300, seed=7)
    out, nfb = ctx.surrogate_eval(img, c["bitmask"], c["lead16"], pr.k, pr.label_off, smp, prm,
                                  margin=0.1)
    ctx.sync()
    P = pr.H * pr.W
    nl = pr.n_labels
    post = out["post"].cpu().numpy().reshape(nl, P)
    post_ex = ex["post"].cpu().numpy().reshape(nl, P)
    perr = np.max(np.abs(post - post_ex))
    agree = np.mean(np.argmax(post, 0) == np.argmax(post_ex, 0))
    assert perr <= 1e-2 and agree >= 0.999, (perr, agree, nfb)
    # fallback pixels are the exact FP32 sum, bit for bit
    neg = out["neglog"].cpu().numpy().reshape(nl, P)
    neg_ex = ex["neglog"].cpu().numpy().reshape(nl, P)
    assert np.all(neg == neg_ex, axis=0).sum() >= nfb
    # the network alone: time and error against the exact FP32 method
    ts = []
    for fn in ("exact", "net"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            if fn == "exact":
                ctx.likelihood(img, c["bitmask"], pr.k, pr.label_off, smp, prm)
            else:
                raw, _ = ctx.surrogate_eval(img, c["bitmask"], c["lead16"], pr.k, pr.label_off,
                                            smp, prm, margin=-1.0, count=False)
        torch.cuda.synchronize()
        ts.append((time.perf_counter() - t0) / 3)
    praw = raw["post"].cpu().numpy().reshape(nl, P)
    raw_err = np.max(np.abs(praw - post_ex))
    raw_agree = np.mean(np.argmax(praw, 0) == np.argmax(post_ex, 0))
    print(f"mode {mode}: guaranteed path: max prob err {perr:.2e}, fallback share {nfb / P:.3f}; "
          f"network alone: {ts[0] / ts[1]:.1f}x faster than the exact FP32 sum, "
          f"max prob err {raw_err:.3f}, argmax agreement {raw_agree:.3f}")
    assert ts[1] < ts[0]
    assert raw_agree > 1.0 / nl  # better than chance


def test_surrogate_against_oracle_sampled(env):
    """Surrogate posteriors vs the FP64 oracle at sampled pixels."""
    cs, ctx, torch = env
    pr = synth.make_problem(192, 224, 3, 1200, p=7, k=98, n_regions=3, seed=33)
    prm = cs.Params.from_synth(pr.params)
    img, c, smp, _ = _exact(env, pr, prm)
    ctx.surrogate_fit(img, c["bitmask"], c["lead16"], pr.k, pr.label_off, smp, prm,
                      frac=0.05, steps=300, seed=3)
    out, nfb = ctx.surrogate_eval(img, c["bitmask"], c["lead16"], pr.k, pr.label_off, smp, prm)
    ctx.sync()
    rng = np.random.default_rng(4)
    P = pr.H * pr.W
    pix = np.unique(rng.integers(0, P, 1500)).astype(np.int32)
    ref = oracle.data_term(pr, pix=pix)
    post = out["post"].cpu().numpy().reshape(pr.n_labels, P)[:, pix]
    assert np.max(np.abs(post - ref["post"])) <= 1e-2
    assert np.mean(np.argmax(post, 0) == np.argmax(ref["post"], 0)) >= 0.999


def test_surrogate_requires_fit(env):
    cs, ctx, torch = env
    pr = synth.make_problem(40, 40, 2, 50, p=5, k=50, seed=5)
    prm = cs.Params.from_synth(pr.params)
    img, c, smp, _ = _exact(env, pr, prm)
    fresh = cs.Context(0)
    with pytest.raises(cs.CsError) as ei:
        fresh.surrogate_eval(img, c["bitmask"], c["lead16"], pr.k, pr.label_off, smp, prm)
    assert ei.value.status == cs.CS_ERR_INVALID_ARG
    fresh.close()


def test_surrogate_save_load_roundtrip(env, tmp_path):
    """A saved surrogate loaded into a fresh context evaluates identically;
    a malformed file is refused."""
    cs, ctx, torch = env
    pr = synth.make_problem(64, 72, 3, 300, p=7, k=98, n_regions=3, seed=41)
    prm = cs.Params.from_synth(pr.params)
    img, c, smp, _ = _exact(env, pr, prm)
    ctx.surrogate_fit(img, c["bitmask"], c["lead16"], pr.k, pr.label_off, smp, prm,
                      frac=0.1, steps=100, seed=5)
    path = str(tmp_path / "net.cssurr")
    ctx.surrogate_save(path)
    a, _ = ctx.surrogate_eval(img, c["bitmask"], c["lead16"], pr.k, pr.label_off, smp, prm,
                              margin=-1.0, count=False)
    other = cs.Context(0)
    other.surrogate_load(path)
    b, _ = other.surrogate_eval(img, c["bitmask"], c["lead16"], pr.k, pr.label_off, smp, prm,
                                margin=-1.0, count=False)
    torch.cuda.synchronize()
    assert torch.equal(a["neglog"], b["neglog"]) and torch.equal(a["post"], b["post"])
    assert np.array_equal(ctx.surrogate_params(), other.surrogate_params())
    bad = tmp_path / "bad.cssurr"
    bad.write_bytes(b"not a surrogate")
    with pytest.raises(cs.CsError) as ei:
        other.surrogate_load(str(bad))
    assert ei.value.status == cs.CS_ERR_INVALID_ARG
    other.close()
