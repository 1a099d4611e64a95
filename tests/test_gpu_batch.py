"""Batches (cs_batch_*): many images with one persistent tensor-core sum.

Every image of a batch must come out bit-identical to cs_data_term on that
image alone (same kernels, same per-pixel arithmetic and sample order), in
every form, with and without CUDA-graph replay and autotuning, when the sum
kernel has the single-image shape; the other shape agrees within the
a-priori bound. One image is also checked against the FP64 oracle at
sampled pixels.
"""
import dataclasses

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


def _problems(k=98, p=7):
    """Uneven shapes: ragged tiles, 1 to 5 labels, labels with a single
    sample, with 1, 128, 129 and several hundred samples."""
    shapes = [(37, 53, 2, 17, 1), (64, 48, 3, 129, 2), (75, 100, 5, [1, 128, 300, 40, 7], 3),
              (130, 17, 1, 64, 4), (20, 300, 4, 90, 5), (9, 9, 2, [1, 1], 6)]
    out = []
    for H, W, nl, m, seed in shapes:
        out.append(synth.make_problem(H, W, nl, m, p=p, k=k, seed=seed, cap_frac=0.9))
    # one operator and patch mask for the whole batch
    return [dataclasses.replace(q, omega=out[0].omega, mask=out[0].mask) for q in out]


def _inputs(torch, probs):
    return [{"img": _dev(torch, q.image), "sample_pix": _dev(torch, q.sample_pix),
             "label_off": q.label_off} for q in probs]


def _single(ctx, cs, torch, q, inp, prm, omega, mask):
    return ctx.data_term(inp["img"], omega, mask, q.label_off, inp["sample_pix"], prm)


def _same(a, b):
    for key in ("neglog", "post"):
        x, y = a[key].cpu().numpy(), b[key].cpu().numpy()
        assert np.array_equal(x, y), (key, float(np.max(np.abs(x - y))))


@pytest.mark.parametrize("precision,mode", [(2, 0), (1, 0), (2, 1), (0, 0)])
def test_batch_matches_single_images(env, precision, mode):
    cs, ctx, torch = env
    probs = _problems()
    prm = cs.Params.from_synth(probs[0].params, precision=precision, mode=mode)
    omega, mask = _dev(torch, probs[0].omega), _dev(torch, probs[0].mask)
    inp = _inputs(torch, probs)
    b = ctx.batch(inp, omega, mask, prm)
    outs = b.run()
    ctx.sync()
    for q, x, o in zip(probs, inp, outs):
        _same(o, _single(ctx, cs, torch, q, x, prm, omega, mask))
    cfg = b.config()
    assert cfg["pairs"] == sum(q.H * q.W * q.n_samples for q in probs)
    b.close()


def test_batch_graph_replay_rereads_inputs(env):
    cs, ctx, torch = env
    probs = _problems()
    prm = cs.Params.from_synth(probs[0].params, precision=2)
    omega, mask = _dev(torch, probs[0].omega), _dev(torch, probs[0].mask)
    inp = _inputs(torch, probs)
    b = ctx.batch(inp, omega, mask, prm, flags=cs.BATCH_GRAPH)
    rng = np.random.default_rng(0)
    for rep in range(3):
        # new image contents and scribble positions in the same buffers
        for q, x in zip(probs, inp):
            x["img"].copy_(_dev(torch, np.clip(q.image * rng.uniform(0.5, 1.0), 0, 1)
                                .astype(np.float32)))
            perm = rng.permutation(q.H * q.W)[: q.n_samples].astype(np.int32)
            x["sample_pix"].copy_(_dev(torch, perm))
        outs = b.run()
        ctx.sync()
        for q, x, o in zip(probs, inp, outs):
            _same(o, _single(ctx, cs, torch, q, x, prm, omega, mask))
    b.close()


def test_batch_autotune(env):
    cs, ctx, torch = env
    probs = _problems()
    prm = cs.Params.from_synth(probs[0].params, precision=2)
    omega, mask = _dev(torch, probs[0].omega), _dev(torch, probs[0].mask)
    inp = _inputs(torch, probs)
    b = ctx.batch(inp, omega, mask, prm, flags=cs.BATCH_AUTOTUNE | cs.BATCH_GRAPH)
    outs = b.run()
    b.run()
    ctx.sync()
    cfg = b.config()
    assert cfg["n_streams"] in (1, 2, 4, 8) and cfg["order"] in (0, 1)
    assert cfg["sum_variant"] in (0, 1)
    assert cfg["tuned_ms"] > 0
    for q, x, o in zip(probs, inp, outs):
        ref = _single(ctx, cs, torch, q, x, prm, omega, mask)
        if cfg["sum_variant"] == 0:
            _same(o, ref)
        else:
            _close(o, ref, prm.l_tol)
    b.close()
    # a second batch with the same shapes reuses the tuned configuration
    b2 = ctx.batch(inp, omega, mask, prm, flags=cs.BATCH_AUTOTUNE)
    assert b2.config()["n_streams"] == cfg["n_streams"]
    assert b2.config()["sum_variant"] == cfg["sum_variant"]
    b2.close()


def _close(a, b, l_tol):
    """Two tensor-core results, each within l_tol max(|L|, 1) of the exact L
    (rows above the a-priori bound are recomputed in FP64), differ by at most
    twice that."""
    x = -a["neglog"].cpu().numpy().astype(np.float64)
    y = -b["neglog"].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(x - y) <= 2 * l_tol * np.maximum(np.abs(y), 1)), float(np.max(np.abs(x - y)))


@pytest.mark.parametrize("precision,mode", [(2, 0), (1, 0), (2, 1)])
def test_batch_sum_shapes(env, precision, mode):
    """Both shapes of the tensor-core sum kernel (two CTAs per SM with 8
    epilogue warps; one CTA per SM with 16 epilogue warps and a deeper sample
    ring): shape 0 bit-identical to the single-image calls, shape 1 within
    the a-priori bound of it; an invalid configuration is refused."""
    cs, ctx, torch = env
    probs = _problems()
    prm = cs.Params.from_synth(probs[0].params, precision=precision, mode=mode)
    omega, mask = _dev(torch, probs[0].omega), _dev(torch, probs[0].mask)
    inp = _inputs(torch, probs)
    b = ctx.batch(inp, omega, mask, prm, flags=cs.BATCH_GRAPH)
    got, shapes = [], []
    for variant in (0, 1):
        b.set_config(2, 0, variant)
        outs = b.run()
        ctx.sync()
        cfg = b.config()
        assert cfg["sum_variant"] == variant
        shapes.append(cfg["sum_shape"])
        got.append([{k: o[k].clone() for k in ("neglog", "post")} for o in outs])
    assert shapes[1]["ctas_per_sm"] == 1 and shapes[1]["epilogue_warps"] == 16
    for q, x, o0, o1 in zip(probs, inp, got[0], got[1]):
        _same(o0, _single(ctx, cs, torch, q, x, prm, omega, mask))
        _close(o1, o0, prm.l_tol)
    with pytest.raises(cs.CsError):
        b.set_config(3, 0, 2)
    b.close()


def test_batch_one_shot_and_oracle(env):
    cs, ctx, torch = env
    probs = _problems()
    prm = cs.Params.from_synth(probs[0].params, precision=2)
    omega, mask = _dev(torch, probs[0].omega), _dev(torch, probs[0].mask)
    inp = _inputs(torch, probs)
    outs = ctx.batch_data_term(inp, omega, mask, prm)
    q, o = probs[2], outs[2]
    rng = np.random.default_rng(1)
    pix = np.unique(rng.integers(0, q.H * q.W, 600)).astype(np.int32)
    ref = oracle.data_term(q, pix=pix)
    nl = q.n_labels
    L = -o["neglog"].cpu().numpy().reshape(nl, -1)[:, pix].astype(np.float64)
    post = o["post"].cpu().numpy().reshape(nl, -1)[:, pix]
    rel = np.max(np.abs(L - ref["L"]) / np.maximum(np.abs(ref["L"]), 1.0))
    assert rel <= 1e-4, rel
    assert np.max(np.abs(post - ref["post"])) <= 1e-2


def test_batch_invalid(env):
    cs, ctx, torch = env
    probs = _problems()[:2]
    prm = cs.Params.from_synth(probs[0].params, precision=2)
    omega, mask = _dev(torch, probs[0].omega), _dev(torch, probs[0].mask)
    inp = _inputs(torch, probs)
    bad = dict(inp[1])
    bad["label_off"] = np.array([0, 5, 5], np.int32)  # second label empty
    with pytest.raises(cs.CsError) as ei:
        ctx.batch([inp[0], bad], omega, mask, prm)
    assert ei.value.status == cs.CS_ERR_INVALID_ARG and "image 1" in str(ei.value)
    with pytest.raises(cs.CsError) as ei:
        ctx.batch([], omega, mask, prm)
    assert ei.value.status == cs.CS_ERR_INVALID_ARG


@pytest.mark.parametrize("precision", [2, 0])
def test_batch_likelihood_with_given_bitmasks(env, precision):
    """cs_batch_likelihood on bitmasks computed beforehand gives what
    cs_likelihood gives on each image."""
    cs, ctx, torch = env
    probs = _problems()
    prm = cs.Params.from_synth(probs[0].params, precision=precision)
    omega, mask = _dev(torch, probs[0].omega), _dev(torch, probs[0].mask)
    inp = _inputs(torch, probs)
    for x in inp:
        x["bitmask"] = ctx.codes(x["img"], omega, mask, prm)["bitmask"]
    outs = ctx.batch_likelihood(inp, probs[0].k, prm)
    for q, x, o in zip(probs, inp, outs):
        ref = ctx.likelihood(x["img"], x["bitmask"], q.k, q.label_off, x["sample_pix"], prm)
        ctx.sync()
        _same(o, ref)
