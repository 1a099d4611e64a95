"""The timeout path of the bounded device waits, on the GPU, without a fault.

Every barrier wait in the solver's cooperative launch and in the
tensor-core sum gives up after a time limit, records a timeout (and the
site) in the context's device error word, raises an abort flag that the
launch's other waits see, and lets the launch end; cs_sync_status then
returns CS_ERR_TIMEOUT and the context stays usable. The test hook
cs_test_wait shortens the limit and makes one wait run out: a grid-barrier
arrival that one solver block skips, or, in the sum, a barrier that nothing
completes, waited on by the MMA-issuing thread of one CTA before it issues
any work (so no tensor-core operation or copy is in flight when the CTA
frees its tensor memory and exits). The next launch on the same context
runs normally and reproduces the earlier result bit for bit.
"""
import re
import time

import numpy as np
import pytest

from paper_1312_4746_gb300 import synth

pytestmark = pytest.mark.gpu

LIMIT_NS = 20_000_000  # 20 ms: far above any normal wait of these launches


@pytest.fixture(scope="module")
def env(cuda_lib):
    import torch

    import paper_1312_4746_gb300 as cs

    ctx = cs.Context(0)
    yield cs, ctx, torch
    ctx.test_wait(0, cs.STALL_NONE)
    ctx.close()


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _inputs(torch, pr):
    return (_dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask),
            _dev(torch, pr.sample_pix))


def test_segment_grid_barrier_timeout(env):
    cs, ctx, torch = env
    pr = synth.make_workload(1)
    img, om, mask, smp = _inputs(torch, pr)
    prm = cs.Params.from_synth(pr.params, precision=cs.FP8)
    f = ctx.data_term(img, om, mask, pr.label_off, smp, prm)["neglog"]
    sp = cs.SegParams.default(lam=2.0, iterations=50)
    ref = ctx.segment(f, img, sp)
    ctx.sync()
    u_ref, lab_ref = ref["u"].clone(), ref["labels"].clone()

    ctx.test_wait(LIMIT_NS, cs.STALL_SEGMENT)
    t0 = time.perf_counter()
    ctx.segment(f, img, sp)
    with pytest.raises(cs.CsError) as ei:
        ctx.sync()
    dt = time.perf_counter() - t0
    assert ei.value.status == cs.CS_ERR_TIMEOUT, ei.value
    assert "site 41" in str(ei.value), ei.value
    assert dt < 0.5, dt  # the shortened limit, not the default 1 s
    print(f"solver: {ei.value} after {dt * 1e3:.1f} ms")

    ctx.test_wait(0, cs.STALL_NONE)
    out = ctx.segment(f, img, sp)
    ctx.sync()
    assert torch.equal(out["u"], u_ref) and torch.equal(out["labels"], lab_ref)


@pytest.mark.parametrize("precision", [1, 2])  # BF16, FP8 texture operands
def test_tensor_core_sum_timeout(env, precision):
    cs, ctx, torch = env
    pr = synth.make_workload(1)
    img, om, mask, smp = _inputs(torch, pr)
    prm = cs.Params.from_synth(pr.params, precision=precision)
    ref = ctx.data_term(img, om, mask, pr.label_off, smp, prm)["neglog"].clone()
    ctx.sync()

    ctx.test_wait(LIMIT_NS, cs.STALL_SUM)
    t0 = time.perf_counter()
    ctx.data_term(img, om, mask, pr.label_off, smp, prm)
    with pytest.raises(cs.CsError) as ei:
        ctx.sync()
    dt = time.perf_counter() - t0
    assert ei.value.status == cs.CS_ERR_TIMEOUT, ei.value
    # the first wait to give up records its site: the stalled one (2) or a
    # wait of the same CTA that depends on it (the sum's sites are 1 .. 11)
    site = int(re.search(r"site (\d+)", str(ei.value)).group(1))
    assert 1 <= site <= 11, ei.value
    assert dt < 0.5, dt
    print(f"tensor-core sum: {ei.value} after {dt * 1e3:.1f} ms")

    ctx.test_wait(0, cs.STALL_NONE)
    out = ctx.data_term(img, om, mask, pr.label_off, smp, prm)
    ctx.sync()
    assert torch.equal(out["neglog"], ref)


def test_stall_is_one_shot_and_checked(env):
    cs, ctx, torch = env
    with pytest.raises(cs.CsError) as ei:
        ctx.test_wait(-1, cs.STALL_NONE)
    assert ei.value.status == cs.CS_ERR_INVALID_ARG
    with pytest.raises(cs.CsError):
        ctx.test_wait(0, 3)
    # an armed stall that a plain FP32 sum does not consume stays armed for
    # the next tensor-core sum only; disarm it here
    ctx.test_wait(0, cs.STALL_SUM)
    ctx.test_wait(0, cs.STALL_NONE)
    pr = synth.make_workload(1)
    img, om, mask, smp = _inputs(torch, pr)
    prm = cs.Params.from_synth(pr.params, precision=cs.FP8)
    ctx.data_term(img, om, mask, pr.label_off, smp, prm)
    ctx.sync()
