"""cs_data_term repeated with the same arguments replays a CUDA graph of its
launches (captured at the second call). Every replay must read the current
contents of its input buffers and give the same bits as a direct call on a
fresh context; other arguments (label offsets, parameters) are new keys."""
import numpy as np
import pytest

from paper_1312_4746_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


@pytest.mark.parametrize("precision", [0, 2])
def test_replay_reads_current_inputs(cuda_lib, precision):
    import torch

    import paper_1312_4746_gb300 as cs

    pr = synth.make_problem(96, 128, 3, 400, p=7, k=98, seed=71)
    prm = cs.Params.from_synth(pr.params, precision=precision)
    rng = np.random.default_rng(5)
    ctx = cs.Context(0)
    img = _dev(torch, pr.image)
    om, mask = _dev(torch, pr.omega), _dev(torch, pr.mask)
    smp = _dev(torch, pr.sample_pix)
    out = None
    for call in range(5):
        if call:  # new contents in the same buffers
            img.copy_(_dev(torch, np.clip(pr.image * rng.uniform(0.6, 1.0), 0, 1).astype(np.float32)))
            perm = rng.permutation(pr.H * pr.W)[: pr.n_samples].astype(np.int32)
            smp.copy_(_dev(torch, perm))
        out = ctx.data_term(img, om, mask, pr.label_off, smp, prm, out=out)
        ctx.sync()
        fresh = cs.Context(0)
        ref = fresh.data_term(img, om, mask, pr.label_off, smp, prm)
        fresh.sync()
        for key in ("neglog", "post"):
            assert torch.equal(out[key], ref[key]), (call, key)
        assert ctx.refined_count() == fresh.refined_count()
        fresh.close()
    # a new label split of the same samples is a new call, not a replay
    off2 = np.array([0, 100, 700, pr.n_samples], np.int32)
    out2 = ctx.data_term(img, om, mask, off2, smp, prm)
    fresh = cs.Context(0)
    ref2 = fresh.data_term(img, om, mask, off2, smp, prm)
    ctx.sync()
    fresh.sync()
    assert torch.equal(out2["neglog"], ref2["neglog"])
    fresh.close()
    ctx.close()
