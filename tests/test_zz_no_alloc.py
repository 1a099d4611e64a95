"""cs_codes_noalloc: the allocation-free codes entry point, for callers that
cannot allocate device memory (inside a stream capture, under a fixed memory
budget owned by another allocator, or where cudaMalloc's implicit device
synchronisation is not acceptable).

Called through the C ABI on two calls in a row, it must give exactly the
bitmask and codes that cs_codes gives in the same (FP32) codes form (the
same tolerance as every other co-support test: bit-exact), and reject sizes
beyond its fixed scratch and the tensor-core codes form.
This file sorts last so that a run stopping at its first failure has run
every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1312_4746_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


@pytest.mark.parametrize("H,W,p,k,seed", [(64, 96, 5, 50, 1001), (61, 45, 7, 98, 3),
                                          (33, 70, 9, 162, 4)])
def test_noalloc_matches_cs_codes(cuda_lib, H, W, p, k, seed):
    import torch

    import paper_1312_4746_gb300 as cs

    L = cs.lib()
    pr = synth.make_problem(H, W, 2, 10, p=p, k=k, seed=seed)
    # the allocation-free entry computes the FP32 CUDA-core form of the codes
    prm = cs.Params.from_synth(pr.params, codes_form=cs.CODES_FP32)
    img, om, mask = _dev(torch, pr.image), _dev(torch, pr.omega), _dev(torch, pr.mask)
    ctx = cs.Context(0)
    ref = ctx.codes(img, om, mask, prm, want_codes=True, want_lead16=True)
    ctx.sync()
    P, Wk = H * W, (k + 31) // 32
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):  # two calls in a row share the same scratch
        bits = torch.full((P, Wk), -1, dtype=torch.int32, device="cuda:0")
        codes = torch.empty((P, k), dtype=torch.float32, device="cuda:0")
        lead = torch.empty((P, 16), dtype=torch.float32, device="cuda:0")
        status = torch.full((2,), 7, dtype=torch.int32, device="cuda:0")
        rc = L.cs_codes_noalloc(cs._ptr(img), H, W, cs._ptr(om), k, cs._ptr(mask),
                                ctypes.byref(prm), cs._ptr(codes), cs._ptr(lead), cs._ptr(bits),
                                cs._ptr(status), stream)
        assert rc == cs.CS_OK, L.cs_last_error(None)
        torch.cuda.synchronize()
        assert status.tolist() == [0, 0]
        assert torch.equal(bits, ref["bitmask"])
        assert torch.equal(codes, ref["codes"])
        assert torch.equal(lead, ref["lead16"])
    ctx.close()


def test_noalloc_rejects_oversize(cuda_lib):
    import paper_1312_4746_gb300 as cs

    L = cs.lib()
    prm = cs.Params.default(p=7)
    dummy = ctypes.c_void_p(16)  # never dereferenced: the call must fail before launching
    rc = L.cs_codes_noalloc(dummy, 2048, 1024, dummy, 98, dummy, ctypes.byref(prm), None, None,
                            dummy, dummy, None)
    assert rc == cs.CS_ERR_INVALID_ARG
    assert b"pixels" in L.cs_last_error(None)
    rc = L.cs_codes_noalloc(dummy, 10, 10, dummy, 2000, dummy, ctypes.byref(prm), None, None,
                            dummy, dummy, None)
    assert rc == cs.CS_ERR_INVALID_ARG
    prm.codes_form = cs.CODES_TC
    rc = L.cs_codes_noalloc(dummy, 10, 10, dummy, 98, dummy, ctypes.byref(prm), None, None,
                            dummy, dummy, None)
    assert rc == cs.CS_ERR_UNSUPPORTED
