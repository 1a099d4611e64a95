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


def test_noalloc_rejects_bad_params(cuda_lib):
    """The same parameter checks as cs_codes: patch order and codes form."""
    import paper_1312_4746_gb300 as cs

    L = cs.lib()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the call must fail before launching
    for field, value in (("patch_order", 2), ("patch_order", -1), ("codes_form", 7)):
        prm = cs.Params.default(p=7)
        setattr(prm, field, value)
        rc = L.cs_codes_noalloc(dummy, 10, 10, dummy, 98, dummy, ctypes.byref(prm), None, None,
                                dummy, dummy, None)
        assert rc == cs.CS_ERR_INVALID_ARG, (field, value)


def test_noalloc_guard_overflow_reported(cuda_lib):
    """More entries needing the exact double-precision recheck than the fixed
    list holds (2^20): a one-pixel checkerboard makes every interior window
    one of two patterns, every operator row is the same unit vector, and tau
    is set to the exact code of one pattern, so about half of all P x k
    entries lie within their FP32 error bound of tau. The call reports the
    overflow in dev_status (code 101, then the number of entries), and a
    normal call afterwards starts from a clean status."""
    import torch

    import oracle
    import paper_1312_4746_gb300 as cs

    L = cs.lib()
    H, W, p, k = 192, 192, 7, 128
    yy, xx = np.mgrid[0:H, 0:W]
    g = np.where((yy + xx) % 2 == 0, 0.8, 0.2).astype(np.float32)
    img = np.repeat(g[:, :, None], 3, axis=2).copy()
    row = np.random.default_rng(5).normal(size=p * p)
    om = np.tile((row / np.linalg.norm(row)).astype(np.float32), (k, 1))
    mask = synth.make_mask(p)
    a, _ = oracle.codes(img, om, mask, p, 0.0, pix=np.array([(H // 2) * W + W // 2], np.int32))
    prm = cs.Params.default(p=p, codes_form=cs.CODES_FP32)
    prm.tau = float(abs(a[0, 0]))
    P, Wk = H * W, (k + 31) // 32
    d_img, d_om, d_mask = _dev(torch, img), _dev(torch, om), _dev(torch, mask)
    bits = torch.empty((P, Wk), dtype=torch.int32, device="cuda:0")
    status = torch.zeros(2, dtype=torch.int32, device="cuda:0")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.cs_codes_noalloc(cs._ptr(d_img), H, W, cs._ptr(d_om), k, cs._ptr(d_mask),
                            ctypes.byref(prm), None, None, cs._ptr(bits), cs._ptr(status), stream)
    assert rc == cs.CS_OK, L.cs_last_error(None)
    torch.cuda.synchronize()
    st = status.tolist()
    assert st[0] == 101 and st[1] > (1 << 20), st
    print(f"guard overflow reported: status {st[0]}, {st[1]} entries for a list of {1 << 20}")
    prm.tau = 0.1  # a normal call on the same scratch: clean status again
    rc = L.cs_codes_noalloc(cs._ptr(d_img), H, W, cs._ptr(d_om), k, cs._ptr(d_mask),
                            ctypes.byref(prm), None, None, cs._ptr(bits), cs._ptr(status), stream)
    assert rc == cs.CS_OK
    torch.cuda.synchronize()
    assert status.tolist() == [0, 0]
