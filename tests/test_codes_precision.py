"""Why the codes GEMM keeps split-BF16 operands rather than FP8 with
per-row scaling: the share of co-support entries that a rigorous error
bound cannot decide (|a_j| within the bound of tau) and that the exact FP64
recheck would then have to recompute.

For unit-norm patches s and operator rows O_j, an e4m3 operand carries a
relative rounding error of at most 2^-4 (3 mantissa bits), so a product
O_jt s_t at most 2^-3 + 2^-8 of itself, and the code a_j = sum_t O_jt s_t at
most that times sum_t |O_jt s_t|. The three-piece BF16 splits leave
2^-24-level errors per product; with the FP32 accumulation, 100 2^-24
sum_t |O_jt s_t| bounds them generously. Computed from the FP64 oracle's
patches and codes of a 9x9-patch problem (k = 162, the 4096 x 4096
workload's operator shape) at sampled pixels; tau = 0.1.
"""
import numpy as np

import oracle
from paper_1312_4746_gb300 import synth


def test_fp8_codes_guard_share():
    pr = synth.make_problem(256, 256, 4, 200, p=9, k=162, seed=1005)
    pix = np.unique(np.random.default_rng(9).integers(0, pr.H * pr.W, 4000)).astype(np.int32)
    s = oracle.patches(pr.image, pr.mask, pr.params.p, pix=pix)  # (cnt, n) unit patches
    a, _ = oracle.codes(pr.image, pr.omega, pr.mask, pr.params.p, 0.1, pix=pix)
    absum = np.abs(s) @ np.abs(pr.omega.astype(np.float64)).T  # sum_t |O_jt s_t|
    near = np.abs(np.abs(a) - 0.1)
    fp8 = float(np.mean(near <= (2.0 ** -3 + 2.0 ** -8) * absum))
    bf16 = float(np.mean(near <= 100 * 2.0 ** -24 * absum))
    print(f"guard share: FP8 per-row scaled {fp8:.3f}, split BF16 {bf16:.2e}")
    assert fp8 > 0.5 and bf16 < 1e-3
