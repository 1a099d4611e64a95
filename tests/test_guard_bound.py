"""The guard pass's tree-sum filter (csrc/k_codes.cu, codes_guard_kernel):
for the same FP64 element values v_t, the index-order evaluation of a code
(the canonical order of Sec. 2's definition: mean, centring, norm, quotient,
dot product, each sum in index order) and the warp-tree evaluation are both
within

    |O_j| (e_s + N u (1 + e_s)),   e_s = 2 u sqrt(N) A / sqrt(ss) + (N/2 + 5) u

of the exact value (u = 2^-53, A = sum |v_t|, ss = sum c_t^2), so a tree
value clear of tau by four times that decides the bit the index-order value
decides. Checked here on random and nearly flat patches against a 60-digit
evaluation; the tree sum is the warp butterfly over 32 lanes with lane l
holding elements l, l + 32, l + 64.
"""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

U = 2.0 ** -53


def seq_sum(xs):
    s = 0.0
    for x in xs:
        s = s + x
    return s


def tree_sum(xs):
    lanes = [0.0] * 32
    for t, x in enumerate(xs):
        lanes[t % 32] = lanes[t % 32] + x
    o = 16
    while o:
        lanes = [lanes[l] + lanes[l ^ o] for l in range(32)]
        o >>= 1
    assert len(set(lanes)) == 1  # every lane holds the same value
    return lanes[0]


def code(v, o, summ):
    n = len(v)
    mu = summ(v) / n
    c = [x - mu for x in v]
    ss = summ([x * x for x in c])
    nrm = math.sqrt(ss)
    s = [x / nrm for x in c]
    return summ([oj * sj for oj, sj in zip(o, s)])


def exact_code(v, o):
    getcontext().prec = 60
    dv = [Decimal(x) for x in v]
    mu = sum(dv) / len(dv)
    c = [x - mu for x in dv]
    nrm = sum(x * x for x in c).sqrt()
    return sum(Decimal(oj) * (x / nrm) for oj, x in zip(o, c))


def bound(v, o):
    n = len(v)
    a_abs = sum(abs(x) for x in v)
    mu = sum(v) / n
    ss = sum((x - mu) ** 2 for x in v)
    es = 2 * U * math.sqrt(n) * a_abs / math.sqrt(ss) + (0.5 * n + 5) * U
    return math.sqrt(sum(x * x for x in o)) * (es + n * U * (1 + es))


@pytest.mark.parametrize("n", [25, 49, 81])
def test_tree_and_index_order_within_bound(n):
    rng = np.random.default_rng(n)
    worst = 0.0
    for trial in range(60):
        base = rng.uniform(0, 1)
        spread = 10.0 ** rng.uniform(-7, 0)  # down to nearly flat patches
        w = np.exp(-rng.uniform(0, 2, n))     # mask-like weights
        v = [float(x) for x in w * (base + spread * rng.standard_normal(n))]
        o = rng.standard_normal(n)
        o = [float(x) for x in o / np.linalg.norm(o)]
        ex = exact_code(v, o)
        eps = bound(v, o)
        for summ in (seq_sum, tree_sum):
            err = abs(Decimal(code(v, o, summ)) - ex)
            assert err <= Decimal(eps), (n, trial, summ.__name__, float(err), eps)
            worst = max(worst, float(err) / eps)
    print(f"n = {n}: worst error / bound {worst:.3f}")
