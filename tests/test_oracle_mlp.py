"""Pins of the FP64 surrogate reference (oracle/mlp.py): analytic gradient vs
central finite differences, silu vs its definition, Adam's first step vs its
closed form, bf16 rounding vs exact bit patterns."""
import numpy as np
from scipy import special

from oracle import mlp


def _params(n, seed=0):
    rng = np.random.default_rng(seed)
    p = {}
    for k, s in mlp.shapes(n).items():
        fan = s[1] if len(s) == 2 else 64
        p[k] = rng.normal(0, 1.0 / np.sqrt(fan), s)
    return p


def test_silu_definition():
    u = np.linspace(-30, 30, 1001)
    np.testing.assert_allclose(mlp.silu(u), u * special.expit(u), rtol=1e-13, atol=1e-300)
    h = 1e-6
    np.testing.assert_allclose(mlp.silu_grad(u), (mlp.silu(u + h) - mlp.silu(u - h)) / (2 * h),
                               rtol=1e-6, atol=1e-9)


def test_gradient_finite_differences():
    """Every parameter block: analytic gradient vs central differences of the
    loss. A dropped activation derivative, a transposed weight or a missing
    bias term fails this."""
    n = 5
    p = _params(n, 1)
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (7, mlp.N_IN))
    T = rng.normal(0, 1, (7, n))
    _, g = mlp.loss_and_grad(p, X, T)
    h = 1e-6
    for k in mlp.LAYERS:
        flat = p[k].reshape(-1)
        idx = rng.choice(flat.size, min(12, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = mlp.loss(p, X, T)
            flat[i] = old - h
            lm = mlp.loss(p, X, T)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[i]) <= 1e-7 + 1e-5 * abs(fd), (k, i, fd)


def test_adam_first_step():
    """First bias-corrected Adam step moves each parameter by -lr * sign(g)
    (to within eps)."""
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -0.25, 4.0])}
    st = {"m": {}, "v": {}}
    mlp.adam_step(p, g, st, lr=0.01)
    np.testing.assert_allclose(p["w"], np.array([1.0, -2.0, 3.0]) - 0.01 * np.sign(g["w"]),
                               rtol=0, atol=1e-9)


def test_bf16_round_bit_patterns():
    vals = np.array([1.0, 1.00390625, 1.005859375, -3.140625, 65504.0, 1e-3], np.float32)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: ties to even -> 1.0
    out = mlp.bf16_round(vals)
    assert out[0] == 1.0 and out[1] == 1.0
    assert out[2] == 1.0078125  # 1 + 1.5 * 2^-8 rounds up
    assert out[3] == -3.140625
    # every output is representable with 8 significant bits
    m, e = np.frexp(out[out != 0])
    assert np.all(np.abs(m * 256 - np.round(m * 256)) == 0)
