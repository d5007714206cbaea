"""Pins of the learned screen's FP64 network oracle.

The exact (unrounded) gradient is checked against central finite differences
of the loss; a network wired as a single linear unit reduces to logistic
regression; BF16 rounding follows round-to-nearest-even on binary32; the
rounded variant stays within BF16 error of the exact one.
"""
import numpy as np
import pytest


def rand_params(rng, orc, scale=0.3):
    return (rng.standard_normal(orc.mlp_nparams()) * scale).astype(np.float32)


def test_bf16_round_to_nearest_even(orc):
    cases = {1.0: 1.0, 1 + 2 ** -8: 1.0, 1 + 3 * 2 ** -8: 1 + 2 ** -6, 1 + 2 ** -7: 1 + 2 ** -7,
             -2.5: -2.5, 3.14159: 3.140625, 1e-40: 1e-40 * 0 + orc.bf16(1e-40)}
    for x, want in cases.items():
        assert orc.bf16(x) == pytest.approx(want, abs=0), x
    rng = np.random.default_rng(1)
    for x in rng.standard_normal(2000).astype(np.float32):
        b = orc.bf16(float(x))
        bits = np.float32(b).view(np.uint32)
        assert bits & 0xFFFF == 0
        # the nearest BF16 neighbour: |x - b| <= half a BF16 ulp of x
        ulp = 2.0 ** (np.floor(np.log2(abs(float(x)))) - 7)
        assert abs(float(x) - b) <= ulp / 2 + 1e-30


def test_exact_gradient_matches_finite_differences(orc):
    rng = np.random.default_rng(2)
    n = 7
    X = rng.standard_normal((n, 12))
    y = (rng.random(n) < 0.4).astype(np.float64)
    P = rng.standard_normal(orc.mlp_nparams()) * 0.3
    G, loss = orc.mlp_grad_exact(P, X, y)
    h = 1e-6
    idx = list(range(0, 768, 37)) + list(range(768, 832, 5)) + list(range(832, 4928, 211)) + \
        list(range(4928, 4992, 7)) + list(range(4992, 5057, 9)) + [5056]
    for k in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[k] += h
        Pm[k] -= h
        fd = (orc.mlp_loss_exact(Pp, X, y) - orc.mlp_loss_exact(Pm, X, y)) / (2 * h)
        assert abs(fd - G[k]) <= 1e-6 * max(1.0, abs(G[k])) + 1e-9, k


def test_single_unit_network_is_logistic_regression(orc):
    rng = np.random.default_rng(3)
    n = 50
    X = np.abs(rng.standard_normal((n, 12)))
    y = (rng.random(n) < 0.5).astype(np.float64)
    w = np.abs(rng.standard_normal(12)) * 0.2
    P = np.zeros(orc.mlp_nparams())
    P[0:768].reshape(12, 64)[:, 0] = w         # W1[:, 0] = w (inputs >= 0: the ReLU passes z)
    P[832 + 0 * 64 + 0] = 1.0                   # W2[0][0] = 1
    P[4992 + 0] = 1.0                           # W3[0] = 1 (W3 starts after b2 at 4928)
    G, loss = orc.mlp_grad_exact(P, X, y)
    z = X @ w
    p = 1 / (1 + np.exp(-z))
    ref_loss = np.mean(-(y * np.log(p) + (1 - y) * np.log(1 - p)))
    assert loss == pytest.approx(ref_loss, rel=1e-12)
    gw = X.T @ (p - y) / n
    assert np.allclose(G[0:768].reshape(12, 64)[:, 0], gw, rtol=1e-10, atol=1e-14)
    assert G[5056] == pytest.approx(np.mean(p - y), rel=1e-10)


def test_bf16_variant_close_to_exact(orc):
    rng = np.random.default_rng(4)
    n = 256
    X = rng.standard_normal((n, 12)).astype(np.float32)
    y = (rng.random(n) < 0.3).astype(np.float32)
    P = rand_params(rng, orc)
    Gb, lb = orc.mlp_grad(P, X, y)
    Ge, le = orc.mlp_grad_exact(P.astype(np.float64), X.astype(np.float64), y.astype(np.float64))
    assert abs(lb - le) <= 2e-2 * abs(le)
    cos = Gb @ Ge / np.linalg.norm(Gb) / np.linalg.norm(Ge)
    assert cos >= 0.999
    p, lf = orc.mlp_forward(P, X, y)
    assert lf == pytest.approx(lb, rel=1e-12)
    assert np.all((p > 0) & (p < 1))
