"""Pins of the HoT surrogate oracle (oracle/mlp.py).

* Backpropagation: the gradient equals central finite differences of the
  loss in FP64, with and without bfloat16 weights.
* bfloat16 rounding: exact on representable values, nearest-even on ties,
  relative error below 2^-8.
* Features and outputs: a field with a single known gradient gives the
  expected scaled gradient in the right slot and zeros elsewhere; the 5
  normalised outputs map back to the HoT components they came from.
* Adam: the first step moves every parameter by lr against the sign of its
  gradient (bias-corrected moments); a convex quadratic is driven to its
  minimum.
"""
import math

import numpy as np
import pytest

from oracle import mlp
from oracle.fields import F_RHO, F_TR, F_TT, F_U, mu_ref_of
from paper_2501_10965_gb300 import workloads as W


@pytest.mark.parametrize("bf16", [False, True])
def test_backprop_matches_finite_differences(bf16):
    rng = np.random.default_rng(0)
    theta = mlp.init_params(1) + 0.01 * rng.standard_normal(mlp.NPARAM)
    X = rng.standard_normal((17, 12))
    Y = 0.3 * rng.standard_normal((17, 5))
    loss, g = mlp.loss_and_grad(theta, X, Y, bf16=False)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    for i in idx:
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, X, Y)[0] - mlp.loss_and_grad(tm, X, Y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])
    if bf16:
        # with rounded weights the backward pass is that of the rounded
        # network: compare against finite differences of the rounded loss in
        # the biases (which are not rounded)
        lb, gb = mlp.loss_and_grad(theta, X, Y, bf16=True)
        layers = mlp.unpack(np.arange(mlp.NPARAM, dtype=float))
        bias_idx = np.concatenate([b.astype(int) for _, b in layers])
        for i in rng.choice(bias_idx, 20, replace=False):
            tp, tm = theta.copy(), theta.copy()
            tp[i] += 1e-6
            tm[i] -= 1e-6
            fd = (mlp.loss_and_grad(tp, X, Y, bf16=True)[0] - mlp.loss_and_grad(tm, X, Y, bf16=True)[0]) / 2e-6
            assert abs(fd - gb[i]) <= 1e-7 * max(1.0, abs(gb[i])) + 1e-9


def test_bf16_rounding():
    exact = np.array([1.0, -2.5, 0.15625, 3.0e38], np.float32)
    assert np.array_equal(mlp.bf16_round(exact)[:3], exact[:3].astype(np.float64))
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert mlp.bf16_round(np.array([1.0 + 2.0 ** -8], np.float32))[0] == 1.0
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: ties to even -> 1 + 2^-6
    assert mlp.bf16_round(np.array([1.0 + 3 * 2.0 ** -8], np.float32))[0] == 1.0 + 2.0 ** -6
    x = np.random.default_rng(2).standard_normal(10000).astype(np.float32)
    r = mlp.bf16_round(x)
    assert np.max(np.abs(r - x) / np.abs(x)) <= 2.0 ** -8


def test_features_of_a_single_gradient():
    cfg = W.couette_1d(kn=0.1, nx=20, ppc=10)
    n = 20
    xc = (np.arange(n) + 0.5) / n
    f = np.zeros((n, 18))
    f[:, F_RHO] = 1.0
    f[:, F_TT] = 1.0
    f[:, F_TR] = 1.0
    f[:, F_U + 1] = 0.2 * xc  # du_y/dx = 0.2
    X, scale = mlp.features(f, np.full(n, 0.05), cfg)
    lam = mu_ref_of(0.1) * math.sqrt(math.pi / 2.0)
    np.testing.assert_allclose(X[:, 4], lam * 0.2, rtol=1e-12)
    others = [0, 1, 2, 3, 5, 6, 7, 8, 9]
    assert np.all(X[:, others] == 0.0)
    np.testing.assert_allclose(X[:, 10], 0.05)
    np.testing.assert_allclose(X[:, 11], 1.0)
    np.testing.assert_allclose(scale[:, 0], 1.0)
    np.testing.assert_allclose(scale[:, 2:], [[1.0, 0.0]] * n)   # grad T = 0 -> e = x


def test_outputs_round_trip():
    rng = np.random.default_rng(3)
    n = 30
    hot = rng.standard_normal((n, 12))
    scale = np.stack([1 + rng.random(n), 1 + rng.random(n), np.zeros(n), np.zeros(n)], axis=1)
    ang = rng.random(n) * 2 * math.pi
    scale[:, 2], scale[:, 3] = np.cos(ang), np.sin(ang)
    Y = mlp.targets(hot, scale)
    np.testing.assert_allclose(mlp.to_hot(Y, scale, hot), hot, rtol=1e-12, atol=1e-12)
    # changing the along-e output only moves q along e
    Y2 = Y.copy()
    Y2[:, 3] += 1.0
    h2 = mlp.to_hot(Y2, scale, hot)
    dq = h2[:, 6:8] - hot[:, 6:8]
    np.testing.assert_allclose(dq, scale[:, 1:2] * scale[:, 2:4], rtol=1e-12, atol=1e-12)


def test_adam():
    opt = mlp.Adam(3, lr=0.01)
    th = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    th1 = opt.step(th, g)
    np.testing.assert_allclose(th1, th - 0.01 * np.sign(g), rtol=0, atol=1e-6)
    opt = mlp.Adam(2, lr=0.05)
    th = np.array([3.0, -1.0])
    for _ in range(2000):
        th = opt.step(th, 2 * (th - np.array([0.5, 0.25])))
    np.testing.assert_allclose(th, [0.5, 0.25], atol=1e-3)
