"""2D higher-order terms, Kn_GLL and the network's inputs on the GPU against
the oracle, from oracle-computed fields fed to both sides.

On a 2D box the HoT kernel uses y-gradients, sigma_xy = -mu (du_x/dy +
du_y/dx), the 2D divergence in the normal stresses, the y components of the
NSF heat fluxes and the 2D gradient magnitudes of Kn_GLL (Eqs.
(ns_constitutive), (hot_constitutive), (Kn_GLL); Sec. 3.1).  The fields come
from the FP64 oracle's own DSMC run of a lid-driven cavity, and from a
smooth analytic field whose every gradient is non-zero; HoT must agree to
relative 1e-11, Kn_GLL to 1e-12 and the mask exactly.  The network's
2D inputs (y-gradients of rho, u_x, u_y, T_t, T_r) are checked through its
output and its loss gradient against the oracle network.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import mlp
from oracle.fields import fields_from_sums, hot_kngll
from paper_2501_10965_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _gpu(cfg):
    from paper_2501_10965_gb300 import dsmc
    return dsmc.Dsmc(cfg)


def _oracle_cavity_fields(kn, nx=14, ny=11, ppc=40, seed=0):
    cfg = W.cavity_2d(nx=nx, ny=ny, ppc=ppc, kn=kn, precision="fp64", seed=seed)
    o = oracle.OracleSim(cfg)
    o.step(60)
    o.step(120, sample=True)
    c = o.constants()
    return cfg, fields_from_sums(o.accumulators(), o.nsamples, c["fnum"], c["vcell"], 2.0)


def _analytic_fields(nx, ny):
    """Smooth fields with non-zero x and y gradients of every quantity."""
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    X, Y = X.ravel(), Y.ravel()
    f = np.zeros((nx * ny, 18))
    f[:, 0] = 1.0 + 0.2 * X - 0.15 * Y + 0.1 * X * Y
    f[:, 1] = 0.3 * Y * Y - 0.1 * X
    f[:, 2] = -0.2 * X * Y + 0.05 * Y
    f[:, 3] = 0.02 * X - 0.03 * Y
    f[:, 4] = 1.0 + 0.3 * X * X + 0.1 * Y
    f[:, 5] = 0.95 + 0.25 * X - 0.2 * Y * Y
    f[:, 6:12] = 0.01 * np.sin(np.outer(X + 2 * Y, np.arange(1, 7)))
    f[:, 12:18] = 0.02 * np.cos(np.outer(3 * X - Y, np.arange(1, 7)))
    return f


def _compare_hot(cfg, F):
    # a threshold in the middle of the Kn_GLL distribution, so that the mask
    # holds both values
    _, kn_o, _ = hot_kngll(F, dict(cfg, kn_ref=0.0))
    cfg = dict(cfg, kn_ref=float(np.median(kn_o)) * 1.0000001)
    hot_o, kn_o, mask_o = hot_kngll(F, cfg)
    g = _gpu(cfg)
    hot_g, kn_g, mask_g = [t.cpu().numpy() for t in g.dsmc_hot(torch.tensor(F, device="cuda"))]
    assert 0 < mask_o.sum() < len(mask_o)
    assert np.allclose(kn_g, kn_o, rtol=1e-12, atol=0.0), np.max(np.abs(kn_g / kn_o - 1))
    assert np.array_equal(mask_g.astype(bool), mask_o)
    scale = np.maximum(np.abs(hot_o).max(0), 1e-300)
    err = np.abs(hot_g - hot_o) / scale
    assert err.max() <= 1e-11, (err.max(0), scale)
    # the y-dependent parts are present: sigma_xy and the y heat fluxes
    assert np.abs(hot_o[mask_o][:, [3, 7, 10]]).max() > 0


@pytest.mark.parametrize("kn", [0.05, 0.1])
def test_hot_kngll_2d_cavity_matches_oracle(kn):
    cfg, F = _oracle_cavity_fields(kn)
    _compare_hot(cfg, F)


def test_hot_kngll_2d_analytic_fields_match_oracle():
    cfg = W.cavity_2d(nx=13, ny=9, ppc=4, kn=0.05, precision="fp64")
    _compare_hot(cfg, _analytic_fields(13, 9))


def test_mlp_2d_inputs_output_and_gradient_match_oracle():
    """The network on 2D cavity fields: its output on the network cells and
    its loss gradient follow the oracle network on the oracle's 12 inputs
    (which include the y-gradients), with the same bfloat16 weights."""
    cfg, F = _oracle_cavity_fields(0.1, nx=16, ny=12, ppc=60, seed=1)
    _, kn_o, _ = hot_kngll(F, dict(cfg, kn_ref=0.0))
    cfg = dict(cfg, kn_ref=float(np.quantile(kn_o, 0.3)) * 1.0000001)
    H, K, m = hot_kngll(F, cfg)
    X, S = mlp.features(F, K, cfg)
    assert np.abs(X[m][:, [1, 3, 5, 7, 9]]).max() > 1e-3  # y-gradient inputs in play
    g = _gpu(cfg)
    f_t = torch.tensor(F, device="cuda")
    hot_t, kn_t, mask_t = g.dsmc_hot(f_t)
    assert np.array_equal(mask_t.cpu().numpy().astype(bool), m)
    theta = mlp.init_params(5).astype(np.float32)
    g.mlp_set_params(theta)
    out, judge = g.mlp_apply(f_t, hot_t, kn_t, mask_t)
    out = out.cpu().numpy()
    # tensor-core inference: bfloat16 layer inputs (see test_gpu_mlp for the bounds)
    Yo, _ = mlp.forward(theta.astype(np.float64), X, bf16=True, bf16_act=True)
    ho = mlp.to_hot(Yo, S, H)
    sc = np.max(np.abs(ho[m][:, [0, 1, 3, 6, 7, 9, 10]]))
    err = np.abs(out[m] - ho[m])
    assert np.sqrt(np.mean(err ** 2)) <= 1e-4 * sc and err.max() <= 4e-3 * sc, (np.sqrt(np.mean(err ** 2)), err.max())
    assert np.array_equal(out[~m], H[~m])
    Y = mlp.targets(H, S)
    loss_g, grad_g = g.mlp_grad(f_t, hot_t, kn_t, mask_t)
    loss_o, grad_o = mlp.loss_and_grad(theta.astype(np.float64), X[m], Y[m], bf16=True)
    assert abs(loss_g - loss_o) <= 1e-4 * loss_o, (loss_g, loss_o)
    # first layer: the weights of the y-gradient inputs get their own gradient
    (gw, gb), (ow, ob) = mlp.unpack(grad_g.astype(np.float64))[0], mlp.unpack(grad_o)[0]
    assert np.max(np.abs(gw - ow)) <= 1e-3 * np.max(np.abs(ow)), np.max(np.abs(gw - ow))
    assert np.max(np.abs(gb - ob)) <= 1e-3 * np.max(np.abs(ob))
