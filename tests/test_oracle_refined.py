"""Pins of the oracle's wall-refined cavity grid (the non-uniform DIG mesh
of Sec. 4.1: cell widths growing geometrically from every wall).

* the mesh: edges sum to the box, the first cell has the requested width,
  widths grow by the stretch factor, volumes are the products of widths;
  cells found by brute force from random points;
* initial counts Iround(rho V_cell / F) and a gas at rest between diffuse
  walls at its own temperature staying uniform in cells of every size
  (a wrong volume or cell lookup piles particles up in some cells);
* gradients exact for linear fields and, inside, for quadratics;
  NSF-consistent linear fields have zero HoT;
* the particle modification: target moments exactly, new particles in
  their cell.
"""
import math

import numpy as np

import oracle
from oracle.fields import box_edges, fields_from_sums, grad_refined, hot_kngll, kappa_coefficients, mu_ref_of
from stats3se import assert_within_3se
from paper_2501_10965_gb300 import workloads as W


def _cfg(**kw):
    base = dict(nx=14, ny=12, ppc=40, kn=0.05, dx_min=0.02, precision="fp64")
    base.update(kw)
    return W.cavity_2d_refined(**base)


def test_refined_edges_volumes_and_cells():
    cfg = W.cavity_2d_refined(precision="fp64")
    e = box_edges(100, 1.0, cfg["stretch"])
    w = np.diff(e)
    assert math.isclose(e[-1], 1.0) and math.isclose(w[0], 0.001, rel_tol=1e-9) and math.isclose(w[-1], 0.001, rel_tol=1e-9)
    assert np.allclose(w[1:50] / w[:49], cfg["stretch"], rtol=1e-12) and np.allclose(w, w[::-1], rtol=1e-12)
    c = _cfg()
    o = oracle.OracleSim(c)
    xe, ye = box_edges(14, 1.0, c["stretch"]), box_edges(12, 1.0, c["stretch"])
    v = o.volumes()
    assert np.allclose(v, np.outer(np.diff(ye), np.diff(xe)).ravel(), rtol=1e-13)
    assert math.isclose(v.sum(), 1.0, rel_tol=1e-13)
    rng = np.random.default_rng(1)
    n = 4000
    x, y = rng.random(n), rng.random(n)
    far = (np.min(np.abs(x[:, None] - xe[None, :]), 1) > 1e-9) & (np.min(np.abs(y[:, None] - ye[None, :]), 1) > 1e-9)
    x, y = x[far], y[far]
    o.set_particles({"x": x, "y": y, "vx": np.zeros(len(x)), "vy": np.zeros(len(x)), "vz": np.zeros(len(x)),
                     "ir": np.ones(len(x))})
    p = o.particles()
    cell = (np.searchsorted(ye, y, side="right") - 1) * 14 + np.searchsorted(xe, x, side="right") - 1
    order = np.lexsort((np.arange(len(x)), cell))
    assert np.array_equal(p["cell"], cell[order])


def test_refined_initial_counts_and_gas_at_rest_stays_uniform():
    """Diffuse walls at the gas temperature, no lid: the gas stays uniform.
    Cells are grouped by area (four classes from the small corner cells to
    the large middle ones); every class's density is 1 within the 3-SE
    bound of 6 independent seeds."""
    dens = []
    for seed in range(6):
        c = _cfg(lid=0.0, seed=seed)
        o = oracle.OracleSim(c)
        v, f = o.volumes(), o.constants()["fnum"]
        if seed == 0:
            cnt = np.bincount(o.particles()["cell"], minlength=14 * 12)
            xm = v / f
            assert np.all((cnt == np.floor(xm)) | (cnt == np.floor(xm) + 1))
        o.step(100)
        o.reset_accumulators()
        o.step(300, sample=True)
        rho = fields_from_sums(o.accumulators(), o.nsamples, f, v, 2.0)[:, 0]
        cls = np.digitize(v, np.quantile(v, [0.25, 0.5, 0.75]))
        dens.append([np.sum((rho * v)[cls == k]) / np.sum(v[cls == k]) for k in range(4)])
    assert_within_3se(np.array(dens) - 1.0, what="class density - 1")


def test_refined_gradient_and_hot_of_linear_fields():
    c = dict(_cfg(), kn_ref=0.0)
    xe, ye = box_edges(14, 1.0, c["stretch"]), box_edges(12, 1.0, c["stretch"])
    xc, yc = 0.5 * (xe[:-1] + xe[1:]), 0.5 * (ye[:-1] + ye[1:])
    X, Y = np.meshgrid(xc, yc)
    x, y = X.ravel(), Y.ravel()
    gx, gy = grad_refined(0.3 + 1.7 * x - 0.6 * y, 14, 12, xe, ye)
    assert np.allclose(gx, 1.7, atol=1e-12) and np.allclose(gy, -0.6, atol=1e-12)
    gx, gy = grad_refined(x * x - 2 * y * y, 14, 12, xe, ye)
    inner = ((X > xc[0]) & (X < xc[-1]) & (Y > yc[0]) & (Y < yc[-1])).ravel()
    assert np.allclose(gx[inner], 2 * x[inner], atol=1e-11) and np.allclose(gy[inner], -4 * y[inner], atol=1e-11)
    n = len(x)
    a = np.array([[0.05, -0.02], [0.03, 0.04]])
    F = np.zeros((n, 18))
    F[:, 0] = 1.0 + 0.1 * x - 0.05 * y
    F[:, 1] = 0.1 + a[0, 0] * x + a[0, 1] * y
    F[:, 2] = -0.2 + a[1, 0] * x + a[1, 1] * y
    F[:, 4] = 1.0 + 0.03 * x + 0.02 * y
    F[:, 5] = 0.9 - 0.01 * x + 0.03 * y
    T = (3 * F[:, 4] + 2 * F[:, 5]) / 5
    mu = mu_ref_of(c["kn"]) * T ** c["omega"]
    div = a[0, 0] + a[1, 1]
    F[:, 6] = -mu * (2 * a[0, 0] - 2 / 3 * div)
    F[:, 7] = -mu * (2 * a[1, 1] - 2 / 3 * div)
    F[:, 8] = -mu * (-2 / 3 * div)
    F[:, 9] = -mu * (a[0, 1] + a[1, 0])
    kt, kr = kappa_coefficients(c["a_matrix"], 2.0)
    F[:, 12], F[:, 13] = -kt * mu * 0.03, -kt * mu * 0.02
    F[:, 15], F[:, 16] = -kr * mu * (-0.01), -kr * mu * 0.03
    hot, kn, mask = hot_kngll(F, c)
    assert mask.all() and np.max(np.abs(hot)) < 1e-12


def test_refined_dig_correct_matches_targets():
    c = _cfg()
    o = oracle.OracleSim(c)
    o.step(3)
    nc = 14 * 12
    rng = np.random.default_rng(2)
    t = np.zeros((nc, 6))
    t[:, 0] = 0.6 + 0.8 * rng.random(nc)
    t[:, 1:4] = 0.2 * rng.standard_normal((nc, 3))
    t[:, 4] = 0.8 + 0.4 * rng.random(nc)
    t[:, 5] = 0.8 + 0.4 * rng.random(nc)
    assert o.dig_correct(t) == 0
    p = o.particles()
    v, f = o.volumes(), o.constants()["fnum"]
    cnt = np.bincount(p["cell"], minlength=nc)
    xm = t[:, 0] * v / f
    assert np.all((cnt == np.floor(xm)) | (cnt == np.floor(xm) + 1))
    full = cnt >= 2
    for j, k in enumerate(("vx", "vy", "vz")):
        assert np.allclose(np.bincount(p["cell"], p[k], nc)[full] / cnt[full], t[full, 1 + j], atol=1e-13)
    xe, ye = box_edges(14, 1.0, c["stretch"]), box_edges(12, 1.0, c["stretch"])
    ix, iy = p["cell"] % 14, p["cell"] // 14
    assert np.all((p["x"] >= xe[ix] - 1e-15) & (p["x"] <= xe[ix + 1] + 1e-15))
    assert np.all((p["y"] >= ye[iy] - 1e-15) & (p["y"] <= ye[iy + 1] + 1e-15))
