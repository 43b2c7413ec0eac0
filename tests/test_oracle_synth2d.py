"""Pins of the 2D synthetic-equation oracle (oracle/synth2d.py).

* Manufactured solutions: for smooth analytic fields (and HoT), the discrete
  residual at every balanced cell converges at second order to the exact
  divergence of the fluxes of Eq. (macroscopic_equation) with
  Eq. (full_constitutive), derived here symbolically from the equations
  (a dropped term, a wrong sign or a swapped index fails it).
* Reduction to 1D: a field that varies along one axis only and solves the 1D
  synthetic equations (pinned against the NSF closed form in
  test_oracle_dig.py) solves the 2D equations up to the fourth-difference
  dissipation, whose effect vanishes with dx; along y exactly as along x.
* The Newton solution: residual at rounding level, total mass, Dirichlet
  cells and corner cells unchanged.
"""
import math

import numpy as np
import pytest

from oracle import synth1d, synth2d
from oracle.fields import F_RHO, F_TR, F_TT, F_U, box_edges, kappa_coefficients, mu_ref_of
from paper_2501_10965_gb300 import workloads as W

sympy = pytest.importorskip("sympy")


def _mms_sources(cfg):
    """Exact sources S_k(x, y) = div F_k (minus the rotational source) for the
    analytic fields below, as numpy functions."""
    x, y = sympy.symbols("x y", real=True)
    d_r, omega, Z = float(cfg["d_r"]), float(cfg["omega"]), float(cfg["z_rot"])
    mu_ref = mu_ref_of(float(cfg["kn"]))
    kt_c, kr_c = kappa_coefficients(cfg["a_matrix"], d_r)
    rho = 1 + sympy.Rational(1, 5) * sympy.sin(x) * sympy.cos(y)
    ux = sympy.Rational(1, 5) * sympy.sin(2 * x) * sympy.cos(y)
    uy = sympy.Rational(3, 20) * sympy.cos(x) * sympy.sin(sympy.Rational(3, 2) * y)
    tt = 1 + sympy.Rational(1, 5) * x * y + sympy.Rational(1, 10) * sympy.sin(y)
    tr = sympy.Rational(11, 10) + sympy.Rational(1, 10) * sympy.cos(x + y)
    h = {
        "sxx": sympy.Rational(1, 100) * sympy.cos(x), "syy": sympy.Rational(1, 100) * sympy.sin(y),
        "sxy": sympy.Rational(1, 50) * x * y, "qtx": sympy.Rational(1, 100) * sympy.sin(x + y),
        "qty": sympy.Rational(1, 100) * sympy.cos(x * y), "qrx": sympy.Rational(1, 200) * x,
        "qry": sympy.Rational(1, 200) * y ** 2,
    }
    T = (3 * tt + d_r * tr) / (3 + d_r)
    mu = mu_ref * T ** omega
    div_u = sympy.diff(ux, x) + sympy.diff(uy, y)
    sxx = -mu * (2 * sympy.diff(ux, x) - sympy.Rational(2, 3) * div_u) + h["sxx"]
    syy = -mu * (2 * sympy.diff(uy, y) - sympy.Rational(2, 3) * div_u) + h["syy"]
    sxy = -mu * (sympy.diff(uy, x) + sympy.diff(ux, y)) + h["sxy"]
    qtx = -kt_c * mu * sympy.diff(tt, x) + h["qtx"]
    qty = -kt_c * mu * sympy.diff(tt, y) + h["qty"]
    qrx = -kr_c * mu * sympy.diff(tr, x) + h["qrx"]
    qry = -kr_c * mu * sympy.diff(tr, y) + h["qry"]
    e = (3 * tt + d_r * tr) / 2 + (ux ** 2 + uy ** 2) / 2
    er = d_r * tr / 2
    p_t = rho * tt
    S = [
        sympy.diff(rho * ux, x) + sympy.diff(rho * uy, y),
        sympy.diff(rho * ux * ux + p_t + sxx, x) + sympy.diff(rho * ux * uy + sxy, y),
        sympy.diff(rho * ux * uy + sxy, x) + sympy.diff(rho * uy * uy + p_t + syy, y),
        sympy.diff(rho * e * ux + p_t * ux + sxx * ux + sxy * uy + qtx + qrx, x)
        + sympy.diff(rho * e * uy + p_t * uy + sxy * ux + syy * uy + qty + qry, y),
        sympy.diff(rho * er * ux + qrx, x) + sympy.diff(rho * er * uy + qry, y)
        - (d_r * rho / 2) * (T - tr) / (Z * mu / (rho * T)),
    ]
    f = lambda e_: sympy.lambdify((x, y), e_, "numpy")
    fields = [f(rho), f(ux), f(uy), f(tt), f(tr)]
    hot = {k: f(v) for k, v in h.items()}
    return fields, hot, [f(s) for s in S]


def _centres(cfg):
    nx, ny = int(cfg["nx"]), int(cfg["ny"])
    if cfg.get("mesh", "box") == "refined":
        ex, ey = box_edges(nx, cfg["lx"], cfg["stretch"]), box_edges(ny, cfg["ly"], cfg["stretch"])
        return np.meshgrid(0.5 * (ex[:-1] + ex[1:]), 0.5 * (ey[:-1] + ey[1:]))
    dx, dy = cfg["lx"] / nx, cfg["ly"] / ny
    return np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dy)


def _discrete_error(cfg, fields, hot, S, mask=None):
    nx, ny = int(cfg["nx"]), int(cfg["ny"])
    X, Y = _centres(cfg)
    q = [np.broadcast_to(fn(X, Y), X.shape).astype(float) for fn in fields]
    x = np.concatenate([a.ravel() for a in q])
    H = np.zeros((ny, nx, 12))
    for col, key in ((0, "sxx"), (1, "syy"), (3, "sxy"), (6, "qtx"), (7, "qty"), (9, "qrx"), (10, "qry")):
        H[..., col] = np.broadcast_to(hot[key](X, Y), X.shape)
    dsmc = np.zeros((nx * ny, 18))
    R = synth2d.residual(x, dsmc, H.reshape(-1, 12), cfg).reshape(5, ny, nx)
    errs = []
    for k in range(5):
        ex = np.broadcast_to(S[k](X, Y), X.shape)
        e = np.abs(R[k, 1:-1, 1:-1] - ex[1:-1, 1:-1])
        errs.append(np.max(e if mask is None else e[mask]))
    return np.array(errs)


def test_manufactured_solution_second_order():
    base = W.cavity_2d(nx=12, ny=10, ppc=10, kn=0.1, lx=1.2, ly=1.0)
    fields, hot, S = _mms_sources(base)
    e1 = _discrete_error(W.with_overrides(base, nx=12, ny=10), fields, hot, S)
    e2 = _discrete_error(W.with_overrides(base, nx=24, ny=20), fields, hot, S)
    e3 = _discrete_error(W.with_overrides(base, nx=48, ny=40), fields, hot, S)
    order12 = np.log2(e1 / e2)
    order23 = np.log2(e2 / e3)
    assert (order23 > 1.8).all(), (e1, e2, e3, order12, order23)
    # and small in absolute terms on the finest grid
    assert (e3 < 2e-3).all(), e3


def test_manufactured_solution_on_the_wall_refined_grid():
    """The same sources on the wall-refined grid (widths growing by q from
    each wall, the cavity case of Sec. 4.1), refined as a mapping: q^(12/nx),
    so that neighbouring widths tend to equal as the grid is refined.  Where
    the mapping is smooth the residual converges at second order, which a
    difference over the wrong distance (a uniform dx, a cell width instead of
    the centre distance) or a balance divided by the wrong width fails.  At
    the middle lines, where the widths stop growing and shrink again (a kink
    in the mapping), the error of the two-point face differences is first
    order: the whole grid converges at first order."""
    q0 = 1.25
    base = W.cavity_2d(nx=12, ny=10, ppc=10, kn=0.1, lx=1.2, ly=1.0)
    fields, hot, S = _mms_sources(base)
    e_all, e_far = [], []
    for nx, ny in ((12, 10), (24, 20), (48, 40)):
        cfg = W.with_overrides(base, nx=nx, ny=ny, mesh="refined", stretch=q0 ** (12.0 / nx))
        w = np.diff(box_edges(nx, 1.2, cfg["stretch"]))
        assert w.max() / w.min() > 2.5  # far from uniform on every grid
        X, Y = _centres(cfg)
        far = ((np.abs(X - 0.6) > 0.1) & (np.abs(Y - 0.5) > 0.1))[1:-1, 1:-1]
        e_all.append(_discrete_error(cfg, fields, hot, S))
        e_far.append(_discrete_error(cfg, fields, hot, S, mask=far))
    far12, far23 = np.log2(e_far[0] / e_far[1]), np.log2(e_far[1] / e_far[2])
    all23 = np.log2(e_all[1] / e_all[2])
    assert (far23 > 1.8).all(), (e_far, far12, far23)
    assert (all23 > 0.9).all(), (e_all, all23)
    assert (e_far[2] < 5e-3).all(), e_far[2]


def test_refined_grid_with_unit_stretch_is_the_uniform_grid():
    cfg = W.cavity_2d(nx=9, ny=7, ppc=10, kn=0.05, lx=1.0, ly=0.8)
    rng = np.random.default_rng(4)
    n = 63
    x = np.concatenate([1 + 0.1 * rng.random(n), 0.1 * rng.standard_normal(2 * n), 1 + 0.1 * rng.random(2 * n)])
    d = np.zeros((n, 18))
    d[:, F_RHO] = 1.0
    d[:, F_TT] = d[:, F_TR] = 1.0
    h = 1e-3 * rng.standard_normal((n, 12))
    R0 = synth2d.residual(x, d, h, cfg)
    R1 = synth2d.residual(x, d, h, W.with_overrides(cfg, mesh="refined", stretch=1.0))
    assert np.allclose(R1, R0, rtol=1e-12, atol=1e-12 * np.abs(R0).max())


def test_newton_solution_on_the_wall_refined_grid():
    """Newton's method on the refined cavity grid: rounding-level residual,
    the sampled total mass sum rho V (cells of different areas), Dirichlet
    and corner cells kept."""
    cfg = W.cavity_2d_refined(nx=12, ny=10, ppc=10, kn=0.05, dx_min=0.03, precision="fp64")
    nx, ny = 12, 10
    n = nx * ny
    X, Y = _centres(cfg)
    d = np.zeros((ny, nx, 18))
    d[..., F_RHO] = 1 + 0.02 * np.cos(np.pi * X)
    d[..., F_U] = 0.05 * np.sin(np.pi * X) * np.cos(np.pi * Y) * np.sin(np.pi * Y)
    d[..., F_U + 1] = -0.05 * np.cos(np.pi * X) * np.sin(np.pi * X) * np.sin(np.pi * Y)
    d[..., F_TT] = 1 + 0.01 * Y
    d[..., F_TR] = 1 + 0.012 * Y
    d = d.reshape(n, 18)
    h = 1e-3 * np.random.default_rng(0).standard_normal((n, 12))
    out, it, res = synth2d.synth_solve_2d(d, h, cfg)
    assert res < 1e-11 and it < 10
    V = np.outer(np.diff(box_edges(ny, 1.0, cfg["stretch"])), np.diff(box_edges(nx, 1.0, cfg["stretch"]))).ravel()
    assert V.max() / V.min() > 4.0
    assert math.isclose((out[:, 0] * V).sum(), (d[:, F_RHO] * V).sum(), rel_tol=1e-13)
    assert not math.isclose(out[:, 0].sum(), d[:, F_RHO].sum(), rel_tol=1e-6)
    ring = np.zeros((ny, nx), bool)
    ring[0, :] = ring[-1, :] = ring[:, 0] = ring[:, -1] = True
    ring = ring.ravel()
    for k, col in ((1, F_U), (2, F_U + 1), (4, F_TT), (5, F_TR)):
        np.testing.assert_allclose(out[ring, k], d[ring, col], rtol=0, atol=1e-13)
    corners = [0, nx - 1, n - nx, n - 1]
    np.testing.assert_allclose(out[corners, 0], d[corners, F_RHO], rtol=0, atol=1e-13)
    assert (out[:, 0] > 0.9).all() and (out[:, 0] < 1.1).all()


def _solve_1d(cfg1):
    n = int(cfg1["nx"])
    t_hot = 1.3663
    xc = (np.arange(n) + 0.5) / n
    d = np.zeros((n, 18))
    d[:, F_RHO] = 1.0
    d[:, F_TT] = 1.0 + (t_hot - 1.0) * xc
    d[:, F_TR] = 1.0 + (t_hot - 1.0) * xc + 0.01
    out, _, res = synth1d.synth_solve_1d(d, np.zeros((n, 12)), cfg1)
    assert res < 1e-10
    return out


def _reduce_1d_diff(axis, n, m):
    cfg1 = W.fourier_1d(nx=n, kn=0.05)
    out1 = _solve_1d(cfg1)
    if axis == "x":
        cfg2 = W.cavity_2d(nx=n, ny=m, ppc=10, kn=0.05, lx=1.0, ly=0.4)
        f2 = np.tile(out1[None, :, :], (m, 1, 1))                       # [ny, nx, 6]
    else:
        cfg2 = W.cavity_2d(nx=m, ny=n, ppc=10, kn=0.05, lx=0.4, ly=1.0)
        f2 = np.tile(out1[:, None, :], (1, m, 1))                       # [ny, nx, 6]
    d = np.zeros((n * m, 18))
    d[:, F_RHO] = f2[..., 0].ravel()
    d[:, F_TT] = f2[..., 4].ravel()
    d[:, F_TR] = f2[..., 5].ravel()
    out2, it, res = synth2d.synth_solve_2d(d, np.zeros((n * m, 12)), cfg2)
    assert res < 1e-10
    diff = max(np.max(np.abs(out2[:, k] / d[:, col] - 1.0)) for k, col in ((0, F_RHO), (4, F_TT), (5, F_TR)))
    return diff, np.max(np.abs(out2[:, 1:3]))


def test_reduces_to_1d_fourier():
    """The 1D Fourier solution (u = 0), tiled along the other axis, solves the
    2D equations up to the fourth-difference dissipation, whose effect
    vanishes as the grid is refined (about 3x per halving of dx); the
    problem along y is the transpose of the one along x, to rounding."""
    dx16, ux16 = _reduce_1d_diff("x", 16, 6)
    dx32, ux32 = _reduce_1d_diff("x", 32, 6)
    dy16, uy16 = _reduce_1d_diff("y", 16, 6)
    assert dx16 < 5e-4 and ux16 < 1e-4, (dx16, ux16)
    assert dx32 < dx16 / 2.5 and ux32 < ux16 / 2.5, (dx16, dx32, ux16, ux32)
    assert abs(dy16 - dx16) < 1e-12 and abs(uy16 - ux16) < 1e-12, (dx16, dy16, ux16, uy16)


def test_newton_solution_properties():
    cfg = W.cavity_2d(nx=10, ny=8, ppc=10, kn=0.05)
    nx, ny = 10, 8
    n = nx * ny
    X, Y = np.meshgrid((np.arange(nx) + 0.5) / nx, (np.arange(ny) + 0.5) / ny)
    d = np.zeros((ny, nx, 18))
    d[..., F_RHO] = 1 + 0.02 * np.cos(np.pi * X)
    d[..., F_U] = 0.05 * np.sin(np.pi * X) * np.cos(np.pi * Y) * np.sin(np.pi * Y)
    d[..., F_U + 1] = -0.05 * np.cos(np.pi * X) * np.sin(np.pi * X) * np.sin(np.pi * Y)
    d[..., F_U + 2] = 0.003
    d[..., F_TT] = 1 + 0.01 * Y
    d[..., F_TR] = 1 + 0.012 * Y
    d = d.reshape(n, 18)
    h = 1e-3 * np.random.default_rng(0).standard_normal((n, 12))
    out, it, res = synth2d.synth_solve_2d(d, h, cfg)
    assert res < 1e-11 and it < 10
    assert math.isclose(out[:, 0].sum(), d[:, F_RHO].sum(), rel_tol=1e-13)
    ring = np.zeros((ny, nx), bool)
    ring[0, :] = ring[-1, :] = ring[:, 0] = ring[:, -1] = True
    ring = ring.ravel()
    for k, col in ((1, F_U), (2, F_U + 1), (4, F_TT), (5, F_TR)):
        np.testing.assert_allclose(out[ring, k], d[ring, col], rtol=0, atol=1e-13)
    corners = [0, nx - 1, n - nx, n - 1]
    np.testing.assert_allclose(out[corners, 0], d[corners, F_RHO], rtol=0, atol=1e-13)
    np.testing.assert_array_equal(out[:, 3], d[:, F_U + 2])
    assert (out[:, 0] > 0.9).all() and (out[:, 0] < 1.1).all()
