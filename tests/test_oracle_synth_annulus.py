"""Pins of the synthetic-equation oracle on the cylinder's annulus
(oracle/synth_annulus.py).

* A uniform state (any velocity, constant HoT) is an exact discrete solution
  in every balanced ring: the face vectors of a cell close (a wrong face
  area, normal or volume leaves a residual of order one).
* Manufactured solutions: for smooth analytic fields and HoT in x, y, the
  discrete residual of the balanced rings converges at second order to the
  exact flux divergence of Eq. (macroscopic_equation) with
  Eq. (full_constitutive), the sources derived symbolically (the same
  sources as the box's pin): a dropped or mis-rotated term, a wrong sign or
  a wrong distance fails it.
* Heat conduction between the cylinder and the outer boundary (u = 0):
  the NSF solution has T^(1 + omega) linear in ln r and a uniform pressure;
  the Newton solution converges to it at second order in the ring width.
* Newton: rounding-level residual; both boundary rings keep their whole
  sampled state.
"""
import math

import numpy as np
import pytest

from oracle import synth_annulus as SA
from oracle.fields import F_RHO, F_TR, F_TT, F_U
from paper_2501_10965_gb300 import workloads as W

sympy = pytest.importorskip("sympy")


def _cfg(nt, nr, **kw):
    base = dict(ntheta=nt, nr=nr, ppc=4, kn=0.1, mach=0.5, r_in=0.5, r_out=1.5, precision="fp64")
    base.update(kw)
    return W.cylinder_2d(**base)


def _centres(cfg):
    nt, nr, R, rc, dth, thc = SA.geometry(cfg)
    r, th = np.meshgrid(rc, thc, indexing="ij")
    return (r * np.cos(th)).ravel(), (r * np.sin(th)).ravel(), r.ravel()


def test_uniform_state_is_an_exact_solution():
    cfg = _cfg(20, 6, dr1=0.05)
    assert cfg["stretch"] > 1.2
    nt, nr = 20, 6
    n = nt * nr
    d = np.zeros((n, 18))
    d[:, F_RHO], d[:, F_U], d[:, F_U + 1], d[:, F_TT], d[:, F_TR] = 1.2, 0.3, -0.1, 1.1, 1.1
    h = np.tile(1e-2 * np.arange(1, 13), (n, 1))
    R = SA.residual(SA.initial_state(d), d, h, cfg).reshape(5, nr, nt)
    assert np.max(np.abs(R[:, 1:-1])) < 1e-13
    assert np.max(np.abs(R[:, 0])) == 0.0 and np.max(np.abs(R[:, -1])) == 0.0


def test_manufactured_solution_second_order():
    from test_oracle_synth2d import _mms_sources
    errs = []
    for nt, nr in ((24, 6), (48, 12), (96, 24)):
        cfg = _cfg(nt, nr)
        fields, hot, S = _mms_sources(cfg)
        x, y, r = _centres(cfg)
        q = [np.broadcast_to(fn(x, y), x.shape).astype(float) for fn in fields]
        X = np.concatenate(q)
        H = np.zeros((nt * nr, 12))
        for col, key in ((0, "sxx"), (1, "syy"), (3, "sxy"), (6, "qtx"), (7, "qty"), (9, "qrx"), (10, "qry")):
            H[:, col] = np.broadcast_to(hot[key](x, y), x.shape)
        Rv = SA.residual(X, np.zeros((nt * nr, 18)), H, cfg).reshape(5, nr, nt)
        e = []
        for k in range(5):
            ex = np.broadcast_to(S[k](x, y), x.shape).reshape(nr, nt)
            e.append(np.max(np.abs(Rv[k, 1:-1] - ex[1:-1])))
        errs.append(np.array(e))
    o12, o23 = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert (o23 > 1.8).all(), (errs, o12, o23)
    assert (errs[2] < 1e-2).all(), errs[2]


def _conduction(nr, t_in=1.6, t_out=1.0, rho_out=1.0):
    """Newton solution of pure conduction between the first ring (T_in) and
    the outer ring (T_out, rho_out), u = 0, no HoT; returns (cfg, centres'
    radii, discrete T_t, T_r, rho, the analytic T)."""
    cfg = _cfg(8, nr)
    nt = 8
    n = nt * nr
    x, y, r = _centres(cfg)
    w = 1.0 + float(cfg["omega"])
    rc = SA.geometry(cfg)[3]
    a = (t_in ** w - t_out ** w) / (math.log(rc[0]) - math.log(rc[-1]))
    b = t_in ** w - a * math.log(rc[0])
    T = (a * np.log(r) + b) ** (1.0 / w)
    d = np.zeros((n, 18))
    d[:, F_TT] = d[:, F_TR] = T
    d[:, F_RHO] = rho_out * t_out / T
    out, it, res = SA.synth_solve_annulus(d, np.zeros((n, 12)), cfg)
    assert res < 1e-11 and it < 10
    return cfg, r, out, T


def test_heat_conduction_to_the_cylinder_second_order():
    """The discrete solution approaches the NSF one as the rings narrow: T
    at second order; the flow and the pressure's departure from uniform that
    the fourth-difference dissipation of the varying density drives (a
    mass flux eps4 lambda d^3 rho balanced by a small radial velocity), and
    with it T_t - T_r, faster than second order; axial symmetry holds
    exactly."""
    eT, eu, ep, er = [], [], [], []
    for nr in (6, 12, 24):
        cfg, r, out, T = _conduction(nr)
        er.append(np.max(np.abs(out[:, 4] - out[:, 5])))
        rad = out[:, 0].reshape(nr, 8)
        assert np.allclose(rad, rad[:, :1], rtol=0, atol=1e-12)  # the same in every sector
        eT.append(np.max(np.abs(out[:, 4] - T)))
        eu.append(np.max(np.hypot(out[:, 1], out[:, 2])))
        ep.append(np.max(np.abs(out[:, 0] * out[:, 4] - 1.0)))
    oT = np.log2(np.array(eT[:-1]) / np.array(eT[1:]))
    ou = np.log2(np.array(eu[:-1]) / np.array(eu[1:]))
    op = np.log2(np.array(ep[:-1]) / np.array(ep[1:]))
    orr = np.log2(np.array(er[:-1]) / np.array(er[1:]))
    assert (oT > 1.8).all(), (eT, oT)
    assert (ou > 2.5).all() and (op > 2.5).all() and (orr > 2.5).all(), (eu, ou, ep, op, er, orr)
    assert eT[0] > 1e-5  # the coarse grid is measurably off the NSF profile


def test_newton_keeps_the_boundary_rings():
    nt, nr = 10, 6
    cfg = _cfg(nt, nr, dr1=0.1)
    n = nt * nr
    x, y, r = _centres(cfg)
    d = np.zeros((n, 18))
    d[:, F_RHO] = 1.0 + 0.05 * np.cos(x)
    d[:, F_U] = 0.2 * (1.0 - 0.5 / r) * np.sin(y)
    d[:, F_U + 1] = -0.1 * x * y
    d[:, F_U + 2] = 0.01
    d[:, F_TT] = 1.0 + 0.1 * np.exp(-r)
    d[:, F_TR] = 1.0 + 0.08 * np.exp(-r)
    h = 1e-3 * np.random.default_rng(1).standard_normal((n, 12))
    out, it, res = SA.synth_solve_annulus(d, h, cfg)
    assert res < 1e-11 and it < 10
    first, outer = np.arange(nt), np.arange(n - nt, n)
    for k, col in ((0, F_RHO), (1, F_U), (2, F_U + 1), (4, F_TT), (5, F_TR)):
        np.testing.assert_allclose(out[first, k], d[first, col], rtol=0, atol=1e-13)
        np.testing.assert_allclose(out[outer, k], d[outer, col], rtol=0, atol=1e-13)
    np.testing.assert_array_equal(out[:, 3], d[:, F_U + 2])
    assert np.abs(out[:, 0] - d[:, F_RHO]).max() > 1e-4  # the interior moved
