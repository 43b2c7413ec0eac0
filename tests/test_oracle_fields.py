"""Pins for the oracle's cell fields (Eq. DSMC_macroscopic), NSF relations,
higher-order terms, Kn_GLL and the stable counting sort."""
import math

import numpy as np

import oracle
from oracle.fields import (fields_from_particles, fields_from_sums, grad_cells, hot_kngll,
                           kappa_coefficients)
from paper_2501_10965_gb300 import workloads as W


def _sums(vx, vy, vz, ir):
    v2 = vx * vx + vy * vy + vz * vz
    return np.array([len(vx), vx.sum(), vy.sum(), vz.sum(), (vx * vx).sum(), (vy * vy).sum(), (vz * vz).sum(),
                     (vx * vy).sum(), (vx * vz).sum(), (vy * vz).sum(), (vx * v2).sum(), (vy * v2).sum(),
                     (vz * v2).sum(), ir.sum(), (ir * vx).sum(), (ir * vy).sum(), (ir * vz).sum()])


def test_fields_from_sums_equal_direct_moments():
    """Raw-sum route == central moments computed directly from the particles
    (brute force), for one sample with a large mean velocity."""
    rng = np.random.default_rng(1)
    for _ in range(5):
        n = int(rng.integers(2, 300))
        vx = 3.0 + 1.3 * rng.standard_normal(n)
        vy = -1.0 + 0.7 * rng.standard_normal(n) ** 3
        vz = 0.2 + rng.standard_normal(n)
        ir = rng.exponential(1.1, n)
        ref = fields_from_particles(vx, vy, vz, ir, fnum=0.003, vcell=0.01, d_r=2.0)
        got = fields_from_sums(_sums(vx, vy, vz, ir)[None, :], 1, 0.003, 0.01, 2.0)[0]
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())


def test_fields_time_average_and_temperature_definitions():
    """Two identical samples give the same fields as one (time average); a
    pure shift of all velocities changes only u; T_r = 2 <I_r> / d_r."""
    rng = np.random.default_rng(2)
    vx, vy, vz = rng.standard_normal((3, 500))
    ir = rng.exponential(0.8, 500)
    s = _sums(vx, vy, vz, ir)
    f1 = fields_from_sums(s[None], 1, 1.0, 1.0, 2.0)[0]
    f2 = fields_from_sums(2 * s[None], 2, 1.0, 1.0, 2.0)[0]
    assert np.allclose(f1, f2, rtol=1e-12, atol=1e-12)
    f3 = fields_from_sums(_sums(vx + 5.0, vy, vz, ir)[None], 1, 1.0, 1.0, 2.0)[0]
    assert np.allclose(np.delete(f3, 1), np.delete(f1, 1), rtol=1e-9, atol=1e-9)
    assert abs(f3[1] - f1[1] - 5.0) < 1e-12
    assert abs(f1[5] - ir.mean()) < 1e-12  # d_r = 2
    assert abs(f1[4] - (np.var(vx) + np.var(vy) + np.var(vz)) / 3) < 1e-12


def test_kappa_from_relaxation_matrix():
    # Eq. (kappa_A) for a diagonal A: kappa_t = 5 mu / (2 A_tt), kappa_r = d_r mu / (2 A_rr)
    kt, kr = kappa_coefficients((2 / 3, 0.0, 0.0, 0.5), 2.0)
    assert abs(kt - 3.75) < 1e-14 and abs(kr - 2.0) < 1e-14
    # a full matrix: check A (kt, kr) = (5, d_r)/2 * 1
    A = np.array([[0.7, 0.1], [0.05, 0.6]])
    kt, kr = kappa_coefficients(A.reshape(-1), 2.0)
    assert np.allclose(A @ np.array([kt, kr]), [2.5, 1.0], atol=1e-14)


def test_gradients_exact_on_linear_fields():
    nx, ny, dx, dy = 7, 5, 0.1, 0.2
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dy)
    f = (3.0 * X - 2.0 * Y + 1.0).reshape(-1)
    gx, gy = grad_cells(f, nx, ny, dx, dy, 2)
    assert np.allclose(gx, 3.0, atol=1e-12) and np.allclose(gy, -2.0, atol=1e-12)


def _cfg2d(**kw):
    return W.cavity_2d(nx=8, ny=6, ppc=1, kn=0.05, kn_ref=0.0, **kw)


def test_hot_is_dsmc_minus_nsf_on_linear_fields():
    """With linear u, T fields the NSF stress and heat fluxes are known in
    closed form (Eq. ns_constitutive); HoT = DSMC - NSF (Eq. hot_constitutive)."""
    cfg = _cfg2d()
    nx, ny = cfg["nx"], cfg["ny"]
    dx, dy = cfg["lx"] / nx, cfg["ly"] / ny
    X, Y = [a.reshape(-1) for a in np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dy)]
    f = np.zeros((nx * ny, 18))
    a, b, c, d, e = 0.3, -0.2, 0.1, 0.25, 0.05
    f[:, 0] = 1.0
    f[:, 1] = a * X + b * Y
    f[:, 2] = c * X + d * Y
    f[:, 3] = e * X
    f[:, 4] = 1.0 + 0.2 * X
    f[:, 5] = 1.0 + 0.1 * Y
    rng = np.random.default_rng(3)
    f[:, 6:] = rng.standard_normal((nx * ny, 12)) * 0.01
    hot, kn, mask = hot_kngll(f, cfg)
    assert mask.all()
    T = (3 * f[:, 4] + 2 * f[:, 5]) / 5
    mu = cfg["kn"] * math.sqrt(2 / math.pi) * T ** cfg["omega"]
    div = a + d
    sig_nsf = np.stack([-mu * (2 * a - 2 / 3 * div), -mu * (2 * d - 2 / 3 * div), -mu * (-2 / 3 * div),
                        -mu * (b + c), -mu * e, np.zeros_like(mu)], 1)
    kt, kr = kappa_coefficients(cfg["a_matrix"], 2.0)
    qt = np.stack([-kt * mu * 0.2, 0 * mu, 0 * mu], 1)
    qr = np.stack([0 * mu, -kr * mu * 0.1, 0 * mu], 1)
    assert np.allclose(hot[:, 0:6], f[:, 6:12] - sig_nsf, atol=1e-13)
    assert np.allclose(hot[:, 6:9], f[:, 12:15] - qt, atol=1e-13)
    assert np.allclose(hot[:, 9:12], f[:, 15:18] - qr, atol=1e-13)


def test_kngll_value_and_mask():
    """Kn_GLL = lambda max(|grad rho|/rho, ...), lambda = mu/(rho T) sqrt(pi T/2)
    (= Kn at rho = T = 1); HoT vanishes exactly where Kn_GLL < Kn_ref."""
    cfg = W.base_config(dim=1, nx=10, ppc=1, kn=0.1, kn_ref=0.02)
    x = (np.arange(10) + 0.5) / 10
    f = np.zeros((10, 18))
    f[:, 0] = 1.0 + 0.1 * x  # |grad rho|/rho = 0.1/rho
    f[:, 4] = 1.0
    f[:, 5] = 1.0
    f[:, 6:] = 0.3
    hot, kn, mask = hot_kngll(f, cfg)
    lam = cfg["kn"] * math.sqrt(2 / math.pi) / f[:, 0] * math.sqrt(math.pi / 2)
    assert np.allclose(kn, lam * 0.1 / f[:, 0], rtol=1e-12)
    assert np.all(mask == (kn >= 0.02))
    cfg["kn_ref"] = 0.0096
    hot, kn, mask = hot_kngll(f, cfg)
    assert 0 < mask.sum() < 10
    assert np.all(hot[~mask] == 0.0) and np.all(hot[mask] != 0.0)


def test_stable_sort_matches_brute_force():
    cfg = W.cavity_2d(nx=7, ny=5, ppc=0, capacity=4000)
    sim = oracle.OracleSim(cfg)
    rng = np.random.default_rng(4)
    n = 3000
    # many particles exactly on a few positions so ties are common
    x = rng.choice(np.linspace(0.01, 0.99, 13), n)
    y = rng.choice(np.linspace(0.01, 0.99, 11), n)
    vx = np.arange(n, dtype=np.float64)  # tags the input order
    sim.set_particles(dict(x=x, y=y, vx=vx, vy=np.zeros(n), vz=np.zeros(n), ir=np.zeros(n)))
    p = sim.particles()
    cell = np.minimum((x * 7).astype(int), 6) + 7 * np.minimum((y * 5).astype(int), 4)
    order = np.argsort(cell, kind="stable")
    assert np.array_equal(p["vx"], vx[order])
    assert np.array_equal(p["cell"], cell[order])
    st = sim.start()
    assert np.array_equal(np.diff(st), np.bincount(cell, minlength=35))
