"""Pins for the oracle's DIG particle modification (Sec. 3.2) and the steady
1D synthetic-equation solver (Eq. macroscopic_equation)."""
import math

import numpy as np
import pytest

import oracle
from oracle.fields import hot_kngll, kappa_coefficients
from oracle.synth1d import residual, synth_solve_1d
from paper_2501_10965_gb300 import workloads as W


def _cell_moments(p, ncells):
    out = np.zeros((ncells, 6))
    for c in range(ncells):
        m = p["cell"] == c
        n = m.sum()
        if n == 0:
            continue
        v = np.stack([p["vx"][m], p["vy"][m], p["vz"][m]], 1)
        u = v.mean(0)
        out[c, 0] = n
        out[c, 1:4] = u
        out[c, 4] = ((v - u) ** 2).sum() / (3 * n)
        out[c, 5] = p["ir"][m].mean()  # d_r = 2: T_r = <I_r>
    return out


def _target(ncells, rng, rho_scale=1.0):
    t = np.zeros((ncells, 6))
    t[:, 0] = rho_scale * (0.7 + 0.6 * rng.random(ncells))
    t[:, 1:4] = rng.standard_normal((ncells, 3)) * 0.3
    t[:, 4] = 0.8 + 0.5 * rng.random(ncells)
    t[:, 5] = 0.7 + 0.6 * rng.random(ncells)
    return t


def test_dig_correct_matches_target_moments_exactly():
    """After steps i-iv every cell holds Iround(rho V / F) particles whose
    instantaneous u, T_t, T_r equal the target (Sec. 3.2 step iv makes this
    exact up to rounding)."""
    cfg = W.fourier_1d(nx=40, ppc=50)
    sim = oracle.OracleSim(cfg)
    sim.step(5)
    rng = np.random.default_rng(5)
    t = _target(40, rng)
    assert sim.dig_correct(t) == 0
    p = sim.particles()
    m = _cell_moments(p, 40)
    c = sim.constants()
    x = t[:, 0] * c["vcell"] / c["fnum"]
    assert np.all((m[:, 0] == np.floor(x)) | (m[:, 0] == np.floor(x) + 1))
    occ = m[:, 0] >= 2
    assert np.allclose(m[occ, 1:4], t[occ, 1:4], atol=1e-13)
    assert np.allclose(m[occ, 4], t[occ, 4], rtol=1e-13)
    assert np.allclose(m[occ, 5], t[occ, 5], rtol=1e-13)
    st = sim.start()
    assert np.array_equal(np.diff(st), m[:, 0].astype(int))
    # positions stay inside their cell
    assert np.all(np.minimum((p["x"] * 40).astype(int), 39) == p["cell"])


def test_dig_correct_particle_count_is_unbiased():
    """E[N_new] = rho V / F (Iround is unbiased, Sec. 3.2 step i)."""
    cfg = W.fourier_1d(nx=400, ppc=20)
    sim = oracle.OracleSim(cfg)
    c = sim.constants()
    t = np.zeros((400, 6))
    t[:, 0] = 1.2345
    t[:, 4] = 1.0
    t[:, 5] = 1.0
    total = 0
    reps = 20
    for _ in range(reps):
        assert sim.dig_correct(t) == 0
        total += sim.n
    x = 1.2345 * c["vcell"] / c["fnum"]
    frac = x - math.floor(x)
    se = math.sqrt(400 * reps * frac * (1 - frac))
    assert abs(total - 400 * reps * x) < 4 * se + 1e-9


def test_dig_replicas_copy_existing_particles():
    """Replicated particles copy (v, I_r) of a pre-existing particle of the same
    cell (Sec. 3.2 step ii), and step iv maps every particle of a cell by the
    same affine map, so after doubling the count each cell holds 30 distinct
    states, each an affine image (one a, b, c per cell) of an old one."""
    cfg = W.fourier_1d(nx=10, ppc=30)
    sim = oracle.OracleSim(cfg)
    p0 = sim.particles()
    t = _cell_moments(p0, 10)
    c = sim.constants()
    t[:, 0] = 2.0 * 30 * c["fnum"] / c["vcell"]  # double the count
    t[:, 4] *= 1.2
    assert sim.dig_correct(t) == 0
    p = sim.particles()
    assert sim.n == 600
    for cell in range(10):
        old = np.stack([p0[k][p0["cell"] == cell] for k in ("vx", "vy", "vz", "ir")], 1)
        new = np.stack([p[k][p["cell"] == cell] for k in ("vx", "vy", "vz", "ir")], 1)
        assert len(new) == 60
        # the first 30 (kept, in order) are the images of the old ones
        a = (new[1, 0] - new[0, 0]) / (old[1, 0] - old[0, 0])
        cc = new[0, 3] / old[0, 3]
        b = new[0, :3] - a * old[0, :3]
        assert np.allclose(new[:30, :3], a * old[:, :3] + b, atol=1e-12)
        assert np.allclose(new[:30, 3], cc * old[:, 3], rtol=1e-12)
        # each replica equals one of the kept particles exactly
        kept = {tuple(r) for r in new[:30]}
        assert all(tuple(r) in kept for r in new[30:])


def test_dig_correct_rejects_non_finite_targets_without_change():
    cfg = W.fourier_1d(nx=10, ppc=10)
    sim = oracle.OracleSim(cfg)
    p0 = sim.particles()
    t = np.ones((10, 6))
    t[3, 4] = np.nan
    assert sim.dig_correct(t) == -3
    t[3, 4] = 1.0
    t[5, 5] = -1.0
    assert sim.dig_correct(t) == -3
    p1 = sim.particles()
    for k in p0:
        assert np.array_equal(p0[k], p1[k])


def test_dig_correct_fills_empty_cells_from_target_maxwellian():
    cfg = W.fourier_1d(nx=4, ppc=10, capacity=10000)
    sim = oracle.OracleSim(cfg)
    t = np.zeros((4, 6))
    t[:, 4:6] = 1.0
    assert sim.dig_correct(t) == 0 and sim.n == 0  # empty every cell first
    c = sim.constants()
    t[:, 0] = 500 * c["fnum"] / c["vcell"]
    t[:, 1:4] = [0.1, 0.2, 0.3]
    t[:, 4] = 1.5
    t[:, 5] = 0.5
    assert sim.dig_correct(t) == 0
    m = _cell_moments(sim.particles(), 4)
    assert np.all(m[:, 0] == 500)
    assert np.allclose(m[:, 1:4], [0.1, 0.2, 0.3], atol=1e-13)
    assert np.allclose(m[:, 4], 1.5, rtol=1e-13) and np.allclose(m[:, 5], 0.5, rtol=1e-13)


def test_dig_correct_copies_of_one_particle_keep_a_equal_to_one():
    """A cell holding one particle that the target refills: its copies all
    share one velocity, so T_t* = 0 and step iv takes a = 1 (reading of the
    degenerate case); every particle then moves to the target velocity
    u_target exactly up to one rounding, and I_r is scaled to T_r.  A mean
    taken as (sum v) / N leaves T_t* at a rounding-sized positive value
    instead, and a = sqrt(T_t / T_t*) ~ 1e8 sends the velocities to
    garbage: this catches it."""
    cfg = W.fourier_1d(nx=4, ppc=10, capacity=10000)
    sim = oracle.OracleSim(cfg)
    c = sim.constants()
    # one particle per cell, velocities whose repeated sums round
    v = np.array([0.1234567891234, -0.7654321987654, 0.333333333333333])
    sim.set_particles({"x": (np.arange(4) + 0.5) / 4, "vx": np.full(4, v[0]), "vy": np.full(4, v[1]),
                       "vz": np.full(4, v[2]), "ir": np.full(4, 0.9)})
    t = np.zeros((4, 6))
    t[:, 0] = 15 * c["fnum"] / c["vcell"]
    t[:, 1:4] = [0.0125, -0.0404, -0.0566]
    t[:, 4] = 1.1
    t[:, 5] = 0.8
    assert sim.dig_correct(t) == 0
    p = sim.particles()
    assert np.all(np.bincount(p["cell"], minlength=4) == 15)
    for j, k in enumerate(("vx", "vy", "vz")):
        assert np.allclose(p[k], t[0, 1 + j], rtol=0, atol=1e-16), (k, p[k])
    assert np.allclose(p["ir"], 0.8, rtol=1e-15)


# ----------------------------------------------------------------------------
# steady synthetic equations, 1D
# ----------------------------------------------------------------------------

def _fake_dsmc(cfg, T_left, T_right, uy_left=0.0, uy_right=0.0, rho=1.0):
    n = cfg["nx"]
    x = (np.arange(n) + 0.5) / n
    f = np.zeros((n, 18))
    f[:, 0] = rho
    f[:, 4] = T_left + (T_right - T_left) * x
    f[:, 5] = f[:, 4]
    f[:, 2] = uy_left + (uy_right - uy_left) * x
    return f


def test_synth_nsf_limit_fourier_closed_form():
    """HoT = 0, u = 0, Dirichlet temperatures in the first and last cell: with
    kappa_t, kappa_r both proportional to mu = mu_ref T^omega, the steady
    solution has T_t = T_r = T with T^(1+omega) linear in x, uniform rho T_t,
    and the DSMC mass (Eq. macroscopic_equation, Eq. ns_constitutive)."""
    cfg = W.fourier_1d(nx=100, kn=0.01)
    f = _fake_dsmc(cfg, 1.0, 1.5)
    f[:, 4] += 0.05 * np.sin(np.linspace(0, 3, 100))  # a non-converged guess
    f[0, 4] = f[0, 5] = 1.0
    f[-1, 4] = f[-1, 5] = 1.5
    hot = np.zeros((100, 12))
    out, it, res = synth_solve_1d(f, hot, cfg)
    assert res < 1e-10 and it < 30
    x = (np.arange(100) + 0.5) / 100
    w = cfg["omega"]
    a0, a1 = 1.0 ** (1 + w), 1.5 ** (1 + w)
    xs = (x - x[0]) / (x[-1] - x[0])
    T_ref = (a0 + (a1 - a0) * xs) ** (1 / (1 + w))
    assert np.max(np.abs(out[:, 4] - T_ref)) < 2e-5
    assert np.max(np.abs(out[:, 5] - T_ref)) < 2e-5
    p = out[:, 0] * out[:, 4]
    assert np.ptp(p) < 1e-12 * p.mean()
    assert abs(out[:, 0].sum() - f[:, 0].sum()) < 1e-12 * f[:, 0].sum()


def test_synth_nsf_limit_couette_uniform_shear():
    """Couette, HoT = 0: sigma_xy = -mu du/dx is uniform; total energy flux
    sigma_xy u_y + q is uniform; viscous heating makes T peak inside."""
    cfg = W.couette_1d(kn=0.01, nx=80)
    f = _fake_dsmc(cfg, 1.0, 1.0, -0.3, 0.3)
    hot = np.zeros((80, 12))
    out, it, res = synth_solve_1d(f, hot, cfg)
    assert res < 1e-10
    dx = 1 / 80
    tt, tr, uy = out[:, 4], out[:, 5], out[:, 2]
    Tf = (3 * (tt[1:] + tt[:-1]) / 2 + 2 * (tr[1:] + tr[:-1]) / 2) / 5
    mu = cfg["kn"] * math.sqrt(2 / math.pi) * Tf ** cfg["omega"]
    s = -mu * np.diff(uy) / dx
    assert np.ptp(s) < 1e-9 * abs(s).max()
    assert tt[40] > tt[0] + 1e-4
    assert abs(uy[40] + uy[39]) < 1e-9  # antisymmetric profile


def test_synth_residual_zero_at_solution_and_hot_enters_as_flux():
    """A uniform HoT_qx shifts the heat flux but not the temperature profile
    (its divergence is zero); a linear HoT_qx acts as a source."""
    cfg = W.fourier_1d(nx=50, kn=0.05)
    f = _fake_dsmc(cfg, 1.0, 1.3)
    hot = np.zeros((50, 12))
    out0, _, _ = synth_solve_1d(f, hot, cfg)
    hot[:, 6] = 0.02
    out1, _, r1 = synth_solve_1d(f, hot, cfg)
    assert r1 < 1e-10
    assert np.allclose(out0, out1, atol=1e-10)
    hot[:, 6] = 0.05 * np.linspace(0, 1, 50)
    out2, _, r2 = synth_solve_1d(f, hot, cfg)
    assert r2 < 1e-10 and np.max(np.abs(out2[:, 4] - out0[:, 4])) > 1e-3
    x = np.concatenate([out2[:, 0], out2[:, 2], out2[:, 3], out2[:, 4], out2[:, 5]])
    assert np.max(np.abs(residual(x, f, hot, cfg))) < 1e-10


def test_dig_correct_empties_a_cell_whose_target_density_is_zero():
    """A target row of zeros (an unsampled cell's fields) empties the cell
    and is accepted although its temperatures are zero; with rho > 0 a zero
    temperature is still rejected."""
    cfg = W.fourier_1d(nx=6, ppc=20)
    sim = oracle.OracleSim(cfg)
    t = _cell_moments(sim.particles(), 6)
    c = sim.constants()
    t[:, 0] = t[:, 0] * c["fnum"] / c["vcell"]
    t[2] = 0.0
    assert sim.dig_correct(t) == 0
    cnt = np.bincount(sim.particles()["cell"], minlength=6)
    assert cnt[2] == 0 and np.all(cnt[[0, 1, 3, 4, 5]] > 0)
    t[3, 4] = 0.0
    p0 = sim.particles()
    assert sim.dig_correct(t) == -3
    assert np.array_equal(sim.particles()["x"], p0["x"])
