"""Pins for the oracle's move stage, wall model and sampled fields, from
free-molecular closed forms and steady-state invariants of 1D flows."""
import math

import numpy as np
import pytest

import oracle
from oracle.fields import fields_from_sums
from paper_2501_10965_gb300 import workloads as W


def test_free_flight_is_exact_and_specular_walls_mirror():
    cfg = W.homogeneous_box(ncells=10, ppc=0, dt=0.1, capacity=16)
    sim = oracle.OracleSim(cfg)
    x = np.array([0.05, 0.5, 0.95, 0.01, 0.99])
    vx = np.array([0.1, -0.3, 0.2, -0.3, 0.25])
    vy = np.array([1.0, 2.0, -1.0, 0.5, 0.0])
    sim.set_particles(dict(x=x, vx=vx, vy=vy, vz=np.zeros(5), ir=np.ones(5)))
    sim.move()
    p = sim.particles()
    order = np.argsort(p["x"])
    got = np.sort(p["x"])
    # free flight for the first three, mirror images for the two that hit
    xf = np.array([0.05 + 0.01, 0.5 - 0.03, 0.95 + 0.02, -(0.01 - 0.03), 1.0 - (0.99 + 0.025 - 1.0)])
    assert np.allclose(got, np.sort(xf), atol=1e-15, rtol=0)
    assert set(np.round(p["vx"], 12)) == set(np.round([0.1, -0.3, 0.2, 0.3, -0.25], 12))
    assert np.all(p["ir"] == 1.0)


def test_diffuse_wall_reemission_statistics():
    """Particles leaving a diffuse wall at T_w: normal speed Rayleigh,
    P(v_n < v) = 1 - exp(-v^2 / (2 T_w)) (flux-weighted half Maxwellian),
    tangential components N(U_w, T_w), I_r exponential with mean T_w (d_r = 2)."""
    from scipy import stats
    Tw, Uw = 2.0, 0.7
    cfg = W.base_config(dim=1, nx=4, ppc=0, dt=1e-3, collisions=False, capacity=100000,
                        walls=[{"kind": "diffuse", "T": Tw, "u": (0.0, Uw, 0.0)},
                               {"kind": "specular", "T": 1.0, "u": (0, 0, 0)}, {"kind": "diffuse", "T": 1, "u": (0, 0, 0)},
                               {"kind": "diffuse", "T": 1, "u": (0, 0, 0)}])
    n = 40000
    sim = oracle.OracleSim(cfg)
    # every particle hits wall 0 after 1e-6 and flies the rest of the step
    sim.set_particles(dict(x=np.full(n, 1e-9), vx=np.full(n, -1e-3), vy=np.zeros(n), vz=np.zeros(n), ir=np.zeros(n)))
    sim.move()
    p = sim.particles()
    assert sim.wall_tally()[0, 0] == n
    assert np.all(p["vx"] > 0)
    assert np.allclose(p["x"], p["vx"] * (1e-3 - 1e-6), rtol=1e-9, atol=1e-15)
    ks = stats.kstest(p["vx"], lambda v: 1 - np.exp(-v * v / (2 * Tw)))
    assert ks.pvalue > 1e-4
    assert abs(np.mean(p["vy"]) - Uw) < 4 * math.sqrt(Tw / n)
    assert abs(np.var(p["vy"]) - Tw) < 4 * Tw * math.sqrt(2.0 / n)
    assert abs(np.mean(p["vz"])) < 4 * math.sqrt(Tw / n)
    assert abs(np.var(p["vz"]) - Tw) < 4 * Tw * math.sqrt(2.0 / n)
    assert stats.kstest(p["ir"] / Tw, "expon").pvalue > 1e-4


def _sample_fields(sim, nsteps):
    sim.reset_accumulators()
    sim.step(nsteps, sample=True)
    c = sim.constants()
    return fields_from_sums(sim.accumulators(), sim.nsamples, c["fnum"], c["vcell"], sim.cfg["d_r"])


@pytest.mark.slow
def test_free_molecular_fourier_heat_flux():
    """Collisionless gas between diffuse walls at T1, T2: the exact heat flux
    is q = n (2 + d_r/2)(T1 - T2) / (sqrt(pi/(2 T1)) + sqrt(pi/(2 T2))), with n
    the mean density; it is uniform across the gap."""
    T1, T2 = 1.0, 2.0
    cfg = W.base_config(dim=1, nx=20, ppc=200, dt=0.01, collisions=False, init_tt=1.5, init_tr=1.5,
                        walls=[{"kind": "diffuse", "T": T1, "u": (0, 0, 0)}, {"kind": "diffuse", "T": T2, "u": (0, 0, 0)},
                               {"kind": "diffuse", "T": 1, "u": (0, 0, 0)}, {"kind": "diffuse", "T": 1, "u": (0, 0, 0)}])
    sim = oracle.OracleSim(cfg)
    sim.step(600)
    f = _sample_fields(sim, 2000)
    q = f[:, 12] + f[:, 15]
    n = f[:, 0].mean()
    d_r = 2.0
    q_ref = n * (2 + d_r / 2) * (T1 - T2) / (math.sqrt(math.pi / (2 * T1)) + math.sqrt(math.pi / (2 * T2)))
    assert abs(q.mean() - q_ref) < 0.02 * abs(q_ref), (q.mean(), q_ref)
    assert np.all(np.abs(q - q_ref) < 0.1 * abs(q_ref))
    # the wall tallies see the same flux: energy delivered per unit time and area
    tal = sim.wall_tally()
    c = sim.constants()
    # (tallies cover warm-up + sampling steps)
    t_total = 2600 * cfg["dt"]
    q_wall0 = -tal[0, 4] * c["fnum"] / t_total
    assert abs(q_wall0 - q_ref) < 0.05 * abs(q_ref)


@pytest.mark.slow
def test_free_molecular_couette_shear_stress():
    """Collisionless gas between diffuse walls moving at -/+U_w, both at T_w:
    sigma_xy = -n U_w sqrt(2 T_w / pi) everywhere; the mean velocity is 0."""
    Uw, Tw = 0.5, 1.0
    cfg = W.base_config(dim=1, nx=20, ppc=200, dt=0.01, collisions=False,
                        walls=[{"kind": "diffuse", "T": Tw, "u": (0, -Uw, 0)}, {"kind": "diffuse", "T": Tw, "u": (0, Uw, 0)},
                               {"kind": "diffuse", "T": 1, "u": (0, 0, 0)}, {"kind": "diffuse", "T": 1, "u": (0, 0, 0)}])
    sim = oracle.OracleSim(cfg)
    sim.step(600)
    f = _sample_fields(sim, 2000)
    n = f[:, 0].mean()
    s_ref = -n * Uw * math.sqrt(2 * Tw / math.pi)
    sxy = f[:, 9]
    assert abs(sxy.mean() - s_ref) < 0.02 * abs(s_ref), (sxy.mean(), s_ref)
    assert abs(f[:, 2].mean()) < 0.02


@pytest.mark.slow
def test_steady_fourier_invariants():
    """Steady 1D heat transfer between walls at 273 K and 373 K, Kn 0.1: the
    total heat flux q_t + q_r and the normal stress p_xx = rho T_t + sigma_xx
    are uniform across the gap (1D steady conservation of energy and
    momentum), checked by the slope of a linear fit against its batch-means
    standard error."""
    cfg = W.fourier_1d()
    sim = oracle.OracleSim(cfg)
    sim.step(3000)
    x = (np.arange(cfg["nx"]) + 0.5) / cfg["nx"]
    slopes_q, slopes_p, qs = [], [], []
    for _ in range(8):
        f = _sample_fields(sim, 400)
        q = f[:, 12] + f[:, 15]
        pxx = f[:, 0] * f[:, 4] + f[:, 6]
        slopes_q.append(np.polyfit(x, q, 1)[0])
        slopes_p.append(np.polyfit(x, pxx, 1)[0])
        qs.append(q.mean())
    for s in (np.array(slopes_q), np.array(slopes_p)):
        se = s.std(ddof=1) / math.sqrt(len(s))
        assert abs(s.mean()) < 3.5 * se + 1e-4, (s.mean(), se)
    assert np.mean(qs) < -0.01  # heat flows from the hot wall (x = 1) to the cold one
