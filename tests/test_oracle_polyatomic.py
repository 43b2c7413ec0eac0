"""Pins of the oracle's general Borgnakke-Larsen exchange (d_r = 3) and of
the VSS scattering law (alpha != 1), Sec. 2.2.

* The rotational fraction of one exchange is Beta(d_r/2, 5/2 - omega): KS
  test against scipy's Beta at d_r = 2 (closed form) and 3 (acceptance-
  rejection).
* A molecule's equilibrium rotational energy is Gamma(d_r/2) x T: KS test of
  the initial state and of the energies re-emitted by diffuse walls.
* With d_r = 3 a homogeneous gas relaxes to equipartition, T_t = T_r, at the
  temperature fixed by energy conservation, (3 T_t0 + 3 T_r0)/6; a partition
  with the wrong Beta parameters ends at another T_r / T_t.
* VSS: the deflection from the pre-collision relative velocity has cos chi
  = 2 u^{1/alpha} - 1 exactly, the new relative speed is the given one, and
  the azimuth turns about the old direction.
* Collisions conserve momentum and energy at d_r = 3, alpha = 1.5.
* The collision frequency at alpha != 1 is the mean thermal speed over
  Bird's VSS mean free path 4 alpha (5-2w)(7-2w) / (5 (alpha+1)(alpha+2)) mu
  / (rho sqrt(2 pi T)).
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle
from paper_2501_10965_gb300 import workloads as W


@pytest.mark.parametrize("d_r", [2.0, 3.0])
def test_bl_partition_is_beta(d_r):
    omega = 0.74
    rng = np.random.default_rng(3)
    n = 20000
    u = rng.random(n)
    x = np.array([oracle.bl_fraction(omega, d_r, 11, k, 7, 3, float(u[k])) for k in range(n)])
    assert np.all((x > 0) & (x < 1))
    ks = stats.kstest(x, stats.beta(d_r / 2.0, 2.5 - omega).cdf)
    assert ks.pvalue > 1e-3, ks
    # a swapped pair of parameters is far off
    if d_r == 3.0:
        assert stats.kstest(x, stats.beta(2.5 - omega, d_r / 2.0).cdf).pvalue < 1e-6
    else:
        # d_r = 2: the inverse CDF of Beta(1, b) at the main uniform
        assert np.allclose(x, 1.0 - u ** (1.0 / (2.5 - omega)), rtol=0, atol=1e-14)


def test_rotational_energy_is_gamma_at_init_and_at_walls():
    cfg = W.homogeneous_box(ncells=40, ppc=250, kn=0.1, d_r=3.0, tt=1.0, tr=1.4, dt=0.01)
    sim = oracle.OracleSim(cfg)
    ir = sim.particles()["ir"]
    assert stats.kstest(ir / 1.4, stats.gamma(1.5).cdf).pvalue > 1e-3
    assert stats.kstest(ir / 1.4, stats.expon().cdf).pvalue < 1e-6  # not the d_r = 2 law
    # collisionless slab between diffuse walls at 0.8: after many crossings
    # every particle's I_r was drawn by a wall at 0.8
    cfg = W.base_config(dim=1, nx=10, ppc=300, d_r=3.0, collisions=False, dt=0.02, init_tt=1.0, init_tr=1.4,
                        walls=[{"kind": "diffuse", "T": 0.8, "u": (0, 0, 0)}] * 4)
    sim = oracle.OracleSim(cfg)
    sim.step(3000)
    ir = sim.particles()["ir"]
    assert stats.kstest(ir / 0.8, stats.gamma(1.5).cdf).pvalue > 1e-3


def test_d_r3_gas_relaxes_to_equipartition():
    """T_t0 = 1.3, T_r0 = 0.6 in a specular box: energy conserved exactly,
    and at equilibrium T_t = T_r = 0.95 within 4 standard errors."""
    cfg = W.homogeneous_box(ncells=100, ppc=100, kn=0.05, d_r=3.0, tt=1.3, tr=0.6, dt=0.004)
    sim = oracle.OracleSim(cfg)
    p0 = sim.particles()
    e0 = np.sum(0.5 * (p0["vx"] ** 2 + p0["vy"] ** 2 + p0["vz"] ** 2) + p0["ir"])
    sim.step(300)
    tt, tr = [], []
    for _ in range(20):
        sim.step(20)
        p = sim.particles()
        v2 = p["vx"] ** 2 + p["vy"] ** 2 + p["vz"] ** 2
        tt.append(np.mean(v2) / 3.0)
        tr.append(2.0 * np.mean(p["ir"]) / 3.0)
    e1 = np.sum(0.5 * v2 + p["ir"])
    assert abs(e1 - e0) < 1e-11 * e0
    n = len(p["ir"])
    teq = (3 * 1.3 + 3 * 0.6) / 6.0
    # snapshot noise of T_t and T_r about T for N particles (Gamma variances)
    assert abs(np.mean(tt) - teq) < 4 * teq * math.sqrt(2.0 / (3 * n))
    assert abs(np.mean(tr) - teq) < 4 * teq * math.sqrt(2.0 / (3 * n))
    assert sim.stats()["n_inel"] > 10000


@pytest.mark.parametrize("alpha", [1.0, 1.5, 0.8])
def test_vss_deflection_law(alpha):
    rng = np.random.default_rng(5)
    for _ in range(200):
        g = rng.standard_normal(3) * 1.7
        gn = 0.3 + rng.random()
        u, v = rng.random(), rng.random()
        h = oracle.scatter(alpha, g, gn, u, v)
        assert abs(np.linalg.norm(h) - 0.5 * gn) < 1e-14
        if alpha != 1.0:
            cos_chi = h @ g / (np.linalg.norm(h) * np.linalg.norm(g))
            assert abs(cos_chi - (2.0 * u ** (1.0 / alpha) - 1.0)) < 1e-13
            # averaged over the azimuth the deflected direction is along g
            hs = np.mean([oracle.scatter(alpha, g, gn, u, (k + 0.5) / 8) for k in range(8)], axis=0)
            assert np.allclose(hs, 0.5 * gn * cos_chi * g / np.linalg.norm(g), atol=1e-13)
    if alpha != 1.0:
        # the distribution of cos chi: P(cos chi <= c) = ((c + 1)/2)^alpha
        g = np.array([0.3, -1.1, 0.4])
        c = np.array([oracle.scatter(alpha, g, 1.0, u, 0.3) @ g / (0.5 * np.linalg.norm(g))
                      for u in rng.random(5000)])
        assert stats.kstest(c, lambda t: ((np.clip(t, -1, 1) + 1) / 2) ** alpha).pvalue > 1e-3


def test_collisions_conserve_momentum_and_energy_d_r3_vss():
    cfg = W.homogeneous_box(ncells=20, ppc=60, kn=0.01, tt=1.7, tr=0.4, dt=0.01, init_u=(0.3, -0.2, 0.1),
                            d_r=3.0, alpha=1.5)
    sim = oracle.OracleSim(cfg)

    def totals():
        p = sim.particles()
        e = 0.5 * (p["vx"] ** 2 + p["vy"] ** 2 + p["vz"] ** 2) + p["ir"]
        return np.stack([np.bincount(p["cell"], weights=a, minlength=20) for a in (p["vx"], p["vy"], p["vz"], e)])

    before = totals()
    for k in range(5):
        sim.set_step(k)
        sim.collide()
    after = totals()
    assert sim.stats()["n_coll"] > 1000 and sim.stats()["n_inel"] > 100
    assert np.max(np.abs(after - before)) / np.abs(before).max() < 1e-13


@pytest.mark.parametrize("alpha,omega", [(1.5, 0.74), (1.2, 0.6)])
def test_vss_collision_frequency_matches_mean_free_path(alpha, omega):
    kn = 0.1
    sim = oracle.OracleSim(W.homogeneous_box(ncells=3, ppc=2, kn=kn, omega=omega, alpha=alpha))
    c_sigma = sim.constants()["c_sigma"]
    a = math.sqrt(2.0)

    def f(g):
        return math.sqrt(2.0 / math.pi) * g * g / a ** 3 * math.exp(-g * g / (2 * a * a))

    mean_sg, _ = integrate.quad(lambda g: c_sigma * g ** (2 - 2 * omega) * f(g), 0, 40 * a)
    mu = kn * math.sqrt(2.0 / math.pi)
    lam = 4 * alpha * (5 - 2 * omega) * (7 - 2 * omega) / (5 * (alpha + 1) * (alpha + 2)) * mu / math.sqrt(2 * math.pi)
    nu_ref = math.sqrt(8.0 / math.pi) / lam
    assert abs(mean_sg - nu_ref) / nu_ref < 1e-9
