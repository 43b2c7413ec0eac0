"""Pins of the oracle's flow past a cylinder (annular mesh, Sec. 4.2).

Each test checks the oracle against something it does not compute itself:

* the mesh: cell volumes sum to the annulus area, and cells found by brute
  force from (r, theta) of random points;
* the inflow sampler: the inverse of the entering particles' normal-speed
  CDF against numerical quadrature of the density z exp(-(z - s)^2);
* the freestream entry: the number of particles entering per step against
  the one-sided flux of a drifting Maxwellian;
* a gas at rest around a cylinder at the gas temperature stays uniform
  (detailed balance of entry, exit and diffuse re-emission);
* free-molecular drag and hit rate on the cylinder against the integral of
  the freestream's one-sided momentum and number fluxes over its surface
  (truncated-normal moments), with diffuse re-emission at T_w.
"""
import math

import numpy as np
import pytest

import oracle
from oracle.fields import fields_from_sums
from paper_2501_10965_gb300 import workloads as W


def _cfg(**kw):
    base = dict(ntheta=24, nr=8, ppc=40, kn=0.1, r_in=0.5, r_out=2.5, dr1=0.25, precision="fp64")
    base.update(kw)
    return W.cylinder_2d(**base)


def _ring_radii(cfg):
    nr, q = int(cfg["ny"]), float(cfg["stretch"])
    j = np.arange(nr + 1)
    f = j / nr if q == 1.0 else (q ** j - 1.0) / (q ** nr - 1.0)
    return cfg["r_in"] + (cfg["r_out"] - cfg["r_in"]) * f


def test_annulus_volumes_and_cells():
    cfg = _cfg(dr1=0.05)  # stretched rings
    assert cfg["stretch"] > 1.05
    nt, nr = int(cfg["nx"]), int(cfg["ny"])
    o = oracle.OracleSim(cfg)
    v = o.volumes()
    assert math.isclose(v.sum(), math.pi * (2.5 ** 2 - 0.5 ** 2), rel_tol=1e-12)
    R = _ring_radii(cfg)
    assert math.isclose(R[1] - R[0], 0.05, rel_tol=1e-9)
    np.testing.assert_allclose(v.reshape(nr, nt), np.repeat((np.pi / nt) * np.diff(R ** 2)[:, None], nt, 1),
                               rtol=1e-12)
    rng = np.random.default_rng(0)
    n = 6000
    r = np.sqrt(rng.uniform(0.5 ** 2, 2.5 ** 2, n))
    th = rng.uniform(0.0, 2.0 * np.pi, n)
    j = np.searchsorted(R, r, side="right") - 1
    k = np.floor(th / (2.0 * np.pi / nt)).astype(int)
    # keep points clear of the cell boundaries (rounding decides there)
    far = (np.min(np.abs(r[:, None] - R[None, :]), axis=1) > 1e-9) & \
          (np.abs(th / (2 * np.pi / nt) - np.round(th / (2 * np.pi / nt))) > 1e-9)
    r, th, j, k = r[far], th[far], j[far], k[far]
    m = len(r)
    # two points outside the outer circle leave at once
    x = np.concatenate([r * np.cos(th), [2.6, 0.0]])
    y = np.concatenate([r * np.sin(th), [0.0, -3.0]])
    ids = np.arange(m + 2, dtype=np.float64)
    o.set_particles({"x": x, "y": y, "vx": ids, "vy": np.zeros(m + 2), "vz": np.zeros(m + 2),
                     "ir": np.ones(m + 2)})
    p = o.particles()
    assert len(p["x"]) == m
    got = p["cell"][np.argsort(p["vx"])]
    np.testing.assert_array_equal(got, j * nt + k)


@pytest.mark.parametrize("s", [-3.0, -1.0, 0.0, 0.7, 2.0, 4.2])
def test_inflow_speed_sampler_inverts_the_flux_cdf(s):
    z = np.linspace(0.0, max(s, 0.0) + 10.0, 400001)
    dens = z * np.exp(-(z - s) ** 2)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(z))])
    total = cdf[-1]
    assert math.isclose(oracle.inflow_ginf(s), total, rel_tol=1e-7)
    cdf /= total
    for u in (0.001, 0.1, 0.37, 0.5, 0.9, 0.999):
        zs = oracle.inflow_speed(s, u)
        ze = float(np.interp(u, cdf, z))
        assert abs(zs - ze) <= 2e-5 * (1.0 + ze), (s, u, zs, ze)


def test_entry_count_is_the_one_sided_flux():
    cfg = _cfg(ntheta=48, nr=4, ppc=10, mach=2.0, collisions=False)
    o = oracle.OracleSim(cfg)
    c = o.constants()
    n0 = o.n
    steps = 2000
    o.step(steps)
    f = o.flow()
    assert o.n == n0 + f["n_in"] - f["n_out"] and f["n_out"] > 0
    nt, U, dt = 48, cfg["fs_u"][0], cfg["dt"]
    th = 2.0 * np.pi * (np.arange(nt) + 0.5) / nt
    un = -U * np.cos(th)  # freestream along x, inward normal -(cos, sin)
    s = un / math.sqrt(2.0)
    erfc = np.vectorize(math.erfc)
    flux = math.sqrt(1.0 / (2.0 * math.pi)) * (np.exp(-s * s) + math.sqrt(math.pi) * s * erfc(-s))
    mu = flux * (2.5 * 2.0 * np.pi / nt) * dt / c["fnum"]
    expect = steps * mu.sum()
    frac = mu - np.floor(mu)
    sd = math.sqrt(steps * float((frac * (1.0 - frac)).sum()))
    got = o.flow()["n_in"]
    assert abs(got - expect) <= 4.0 * sd + 0.002 * expect, (got, expect, sd)


def _ring_density(o, cfg, nsamples):
    nt, nr = int(cfg["nx"]), int(cfg["ny"])
    acc = o.accumulators()
    c = o.constants()
    N = acc[:, 0].reshape(nr, nt).sum(1)
    area = o.volumes().reshape(nr, nt).sum(1)
    return N * c["fnum"] / (nsamples * area)


def test_gas_at_rest_around_a_cylinder_at_its_temperature_stays_uniform():
    cfg = _cfg(ntheta=48, nr=6, ppc=40, mach=0.0, t_wall=1.0, kn=0.1)
    o = oracle.OracleSim(cfg)
    n0 = o.n
    o.step(200)
    batches, dens, temps, counts = 16, [], [], []
    for _ in range(batches):
        o.reset_accumulators()
        o.step(100, sample=True)
        dens.append(_ring_density(o, cfg, 100))
        f = fields_from_sums(o.accumulators(), 100, o.constants()["fnum"], o.volumes(), 2.0)
        T = (3.0 * f[:, 4] + 2.0 * f[:, 5]) / 5.0
        temps.append(np.mean(T))
        counts.append(o.n)
    dens = np.array(dens)
    m, se = dens.mean(0), dens.std(0, ddof=1) / math.sqrt(batches)
    assert (np.abs(m - 1.0) <= 4.0 * se + 0.005).all(), (m, se)
    assert abs(np.mean(temps) - 1.0) <= 0.01, np.mean(temps)
    assert abs(np.mean(counts) / n0 - 1.0) <= 0.01, (np.mean(counts), n0)


def _free_molecular_cylinder(rho, U, T, Tw, R, nphi=20000):
    """Force (x) and hit rate per unit length on a cylinder of radius R in a
    freestream (rho, U along x, T), free-molecular, diffuse re-emission at Tw
    from a resting wall.  At the surface point with outward normal n =
    (cos phi, sin phi) the speed into the wall w = -c.n is N(mu, T) with mu =
    -U cos phi; its one-sided moments are the truncated-normal moments
    E[w; w > 0] = mu Phi + sd phi_n, E[w^2; w > 0] = (mu^2 + T) Phi + mu sd phi_n."""
    phi = (np.arange(nphi) + 0.5) * (2.0 * np.pi / nphi)
    sd = math.sqrt(T)
    mu = -U * np.cos(phi)
    a = mu / sd
    Phi = 0.5 * (1.0 + np.vectorize(math.erf)(a / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * a * a) / math.sqrt(2.0 * math.pi)
    g1 = mu * Phi + sd * pdf
    g2 = (mu * mu + T) * Phi + mu * sd * pdf
    gamma = rho * g1
    # momentum delivered per unit area: incoming normal (-n) and tangential
    # (t = (-sin, cos), U.t = -U sin phi) parts, minus the re-emitted mean
    # momentum sqrt(pi Tw / 2) n per emitted particle
    fx = -rho * g2 * np.cos(phi) + U * np.sin(phi) ** 2 * gamma - gamma * math.sqrt(math.pi * Tw / 2.0) * np.cos(phi)
    dphi = 2.0 * np.pi / nphi
    return float(fx.sum() * R * dphi), float(gamma.sum() * R * dphi)


def test_free_molecular_drag_and_hit_rate_on_the_cylinder():
    cfg = _cfg(ntheta=48, nr=6, ppc=40, mach=2.0, t_wall=2.0, collisions=False)
    o = oracle.OracleSim(cfg)
    c = o.constants()
    U, dt = cfg["fs_u"][0], cfg["dt"]
    fx_ref, hits_ref = _free_molecular_cylinder(1.0, U, 1.0, 2.0, 0.5)
    batches, K = 20, 300
    fx, hits = [], []
    for _ in range(batches):
        w0 = o.wall_tally()[0].copy()
        o.step(K)
        d = o.wall_tally()[0] - w0
        fx.append(d[1] * c["fnum"] / (K * dt))
        hits.append(d[0] * c["fnum"] / (K * dt))
    for got, ref in ((np.array(fx), fx_ref), (np.array(hits), hits_ref)):
        m, se = got.mean(), got.std(ddof=1) / math.sqrt(batches)
        assert abs(m - ref) <= 4.0 * se + 0.003 * abs(ref), (m, se, ref)
    assert o.stats()["n_maxhit"] == 0


def test_specular_cylinder_and_empty_freestream():
    """Degenerate settings: a specular cylinder conserves every hit's energy
    (the energy delivered to it stays at rounding level) and an empty
    freestream (fs_rho = 0) lets nothing in, so the gas only drains."""
    cfg = _cfg(ntheta=24, nr=4, ppc=20, mach=2.0, collisions=False, fs_rho=0.0)
    cfg["walls"][0] = dict(cfg["walls"][0], kind="specular")
    o = oracle.OracleSim(cfg)
    n0 = o.n
    e_hit = []
    for _ in range(20):
        o.step(20)
        e_hit.append(o.wall_tally()[0].copy())
    f = o.flow()
    w = o.wall_tally()[0]
    assert f["n_in"] == 0 and f["n_out"] > 0 and o.n == n0 - f["n_out"]
    assert w[0] > 100  # hits
    # energy delivered: rounding only (|dE| per hit ~ 1e-15 of the particle energy)
    assert abs(w[4]) < 1e-11 * w[0], w
    # momentum delivered is along the normals: the z component never changes
    assert w[3] == 0.0


# ---------------------------------------------------------------------------
# Higher-order terms, Kn_GLL and the particle modification on the annulus
# (Sec. 3.1, 3.2 on the cylinder case of Sec. 4.2)
# ---------------------------------------------------------------------------

def _centres(cfg):
    nt, nr = int(cfg["nx"]), int(cfg["ny"])
    R = _ring_radii(cfg)
    rc = 0.5 * (R[:-1] + R[1:])
    th = 2 * np.pi * (np.arange(nt) + 0.5) / nt
    r2, t2 = np.meshgrid(rc, th, indexing="ij")
    return (r2 * np.cos(t2)).ravel(), (r2 * np.sin(t2)).ravel(), r2.ravel(), t2.ravel()


def test_annulus_gradient_exact_for_linear_and_radial_quadratic_fields():
    from oracle.fields import grad_annulus, ring_edges
    cfg = _cfg(dr1=0.05, ntheta=30, nr=9)
    nt, nr = int(cfg["nx"]), int(cfg["ny"])
    R = ring_edges(cfg)
    np.testing.assert_allclose(R, _ring_radii(cfg), rtol=1e-14)
    x, y, r, th = _centres(cfg)
    gx, gy = grad_annulus(0.7 + 1.3 * x - 0.4 * y, nt, nr, R)
    assert np.allclose(gx, 1.3, atol=1e-12) and np.allclose(gy, -0.4, atol=1e-12)
    # f = r^2 - 3 r: d/dr = 2 r - 3 exact inside (three-point formula on
    # stretched rings), first order in the first and last ring
    gx, gy = grad_annulus(r * r - 3 * r, nt, nr, R)
    inner = slice(nt, (nr - 1) * nt)
    d = 2 * r - 3
    assert np.allclose(gx[inner], (d * np.cos(th))[inner], atol=1e-11)
    assert np.allclose(gy[inner], (d * np.sin(th))[inner], atol=1e-11)


def test_annulus_hot_and_kngll_of_linear_fields():
    """Linear u and T_t, T_r in x, y: the NSF stress and heat fluxes from the
    analytic gradients; fields carrying those NSF values have zero HoT, and
    an added stress shows up as HoT unchanged.  Kn_GLL from the analytic
    gradients too."""
    from oracle.fields import hot_kngll, kappa_coefficients, mu_ref_of
    cfg = dict(_cfg(dr1=0.05, ntheta=30, nr=9), kn_ref=0.0)
    x, y, r, th = _centres(cfg)
    n = len(x)
    a = np.array([[0.05, -0.02], [0.03, 0.04]])  # du_i/dx_j
    F = np.zeros((n, 18))
    F[:, 0] = 1.0 + 0.1 * x - 0.05 * y
    F[:, 1] = 0.1 + a[0, 0] * x + a[0, 1] * y
    F[:, 2] = -0.2 + a[1, 0] * x + a[1, 1] * y
    F[:, 4] = 1.0 + 0.03 * x + 0.02 * y
    F[:, 5] = 0.9 - 0.01 * x + 0.03 * y
    T = (3 * F[:, 4] + 2 * F[:, 5]) / 5
    mu = mu_ref_of(cfg["kn"]) * T ** cfg["omega"]
    div = a[0, 0] + a[1, 1]
    sig = np.zeros((n, 6))
    sig[:, 0] = -mu * (2 * a[0, 0] - 2 / 3 * div)
    sig[:, 1] = -mu * (2 * a[1, 1] - 2 / 3 * div)
    sig[:, 2] = -mu * (-2 / 3 * div)
    sig[:, 3] = -mu * (a[0, 1] + a[1, 0])
    kt, kr = kappa_coefficients(cfg["a_matrix"], 2.0)
    F[:, 6:12] = sig
    F[:, 12], F[:, 13] = -kt * mu * 0.03, -kt * mu * 0.02
    F[:, 15], F[:, 16] = -kr * mu * (-0.01), -kr * mu * 0.03
    hot, kn, mask = hot_kngll(F, cfg)
    assert mask.all() and np.max(np.abs(hot)) < 1e-12
    F2 = F.copy()
    F2[:, 9] += 0.01  # an extra shear stress
    hot2, _, _ = hot_kngll(F2, cfg)
    assert np.allclose(hot2[:, 3], 0.01, atol=1e-12)
    # Kn_GLL with the analytic gradients: here the density term is the
    # largest of the four in every cell (checked), and it is exact for a
    # linear density
    lam = mu / (F[:, 0] * T) * np.sqrt(np.pi * T / 2)
    g_rho = np.hypot(0.1, -0.05) / F[:, 0]
    sp = np.hypot(F[:, 1], F[:, 2])
    gsp = np.hypot((F[:, 1] * a[0, 0] + F[:, 2] * a[1, 0]) / sp, (F[:, 1] * a[0, 1] + F[:, 2] * a[1, 1]) / sp)
    others = np.stack([gsp / np.maximum(sp, np.sqrt(1.4 * T)), np.hypot(0.03, 0.02) / F[:, 4],
                       np.hypot(-0.01, 0.03) / F[:, 5]])
    assert np.all(g_rho > 1.2 * others.max(0))
    assert np.allclose(kn, lam * g_rho, rtol=1e-12, atol=0)


def test_annulus_dig_correct_matches_targets_with_cell_volumes():
    """Sec. 3.2 on the annulus: every cell holds Iround(rho V_cell / F)
    particles (its own volume), their instantaneous u, T_t, T_r equal the
    target, and new particles lie inside their sector."""
    cfg = _cfg(dr1=0.05, ntheta=24, nr=8, ppc=30)
    sim = oracle.OracleSim(cfg)
    sim.step(3)
    nc = 24 * 8
    rng = np.random.default_rng(7)
    t = np.zeros((nc, 6))
    t[:, 0] = 0.6 + 0.8 * rng.random(nc)
    t[:, 1:4] = 0.3 * rng.standard_normal((nc, 3))
    t[:, 4] = 0.8 + 0.5 * rng.random(nc)
    t[:, 5] = 0.7 + 0.5 * rng.random(nc)
    t[5, 0] = 0.0
    assert sim.dig_correct(t) == 0
    t[5, 0] = 1.5  # refill the emptied cell from its target Maxwellian
    assert sim.dig_correct(t) == 0
    p = sim.particles()
    v = sim.volumes()
    fnum = sim.constants()["fnum"]
    cnt = np.bincount(p["cell"], minlength=nc)
    xm = t[:, 0] * v / fnum
    assert np.all((cnt == np.floor(xm)) | (cnt == np.floor(xm) + 1))
    full = cnt >= 2
    for j, k in enumerate(("vx", "vy", "vz")):
        m = np.bincount(p["cell"], p[k], nc)[full] / cnt[full]
        assert np.allclose(m, t[full, 1 + j], atol=1e-13)
    c2 = sum(np.bincount(p["cell"], (p[k] - t[p["cell"], 1 + j]) ** 2, nc) for j, k in enumerate(("vx", "vy", "vz")))
    # a cell refilled by copies of one particle has T_t* = 0: only its mean
    # is shifted (a = 1)
    spread = full & (c2 > 1e-20)
    assert spread.sum() > 0.9 * full.sum()
    assert np.allclose(c2[spread] / (3 * cnt[spread]), t[spread, 4], rtol=1e-12)
    assert np.allclose(np.bincount(p["cell"], p["ir"], nc)[full] / cnt[full], t[full, 5], rtol=1e-12)
    R = _ring_radii(cfg)
    r = np.hypot(p["x"], p["y"])
    th = np.mod(np.arctan2(p["y"], p["x"]), 2 * np.pi)
    ring, sec = p["cell"] // 24, p["cell"] % 24
    assert np.all((r >= R[ring] - 1e-12) & (r <= R[ring + 1] + 1e-12))
    ks = th / (2 * np.pi / 24)
    assert np.all((ks >= sec - 1e-9) & (ks <= sec + 1 + 1e-9) | (ks > 23.999999) & (sec == 0))
