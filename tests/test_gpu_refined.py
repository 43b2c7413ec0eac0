"""GPU lid-driven cavity on the wall-refined grid of Sec. 4.1 (cell widths
growing geometrically from every wall) against the oracle.

FP64-deterministic layout: volumes, particle states, (sigma g)_max, event
counts and wall tallies equal the oracle's over 10 steps (relative 1e-12);
the higher-order terms and Kn_GLL from the oracle's sampled fields (the
three-point formula on unequal spacing) to relative 1e-11; the particle
modification over two rounds with steps in between.  FP32 layout: a gas at
rest stays uniform in cells whose areas differ 25-fold (replicas, 3-SE
bound), the particle count is conserved, and the modification follows the
oracle given the GPU's own particles.  The 2D synthetic solve on the refined
grid: the oracle's converged solution (smooth states, and sampled cavity
fields with their HoT), one DIG iteration, and the paper's 100 x 100 grid
with a first cell of 0.001, whose solution zeroes the oracle's residual.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2501_10965_gb300 import workloads as W
from stats3se import assert_within_3se

pytestmark = pytest.mark.gpu

KEYS = ("x", "y", "vx", "vy", "vz", "ir")
NX, NY = 14, 12


def _gpu(cfg):
    from paper_2501_10965_gb300 import dsmc
    return dsmc.Dsmc(cfg)


def _np(p):
    return {k: v.cpu().numpy() for k, v in p.items()}


def _compare_states(g, o, rtol=1e-12, what=""):
    assert len(g["x"]) == len(o["x"]), f"{what}: particle count {len(g['x'])} vs {len(o['x'])}"
    assert np.array_equal(g["cell"], o["cell"]), f"{what}: cell order differs"
    for k in KEYS:
        err = np.abs(g[k] - o[k]) / np.maximum(np.abs(o[k]), 1.0)
        i = int(np.argmax(err)) if len(err) else 0
        assert len(err) == 0 or err.max() <= rtol, f"{what}: {k} differs at {i}: {g[k][i]!r} vs {o[k][i]!r}"


def _cfg(**kw):
    base = dict(nx=NX, ny=NY, ppc=30, kn=0.05, dx_min=0.02, lid=0.5, precision="fp64")
    base.update(kw)
    return W.cavity_2d_refined(**base)


def test_refined_cavity_steps_match_oracle_fp64():
    cfg = _cfg()
    g, o = _gpu(cfg), oracle.OracleSim(cfg)
    v = o.volumes()
    np.testing.assert_allclose(g.volumes(), v, rtol=1e-14)
    assert v.max() / v.min() > 10.0
    _compare_states(_np(g.get_particles()), o.particles(), what="init")
    for k in range(10):
        g.dsmc_step(1)
        o.step(1)
        _compare_states(_np(g.get_particles()), o.particles(), what=f"step {k}")
    assert np.allclose(g.sgmax().cpu().numpy(), o.sgmax(), rtol=1e-12, atol=0)
    gs, os_ = g.stats(), o.stats()
    for key in ("n_cand", "n_coll", "n_clip", "n_inel", "n_hits", "n_maxhit"):
        assert gs[key] == os_[key], (key, gs[key], os_[key])
    assert gs["n_hits"] > 0 and gs["n_coll"] > 0
    np.testing.assert_allclose(np.array(g.wall_tally()), o.wall_tally(), rtol=1e-11, atol=1e-12)


def _oracle_fields(cfg, steps=60, sample=200):
    from oracle.fields import fields_from_sums
    o = oracle.OracleSim(cfg)
    o.step(steps)
    o.reset_accumulators()
    o.step(sample, sample=True)
    c = o.constants()
    return fields_from_sums(o.accumulators(), o.nsamples, c["fnum"], o.volumes(), 2.0)


def test_hot_kngll_on_refined_box_matches_oracle():
    from oracle.fields import hot_kngll
    cfg = _cfg()
    F = _oracle_fields(cfg)
    _, kn_o, _ = hot_kngll(F, dict(cfg, kn_ref=0.0))
    cfg = dict(cfg, kn_ref=float(np.nanmedian(kn_o)) * 1.0000001)
    hot_o, kn_o, mask_o = hot_kngll(F, cfg)
    g = _gpu(cfg)
    hot_g, kn_g, mask_g = [t.cpu().numpy() for t in g.dsmc_hot(torch.tensor(F, device="cuda"))]
    assert 0 < mask_o.sum() < len(mask_o) and np.isfinite(kn_o).sum() > 0.95 * len(kn_o)
    assert np.allclose(kn_g, kn_o, rtol=1e-12, atol=0.0, equal_nan=True)
    assert np.array_equal(mask_g.astype(bool), mask_o)
    scale = np.maximum(np.abs(hot_o).max(0), 1e-300)
    assert (np.abs(hot_g - hot_o) / scale).max() <= 1e-11


def _targets(nc, rng):
    t = np.zeros((nc, 6))
    t[:, 0] = 0.6 + 0.8 * rng.random(nc)
    t[:, 1:4] = 0.3 * rng.standard_normal((nc, 3))
    t[:, 4] = 0.8 + 0.5 * rng.random(nc)
    t[:, 5] = 0.7 + 0.5 * rng.random(nc)
    t[NX + 3, 0] = 0.0  # empty a cell; the second modification refills it
    return t


def test_dig_correct_on_refined_box_matches_oracle_fp64():
    """Sec. 3.2 with per-cell volumes (target counts Iround(rho V_cell / F))
    and new particles uniform in their cell's rectangle."""
    cfg = _cfg()
    g, o = _gpu(cfg), oracle.OracleSim(cfg)
    g.dsmc_step(3)
    o.step(3)
    t = _targets(NX * NY, np.random.default_rng(3))
    for rep in range(2):
        g.dig_correct(torch.tensor(t, device="cuda"))
        assert o.dig_correct(t) == 0
        _compare_states(_np(g.get_particles()), o.particles(), what=f"dig {rep}")
        g.dsmc_step(2)
        o.step(2)
        _compare_states(_np(g.get_particles()), o.particles(), what=f"dig {rep} + 2 steps")
        t[NX + 3, 0] = 1.2


def test_dig_correct_on_refined_box_fp32_follows_the_oracle():
    cfg = _cfg(precision="fp32")
    g = _gpu(cfg)
    g.dsmc_step(4)
    t = _targets(NX * NY, np.random.default_rng(4))
    p = _np(g.get_particles())
    o = oracle.OracleSim(dict(cfg, precision="fp64"))
    o.set_particles({k: p[k] for k in KEYS})
    assert np.array_equal(o.particles()["cell"], p["cell"])
    o.set_step(0, dig_iter=0)
    g.dig_correct(torch.tensor(t, device="cuda"))
    assert o.dig_correct(t) == 0
    a, b = _np(g.get_particles()), o.particles()
    assert np.array_equal(a["cell"], b["cell"])
    for k in KEYS:
        err = np.abs(a[k] - b[k]) / np.maximum(np.abs(b[k]), 1.0)
        assert err.max() <= 1e-6, (k, err.max())


def test_refined_fp32_gas_at_rest_stays_uniform():
    """No lid, walls at the gas temperature, 8 replicas of a 40 x 40 grid
    whose corner cells are 25 times smaller than the middle ones: the
    particle count is conserved, and the density of each quartile of cell
    areas, the domain's temperature and the collision rate N nu dt / 2 stay
    at their equilibrium values within the replicas' 3-SE bound (3 % for the
    rate)."""
    nrep, rels, temps, ratios = 8, [], [], []
    for rep in range(nrep):
        cfg = _cfg(nx=40, ny=40, ppc=40, lid=0.0, dx_min=0.005, precision="fp32", seed=rep)
        g = _gpu(cfg)
        c = g.constants()
        n0 = g.num_particles()
        vol = g.volumes()
        assert vol.max() / vol.min() > 20.0
        cls = np.digitize(vol, np.quantile(vol, [0.25, 0.5, 0.75]))
        g.dsmc_step(100)
        g.dsmc_sample(reset=True)
        c0, nsum, tsnap = g.stats()["n_coll"], 0, []
        for blk in range(40):
            nsum += 10 * g.num_particles()
            g.dsmc_step(10, sample=True)
            if blk % 4 == 3:
                pp = _np(g.get_particles())
                tt = np.mean(pp["vx"] ** 2 + pp["vy"] ** 2 + pp["vz"] ** 2) / 3.0
                tsnap.append((3.0 * tt + 2.0 * np.mean(pp["ir"])) / 5.0)
        assert g.num_particles() == n0
        f = g.dsmc_sample(reset=True).cpu().numpy()
        rels.append([np.sum((f[:, 0] * vol)[cls == k]) / np.sum(vol[cls == k]) for k in range(4)])
        temps.append(np.mean(tsnap))
        ratios.append((g.stats()["n_coll"] - c0) / (0.5 * c["k_visc"] / c["mu_ref"] * cfg["dt"] * nsum))
    assert abs(np.mean(ratios) - 1.0) < 0.03, ratios
    assert_within_3se(np.array(rels) - 1.0, what="density by cell-area quartile")
    assert_within_3se(np.array(temps) - 1.0, what="temperature")


# ---------------------------------------------------------------------------
# the 2D synthetic solve on the wall-refined grid
# ---------------------------------------------------------------------------

def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _smooth_refined(cfg, seed=0, hot_amp=1e-3):
    from oracle.fields import F_RHO, F_TR, F_TT, F_U, box_edges
    nx, ny = int(cfg["nx"]), int(cfg["ny"])
    ex, ey = box_edges(nx, cfg["lx"], cfg["stretch"]), box_edges(ny, cfg["ly"], cfg["stretch"])
    X, Y = np.meshgrid(0.5 * (ex[:-1] + ex[1:]), 0.5 * (ey[:-1] + ey[1:]))
    d = np.zeros((ny, nx, 18))
    d[..., F_RHO] = 1 + 0.02 * np.cos(np.pi * X)
    d[..., F_U] = 0.05 * np.sin(np.pi * X) * np.cos(np.pi * Y) * np.sin(np.pi * Y)
    d[..., F_U + 1] = -0.05 * np.cos(np.pi * X) * np.sin(np.pi * X) * np.sin(np.pi * Y)
    d[..., F_U + 2] = 0.003
    d[..., F_TT] = 1 + 0.01 * Y
    d[..., F_TR] = 1 + 0.012 * Y
    return d.reshape(nx * ny, 18), hot_amp * np.random.default_rng(seed).standard_normal((nx * ny, 12))


def _scfg(nx, ny, **kw):
    base = dict(nx=nx, ny=ny, ppc=4, kn=0.05, dx_min=0.04, precision="fp64", synth2d=True, synth_tol=1e-12, n_m=50)
    base.update(kw)
    return W.cavity_2d_refined(**base)


@pytest.mark.parametrize("nx,ny", [(10, 8), (7, 11)])
def test_synth_solve_on_refined_box_matches_oracle(nx, ny):
    from oracle import synth2d
    cfg = _scfg(nx, ny)
    d, h = _smooth_refined(cfg)
    g = _gpu(cfg)
    out_g, it_g, res_g = g.synth_solve(_dev(d), _dev(h))
    out_o, it_o, res_o = synth2d.synth_solve_2d(d, h, cfg, tol=1e-12, max_iter=50)
    assert res_g < 1e-11 and res_o < 1e-11, (res_g, res_o)
    assert abs(it_g - it_o) <= 1, (it_g, it_o)
    np.testing.assert_allclose(out_g.cpu().numpy(), out_o, rtol=0, atol=1e-10)


def test_synth_solve_of_sampled_refined_cavity_matches_oracle():
    """Fields sampled by the GPU on the refined cavity with their HoT and
    Kn_GLL mask, solved on both sides; the solution keeps the sampled mass
    sum rho V and the wall cells' u, T."""
    from oracle import synth2d
    from oracle.fields import F_RHO, F_TR, F_TT, F_U
    nx, ny = 14, 11
    cfg = _scfg(nx, ny, ppc=60, kn=0.1, lid=0.5)
    g = _gpu(cfg)
    g.dsmc_step(150)
    g.dsmc_step(150, sample=True)
    f = g.dsmc_sample(reset=False)
    hot, _, mask = g.dsmc_hot(f)
    out_g, it_g, res_g = g.synth_solve(f, hot)
    F, H = f.cpu().numpy(), hot.cpu().numpy()
    out_o, it_o, res_o = synth2d.synth_solve_2d(F, H, cfg, tol=1e-12, max_iter=50)
    assert res_g < 1e-10 and res_o < 1e-10, (res_g, res_o)
    np.testing.assert_allclose(out_g.cpu().numpy(), out_o, rtol=0, atol=1e-9)
    O, V = out_g.cpu().numpy(), g.volumes()
    assert abs((O[:, 0] * V).sum() / (F[:, F_RHO] * V).sum() - 1.0) < 1e-12
    ring = np.zeros((ny, nx), bool)
    ring[0, :] = ring[-1, :] = ring[:, 0] = ring[:, -1] = True
    ring = ring.ravel()
    for k, col in ((1, F_U), (2, F_U + 1), (4, F_TT), (5, F_TR)):
        np.testing.assert_allclose(O[ring, k], F[ring, col], rtol=0, atol=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_dig_iteration_on_refined_cavity(precision):
    """One DIG iteration on the refined cavity (steps, sample, HoT, the 2D
    synthetic solve, the modification): the particles number the sum of
    Iround(rho V_c / F) over cells of their own volumes (within 6 sigma of
    the stochastic rounding), and the target keeps the sampled mass."""
    from paper_2501_10965_gb300 import dig
    cfg = _scfg(12, 10, ppc=50, kn=0.05, synth_tol=1e-8, precision=precision)
    g = _gpu(cfg)
    g.dsmc_step(100)
    r = dig.dig_iteration(g, 100)
    assert r["synth_status"] == 0 and r["synth_resid"] < 1e-8
    t = r["target"].cpu().numpy()
    V, c = g.volumes(), g.constants()
    m = t[:, 0] * V / c["fnum"]
    frac = m - np.floor(m)
    sd = np.sqrt(np.sum(frac * (1.0 - frac)))
    assert abs(g.num_particles() - m.sum()) <= 6.0 * sd + 1.0, (g.num_particles(), m.sum(), sd)
    assert abs((t[:, 0] * V).sum() / (r["fields"][:, 0].cpu().numpy() * V).sum() - 1.0) < 1e-8


def test_paper_refined_grid_solution_satisfies_the_oracle_equations():
    """Sec. 4.1's DIG grid: 100 x 100 cells, first cell 0.001 at every wall
    (50 000 unknowns; the oracle's Newton solver is too slow here): the GPU's
    converged solution zeroes the oracle's residual at every cell (1e-9),
    keeps the sampled mass sum rho V and the wall and corner cells."""
    from oracle import synth2d
    from oracle.fields import F_RHO, F_TR, F_TT, F_U
    nx = ny = 100
    cfg = _scfg(nx, ny, ppc=2, dx_min=0.001, synth_tol=1e-10)
    d, h = _smooth_refined(cfg, seed=5)
    g = _gpu(cfg)
    out, it, res = g.synth_solve(_dev(d), _dev(h))
    assert res < 1e-9 and it <= 12
    O, V = out.cpu().numpy(), g.volumes()
    x = np.concatenate([O[:, 0], O[:, 1], O[:, 2], O[:, 4], O[:, 5]])
    R = synth2d.residual(x, d, h, cfg)
    assert np.max(np.abs(R)) < 1e-9, np.max(np.abs(R))
    assert abs((O[:, 0] * V).sum() / (d[:, F_RHO] * V).sum() - 1.0) < 1e-12
    ring = np.zeros((ny, nx), bool)
    ring[0, :] = ring[-1, :] = ring[:, 0] = ring[:, -1] = True
    ring = ring.ravel()
    for k, col in ((1, F_U), (2, F_U + 1), (4, F_TT), (5, F_TR)):
        np.testing.assert_allclose(O[ring, k], d[ring, col], rtol=0, atol=1e-12)
    corners = [0, nx - 1, nx * (ny - 1), nx * ny - 1]
    np.testing.assert_allclose(O[corners, 0], d[corners, F_RHO], rtol=0, atol=1e-12)
