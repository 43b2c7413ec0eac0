"""GPU parity of the 2D synthetic solve (synth_solve on a 2D box, Sec. 3
step 3) with the oracle's Newton solver (oracle/synth2d.py).

Both sides solve the same discrete equations (finite volumes with the
fourth-difference dissipation, Dirichlet wall cells, fixed corner cells, the
total-mass row) by Newton's method from the sampled fields with a
central-difference Jacobian; the GPU factorises it as a band with partial
pivoting, the oracle with a sparse direct solve.  Converged to a relative
update of 1e-12, the outputs agree to rounding; after a single Newton step
(n_m = 1) they agree to the Jacobian's rounding.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import synth2d
from oracle.fields import F_RHO, F_TR, F_TT, F_U
from paper_2501_10965_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _gpu(cfg):
    from paper_2501_10965_gb300 import dsmc
    return dsmc.Dsmc(cfg)


def _cfg(nx, ny, **kw):
    base = dict(nx=nx, ny=ny, ppc=4, kn=0.05, precision="fp64", synth2d=True, synth_tol=1e-12, n_m=50)
    base.update(kw)
    return W.cavity_2d(**base)


def _smooth(nx, ny, seed=0, hot_amp=1e-3):
    """A recirculating cavity-like state with random HoT (the oracle's pinned
    Newton test uses the same recipe)."""
    n = nx * ny
    X, Y = np.meshgrid((np.arange(nx) + 0.5) / nx, (np.arange(ny) + 0.5) / ny)
    d = np.zeros((ny, nx, 18))
    d[..., F_RHO] = 1 + 0.02 * np.cos(np.pi * X)
    d[..., F_U] = 0.05 * np.sin(np.pi * X) * np.cos(np.pi * Y) * np.sin(np.pi * Y)
    d[..., F_U + 1] = -0.05 * np.cos(np.pi * X) * np.sin(np.pi * X) * np.sin(np.pi * Y)
    d[..., F_U + 2] = 0.003
    d[..., F_TT] = 1 + 0.01 * Y
    d[..., F_TR] = 1 + 0.012 * Y
    h = hot_amp * np.random.default_rng(seed).standard_normal((n, 12))
    return d.reshape(n, 18), h


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


# (10, 8), (16, 5), (24, 20): nx > ny, so the band numbers cells along y
# first; (7, 11): along x first; (24, 20): 2400 unknowns, kl = 204
@pytest.mark.parametrize("nx,ny", [(10, 8), (7, 11), (16, 5), (24, 20)])
def test_converged_solution_matches_oracle(nx, ny):
    cfg = _cfg(nx, ny)
    d, h = _smooth(nx, ny)
    g = _gpu(cfg)
    out_g, it_g, res_g = g.synth_solve(_dev(d), _dev(h))
    out_o, it_o, res_o = synth2d.synth_solve_2d(d, h, cfg, tol=1e-12, max_iter=50)
    assert res_g < 1e-11 and res_o < 1e-11, (res_g, res_o)
    assert abs(it_g - it_o) <= 1, (it_g, it_o)
    np.testing.assert_allclose(out_g.cpu().numpy(), out_o, rtol=0, atol=1e-10)


def test_single_newton_step_matches_oracle():
    """n_m = 1: the first Newton update from the sampled fields (status
    NOT_CONVERGED, outputs written) equals the oracle's first iterate."""
    nx, ny = 12, 9
    cfg = _cfg(nx, ny, n_m=1)
    d, h = _smooth(nx, ny, seed=3, hot_amp=3e-3)
    g = _gpu(cfg)
    out_g, it_g, _ = g.synth_solve(_dev(d), _dev(h), allow_not_converged=True)
    assert g.last_synth_status == -4 and it_g == 1
    out_o, it_o, _ = synth2d.synth_solve_2d(d, h, cfg, tol=1e-12, max_iter=1)
    assert it_o == 1
    o = out_g.cpu().numpy()
    assert np.abs(o - d[:, [F_RHO, F_U, F_U + 1, F_U + 2, F_TT, F_TR]]).max() > 1e-4  # it moved
    np.testing.assert_allclose(o, out_o, rtol=0, atol=1e-10)


@pytest.mark.parametrize("kn", [0.05, 0.1])
def test_sampled_cavity_fields_and_hot_match_oracle(kn):
    """The DIG inputs as they come: fields sampled by the GPU DSMC step on a
    lid-driven cavity and their HoT with the Kn_GLL mask (at Kn 0.1 part of
    the cells keep their HoT), solved on both sides."""
    nx, ny = 14, 11
    cfg = _cfg(nx, ny, ppc=60, kn=kn)
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
    # the solution keeps the sampled total mass and the wall cells' u, T
    O = out_g.cpu().numpy()
    assert abs(O[:, 0].sum() / F[:, F_RHO].sum() - 1.0) < 1e-12
    ring = np.zeros((ny, nx), bool)
    ring[0, :] = ring[-1, :] = ring[:, 0] = ring[:, -1] = True
    ring = ring.ravel()
    for k, col in ((1, F_U), (2, F_U + 1), (4, F_TT), (5, F_TR)):
        np.testing.assert_allclose(O[ring, k], F[ring, col], rtol=0, atol=1e-12)


def test_without_synth2d_workspace_is_rejected():
    from paper_2501_10965_gb300 import dsmc
    cfg = _cfg(8, 6, synth2d=False)
    g = _gpu(cfg)
    d, h = _smooth(8, 6)
    with pytest.raises(dsmc.DsmcError) as e:
        g.synth_solve(_dev(d), _dev(h))
    assert e.value.code == -1


def test_dig_iteration_on_a_cavity():
    """One DIG iteration on a 2D cavity (steps, sample, HoT, 2D synthetic
    solve, particle modification): the particles afterwards number the sum
    over cells of Iround(rho V / F) (stochastic rounding: within 6 sigma of
    the sum of rho V / F), and the target keeps the sampled mass."""
    from paper_2501_10965_gb300 import dig
    nx, ny = 12, 10
    cfg = _cfg(nx, ny, ppc=50, kn=0.05, synth_tol=1e-8)
    g = _gpu(cfg)
    g.dsmc_step(100)
    r = dig.dig_iteration(g, 100)
    assert r["synth_status"] == 0 and r["synth_resid"] < 1e-8
    t = r["target"].cpu().numpy()
    c = g.constants()
    m = t[:, 0] * c["vcell"] / c["fnum"]
    frac = m - np.floor(m)
    sd = np.sqrt(np.sum(frac * (1.0 - frac)))
    assert abs(g.num_particles() - m.sum()) <= 6.0 * sd + 1.0, (g.num_particles(), m.sum(), sd)
    assert abs(t[:, 0].sum() / r["fields"][:, 0].sum().item() - 1.0) < 1e-8


@pytest.mark.parametrize("nx,ny", [(100, 100), (60, 50), (130, 128)])
def test_full_size_cavity_solution_satisfies_the_oracle_equations(nx, ny):
    """The paper's cavity grid, 100 x 100 cells (50 000 unknowns), where the
    oracle's Newton solver is too slow to run: the GPU's converged solution
    makes the oracle's residual of the discrete equations vanish at every
    cell (to 1e-9, against O(100) terms), keeps the sampled total mass, and
    keeps the wall cells' u, T and the corner cells' whole state.  (60 x 50:
    panels of 536 rows, two rows of each thread in the panel factorisation's
    registers; 100 x 100: 1 036 rows, three; 130 x 128: windows of 41
    blocks of 32 rows, more than one pass of a substitution group's warps
    over a CTA's blocks.)"""
    cfg = _cfg(nx, ny, ppc=2, synth_tol=1e-10)
    d, h = _smooth(nx, ny, seed=5)
    g = _gpu(cfg)
    out, it, res = g.synth_solve(_dev(d), _dev(h))
    assert res < 1e-9 and it <= 10
    O = out.cpu().numpy()
    x = np.concatenate([O[:, 0], O[:, 1], O[:, 2], O[:, 4], O[:, 5]])
    R = synth2d.residual(x, d, h, cfg)
    assert np.max(np.abs(R)) < 1e-9, np.max(np.abs(R))
    assert abs(O[:, 0].sum() / d[:, F_RHO].sum() - 1.0) < 1e-12
    ring = np.zeros((ny, nx), bool)
    ring[0, :] = ring[-1, :] = ring[:, 0] = ring[:, -1] = True
    ring = ring.ravel()
    for k, col in ((1, F_U), (2, F_U + 1), (4, F_TT), (5, F_TR)):
        np.testing.assert_allclose(O[ring, k], d[ring, col], rtol=0, atol=1e-12)
    corners = [0, nx - 1, nx * (ny - 1), nx * ny - 1]
    np.testing.assert_allclose(O[corners, 0], d[corners, F_RHO], rtol=0, atol=1e-12)


def test_factorisation_reused_across_solves_gives_the_same_solution():
    """dsmc_synth_reuse: a solve of another state that starts from the
    previous solve's factorisation converges to the solution a fresh solve
    finds (to the tolerance); a handle without the 2D solve refuses it."""
    nx, ny = 24, 20
    cfg = _cfg(nx, ny, synth_tol=1e-10)
    d1, h1 = _smooth(nx, ny, seed=1)
    d2, h2 = _smooth(nx, ny, seed=2, hot_amp=2e-3)
    g = _gpu(cfg)
    g.synth_reuse(True)
    g.synth_solve(_dev(d1), _dev(h1))
    out_r, it_r, res_r = g.synth_solve(_dev(d2), _dev(h2))
    out_f, it_f, res_f = _gpu(cfg).synth_solve(_dev(d2), _dev(h2))
    assert res_r < 1e-9 and res_f < 1e-9
    np.testing.assert_allclose(out_r.cpu().numpy(), out_f.cpu().numpy(), rtol=0, atol=1e-8)
    # and Newton from the previous solution as well (bit 1)
    gw = _gpu(cfg)
    gw.synth_reuse(True, warm=True)
    gw.synth_solve(_dev(d1), _dev(h1))
    out_w, it_w, res_w = gw.synth_solve(_dev(d2), _dev(h2))
    assert res_w < 1e-9
    np.testing.assert_allclose(out_w.cpu().numpy(), out_f.cpu().numpy(), rtol=0, atol=1e-8)
    with pytest.raises(RuntimeError):
        _gpu(W.fourier_1d(precision="fp64")).synth_reuse(True)
