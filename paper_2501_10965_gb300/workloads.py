"""Seeded synthetic workloads shaped like the paper's cases.

This module only states inputs: geometry, gas constants, wall states, initial
state, time step and seed, as plain numbers.  It holds none of the method's
arithmetic, so that both the CUDA library and the independent CPU oracle can be
driven from the same description.

Units follow Sec. 2 of the paper: lengths in L0, density in rho0, temperature
in T0 and speed in sqrt(R T0).  For the N2-like gas, R = k/m with
m = 4.65e-26 kg (Sec. 4), so sqrt(R * 273 K) = 284.7 m/s.

The time step follows the rule dt = CFL * dx_min / sqrt(T_max): a particle at
the thermal speed crosses at most a fraction CFL of a cell per step; every
workload below also keeps dt under the mean collision time, as Sec. 4 asks.
"""
from __future__ import annotations

import copy
import math

K_BOLTZMANN = 1.380649e-23
N2_MASS = 4.65e-26            # kg, Sec. 4
T_REF_K = 273.0               # K, reference temperature of the 1D and cavity cases
R_N2 = K_BOLTZMANN / N2_MASS  # J/(kg K)
SPEED_REF = math.sqrt(R_N2 * T_REF_K)  # m/s


def _wall(kind="diffuse", T=1.0, u=(0.0, 0.0, 0.0)):
    return {"kind": kind, "T": float(T), "u": tuple(float(v) for v in u)}


def base_config(**kw) -> dict:
    """Defaults: N2-like gas (omega 0.74, alpha 1, d_r 2, Z_rot 5), unit box."""
    cfg = {
        "dim": 1, "nx": 100, "ny": 1, "ppc": 100,
        "lx": 1.0, "ly": 1.0,
        "kn": 0.1, "omega": 0.74, "alpha": 1.0, "z_rot": 5.0, "d_r": 2.0,
        # heat-flux relaxation matrix A (A_tt, A_tr, A_rt, A_rr); the paper
        # prints no values, these give kappa_t = 15/4 mu, kappa_r = 1.32 mu
        "a_matrix": (2.0 / 3.0, 0.0, 0.0, 1.0 / 1.32),
        "dt": 1e-3,
        "walls": [_wall(), _wall(), _wall(), _wall()],
        "init_rho": 1.0, "init_tt": 1.0, "init_tr": 1.0, "init_u": (0.0, 0.0, 0.0),
        "collisions": True,
        "precision": "fp64",
        "seed": 0,
        "capacity": 0,
        "n_s": 100, "n_m": 2000,
        "kn_ref": 0.01,
        "synth_tol": 1e-5,
        "bin_slack": 2.0,
        # mesh "box": the Cartesian box above; "annulus": r_in <= r <= r_out
        # around a cylinder (nx angular x ny radial cells, radial widths
        # growing by `stretch` per ring), wall 0 the cylinder, freestream
        # (fs_rho, fs_t, fs_u) entering through the outer circle;
        # "refined": the box with cell widths growing by `stretch` from both
        # walls of each axis to the middle
        "mesh": "box",
        "r_in": 0.5, "r_out": 5.5, "stretch": 1.0,
        "fs_rho": 1.0, "fs_t": 1.0, "fs_u": (0.0, 0.0, 0.0),
    }
    cfg.update(kw)
    return cfg


def fourier_1d(**kw) -> dict:
    """1D planar Fourier heat transfer: 100 cells x 100 particles, walls at
    273 K and 373 K, uniform initial Maxwellian at 323 K, Kn 0.1, FP64,
    Philox seed 0 (4000 steps in the full run)."""
    t_hot = 373.0 / T_REF_K
    t0 = 323.0 / T_REF_K
    dx = 1.0 / 100
    cfg = base_config(dim=1, nx=100, ppc=100, kn=0.1, z_rot=5.0,
                      walls=[_wall(T=1.0), _wall(T=t_hot), _wall(), _wall()],
                      init_tt=t0, init_tr=t0, precision="fp64", seed=0,
                      dt=0.3 * dx / math.sqrt(t_hot), n_s=100)
    cfg.update(kw)
    return cfg


def couette_1d(kn: float = 0.1, **kw) -> dict:
    """1D Couette flow: 200 cells x 200 particles, walls moving at -/+100 m/s
    (tangential, y) at 273 K; DIG every 50 steps; FP32 particles."""
    uw = 100.0 / SPEED_REF
    dx = 1.0 / 200
    cfg = base_config(dim=1, nx=200, ppc=200, kn=kn, z_rot=5.0,
                      walls=[_wall(T=1.0, u=(0.0, -uw, 0.0)), _wall(T=1.0, u=(0.0, uw, 0.0)),
                             _wall(), _wall()],
                      precision="fp32", dt=0.3 * dx, n_s=50)
    cfg.update(kw)
    return cfg


def cavity_2d(nx: int = 100, ny: int = 100, ppc: int = 50, kn: float = 0.01,
              lid_mps: float = 50.0, lx: float = 1.0, ly: float = 1.0, **kw) -> dict:
    """2D lid-driven cavity: diffuse walls at 273 K, the top wall (y = ly)
    slides along +x.  Defaults: 100 x 100 cells, 50 particles per cell,
    Kn 0.01, lid 50 m/s, Kn_ref 0.05, FP32."""
    ulid = lid_mps / SPEED_REF
    dxm = min(lx / nx, ly / ny)
    cfg = base_config(dim=2, nx=nx, ny=ny, ppc=ppc, lx=lx, ly=ly, kn=kn, z_rot=5.0,
                      walls=[_wall(), _wall(), _wall(), _wall(u=(ulid, 0.0, 0.0))],
                      precision="fp32", dt=0.3 * dxm, kn_ref=0.05, n_s=100)
    cfg.update(kw)
    return cfg


def cavity_2d_20m(**kw) -> dict:
    """Throughput workload at the cylinder case's scale (400 x 300 cells,
    ~167 particles per cell, 20.0 M particles, Kn 0.01, FP32): a 4:3 cavity
    with square cells and a 50 m/s lid."""
    cfg = cavity_2d(nx=400, ny=300, ppc=167, kn=0.01, lx=4.0 / 3.0, ly=1.0)
    cfg.update(kw)
    return cfg


def radial_stretch(dr1: float, nr: int, span: float) -> float:
    """Ratio q > 1 of consecutive radial widths with first width dr1 and nr
    rings spanning `span`: dr1 (q^nr - 1) / (q - 1) = span (bisection)."""
    if dr1 * nr >= span:
        return 1.0
    lo, hi = 1.0 + 1e-12, 2.0
    while dr1 * (hi ** nr - 1.0) / (hi - 1.0) < span:
        lo, hi = hi, 2.0 * hi
    for _ in range(200):
        q = 0.5 * (lo + hi)
        if dr1 * (q ** nr - 1.0) / (q - 1.0) > span:
            hi = q
        else:
            lo = q
    return 0.5 * (lo + hi)


def cylinder_2d(ntheta: int = 400, nr: int = 300, ppc: int = 167, kn: float = 0.01, mach: float = 5.0,
                t_wall: float = 2.5, r_in: float = 0.5, r_out: float = 5.5, dr1: float | None = None,
                **kw) -> dict:
    """Hypersonic flow past a cylinder of diameter 1 (L0): Mach 5 N2-like
    freestream at 200 K (the temperature unit here), diffuse cylinder wall at
    500 K, annular mesh r in [0.5, 5.5] of ntheta x nr cells whose radial
    widths grow geometrically from dr1 (default 0.2 of the freestream mean
    free path, Kn L0), ~ppc particles per cell on average, FP32.  The gas
    starts as the uniform freestream; the freestream enters through the outer
    circle and particles leave through it."""
    gamma = 7.0 / 5.0
    u_inf = mach * math.sqrt(gamma * 1.0)
    dr1 = 0.2 * kn if dr1 is None else dr1
    q = radial_stretch(dr1, nr, r_out - r_in)
    dr_min = dr1 if q > 1.0 else (r_out - r_in) / nr
    dx_min = min(dr_min, r_in * 2.0 * math.pi / ntheta)
    t_max = max(1.0, t_wall)
    tau = kn * math.sqrt(math.pi / 8.0)
    dt = min(0.3 * dx_min / (u_inf + 3.0 * math.sqrt(t_max)), 0.5 * tau)
    cfg = base_config(dim=2, nx=ntheta, ny=nr, ppc=ppc, kn=kn, z_rot=5.0, mesh="annulus",
                      lx=2.0 * math.pi, ly=r_out - r_in, r_in=r_in, r_out=r_out, stretch=q,
                      walls=[_wall(T=t_wall), _wall(), _wall(), _wall()],
                      init_u=(u_inf, 0.0, 0.0), fs_rho=1.0, fs_t=1.0, fs_u=(u_inf, 0.0, 0.0),
                      precision="fp32", dt=dt, kn_ref=0.05, n_s=100)
    cfg.update(kw)
    return cfg


def refined_stretch(n: int, length: float, d_min: float) -> float:
    """Growth factor q of the wall-refined box whose first cell at each wall
    (of n along an axis of this length, widths proportional to
    q^min(i, n-1-i)) is d_min wide (bisection)."""
    def first(q):
        m = [min(i, n - 1 - i) for i in range(n)]
        return length / sum(q ** k for k in m)
    if first(1.0) <= d_min:
        raise ValueError("refined_stretch: a uniform grid's cells are already at most d_min wide")
    lo, hi = 1.0, 2.0
    while first(hi) > d_min:
        lo, hi = hi, 2.0 * hi
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if first(mid) > d_min:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def cavity_2d_refined(nx: int = 100, ny: int = 100, ppc: int = 50, kn: float = 0.01, dx_min: float = 0.001,
                      lid: float = 50.0 / SPEED_REF, **kw) -> dict:
    """Lid-driven cavity on the wall-refined grid of Sec. 4.1 (the DIG mesh
    of its Kn 0.01 case: 100 x 100 cells, first cell 0.001 at every wall),
    ~ppc particles per cell on average (cell populations follow the cell
    areas), lid at 50 m/s (0.176), diffuse walls at T0, FP32; dt from the
    smallest cell."""
    q = refined_stretch(nx, 1.0, dx_min)
    dt = min(0.3 * dx_min / (lid + 3.0), 0.5 * kn * math.sqrt(math.pi / 8.0))
    cfg = base_config(dim=2, nx=nx, ny=ny, ppc=ppc, kn=kn, mesh="refined", stretch=q, lx=1.0, ly=1.0,
                      walls=[_wall(), _wall(), _wall(), _wall(u=(lid, 0.0, 0.0))],
                      precision="fp32", dt=dt, kn_ref=0.05, n_s=100)
    cfg.update(kw)
    return cfg


def homogeneous_box(ncells: int = 100, ppc: int = 100, kn: float = 0.1, tt: float = 1.0,
                    tr: float = 1.0, dt: float = 2e-3, **kw) -> dict:
    """Spatially homogeneous gas: a 1D box with specular walls, so no wall
    changes the state and every cell is an independent sample."""
    cfg = base_config(dim=1, nx=ncells, ppc=ppc, kn=kn,
                      walls=[_wall("specular"), _wall("specular"), _wall(), _wall()],
                      init_tt=tt, init_tr=tr, dt=dt, precision="fp64")
    cfg.update(kw)
    return cfg


def with_overrides(cfg: dict, **kw) -> dict:
    out = copy.deepcopy(cfg)
    out.update(kw)
    return out


def ensemble_1d(ncases: int = 64, seed: int = 0, **kw) -> list:
    """Batched ensemble: `ncases` independent 1D cases drawn with a seeded
    generator: cells uniform in 50..800, particles per cell uniform in 50..200,
    Kn log-uniform in [1e-3, 1], Z_rot in {2, 5, 10}; even cases are Fourier
    (walls at 273 K / 373 K), odd ones Couette (walls at -/+100 m/s, 273 K);
    FP32 particles; case k has Philox seed `seed` + k."""
    import numpy as np
    rng = np.random.default_rng(seed)
    cases = []
    for k in range(ncases):
        nx = int(rng.integers(50, 801))
        ppc = int(rng.integers(50, 201))
        kn = float(10 ** rng.uniform(-3, 0))
        z = float(rng.choice([2.0, 5.0, 10.0]))
        # dt: CFL rule, capped at half the mean free time Kn sqrt(pi/8)
        tau = kn * math.sqrt(math.pi / 8.0)
        if k % 2 == 0:
            c = fourier_1d(nx=nx, ppc=ppc, kn=kn, z_rot=z, precision="fp32",
                           dt=min(0.3 * (1.0 / nx) / math.sqrt(373.0 / T_REF_K), 0.5 * tau))
        else:
            c = couette_1d(kn=kn, nx=nx, ppc=ppc, z_rot=z, dt=min(0.3 * (1.0 / nx), 0.5 * tau))
        c["seed"] = seed + k
        c.update(kw)
        cases.append(c)
    return cases


def replicas(cfg: dict, n: int, seed0: int = 0) -> list:
    """`n` copies of one workload with Philox seeds seed0, seed0 + 1, ..."""
    return [dict(copy.deepcopy(cfg), seed=seed0 + r) for r in range(n)]

def smooth_cavity_state(nx: int, ny: int, seed: int = 0, hot_amp: float = 1e-3, xc=None, yc=None):
    """A smooth recirculating cavity-like state as sampled fields (ncells x
    18: rho 1 + 0.02 cos(pi x), a single vortex of amplitude 0.05 in (u_x,
    u_y), u_z 0.003, T_t 1 + 0.01 y, T_r 1 + 0.012 y) and seeded normal HoT
    of amplitude hot_amp (ncells x 12), at the cell centres xc (nx), yc (ny)
    (default: the uniform grid's), for timing and checking the synthetic
    solve."""
    import numpy as np
    if xc is None:
        xc = (np.arange(nx) + 0.5) / nx
    if yc is None:
        yc = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(np.asarray(xc), np.asarray(yc))
    d = np.zeros((ny, nx, 18))
    d[..., 0] = 1 + 0.02 * np.cos(np.pi * X)
    d[..., 1] = 0.05 * np.sin(np.pi * X) * np.cos(np.pi * Y) * np.sin(np.pi * Y)
    d[..., 2] = -0.05 * np.cos(np.pi * X) * np.sin(np.pi * X) * np.sin(np.pi * Y)
    d[..., 3] = 0.003
    d[..., 4] = 1 + 0.01 * Y
    d[..., 5] = 1 + 0.012 * Y
    h = hot_amp * np.random.default_rng(seed).standard_normal((nx * ny, 12))
    return d.reshape(nx * ny, 18), h
