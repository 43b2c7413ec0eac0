"""Independent CPU oracle for the DIG / polyatomic DSMC hot path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``; never by the product path.  It
shares no code with the CUDA library.

* ``OracleSim``      -- particle stages in plain C, FP64 (dsmc_oracle.c)
* ``fields``         -- Eq. (DSMC_macroscopic) moments, Eq. (ns_constitutive),
                        Eq. (hot_constitutive), Eq. (Kn_GLL) in numpy
* ``synth1d``        -- steady 1D synthetic equations, Eq. (macroscopic_equation),
                        solved by Newton's method
"""
from __future__ import annotations

import ctypes
import numpy as np

from . import build as _build

_lib = None

OR_TAGS = {"init": 1, "wall": 2, "ntc": 3, "coll": 4, "dig_n": 5, "dig_sel": 6, "dig_pos": 7, "inj": 8}


class OrConfig(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("ppc", ctypes.c_int32),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("kn", ctypes.c_double), ("omega", ctypes.c_double), ("alpha", ctypes.c_double),
        ("z_rot", ctypes.c_double), ("d_r", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("wall_kind", ctypes.c_int32 * 4),
        ("wall_t", ctypes.c_double * 4),
        ("wall_u", (ctypes.c_double * 3) * 4),
        ("init_rho", ctypes.c_double), ("init_tt", ctypes.c_double), ("init_tr", ctypes.c_double),
        ("init_u", ctypes.c_double * 3),
        ("collisions", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("capacity", ctypes.c_int64),
        ("mesh", ctypes.c_int32), ("pad1", ctypes.c_int32),
        ("r_in", ctypes.c_double), ("r_out", ctypes.c_double), ("stretch", ctypes.c_double),
        ("fs_rho", ctypes.c_double), ("fs_t", ctypes.c_double), ("fs_u", ctypes.c_double * 3),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        L.or_create.argtypes = [ctypes.POINTER(OrConfig), ctypes.POINTER(P)]
        L.or_create.restype = ctypes.c_int
        L.or_destroy.argtypes = [P]
        for name in ("or_move", "or_sort", "or_collide", "or_sample", "or_reset_acc"):
            getattr(L, name).argtypes = [P]
            getattr(L, name).restype = None
        L.or_step.argtypes = [P, ctypes.c_int, ctypes.c_int]
        L.or_num_particles.argtypes = [P]
        L.or_num_particles.restype = ctypes.c_int64
        L.or_num_cells.argtypes = [P]
        L.or_num_cells.restype = ctypes.c_int
        L.or_get_step.argtypes = [P]
        L.or_get_step.restype = ctypes.c_uint32
        L.or_get_nsamples.argtypes = [P]
        L.or_get_nsamples.restype = ctypes.c_int64
        L.or_get_particles.argtypes = [P] + [P] * 7
        L.or_get_start.argtypes = [P, P]
        L.or_set_particles.argtypes = [P, ctypes.c_int64] + [P] * 6
        L.or_set_particles.restype = ctypes.c_int
        L.or_get_acc.argtypes = [P, P]
        L.or_get_sgmax.argtypes = [P, P]
        L.or_set_sgmax.argtypes = [P, P]
        L.or_set_step.argtypes = [P, ctypes.c_uint32, ctypes.c_uint32]
        L.or_get_stats.argtypes = [P, P]
        L.or_get_wall.argtypes = [P, P]
        L.or_constants.argtypes = [P, P]
        L.or_dig_correct.argtypes = [P, P]
        L.or_dig_correct.restype = ctypes.c_int
        L.or_philox.argtypes = [ctypes.c_uint32] * 6 + [P]
        L.or_uniform.argtypes = [ctypes.c_uint64] + [ctypes.c_uint32] * 5
        L.or_uniform.restype = ctypes.c_double
        L.or_iround_pub.argtypes = [ctypes.c_double, ctypes.c_double]
        L.or_iround_pub.restype = ctypes.c_int64
        for name in ("or_inflow_ginf_pub",):
            getattr(L, name).argtypes = [ctypes.c_double]
            getattr(L, name).restype = ctypes.c_double
        L.or_inflow_speed_pub.argtypes = [ctypes.c_double, ctypes.c_double]
        L.or_inflow_speed_pub.restype = ctypes.c_double
        L.or_bl_fraction_pub.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_uint64] + [ctypes.c_uint32] * 3 + [
            ctypes.c_double, ctypes.c_uint32]
        L.or_bl_fraction_pub.restype = ctypes.c_double
        L.or_scatter_pub.argtypes = [ctypes.c_double] * 7 + [P]
        L.or_scatter_pub.restype = None
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def philox_block(c0, c1, c2, c3, k0, k1) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    lib().or_philox(c0, c1, c2, c3, k0, k1, _ptr(out))
    return out


def inflow_speed(s: float, u: float) -> float:
    """Scaled inward normal speed z = v_n / sqrt(2T) of an entering particle
    whose CDF value is u (speed ratio s of the normal drift)."""
    return lib().or_inflow_speed_pub(s, u)


def inflow_ginf(s: float) -> float:
    return lib().or_inflow_ginf_pub(s)


def bl_fraction(omega: float, d_r: float, seed: int, k: int, cell: int, step: int, u: float,
                jx: int = 2048) -> float:
    """Fraction of E_c kept as rotational energy in one Borgnakke-Larsen
    exchange of candidate k of (cell, step), main uniform u (Beta(d_r/2,
    5/2 - omega))."""
    return lib().or_bl_fraction_pub(omega, d_r, seed, k, cell, step, u, jx)


def scatter(alpha: float, g, gn: float, u: float, v: float) -> np.ndarray:
    """Half the post-collision relative velocity for the pre-collision
    relative velocity g, new magnitude gn and the two scattering uniforms."""
    out = np.zeros(3)
    lib().or_scatter_pub(alpha, float(g[0]), float(g[1]), float(g[2]), gn, u, v, _ptr(out))
    return out


def uniform(seed, tag, c0, c1, c2, j) -> float:
    return lib().or_uniform(seed, tag, c0, c1, c2, j)


def iround(x: float, u: float) -> int:
    return int(lib().or_iround_pub(x, u))


def make_config(cfg: dict) -> OrConfig:
    c = OrConfig()
    c.dim, c.nx, c.ny, c.ppc = int(cfg["dim"]), int(cfg["nx"]), int(cfg.get("ny", 1)), int(cfg["ppc"])
    c.lx, c.ly = float(cfg["lx"]), float(cfg.get("ly", 1.0))
    c.kn, c.omega, c.alpha = float(cfg["kn"]), float(cfg["omega"]), float(cfg["alpha"])
    c.z_rot, c.d_r, c.dt = float(cfg["z_rot"]), float(cfg["d_r"]), float(cfg["dt"])
    for w, wall in enumerate(cfg["walls"][:4]):
        c.wall_kind[w] = 0 if wall["kind"] == "diffuse" else 1
        c.wall_t[w] = float(wall["T"])
        for k in range(3):
            c.wall_u[w][k] = float(wall["u"][k])
    c.init_rho, c.init_tt, c.init_tr = float(cfg["init_rho"]), float(cfg["init_tt"]), float(cfg["init_tr"])
    for k in range(3):
        c.init_u[k] = float(cfg["init_u"][k])
    c.collisions = 1 if cfg.get("collisions", True) else 0
    c.seed = int(cfg.get("seed", 0))
    c.capacity = int(cfg.get("capacity", 0) or 0)
    c.mesh = {"box": 0, "annulus": 1, "refined": 2}[cfg.get("mesh", "box")]
    c.r_in, c.r_out = float(cfg.get("r_in", 0.5)), float(cfg.get("r_out", 5.5))
    c.stretch = float(cfg.get("stretch", 1.0))
    c.fs_rho, c.fs_t = float(cfg.get("fs_rho", 1.0)), float(cfg.get("fs_t", 1.0))
    for k in range(3):
        c.fs_u[k] = float(cfg.get("fs_u", (0.0, 0.0, 0.0))[k])
    return c


class OracleSim:
    """The oracle's particle system (FP64, compact cell-sorted layout)."""

    NMOM = 17

    def __init__(self, cfg: dict):
        self.cfg = dict(cfg)
        self._c = make_config(cfg)
        h = ctypes.c_void_p()
        rc = lib().or_create(ctypes.byref(self._c), ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"or_create failed: {rc}")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_destroy(self._h)
            self._h = None

    # --- stages -------------------------------------------------------------
    def move(self):
        lib().or_move(self._h)

    def sort(self):
        lib().or_sort(self._h)

    def collide(self):
        lib().or_collide(self._h)

    def sample(self):
        lib().or_sample(self._h)

    def step(self, nsteps: int = 1, sample: bool = False):
        lib().or_step(self._h, int(nsteps), 1 if sample else 0)

    def dig_correct(self, target: np.ndarray) -> int:
        t = np.ascontiguousarray(target, dtype=np.float64).reshape(self.ncells, 6)
        return lib().or_dig_correct(self._h, _ptr(t))

    # --- state --------------------------------------------------------------
    @property
    def n(self) -> int:
        return int(lib().or_num_particles(self._h))

    @property
    def ncells(self) -> int:
        return int(lib().or_num_cells(self._h))

    @property
    def step_index(self) -> int:
        return int(lib().or_get_step(self._h))

    @property
    def nsamples(self) -> int:
        return int(lib().or_get_nsamples(self._h))

    def particles(self) -> dict:
        n = self.n
        arrs = {k: np.zeros(n, np.float64) for k in ("x", "y", "vx", "vy", "vz", "ir")}
        cell = np.zeros(n, np.int32)
        lib().or_get_particles(self._h, *[_ptr(arrs[k]) for k in ("x", "y", "vx", "vy", "vz", "ir")], _ptr(cell))
        arrs["cell"] = cell
        return arrs

    def set_particles(self, p: dict):
        n = len(p["x"])
        a = {k: np.ascontiguousarray(p.get(k, np.zeros(n)), dtype=np.float64) for k in ("x", "y", "vx", "vy", "vz", "ir")}
        rc = lib().or_set_particles(self._h, n, *[_ptr(a[k]) for k in ("x", "y", "vx", "vy", "vz", "ir")])
        if rc != 0:
            raise ValueError(f"or_set_particles failed: {rc}")

    def start(self) -> np.ndarray:
        out = np.zeros(self.ncells + 1, np.int64)
        lib().or_get_start(self._h, _ptr(out))
        return out

    def accumulators(self) -> np.ndarray:
        out = np.zeros((self.ncells, self.NMOM), np.float64)
        lib().or_get_acc(self._h, _ptr(out))
        return out

    def reset_accumulators(self):
        lib().or_reset_acc(self._h)

    def sgmax(self) -> np.ndarray:
        out = np.zeros(self.ncells, np.float64)
        lib().or_get_sgmax(self._h, _ptr(out))
        return out

    def set_sgmax(self, v: np.ndarray):
        v = np.ascontiguousarray(v, dtype=np.float64)
        lib().or_set_sgmax(self._h, _ptr(v))

    def set_step(self, step: int, dig_iter: int = 0):
        lib().or_set_step(self._h, int(step), int(dig_iter))

    def stats(self) -> dict:
        out = np.zeros(6, np.int64)
        lib().or_get_stats(self._h, _ptr(out))
        return dict(zip(("n_cand", "n_coll", "n_clip", "n_inel", "n_hits", "n_maxhit"), out.tolist()))

    def volumes(self) -> np.ndarray:
        """Cell volumes (areas per unit depth in 2D)."""
        out = np.zeros(self.ncells, np.float64)
        lib().or_get_vol(self._h, _ptr(out))
        return out

    def flow(self) -> dict:
        """Particles that entered through the outer circle and that left
        (annulus)."""
        out = np.zeros(2, np.int64)
        lib().or_get_flow(self._h, _ptr(out))
        return {"n_in": int(out[0]), "n_out": int(out[1])}

    def wall_tally(self) -> np.ndarray:
        out = np.zeros((4, 5), np.float64)
        lib().or_get_wall(self._h, _ptr(out))
        return out

    def constants(self) -> dict:
        out = np.zeros(8, np.float64)
        lib().or_constants(self._h, _ptr(out))
        return dict(zip(("dx", "dy", "vcell", "fnum", "mu_ref", "k_visc", "c_sigma", "p_inel"), out.tolist()))
