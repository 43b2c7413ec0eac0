"""Python binding of the C ABI declared in ``include/dig_dsmc.h``.

Argument marshalling only: every step of the path runs in the CUDA library
``_build/libdigdsmc.so``.  PyTorch supplies device memory (the workspace and
the field buffers) and the CUDA stream.  There is no CPU fallback: if the
library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

DSMC_OK = 0
ERRORS = {-1: "DSMC_ERR_ARG", -2: "DSMC_ERR_CAPACITY", -3: "DSMC_ERR_NUMERIC",
          -4: "DSMC_ERR_NOT_CONVERGED", -5: "DSMC_ERR_TIMEOUT", -6: "DSMC_ERR_CUDA"}
ABI_VERSION = 2
NFIELDS, NHOT, NTARGET, NMOM = 18, 12, 6, 17
PREC = {"fp64": 0, "fp32": 1}
WALL = {"diffuse": 0, "specular": 1}
MESH = {"box": 0, "annulus": 1, "refined": 2}

# every symbol the header declares
SYMBOLS = ["dsmc_workspace_size", "dsmc_init", "dsmc_destroy", "dsmc_last_error", "dsmc_step", "dsmc_sample",
           "dsmc_hot", "synth_solve", "dsmc_synth_reuse", "dig_correct", "dsmc_num_particles", "dsmc_get_particles",
           "dsmc_set_particles", "dsmc_get_accumulators", "dsmc_get_sgmax", "dsmc_set_sgmax",
           "dsmc_get_counters", "dsmc_set_counters", "dsmc_get_stats", "dsmc_get_wall_tally",
           "dsmc_get_constants", "synth_solve_noalloc", "dsmc_batch_workspace_size", "dsmc_batch_init",
           "hot_mlp_init", "hot_mlp_set_params", "hot_mlp_get_params", "hot_mlp_grad", "hot_mlp_train",
           "hot_mlp_apply", "dsmc_get_launch_config", "dsmc_get_flow", "dsmc_get_volumes",
           "hot_mlp_apply_judged", "hot_mlp_judge_reset", "dsmc_get_launch_shape"]
MLP_NPARAM = 9477


class DsmcConfig(ctypes.Structure):
    _fields_ = [
        ("version", ctypes.c_int32), ("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("ppc", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("kn", ctypes.c_double), ("omega", ctypes.c_double), ("alpha", ctypes.c_double),
        ("z_rot", ctypes.c_double), ("d_r", ctypes.c_double),
        ("a_matrix", ctypes.c_double * 4),
        ("dt", ctypes.c_double),
        ("wall_kind", ctypes.c_int32 * 4),
        ("wall_t", ctypes.c_double * 4),
        ("wall_u", (ctypes.c_double * 3) * 4),
        ("init_rho", ctypes.c_double), ("init_tt", ctypes.c_double), ("init_tr", ctypes.c_double),
        ("init_u", ctypes.c_double * 3),
        ("collisions", ctypes.c_int32), ("n_s", ctypes.c_int32), ("n_m", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("kn_ref", ctypes.c_double), ("synth_tol", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("capacity", ctypes.c_int64),
        ("bin_slack", ctypes.c_double),
        ("mesh", ctypes.c_int32), ("synth2d", ctypes.c_int32),
        ("r_in", ctypes.c_double), ("r_out", ctypes.c_double), ("stretch", ctypes.c_double),
        ("fs_rho", ctypes.c_double), ("fs_t", ctypes.c_double), ("fs_u", ctypes.c_double * 3),
    ]


_lib = None


class DsmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or _build.is_stale():
        if not build_if_missing:
            raise OSError(f"CUDA library not built: {path}")
        _build.build()
    L = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    H = ctypes.c_void_p
    sig = {
        "dsmc_workspace_size": ([P, P], ctypes.c_int),
        "dsmc_init": ([P, P, ctypes.c_size_t, P, P], ctypes.c_int),
        "dsmc_destroy": ([H], ctypes.c_int),
        "dsmc_last_error": ([H], ctypes.c_char_p),
        "dsmc_step": ([H, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "dsmc_sample": ([H, P, ctypes.c_int], ctypes.c_int),
        "dsmc_hot": ([H, P, P, P, P], ctypes.c_int),
        "synth_solve": ([H, P, P, P, P, P], ctypes.c_int),
        "dsmc_synth_reuse": ([H, ctypes.c_int], ctypes.c_int),
        "dig_correct": ([H, P], ctypes.c_int),
        "dsmc_num_particles": ([H, P], ctypes.c_int),
        "dsmc_get_particles": ([H, P, P, P, P, P, P, P, I64, P], ctypes.c_int),
        "dsmc_set_particles": ([H, I64, P, P, P, P, P, P], ctypes.c_int),
        "dsmc_get_accumulators": ([H, P, P], ctypes.c_int),
        "dsmc_get_sgmax": ([H, P], ctypes.c_int),
        "dsmc_set_sgmax": ([H, P], ctypes.c_int),
        "dsmc_get_counters": ([H, P, P], ctypes.c_int),
        "dsmc_set_counters": ([H, ctypes.c_uint32, ctypes.c_uint32], ctypes.c_int),
        "dsmc_get_stats": ([H, P], ctypes.c_int),
        "dsmc_get_wall_tally": ([H, P], ctypes.c_int),
        "dsmc_get_constants": ([H, P], ctypes.c_int),
        "synth_solve_noalloc": ([P, P, P, P, P, P, P], ctypes.c_int),
        "dsmc_batch_workspace_size": ([P, ctypes.c_int, P], ctypes.c_int),
        "dsmc_batch_init": ([P, ctypes.c_int, P, ctypes.c_size_t, P, P], ctypes.c_int),
        "hot_mlp_init": ([H, ctypes.c_uint64], ctypes.c_int),
        "dsmc_get_launch_config": ([H, P], ctypes.c_int),
        "dsmc_get_flow": ([H, P], ctypes.c_int),
        "dsmc_get_volumes": ([H, P], ctypes.c_int),
        "hot_mlp_set_params": ([H, P], ctypes.c_int),
        "hot_mlp_get_params": ([H, P], ctypes.c_int),
        "hot_mlp_grad": ([H, P, P, P, P, P, P], ctypes.c_int),
        "hot_mlp_train": ([H, P, P, P, P, ctypes.c_int, ctypes.c_double, P], ctypes.c_int),
        "hot_mlp_apply": ([H, P, P, P, P, P, P], ctypes.c_int),
        "hot_mlp_apply_judged": ([H, P, P, P, P, P, D, ctypes.c_int, D, P, P, P], ctypes.c_int),
        "hot_mlp_judge_reset": ([H], ctypes.c_int),
        "dsmc_get_launch_shape": ([H, P, P], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def make_config(cfg: dict) -> DsmcConfig:
    c = DsmcConfig()
    c.version = ABI_VERSION
    c.dim, c.nx, c.ny, c.ppc = int(cfg["dim"]), int(cfg["nx"]), int(cfg.get("ny", 1)), int(cfg["ppc"])
    c.precision = PREC[cfg.get("precision", "fp32")]
    c.lx, c.ly = float(cfg["lx"]), float(cfg.get("ly", 1.0))
    c.kn, c.omega, c.alpha = float(cfg["kn"]), float(cfg["omega"]), float(cfg["alpha"])
    c.z_rot, c.d_r = float(cfg["z_rot"]), float(cfg["d_r"])
    for k in range(4):
        c.a_matrix[k] = float(cfg["a_matrix"][k])
    c.dt = float(cfg["dt"])
    for w, wall in enumerate(cfg["walls"][:4]):
        c.wall_kind[w] = WALL[wall["kind"]]
        c.wall_t[w] = float(wall["T"])
        for k in range(3):
            c.wall_u[w][k] = float(wall["u"][k])
    c.init_rho, c.init_tt, c.init_tr = float(cfg["init_rho"]), float(cfg["init_tt"]), float(cfg["init_tr"])
    for k in range(3):
        c.init_u[k] = float(cfg["init_u"][k])
    c.collisions = 1 if cfg.get("collisions", True) else 0
    c.n_s, c.n_m = int(cfg.get("n_s", 100)), int(cfg.get("n_m", 2000))
    c.kn_ref, c.synth_tol = float(cfg.get("kn_ref", 0.01)), float(cfg.get("synth_tol", 1e-5))
    c.seed = int(cfg.get("seed", 0))
    c.capacity = int(cfg.get("capacity", 0) or 0)
    c.bin_slack = float(cfg.get("bin_slack", 2.0))
    c.mesh = MESH[cfg.get("mesh", "box")]
    c.synth2d = 1 if cfg.get("synth2d", False) else 0
    c.r_in, c.r_out = float(cfg.get("r_in", 0.5)), float(cfg.get("r_out", 5.5))
    c.stretch = float(cfg.get("stretch", 1.0))
    c.fs_rho, c.fs_t = float(cfg.get("fs_rho", 1.0)), float(cfg.get("fs_t", 1.0))
    for k in range(3):
        c.fs_u[k] = float(cfg.get("fs_u", (0.0, 0.0, 0.0))[k])
    return c


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _ncells(cfg: dict) -> int:
    return int(cfg["nx"]) * (int(cfg.get("ny", 1)) if int(cfg["dim"]) == 2 else 1)


class Dsmc:
    """One simulation, or a batch of independent ones (a list of configs),
    held by a handle of the C library plus its torch-owned workspace.  In a
    batch the cells are numbered case after case (``cell0`` gives the
    offsets)."""

    def __init__(self, cfg, device="cuda", stream: torch.cuda.Stream | None = None):
        L = load()
        cfgs = list(cfg) if isinstance(cfg, (list, tuple)) else [cfg]
        self.cfgs = [dict(c) for c in cfgs]
        self.cfg = self.cfgs[0]
        arr = (DsmcConfig * len(cfgs))(*[make_config(c) for c in cfgs])
        self._c = arr
        n = len(cfgs)
        nbytes = ctypes.c_size_t()
        self._check(L.dsmc_batch_workspace_size(arr, n, ctypes.byref(nbytes)), None)
        self.device = torch.device(device)
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        self._check(L.dsmc_batch_init(arr, n, _ptr(self.workspace), nbytes.value,
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), None)
        self._h = h
        self.ncases = n
        self.cell0 = [0]
        for c in self.cfgs:
            self.cell0.append(self.cell0[-1] + _ncells(c))
        self.ncells = self.cell0[-1]

    def _check(self, rc, h="self", allow=()):
        if rc == DSMC_OK or rc in allow:
            return rc
        L = load()
        hh = self._h if h == "self" else h
        msg = L.dsmc_last_error(hh).decode() if hh is not None else "invalid configuration"
        raise DsmcError(rc, msg)

    def close(self):
        if getattr(self, "_h", None):
            load().dsmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- the hot path ---------------------------------------------------------
    def dsmc_step(self, nsteps: int = 1, sample: bool = False):
        self._check(load().dsmc_step(self._h, int(nsteps), 1 if sample else 0))

    def dsmc_sample(self, reset: bool = True, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.ncells, NFIELDS), dtype=torch.float64, device=self.device)
        self._check(load().dsmc_sample(self._h, _ptr(out), 1 if reset else 0))
        return out

    def dsmc_hot(self, fields: torch.Tensor):
        hot = torch.empty((self.ncells, NHOT), dtype=torch.float64, device=self.device)
        kn = torch.empty(self.ncells, dtype=torch.float64, device=self.device)
        mask = torch.empty(self.ncells, dtype=torch.uint8, device=self.device)
        self._check(load().dsmc_hot(self._h, _ptr(fields.contiguous()), _ptr(hot), _ptr(kn), _ptr(mask)))
        return hot, kn, mask

    def synth_solve(self, fields: torch.Tensor, hot: torch.Tensor, allow_not_converged: bool = False,
                    allow_fallback: bool = False):
        """Returns (targets, iterations, max residual); with allow_fallback a
        slab without an admissible solution keeps its sampled fields instead
        of raising (the status is in self.last_synth_status)."""
        out = torch.empty((self.ncells, NTARGET), dtype=torch.float64, device=self.device)
        it = ctypes.c_int()
        res = ctypes.c_double()
        rc = load().synth_solve(self._h, _ptr(fields.contiguous()), _ptr(hot.contiguous()), _ptr(out),
                                ctypes.byref(it), ctypes.byref(res))
        allow = ((-4,) if allow_not_converged else ()) + ((-3,) if allow_fallback else ())
        self._check(rc, allow=allow)
        self.last_synth_status = rc
        return out, it.value, res.value

    def synth_reuse(self, on: bool = True, warm: bool = False):
        """2D: let each synth_solve start from the previous call's
        factorisation (and with warm, Newton from its solution)."""
        self._check(load().dsmc_synth_reuse(self._h, (1 if on else 0) | (2 if warm else 0)))

    def launch_config(self) -> int:
        """Warps (cells) per CTA of the FP32 fused step chosen by the tuner."""
        v = ctypes.c_int()
        self._check(load().dsmc_get_launch_config(self._h, ctypes.byref(v)))
        return v.value

    def launch_shape(self) -> tuple:
        """(warps per CTA, tile) of the FP32 fused step chosen by the tuner."""
        w, t = ctypes.c_int(), ctypes.c_int()
        self._check(load().dsmc_get_launch_shape(self._h, ctypes.byref(w), ctypes.byref(t)))
        return w.value, t.value

    # ---- HoT surrogate network (see the header) ----
    def mlp_init(self, seed: int = 0):
        self._check(load().hot_mlp_init(self._h, ctypes.c_uint64(seed)))

    def mlp_set_params(self, params):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        assert a.size == MLP_NPARAM
        self._check(load().hot_mlp_set_params(self._h, a.ctypes.data_as(ctypes.c_void_p)))

    def mlp_get_params(self):
        import numpy as np
        a = np.zeros(MLP_NPARAM, np.float32)
        self._check(load().hot_mlp_get_params(self._h, a.ctypes.data_as(ctypes.c_void_p)))
        return a

    def mlp_grad(self, fields, hot, kngll, mask):
        """(loss, gradient [MLP_NPARAM] as numpy float32) over the mask cells."""
        import numpy as np
        g = np.zeros(MLP_NPARAM, np.float32)
        loss = ctypes.c_double()
        self._check(load().hot_mlp_grad(self._h, _ptr(fields.contiguous()), _ptr(hot.contiguous()),
                                        _ptr(kngll.contiguous()), _ptr(mask.contiguous()),
                                        g.ctypes.data_as(ctypes.c_void_p), ctypes.byref(loss)))
        return loss.value, g

    def mlp_train(self, fields, hot, kngll, mask, nsteps: int, lr: float = 1e-3) -> float:
        loss = ctypes.c_double()
        self._check(load().hot_mlp_train(self._h, _ptr(fields.contiguous()), _ptr(hot.contiguous()),
                                         _ptr(kngll.contiguous()), _ptr(mask.contiguous()), int(nsteps),
                                         float(lr), ctypes.byref(loss)))
        return loss.value

    def mlp_apply_judged(self, fields, hot, kngll, mask, group=None, z: float = 3.0, min_samples: int = 4,
                         rel: float = 0.1):
        """(HoT [ncells x 12], judge, cells given the network's HoT): the
        network where its group's running residuals against the DSMC HoT
        bound its bias below rel of the DSMC terms (with z standard errors of
        confidence), the DSMC HoT elsewhere."""
        out = torch.empty_like(hot)
        judge = ctypes.c_double()
        nnet = ctypes.c_int64()
        g = group.to(device=self.device, dtype=torch.int32).contiguous() if group is not None else None
        self._check(load().hot_mlp_apply_judged(self._h, _ptr(fields.contiguous()), _ptr(hot.contiguous()),
                                                _ptr(kngll.contiguous()), _ptr(mask.contiguous()), _ptr(g),
                                                float(z), int(min_samples), float(rel), _ptr(out), ctypes.byref(judge),
                                                ctypes.byref(nnet)))
        return out, judge.value, nnet.value

    def mlp_judge_reset(self):
        self._check(load().hot_mlp_judge_reset(self._h))

    def mlp_apply(self, fields, hot, kngll, mask):
        """(HoT for the synthetic equations [ncells x 12], judge)."""
        out = torch.empty_like(hot)
        judge = ctypes.c_double()
        self._check(load().hot_mlp_apply(self._h, _ptr(fields.contiguous()), _ptr(hot.contiguous()),
                                         _ptr(kngll.contiguous()), _ptr(mask.contiguous()), _ptr(out),
                                         ctypes.byref(judge)))
        return out, judge.value

    def dig_correct(self, target: torch.Tensor):
        self._check(load().dig_correct(self._h, _ptr(target.contiguous())))

    # --- state access ---------------------------------------------------------
    def num_particles(self) -> int:
        n = ctypes.c_int64()
        self._check(load().dsmc_num_particles(self._h, ctypes.byref(n)))
        return n.value

    def get_particles(self) -> dict:
        n = self.num_particles()
        cap = max(n, 1)
        arrs = {k: torch.empty(cap, dtype=torch.float64, device=self.device) for k in ("x", "y", "vx", "vy", "vz", "ir")}
        cell = torch.empty(cap, dtype=torch.int32, device=self.device)
        got = ctypes.c_int64()
        self._check(load().dsmc_get_particles(self._h, *[_ptr(arrs[k]) for k in ("x", "y", "vx", "vy", "vz", "ir")],
                                              _ptr(cell), cap, ctypes.byref(got)))
        out = {k: v[:got.value] for k, v in arrs.items()}
        out["cell"] = cell[:got.value]
        return out

    def set_particles(self, p: dict):
        n = int(p["x"].numel())
        t = {k: p[k].to(device=self.device, dtype=torch.float64).contiguous() for k in ("x", "vx", "vy", "vz", "ir")}
        t["y"] = (p["y"] if "y" in p else torch.zeros(n)).to(device=self.device, dtype=torch.float64).contiguous()
        self._check(load().dsmc_set_particles(self._h, n, *[_ptr(t[k]) for k in ("x", "y", "vx", "vy", "vz", "ir")]))

    def accumulators(self):
        out = torch.empty((self.ncells, NMOM), dtype=torch.float64, device=self.device)
        ns = ctypes.c_int64()
        self._check(load().dsmc_get_accumulators(self._h, _ptr(out), ctypes.byref(ns)))
        return out, ns.value

    def sgmax(self) -> torch.Tensor:
        out = torch.empty(self.ncells, dtype=torch.float64, device=self.device)
        self._check(load().dsmc_get_sgmax(self._h, _ptr(out)))
        return out

    def set_sgmax(self, v: torch.Tensor):
        v = v.to(device=self.device, dtype=torch.float64).contiguous()
        self._check(load().dsmc_set_sgmax(self._h, _ptr(v)))

    def counters(self):
        s, d = ctypes.c_uint32(), ctypes.c_uint32()
        self._check(load().dsmc_get_counters(self._h, ctypes.byref(s), ctypes.byref(d)))
        return s.value, d.value

    def set_counters(self, step: int, dig_iter: int = 0):
        self._check(load().dsmc_set_counters(self._h, int(step), int(dig_iter)))

    def stats(self) -> dict:
        out = (ctypes.c_int64 * 8)()
        self._check(load().dsmc_get_stats(self._h, out))
        return dict(zip(("n_cand", "n_coll", "n_clip", "n_inel", "n_hits", "n_maxhit", "n_overflow", "n_rebuild"),
                        list(out)))

    def flow(self) -> dict:
        """Annulus: particles that entered through the outer circle and that
        left through it since the start."""
        out = np.zeros(2, np.int64)
        self._check(load().dsmc_get_flow(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return {"n_in": int(out[0]), "n_out": int(out[1])}

    def volumes(self) -> np.ndarray:
        """Cell volumes (areas per unit depth in 2D)."""
        out = np.zeros(self.ncells, np.float64)
        self._check(load().dsmc_get_volumes(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def wall_tally(self):
        out = (ctypes.c_double * 20)()
        self._check(load().dsmc_get_wall_tally(self._h, out))
        return [list(out[5 * w:5 * w + 5]) for w in range(4)]

    def constants(self) -> dict:
        out = (ctypes.c_double * 8)()
        self._check(load().dsmc_get_constants(self._h, out))
        return dict(zip(("dx", "dy", "vcell", "fnum", "mu_ref", "k_visc", "c_sigma", "p_inel"), list(out)))


def synth_solve_noalloc(cfg: dict, fields: torch.Tensor, hot: torch.Tensor, out: torch.Tensor | None = None,
                        stream: torch.cuda.Stream | None = None):
    """The 1D synthetic solve without a handle or workspace (see the header):
    for callers that cannot allocate device memory.  Returns (out, iterations,
    max residual, status code)."""
    L = load()
    c = make_config(cfg)
    if out is None:
        out = torch.empty((int(cfg["nx"]), NTARGET), dtype=torch.float64, device=fields.device)
    st = stream if stream is not None else torch.cuda.current_stream(fields.device)
    it = ctypes.c_int()
    res = ctypes.c_double()
    rc = L.synth_solve_noalloc(ctypes.byref(c), _ptr(fields.contiguous()), _ptr(hot.contiguous()), _ptr(out),
                               ctypes.c_void_p(st.cuda_stream), ctypes.byref(it), ctypes.byref(res))
    return out, it.value, res.value, rc
