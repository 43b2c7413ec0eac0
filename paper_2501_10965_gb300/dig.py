"""DIG outer loop and the time-to-steady measurement (host orchestration).

One DIG iteration (Sec. 3, steps 2-4, Fig. flowchart): N_s DSMC steps with
sampling, the time-averaged fields M^{n+1/2} and their higher-order terms
(Eq. DSMC_macroscopic, Eq. hot_constitutive, Kn_GLL mask of Sec. 3.1), the
steady synthetic equations (Eq. macroscopic_equation) for M^{n+1}, and the
particle modification of Sec. 3.2.  Every step runs in the CUDA library; this
module only sequences the calls.

Time to steady state: err(t) = ||F_W(t) - F_ref|| / ||F_ref|| for the flow
velocity and the total temperature, where F_W is the average over an
ensemble of independent replicas and over a window of W steps, on coarse
bins of cells (the noise floor is reported), and F_ref the long-run
plain-DSMC solution.  A run is steady from the first window after which the
error stays at or below the threshold for three consecutive windows.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import dsmc


def dig_iteration(sim: "dsmc.Dsmc", n_s: int, allow_not_converged: bool = True) -> dict:
    """N_s DSMC steps, sample, HoT, synthetic solve, particle modification."""
    sim.dsmc_step(n_s, sample=True)
    f = sim.dsmc_sample(reset=True)
    hot, kn, mask = sim.dsmc_hot(f)
    out, iters, res = sim.synth_solve(f, hot, allow_not_converged=allow_not_converged, allow_fallback=True)
    sim.dig_correct(out)
    return {"fields": f, "target": out, "synth_iters": iters, "synth_resid": res,
            "synth_status": sim.last_synth_status, "mask_fraction": float(mask.float().mean().item())}


def total_temperature(f: np.ndarray, d_r: float = 2.0) -> np.ndarray:
    return (3.0 * f[..., 4] + d_r * f[..., 5]) / (3.0 + d_r)


def binned(a: np.ndarray, nbins: int) -> np.ndarray:
    n = a.shape[-1]
    k = n // nbins
    return a[..., : k * nbins].reshape(*a.shape[:-1], nbins, k).mean(-1)


class Ensemble:
    """R independent replicas of one workload (seeds seed0 + r)."""

    def __init__(self, cfg: dict, replicas: int, seed0: int = 0):
        self.cfg = dict(cfg)
        self.sims = [dsmc.Dsmc(dict(cfg, seed=seed0 + r)) for r in range(replicas)]
        self.steps = 0
        self.wall = 0.0  # GPU wall time spent in the method's calls, seconds

    def _timed(self, fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        self.wall += time.perf_counter() - t0
        return out

    def advance_plain(self, nsteps: int) -> np.ndarray:
        def run():
            fs = []
            for s in self.sims:
                s.dsmc_step(nsteps, sample=True)
                fs.append(s.dsmc_sample(reset=True))
            return fs
        fs = self._timed(run)
        self.steps += nsteps
        return torch.stack(fs).cpu().numpy()

    def advance_dig(self, n_s: int) -> np.ndarray:
        def run():
            return [dig_iteration(s, n_s)["fields"] for s in self.sims]
        fs = self._timed(run)
        self.steps += n_s
        return torch.stack(fs).cpu().numpy()


def window_error(fs: np.ndarray, ref_u: np.ndarray, ref_t: np.ndarray, flow_axis: int, nbins: int):
    """Relative L2 errors of the ensemble-averaged, binned flow velocity and
    total temperature."""
    mean = fs.mean(0)
    u = binned(mean[:, 1 + flow_axis], nbins)
    t = binned(total_temperature(mean), nbins)
    eu = np.linalg.norm(u - ref_u) / np.linalg.norm(ref_u)
    et = np.linalg.norm(t - ref_t) / np.linalg.norm(ref_t)
    return float(eu), float(et)


def time_to_steady(errors: list, threshold: float, consecutive: int = 3):
    """Index of the first window after which the error stays <= threshold for
    `consecutive` windows, or None."""
    run = 0
    for i, e in enumerate(errors):
        if e <= threshold:
            run += 1
            if run >= consecutive:
                return i - consecutive + 1
        else:
            run = 0
    return None


def reference_solution(cfg: dict, replicas: int, transient_steps: int, average_steps: int, window: int,
                       flow_axis: int, nbins: int, seed0: int = 1000):
    """Long-run plain-DSMC average: `transient_steps` discarded, then the
    average over `average_steps` and the replicas."""
    ens = Ensemble(cfg, replicas, seed0)
    done = 0
    while done < transient_steps:
        k = min(window * 20, transient_steps - done)
        for s in ens.sims:
            s.dsmc_step(k, sample=False)
        done += k
    acc = None
    nwin = max(1, average_steps // window)
    for _ in range(nwin):
        fs = ens.advance_plain(window)
        acc = fs.mean(0) if acc is None else acc + fs.mean(0)
    mean = acc / nwin
    return binned(mean[:, 1 + flow_axis], nbins), binned(total_temperature(mean), nbins), mean


def measure(cfg: dict, method: str, replicas: int, window: int, max_steps: int, ref_u, ref_t, flow_axis: int,
            nbins: int, threshold: float = 0.01, seed0: int = 0) -> dict:
    """Run `method` ("plain" or "dig") from the uniform initial state and
    record err(t) per window; returns the time to steady (steps and GPU wall
    seconds) and the error history."""
    ens = Ensemble(cfg, replicas, seed0)
    eu_hist, et_hist, walls, steps = [], [], [], []
    n_s = int(cfg["n_s"])
    while ens.steps < max_steps:
        if method == "dig":
            fs = np.stack([ens.advance_dig(n_s) for _ in range(max(1, window // n_s))]).mean(0)
        else:
            fs = ens.advance_plain(window)
        eu, et = window_error(fs, ref_u, ref_t, flow_axis, nbins)
        eu_hist.append(eu)
        et_hist.append(et)
        walls.append(ens.wall)
        steps.append(ens.steps)
        i = time_to_steady([max(a, b) for a, b in zip(eu_hist, et_hist)], threshold)
        if i is not None:
            return {"method": method, "steady_step": steps[i], "steady_wall_s": walls[i],
                    "err_u": eu_hist, "err_T": et_hist, "steps": steps, "wall": walls}
    return {"method": method, "steady_step": None, "steady_wall_s": None, "err_u": eu_hist, "err_T": et_hist,
            "steps": steps, "wall": walls}
