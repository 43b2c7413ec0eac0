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


def target_as_fields(target: torch.Tensor) -> torch.Tensor:
    """Cell fields (ncells x 18) holding a synthetic solution's rho, u, T_t,
    T_r (stress and heat-flux slots zero): the smooth state the HoT network
    reads its inputs from."""
    f = torch.zeros((target.shape[0], dsmc.NFIELDS), dtype=torch.float64, device=target.device)
    f[:, :6] = target
    return f


def dig_iteration(sim: "dsmc.Dsmc", n_s: int, allow_not_converged: bool = True,
                  hot_model: bool = False, prev_target: torch.Tensor | None = None,
                  hot_group: torch.Tensor | None = None, judge_z: float = 3.0, judge_min: int = 4,
                  judge_rel: float = 0.1) -> dict:
    """N_s DSMC steps, sample, HoT, synthetic solve, particle modification.

    With hot_model, the higher-order terms where Kn_GLL >= Kn_ref are the
    handle's HoT network evaluated on the previous synthetic solution (a
    smooth state; the sampled fields' gradients are dominated by noise),
    judged against the sampled HoT: a cell takes the network's terms only
    once the running residuals of its group (hot_group, e.g. the same cell
    of every replica) bound the network's bias below judge_rel of the
    sampled terms with judge_z standard errors of confidence, and the
    sampled HoT otherwise; the first iteration, with no previous solution,
    uses the sampled HoT."""
    sim.dsmc_step(n_s, sample=True)
    f = sim.dsmc_sample(reset=True)
    hot, kn, mask = sim.dsmc_hot(f)
    judge, nnet = None, None
    if hot_model and prev_target is not None:
        fs = target_as_fields(prev_target)
        _, kn_s, mask_s = sim.dsmc_hot(fs)
        hot, judge, nnet = sim.mlp_apply_judged(fs, hot, kn_s, mask_s, group=hot_group, z=judge_z,
                                                min_samples=judge_min, rel=judge_rel)
    out, iters, res = sim.synth_solve(f, hot, allow_not_converged=allow_not_converged, allow_fallback=True)
    # a target the modification refuses (a sampled cell with particles but a
    # zero temperature, as a nearly empty cell of an early wake has) leaves
    # the particles as they are: the iteration is plain DSMC
    modified = True
    try:
        sim.dig_correct(out)
    except dsmc.DsmcError as e:
        if e.code != -3:
            raise
        modified = False
    # the HoT mask stays on the device (reducing it here would put a host
    # round trip, and the first use of a framework kernel, into the loop)
    return {"fields": f, "target": out, "synth_iters": iters, "synth_resid": res,
            "synth_status": sim.last_synth_status, "mask": mask, "judge": judge, "network_cells": nnet,
            "modified": modified}


def total_temperature(f: np.ndarray, d_r: float = 2.0) -> np.ndarray:
    return (3.0 * f[..., 4] + d_r * f[..., 5]) / (3.0 + d_r)


def binned(a: np.ndarray, nbins: int) -> np.ndarray:
    n = a.shape[-1]
    k = n // nbins
    return a[..., : k * nbins].reshape(*a.shape[:-1], nbins, k).mean(-1)


class Ensemble:
    """R independent replicas of one 1D workload (seeds seed0 + r), held in
    one batched handle so that each stage is one launch for all of them."""

    def __init__(self, cfg: dict, replicas: int, seed0: int = 0, hot_params=None):
        from . import workloads
        self.cfg = dict(cfg)
        self.R = replicas
        self.nx = int(cfg["nx"])
        self.sim = dsmc.Dsmc(workloads.replicas(cfg, replicas, seed0))
        self.hot_model = hot_params is not None
        self.group = None
        if self.hot_model:
            self.sim.mlp_set_params(hot_params)
            # the judge pools the same cell of every replica
            self.group = (torch.arange(self.R * self.nx, dtype=torch.int32) % self.nx).to(self.sim.device)
        self.target = None
        self.steps = 0
        self.wall = 0.0  # GPU wall time spent in the method's calls, seconds

    def _timed(self, fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        self.wall += time.perf_counter() - t0
        return out

    def _per_replica(self, f: torch.Tensor) -> np.ndarray:
        return f.cpu().numpy().reshape(self.R, self.nx, -1)

    def advance_plain(self, nsteps: int) -> np.ndarray:
        def run():
            self.sim.dsmc_step(nsteps, sample=True)
            return self.sim.dsmc_sample(reset=True)
        f = self._timed(run)
        self.steps += nsteps
        return self._per_replica(f)

    def advance_quiet(self, nsteps: int):
        self._timed(lambda: self.sim.dsmc_step(nsteps, sample=False))
        self.steps += nsteps

    def advance_dig(self, n_s: int) -> np.ndarray:
        r = self._timed(lambda: dig_iteration(self.sim, n_s, hot_model=self.hot_model, prev_target=self.target,
                                              hot_group=self.group))
        self.target = r["target"]
        self.last = r
        self.steps += n_s
        return self._per_replica(r["fields"])


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
        ens.advance_quiet(k)
        done += k
    wins = []
    nwin = max(1, average_steps // window)
    for _ in range(nwin):
        wins.append(ens.advance_plain(window).mean(0))
    mean = np.mean(wins, axis=0)
    ref_u = binned(mean[:, 1 + flow_axis], nbins)
    ref_t = binned(total_temperature(mean), nbins)
    # noise floor of the window error at steady state: median over the
    # averaging windows of their error against the long-run mean
    floor = [max(window_error(w[None], ref_u, ref_t, flow_axis, nbins)) for w in wins]
    return ref_u, ref_t, mean, float(np.median(floor))


def measure(cfg: dict, method: str, replicas: int, window: int, max_steps: int, ref_u, ref_t, flow_axis: int,
            nbins: int, threshold: float = 0.01, seed0: int = 0, hot_params=None) -> dict:
    """Run `method` ("plain", "dig" or "dig_mlp": DIG with the HoT network of
    parameters hot_params) from the uniform initial state and record err(t)
    per window; returns the time to steady (steps and GPU wall seconds) and
    the error history."""
    ens = Ensemble(cfg, replicas, seed0, hot_params=hot_params if method == "dig_mlp" else None)
    eu_hist, et_hist, walls, steps = [], [], [], []
    n_s = int(cfg["n_s"])
    while ens.steps < max_steps:
        if method in ("dig", "dig_mlp"):
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


def time_to_steady_dig_vs_plain(cfg: dict, replicas: int = 800, window: int = 100, nbins: int = 20,
                                transient: int = 50000, average: int = 15000, threshold: float = 0.01,
                                max_dig: int = 6000, max_plain: int = 60000, hot_params=None) -> dict:
    """Time to steady state at `threshold` field error, DIG against plain
    DSMC, both on the GPU from the same uniform initial state, ensemble of
    `replicas` (one batched handle) against the long-run plain-DSMC reference
    of an independent ensemble."""
    t0 = time.perf_counter()
    ref_u, ref_t, _, floor = reference_solution(cfg, replicas, transient, average, window, 1, nbins)
    t_ref = time.perf_counter() - t0
    out = {"replicas": replicas, "particles": replicas * int(cfg["nx"]) * int(cfg["ppc"]), "window": window,
           "bins": nbins, "threshold": threshold, "noise_floor": floor, "reference_wall_s": t_ref}
    methods = [("dig", max_dig), ("plain", max_plain)]
    if hot_params is not None:
        methods.insert(1, ("dig_mlp", max_dig))
    for method, cap in methods:
        r = measure(cfg, method, replicas, window, cap, ref_u, ref_t, 1, nbins, threshold, hot_params=hot_params)
        out[method] = {"steady_step": r["steady_step"], "steady_wall_s": r["steady_wall_s"],
                       "final_err_u": r["err_u"][-1], "final_err_T": r["err_T"][-1]}
    pl = out["plain"]
    for m, suffix in (("dig", ""), ("dig_mlp", "_mlp")):
        d = out.get(m)
        if d and d["steady_wall_s"] and pl["steady_wall_s"]:
            out["speedup_wall" + suffix] = pl["steady_wall_s"] / d["steady_wall_s"]
            out["speedup_steps" + suffix] = pl["steady_step"] / d["steady_step"]
    return out


def train_hot_model_on_dig(cfgs: list, replicas: int = 64, iterations: int = 40, n_s: int | None = None,
                           rounds: int = 10, steps_per_round: int = 100, lrs=(2e-3, 5e-4), seed0: int = 7000,
                           init_seed: int = 0):
    """Train the HoT network on the states it serves inside DIG.  Plain DIG
    (no network) runs on `replicas` copies of each configuration (seeds from
    seed0, independent of the runs the network will serve); after every
    iteration the previous synthetic target -- a smooth state, the network's
    input when it is coupled into DIG -- is paired with the HoT of the DSMC
    window that followed it (noisy: the network learns its mean over copies
    and iterations).  Features and labels come from a handle of the same
    cells with Kn_ref 0 (every cell a training cell), which also holds and
    trains the network (Adam, full batch per iteration's pairs, `rounds`
    rounds of `steps_per_round` steps, step size lrs[0] then lrs[1]).
    Returns (parameters as float32 numpy, a dict with the data's size and the
    last loss)."""
    from . import workloads
    cases = []
    for k, c in enumerate(cfgs):
        cases += workloads.replicas(c, replicas, seed0 + 1000 * k)
    g = dsmc.Dsmc(cases)
    lab = dsmc.Dsmc([dict(c, kn_ref=0.0, ppc=1) for c in cases])
    lab.mlp_init(init_seed)
    ns = int(n_s if n_s is not None else cfgs[0].get("n_s", 50))
    data, prev = [], None
    for _ in range(iterations):
        r = dig_iteration(g, ns, allow_not_converged=True)
        if prev is not None:
            fs = target_as_fields(prev)
            _, kn_s, mask_s = lab.dsmc_hot(fs)
            hot_w, _, _ = lab.dsmc_hot(r["fields"])
            data.append((fs, hot_w, kn_s, mask_s))
        prev = r["target"]
    del g
    loss = None
    for rr in range(rounds):
        lr = lrs[0] if rr < rounds // 2 else lrs[1]
        for fs, hot_w, kn_s, mask_s in data:
            loss = lab.mlp_train(fs, hot_w, kn_s, mask_s, steps_per_round, lr)
    params = lab.mlp_get_params()
    info = {"cases": len(cases), "cells": lab.ncells, "pairs": len(data), "loss": loss}
    del lab
    return params, info


def train_hot_model(cfgs: list, replicas: int = 32, snapshots=(100, 300, 700, 1500, 3000, 6000),
                    window: int = 200, rounds: int = 20, steps_per_round: int = 100,
                    lrs=(2e-3, 5e-4), seed0: int = 5000, init_seed: int = 0):
    """Train the HoT network on the method's own DSMC samples.  Every
    configuration in cfgs runs as `replicas` independent copies (seeds from
    seed0, independent of the runs the network will serve), all in one
    batched handle, from the uniform start; at each of `snapshots` (steps
    from the start) a `window`-step sample is taken and averaged over the
    copies of its configuration, so that the network learns HoT as a function
    of clean inputs (a single run's gradients are dominated by sampling
    noise), over the transient as well as the steady state.  Training: Adam,
    full batch per snapshot, cycling through the snapshots for `rounds`
    rounds of `steps_per_round` steps, the step size going from lrs[0] to
    lrs[1] halfway; every cell is a training cell (Kn_ref 0).
    Returns (parameters as float32 numpy, a dict with the data's size and the
    last loss)."""
    from . import workloads
    cases = []
    for k, c in enumerate(cfgs):
        cases += workloads.replicas(dict(c, kn_ref=0.0), replicas, seed0 + 1000 * k)
    g = dsmc.Dsmc(cases)
    g.mlp_init(init_seed)
    nc = [int(c["nx"]) * (int(c.get("ny", 1)) if int(c["dim"]) == 2 else 1) for c in cfgs]
    data = []
    done = 0
    for t in snapshots:
        if t - window > done:
            g.dsmc_step(t - window - done)
            done = t - window
        g.dsmc_sample(reset=True)
        g.dsmc_step(window, sample=True)
        done += window
        f = g.dsmc_sample(reset=True)
        # average over the copies of each configuration, written back to all
        parts, o = [], 0
        for n in nc:
            blk = f[o:o + replicas * n].view(replicas, n, -1)
            parts.append(blk.mean(0, keepdim=True).expand(replicas, n, blk.shape[-1]).reshape(replicas * n, -1))
            o += replicas * n
        fa = torch.cat(parts).contiguous()
        hot, kn, mask = g.dsmc_hot(fa)
        data.append((fa, hot, kn, mask))
    loss = None
    for r in range(rounds):
        lr = lrs[0] if r < rounds // 2 else lrs[1]
        for fa, hot, kn, mask in data:
            loss = g.mlp_train(fa, hot, kn, mask, steps_per_round, lr)
    params = g.mlp_get_params()
    info = {"cases": len(cases), "cells": g.ncells, "snapshots": len(data), "loss": loss}
    del g
    return params, info


def binned2d(a: np.ndarray, nx: int, ny: int, bx: int, by: int) -> np.ndarray:
    """Means over blocks of bx x by cells of a cell field (cell j nx + i)."""
    g = a.reshape(ny, nx)[: (ny // by) * by, : (nx // bx) * bx]
    return g.reshape(ny // by, by, nx // bx, bx).mean(axis=(1, 3))


def time_to_steady_2d(cfg: dict, window: int = 200, bx: int = 5, by: int = 5, transient: int = 15000,
                      average: int = 10000, threshold: float = 0.01, max_dig: int = 4000,
                      max_plain: int = 20000, reuse_factorisation: bool = True, warm_start: bool = True) -> dict:
    """Time to steady state of a 2D case, DIG against plain DSMC, from the
    same uniform initial state.  The 2D synthetic solve takes one case per
    handle, so each method runs one handle (many particles per cell instead
    of an ensemble).  err(t) = the relative L2 errors of the flow velocity
    (both components) and the total temperature, averaged over a window of
    steps and over blocks of bx x by cells, against the long-run plain-DSMC
    average of an independent handle (seed + 1000); the noise floor is the
    median window error of that handle's averaging phase, and a run is
    steady from the first window after which the larger error stays at or
    below max(threshold, 1.5 x floor) for three windows.  With
    reuse_factorisation each DIG synthetic solve starts from the previous
    solve's factorisation, with warm_start Newton from its solution
    (dsmc_synth_reuse)."""
    nx, ny = int(cfg["nx"]), int(cfg["ny"])

    def reduce(f):
        u = np.stack([binned2d(f[:, 1], nx, ny, bx, by), binned2d(f[:, 2], nx, ny, bx, by)])
        return u, binned2d(total_temperature(f), nx, ny, bx, by)

    def err(f, ref_u, ref_t):
        u, t = reduce(f)
        return (float(np.linalg.norm(u - ref_u) / np.linalg.norm(ref_u)),
                float(np.linalg.norm(t - ref_t) / np.linalg.norm(ref_t)))

    t0 = time.perf_counter()
    ref = dsmc.Dsmc(dict(cfg, seed=int(cfg.get("seed", 0)) + 1000))
    ref.dsmc_step(transient, sample=False)
    wins = []
    for _ in range(max(1, average // window)):
        ref.dsmc_step(window, sample=True)
        wins.append(ref.dsmc_sample(reset=True).cpu().numpy())
    mean = np.mean(wins, axis=0)
    ref_u, ref_t = reduce(mean)
    floor = float(np.median([max(err(w, ref_u, ref_t)) for w in wins]))
    del ref
    thr = max(threshold, 1.5 * floor)
    out = {"cells": f"{nx} x {ny}", "particles": nx * ny * int(cfg["ppc"]), "window": window,
           "bins": f"{bx} x {by} cells", "noise_floor": floor, "threshold": thr, "reference_wall_s": time.perf_counter() - t0}
    n_s = int(cfg["n_s"])
    for method, cap in (("dig", max_dig), ("plain", max_plain)):
        sim = dsmc.Dsmc(cfg)
        if method == "dig" and (reuse_factorisation or warm_start):
            sim.synth_reuse(reuse_factorisation, warm=warm_start)
        hist, steps, walls, wall, nsteps = [], [], [], 0.0, 0
        steady = None
        solves = []  # (status, Newton iterations) of the DIG iterations' synthetic solves
        while nsteps < cap:
            torch.cuda.synchronize()
            ta = time.perf_counter()
            if method == "dig":
                fs = []
                for _ in range(max(1, window // n_s)):
                    r = dig_iteration(sim, n_s)
                    fs.append(r["fields"].cpu().numpy())
                    solves.append((int(r["synth_status"]), int(r["synth_iters"]), bool(r["modified"])))
                f = np.mean(fs, axis=0)
                nsteps += n_s * len(fs)
            else:
                sim.dsmc_step(window, sample=True)
                f = sim.dsmc_sample(reset=True).cpu().numpy()
                nsteps += window
            torch.cuda.synchronize()
            wall += time.perf_counter() - ta
            hist.append(max(err(f, ref_u, ref_t)))
            steps.append(nsteps)
            walls.append(wall)
            i = time_to_steady(hist, thr)
            if i is not None:
                steady = i
                break
        out[method] = {"steady_step": steps[steady] if steady is not None else None,
                       "steady_wall_s": walls[steady] if steady is not None else None,
                       "errors": [round(e, 4) for e in hist], "final_error": hist[-1] if hist else None}
        if solves:
            out[method]["synth_solves"] = len(solves)
            out[method]["synth_not_converged"] = sum(1 for st, _, _ in solves if st != 0)
            out[method]["synth_mean_newton_steps"] = float(np.mean([it for _, it, _ in solves]))
            out[method]["modifications_skipped"] = sum(1 for _, _, mod in solves if not mod)
        del sim
    d, p = out["dig"], out["plain"]
    if d["steady_step"] and p["steady_step"]:
        out["speedup_steps"] = p["steady_step"] / d["steady_step"]
        out["speedup_wall"] = p["steady_wall_s"] / d["steady_wall_s"]
    return out
