"""Throughput benchmark of the DSMC hot path on one GB300, plus the time to
steady state of DIG against plain DSMC.

A step is one DSMC time step of the whole particle path (free flight with
diffuse walls, cell indexing and bin sort, NTC/VHS/Borgnakke-Larsen
collisions, cell sampling, and on the annulus the freestream entry) over the
workload's full particle state, which stays resident in HBM.  The default
workload is the paper's hypersonic cylinder case: Mach 5 N2-like freestream
at 200 K past a diffuse cylinder at 500 K, annular mesh of 400 x 300 cells
(geometrically stretched rings), ~167 particles per cell (20.0 M particles),
Kn 0.01, FP32 particles with FP64 moment accumulators.  `cavity2d_20m` is a
lid-driven cavity of the same size.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead, on a
bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

ALGO_BYTES_PER_PARTICLE_STEP = {("fp32", 2): 48, ("fp32", 1): 40, ("fp64", 2): 96, ("fp64", 1): 80}
# DRAM bytes (read + write) per particle-step of k_fused, from one ncu capture
# of the current kernel, scaled to a launch of the workload by its particle
# count; keyed by (precision, dim, mesh).  Box: the 300 x 225-cell, 11.27
# M-particle cavity (dram__bytes_read.sum 336.42 MB + dram__bytes_write.sum
# 243.00 MB for one launch of the current kernel, `--workload cavity2d_11m
# --profile-steps 4 --warmup 3`, third fused launch).  Re-measure whenever
# k_fused changes.
# Annulus: the 300 x 225-cell, 11.27 M-particle cylinder case
# (dram__bytes_read.sum 352.24 MB + dram__bytes_write.sum 279.16 MB for one
# launch of the current kernel, `--workload cylinder2d_11m --profile-steps 4
# --warmup 3`, third fused launch).
NCU_TRAFFIC_BYTES_PER_PARTICLE_STEP = {("fp32", 2, "box"): 579425536 / 11272500,
                                       ("fp32", 2, "annulus"): 631403520 / 11272500}
METRIC = "particle-steps/s"


def workload(name: str) -> dict:
    from paper_2501_10965_gb300 import workloads as W
    if name == "cylinder2d_20m":
        return W.cylinder_2d()
    if name == "cylinder2d_11m":
        return W.cylinder_2d(ntheta=300, nr=225)
    if name == "cavity2d_20m":
        return W.cavity_2d_20m()
    if name == "cavity2d_11m":
        return W.cavity_2d(nx=300, ny=225, ppc=167, kn=0.01, lx=4.0 / 3.0, ly=1.0)
    if name == "cavity2d_500k":
        return W.cavity_2d()
    if name == "couette1d_40k":
        return W.couette_1d(kn=0.01)
    raise SystemExit(f"unknown workload {name}")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_config(cfg: dict, rank: int) -> dict:
    """Rank r runs its own seeded copy of the workload (independent
    replicas, no data-path exchange): Philox seed + 1000 r."""
    out = dict(cfg)
    out["seed"] = int(cfg.get("seed", 0)) + 1000 * rank
    return out


def over_ranks(x: float, world: int, op: str, device=None) -> float:
    """max or sum of a per-rank number over the process group (identity on
    one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(particles: float, steps: int, t_max: float, world: int, device=None) -> float:
    """Whole-job particle-steps/s: the particles of every rank over the
    slowest rank's time."""
    return over_ranks(particles, world, "sum", device) * steps / t_max


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = sorted(v for v in (num(r[1]) for r in rows) if v is not None)
        smax = max((v for v in (num(r[2]) for r in rows) if v is not None), default=None)
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        load = [v for v in sm if smax is None or v > 0.3 * smax] or sm
        return {"sm_mhz": load[len(load) // 2] if load else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(rows)}


def _events_time(fn, stream) -> float:
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def _oracle_sample(cfg: dict) -> dict:
    """The bounded sample of the workload the oracle is timed on: the same
    gas, Kn, particles per cell and time step on a smaller box of cells."""
    sub = dict(cfg)
    sub["precision"] = "fp64"
    if cfg.get("mesh") == "annulus":
        # the same annulus, gas, Kn, particles per cell and time step on 40 x 30 cells
        from paper_2501_10965_gb300 import workloads as W
        sub = W.cylinder_2d(ntheta=40, nr=30, ppc=int(cfg["ppc"]), kn=float(cfg["kn"]), r_in=float(cfg["r_in"]),
                            r_out=float(cfg["r_out"]), dt=float(cfg["dt"]), precision="fp64")
    elif int(cfg["dim"]) == 2:
        sub["nx"], sub["ny"] = 40, 30
        sub["lx"] = float(cfg["lx"]) * 40 / int(cfg["nx"])
        sub["ly"] = float(cfg["ly"]) * 30 / int(cfg["ny"])
    return sub


def _oracle_rate(sub: dict, budget_s: float):
    """(particle-steps, seconds, particles) of the oracle on sub for about
    budget_s seconds (one thread)."""
    import oracle
    sim = oracle.OracleSim(sub)
    n = sim.n
    sim.step(2, sample=True)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        sim.step(5, sample=True)
        steps += 5
    return n * steps, time.perf_counter() - t0, n


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(cfg: dict, budget_s: float = 12.0, all_cores: bool = True) -> dict:
    """The oracle, as it stands, on a bounded sample of the workload (one
    thread), and the same sample as independent seeded copies on every host
    core the process may use (spawned workers, aggregate throughput)."""
    sub = _oracle_sample(cfg)
    ps, dt, n = _oracle_rate(sub, budget_s)
    cells = int(sub["nx"]) * (int(sub.get("ny", 1)) if int(sub["dim"]) == 2 else 1)
    out = {"value": ps / dt, "unit": METRIC, "cores": 1, "kind": "oracle",
           "sample": f"{cells} cells x {sub['ppc']} particles ({n} particles), {ps // n} steps, {dt:.1f} s, "
                     f"FP64 single-threaded C oracle, same gas/Kn/ppc/dt as the workload",
           "cpu_model": cpu_model()}
    if not all_cores:
        return out
    try:
        import concurrent.futures
        import multiprocessing
        ncores = len(os.sched_getaffinity(0))
        subs = [dict(sub, seed=int(sub.get("seed", 0)) + 17 * (k + 1)) for k in range(ncores)]
        with concurrent.futures.ProcessPoolExecutor(max_workers=ncores,
                                                    mp_context=multiprocessing.get_context("spawn")) as ex:
            res = list(ex.map(_oracle_rate, subs, [budget_s / 2] * ncores))
        out["all_cores"] = {"value": sum(r[0] / r[1] for r in res), "unit": METRIC, "cores": ncores,
                            "sample": f"{ncores} independent seeded copies of the sample, one per core, "
                                      f"{budget_s / 2:.0f} s each"}
    except Exception as e:  # the single-thread figure stands on its own
        out["all_cores"] = {"unavailable": str(e)[:200]}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cfg = workload(args.workload)
    per_step = []
    for _ in range(args.warmup):
        cpu_baseline(cfg, budget_s=1.0, all_cores=False)
    tot = 0.0
    for _ in range(args.steps):
        r = cpu_baseline(cfg, budget_s=max(2.0, 30.0 / max(args.steps, 1)), all_cores=False)
        per_step.append(r["value"])
        tot += r["value"]
    v = tot / len(per_step)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "sample": r["sample"]},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": r["sample"]},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Initialise, run the warm-up steps and then --profile-steps steps of the
    workload, nothing else (a short, fixed launch sequence for ncu)."""
    import torch

    from paper_2501_10965_gb300 import dsmc
    cfg = workload(args.workload)
    sim = dsmc.Dsmc(cfg)
    sim.dsmc_step(args.warmup, sample=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.dsmc_step(args.profile_steps, sample=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    print(json.dumps({"profile_steps": args.profile_steps, "workload": args.workload,
                      "particles": sim.num_particles(), "wall_s": dt, "stats": sim.stats()}), flush=True)


def run_adaptive_region(args):
    """The adaptive treatment of Sec. 3.1 on the flow past the cylinder, on
    the paper's meshes (Sec. 4.2: Kn 0.1 on 100 x 64 cells, Kn 0.01 on 300 x
    200; 200 particles per cell; wall at the freestream temperature;
    Kn_ref 0.01): the equilibrium area fraction (cells with Kn_GLL <
    Kn_ref, weighted by area) from fields sampled over the last third of
    each of three domain transits (11 L0 at the freestream speed)."""
    import torch

    from paper_2501_10965_gb300 import dsmc, workloads as W
    out = []
    for kn, nt, nr in ((0.1, 100, 64), (0.01, 300, 200)):
        cfg = W.cylinder_2d(ntheta=nt, nr=nr, ppc=200, kn=kn, t_wall=1.0, kn_ref=0.01)
        sim = dsmc.Dsmc(cfg)
        u_inf = float(cfg["fs_u"][0])
        transit = int(math.ceil(2.0 * float(cfg["r_out"]) / u_inf / float(cfg["dt"])))
        vol = sim.volumes()
        fr = []
        t0 = time.perf_counter()
        for _ in range(3):
            sim.dsmc_step(transit - transit // 3)
            sim.dsmc_sample(reset=True)
            sim.dsmc_step(transit // 3, sample=True)
            f = sim.dsmc_sample(reset=True)
            _, kngll, mask = sim.dsmc_hot(f)
            m = mask.cpu().numpy().astype(bool)
            fr.append(float(vol[~m].sum() / vol.sum()))
        torch.cuda.synchronize()
        out.append({"kn": kn, "mesh": f"{nt} x {nr}", "particles": sim.num_particles(), "steps_per_transit": transit,
                    "equilibrium_fraction_after_transit": fr, "wall_s": time.perf_counter() - t0,
                    "paper": 0.44 if kn == 0.1 else 0.79})
        del sim
        torch.cuda.empty_cache()
    print(json.dumps({"adaptive_region": out, "kn_ref": 0.01}), flush=True)


def run_synth2d(args):
    """The 2D synthetic solve (Sec. 3 step 3) on its own: a smooth
    recirculating cavity state with seeded HoT (workloads.smooth_cavity_state)
    solved to a relative update of 1e-10 on nx x ny cells (uniform, or the
    wall-refined grid of Sec. 4.1 with a first cell of 0.001), timed on the
    host around the call (it synchronises), best of --synth2d-reps; on the
    uniform grid also a solve of a second state (seed 6) that starts from
    the factorisation the first state's solve left, as DIG's iterations do
    with dsmc_synth_reuse."""
    import numpy as np
    import torch

    from paper_2501_10965_gb300 import dsmc, workloads as W
    nx, ny = (int(v) for v in args.synth2d.lower().split("x"))
    refined = args.synth2d_refined
    if refined:
        cfg = W.cavity_2d_refined(nx=nx, ny=ny, ppc=2, kn=0.05, dx_min=0.001, precision="fp64", synth2d=True,
                                  synth_tol=1e-10, n_m=50)
        q = float(cfg["stretch"])

        def centres(n):
            w = q ** np.minimum(np.arange(n), n - 1 - np.arange(n)).astype(np.float64)
            e = np.concatenate([[0.0], np.cumsum(w / w.sum())])
            return 0.5 * (e[:-1] + e[1:])
        d, h = W.smooth_cavity_state(nx, ny, seed=5, xc=centres(nx), yc=centres(ny))
    else:
        cfg = W.cavity_2d(nx=nx, ny=ny, ppc=2, kn=0.05, precision="fp64", synth2d=True, synth_tol=1e-10, n_m=50)
        d, h = W.smooth_cavity_state(nx, ny, seed=5)
    sim = dsmc.Dsmc(cfg)
    D = torch.tensor(d, dtype=torch.float64, device="cuda")
    H = torch.tensor(h, dtype=torch.float64, device="cuda")
    ts, it, res = [], 0, 0.0
    for _ in range(max(1, args.synth2d_reps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, it, res = sim.synth_solve(D, H)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    line = {"synth2d": f"{nx} x {ny}", "refined": refined, "unknowns": 5 * nx * ny,
            "ms_per_solve": 1e3 * min(ts), "all_ms": [1e3 * t for t in ts], "newton_steps": it, "max_residual": res}
    # as in DIG: a solve of another state (seed 6) that starts from the
    # factorisation the previous solve left (dsmc_synth_reuse)
    if not refined:
        d2, h2 = W.smooth_cavity_state(nx, ny, seed=6)
        D2 = torch.tensor(d2, dtype=torch.float64, device="cuda")
        H2 = torch.tensor(h2, dtype=torch.float64, device="cuda")
        sim.synth_reuse(True)
        tr = []
        for rep in range(max(1, args.synth2d_reps)):
            sim.synth_solve(D if rep % 2 else D2, H if rep % 2 else H2)  # leaves a factorisation of the other state
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, it2, _ = sim.synth_solve(D2 if rep % 2 else D, H2 if rep % 2 else H)
            torch.cuda.synchronize()
            tr.append(time.perf_counter() - t0)
        line.update(ms_per_solve_reused=1e3 * min(tr), newton_steps_reused=it2)
        # and Newton from the previous solution too
        sim.synth_reuse(True, warm=True)
        tw = []
        for rep in range(max(1, args.synth2d_reps)):
            sim.synth_solve(D if rep % 2 else D2, H if rep % 2 else H2)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, it3, _ = sim.synth_solve(D2 if rep % 2 else D, H2 if rep % 2 else H)
            torch.cuda.synchronize()
            tw.append(time.perf_counter() - t0)
        line.update(ms_per_solve_warm=1e3 * min(tw), newton_steps_warm=it3)
    print(json.dumps(line), flush=True)


def run_tts2d(args):
    """DIG against plain DSMC on 2D lid-driven cavities, steps and GPU wall
    time to steady state (dig.time_to_steady_2d), from the same uniform
    state, lid 100 m/s, N_s = 100, FP32 particles, cells of the mean free
    path: Kn 0.02 on 50 x 50 cells (1000 per cell, 2.5 M particles; windows
    of 200 steps, bins of 5 x 5 cells) and Kn 0.01 on 100 x 100 (500 per
    cell, 5 M; windows of 500 steps, bins of 10 x 10 cells), where viscous
    diffusion takes four times longer; and the flow past the cylinder at Kn
    0.1 on the paper's 100 x 64 annulus, at Mach 5 and Mach 0.5."""
    from paper_2501_10965_gb300 import dig, workloads as W
    out = []
    for kn, n, ppc, window, b, transient, average, max_plain in ((0.02, 50, 1000, 200, 5, 15000, 10000, 20000),
                                                                 (0.01, 100, 500, 500, 10, 40000, 20000, 40000)):
        if args.tts2d_case and args.tts2d_case != str(kn):
            continue
        cfg = W.cavity_2d(nx=n, ny=n, ppc=ppc, kn=kn, lid_mps=100.0, synth2d=True, synth_tol=1e-8, n_m=50)
        r = dig.time_to_steady_2d(cfg, window=window, bx=b, by=b, transient=transient, average=average,
                                  max_dig=4000, max_plain=max_plain)
        out.append(dict(r, case="cavity", kn=kn, lid_mps=100.0, n_s=int(cfg["n_s"]), kn_ref=float(cfg["kn_ref"])))
        print(json.dumps({"time_to_steady_2d": out[-1]}), flush=True)
    # the flow past the cylinder at Kn 0.1 on the paper's 100 x 64 mesh
    # (Sec. 4.2), 100 particles per cell (0.64 M), the wall at the freestream
    # temperature, Kn_ref 0.01 as in the paper: Mach 5 (the paper's case;
    # windows of 500 steps, a transit of the domain takes ~2 760) and Mach
    # 0.5 (windows of 1 000 steps, a transit ~11 100); bins of 10 sectors x
    # 8 rings
    for mach, window, transient, average, max_plain in ((5.0, 500, 15000, 15000, 25000),
                                                        (0.5, 1000, 60000, 30000, 80000)):
        if args.tts2d_case and args.tts2d_case != f"cylinder{mach:g}":
            continue
        cfg = W.cylinder_2d(ntheta=100, nr=64, ppc=100, kn=0.1, mach=mach, t_wall=1.0, kn_ref=0.01, synth2d=True,
                            synth_tol=1e-8, n_m=50)
        r = dig.time_to_steady_2d(cfg, window=window, bx=10, by=8, transient=transient, average=average,
                                  max_dig=6000, max_plain=max_plain)
        out.append(dict(r, case="cylinder", kn=0.1, mach=mach, n_s=int(cfg["n_s"]), kn_ref=0.01))
        print(json.dumps({"time_to_steady_2d": out[-1]}), flush=True)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2501_10965_gb300 import dsmc

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", rank=rank, world_size=world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # independent replicas: every rank runs its own seeded copy of the workload
    cfg = replica_config(workload(args.workload), rank)
    prec = cfg["precision"]
    dim = int(cfg["dim"])
    stream = torch.cuda.current_stream(dev)
    sim = dsmc.Dsmc(cfg, device=dev, stream=stream)
    n = sim.num_particles()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (untimed)
    sim.dsmc_step(max(args.warmup, 3), sample=True)
    reb0 = sim.stats()["n_rebuild"]
    barrier()
    with ClockSampler(local) as clk:
        barrier()
        t = _events_time(lambda: sim.dsmc_step(args.steps, sample=True), stream)
        barrier()
    clocks = clk.summary()
    reb1 = sim.stats()["n_rebuild"]
    t = over_ranks(t, world, "max", dev)
    # particle-steps: the count changes on the annulus (entry and exit), so
    # the mean of the counts before and after the timed steps
    n_end = sim.num_particles()
    n_mean = 0.5 * (n + n_end)
    value = job_throughput(n_mean, args.steps, t, world, dev)
    cfg_line_shape = sim.launch_shape()

    # average duration of one fused step kernel: difference of two runs with
    # different step counts on the launching stream (the constant parts --
    # the first move-only and last collide-only launch and the bin check --
    # cancel)
    k1, k2 = 4, 4 + max(8, min(args.steps // 2, 200))
    t1 = min(_events_time(lambda: sim.dsmc_step(k1, sample=True), stream) for _ in range(2))
    t2 = min(_events_time(lambda: sim.dsmc_step(k2, sample=True), stream) for _ in range(2))
    per_launch = (t2 - t1) / (k2 - k1)
    n = sim.num_particles()
    algo = ALGO_BYTES_PER_PARTICLE_STEP[(prec, dim)] * n
    mesh = cfg.get("mesh", "box")
    peaks = measured_peaks()
    achieved = algo / per_launch / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": args.traffic if args.traffic is not None else (
                    NCU_TRAFFIC_BYTES_PER_PARTICLE_STEP[(prec, dim, mesh)] * n
                    if (prec, dim, mesh) in NCU_TRAFFIC_BYTES_PER_PARTICLE_STEP else None),
                "kernel": "k_fused (collide + sample + move + bin append, one launch per step)",
                "algorithmic_bytes_per_launch": algo, "launch_ms": per_launch * 1e3,
                "peak_source": peaks["source"] + " (MEASURED_PEAKS.json hbm_gbs, burst copy)"}

    # end to end through the C ABI with host buffers: upload the particle
    # state from pinned host memory, K steps, download the sampled fields
    p = sim.get_particles()
    host = {k: v.to("cpu").pin_memory() for k, v in p.items() if k != "cell"}
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    fields_host = torch.empty((sim.ncells, dsmc.NFIELDS), dtype=torch.float64).pin_memory()
    d2h = fields_host.numel() * fields_host.element_size()

    def e2e():
        dev_p = {k: v.to(dev, non_blocking=True) for k, v in host.items()}
        sim.set_particles(dev_p)
        sim.dsmc_sample(reset=True)
        sim.dsmc_step(args.steps, sample=True)
        f = sim.dsmc_sample(reset=True)
        fields_host.copy_(f, non_blocking=True)
    barrier()
    n_up = len(host["x"])
    te = over_ranks(_events_time(e2e, stream), world, "max", dev)
    e2e_value = job_throughput(0.5 * (n_up + sim.num_particles()), args.steps, te, world, dev)
    stats = sim.stats()
    ncells = sim.ncells

    # per dsmc_step(K): one move-only launch, K - 1 fused launches and one
    # collide-and-sample launch, plus on the annulus the entry kernel after
    # each of the K moves; a bin rebuild adds 5
    gpu_launches = (args.steps + 1) + (args.steps if cfg.get("mesh") == "annulus" else 0) + 5 * (reb1 - reb0)

    # batched ensemble: 64 independent 1D cases of uneven size in one handle
    # (one launch per step for all of them), device-resident
    ens = None
    if rank == 0 and not args.no_ensemble:
        from paper_2501_10965_gb300 import workloads as Wk
        ge = dsmc.Dsmc(Wk.ensemble_1d(64))
        ge.dsmc_step(10, sample=True)
        ke = 200
        t_e = _events_time(lambda: ge.dsmc_step(ke, sample=True), stream)
        ne = ge.num_particles()
        ens = {"workload": "64 1D cases (Fourier/Couette alternating), 50..800 cells, 50..200 particles per cell, "
                           "Kn 1e-3..1, Z 2/5/10, FP32; seeds 0..63",
               "cells": ge.ncells, "particles": ne, "steps": ke, "value": ne * ke / t_e, "unit": METRIC,
               "ms_per_step": t_e / ke * 1e3}
        del ge
        torch.cuda.empty_cache()
    tts = None
    if rank == 0 and not args.no_time_to_steady:
        from paper_2501_10965_gb300 import dig, workloads as Wk
        del sim, p, fields_host
        torch.cuda.empty_cache()
        cfg_tts = Wk.couette_1d(kn=0.01, kn_ref=0.1)
        # the HoT network for "dig_mlp": trained on plain DIG's own states
        # (independent seeds), judged cell by cell against the DSMC terms
        t_train = time.perf_counter()
        params, tinfo = dig.train_hot_model_on_dig([cfg_tts], replicas=64, iterations=40)
        t_train = time.perf_counter() - t_train
        tts = dig.time_to_steady_dig_vs_plain(cfg_tts, replicas=args.tts_replicas, hot_params=params)
        tts["workload"] = ("1D Couette, Kn 0.01, 200 cells x 200 particles, walls -/+100 m/s; DIG every 50 steps, "
                           "Kn_ref 0.1; ensemble of replicas in one batched handle; dig_mlp: DIG with the HoT "
                           "network judged against the DSMC terms (z 3, pooled over the replicas of a cell)")
        tts["network_training"] = dict(tinfo, wall_s=t_train)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64",
                "data": "synthetic",
                "config": {"workload": args.workload, "cells": ncells, "particles": n_mean,
                           "particles_per_cell": cfg["ppc"], "kn": cfg["kn"], "dt": cfg["dt"],
                           "precision": prec + " particles, fp64 compensated moments",
                           "l2": "inputs larger than L2 (particle state %.2f GB)" % (n * 24 / 1e9),
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "fused_warps_per_cta": cfg_line_shape[0], "fused_tile": cfg_line_shape[1]},
                "roofline": roofline, "clocks": clocks, "gpu_launches": gpu_launches,
                "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": h2d / args.steps,
                        "d2h_bytes_per_step": d2h / args.steps},
                "cpu_baseline": cpu,
                "time_to_steady": tts,
                "ensemble64": ens,
                "stats": stats}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="cylinder2d_20m")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per fused launch from an ncu capture of the current kernel")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-time-to-steady", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--tts-replicas", type=int, default=800)
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="only run warm-up + this many steps (for profiler captures)")
    ap.add_argument("--adaptive-region", action="store_true",
                    help="only measure the equilibrium area fraction of the cylinder cases")
    ap.add_argument("--synth2d", default="",
                    help="only time the 2D synthetic solve on NXxNY cells (e.g. 100x100)")
    ap.add_argument("--synth2d-refined", action="store_true", help="on the wall-refined grid")
    ap.add_argument("--synth2d-reps", type=int, default=3)
    ap.add_argument("--tts2d", action="store_true",
                    help="only measure DIG against plain DSMC to steady state on 2D cavities")
    ap.add_argument("--tts2d-case", default="",
                    help="only one case: 0.02, 0.01 (cavities), cylinder5 or cylinder0.5")
    args = ap.parse_args()
    if args.tts2d:
        run_tts2d(args)
    elif args.synth2d:
        run_synth2d(args)
    elif args.adaptive_region:
        run_adaptive_region(args)
    elif args.profile_steps > 0:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
