"""FP32 particle state against the FP64 oracle, field by field, on the 1D
Couette flow of 200 cells x 200 particles (walls at -/+100 m/s, 273 K) at
Kn 0.01, 0.1 and 1: the FP32 layout (FP32 particles, compensated FP64
moment accumulators) and the FP64 oracle run the same case from the same
uniform start with independent seeds; the time-averaged rho, u_y, T_t, T_r,
sigma_xy, q_t,x and q_r,x of every cell over the same window agree within 3
standard errors of the seeds' spread, and so do their domain means.

With ``-s`` the test prints, per Kn and field, the FP64 domain mean, the
FP32 - FP64 difference of the domain means with its standard error, and
the largest |difference| / SE over the cells: the error statement of the
FP32 layout.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle_runs
from paper_2501_10965_gb300 import workloads as W
from stats3se import assert_within_3se

pytestmark = pytest.mark.gpu

FIELDS = (("rho", 0), ("u_y", 2), ("T_t", 4), ("T_r", 5), ("sigma_xy", 9), ("q_t,x", 12), ("q_r,x", 15))
# transient steps before the window, steps in the window
WINDOWS = {0.01: (3000, 2000), 0.1: (1500, 2000), 1.0: (1500, 2000)}


def _gpu_run(kn, seed, warm, ns):
    from paper_2501_10965_gb300 import dsmc
    g = dsmc.Dsmc(W.couette_1d(kn=kn, precision="fp32", seed=seed))
    g.dsmc_step(warm)
    g.dsmc_sample(reset=True)
    g.dsmc_step(ns, sample=True)
    return g.dsmc_sample(reset=True).cpu().numpy()


@pytest.mark.parametrize("kn", sorted(WINDOWS))
def test_fp32_fields_against_fp64_oracle(kn):
    warm, ns = WINDOWS[kn]
    # the oracle's seeds run in spawned worker processes while the GPU runs
    with oracle_runs.pool(4) as ex:
        jobs = [ex.submit(oracle_runs.couette_fields, kn, s, warm, ns) for s in range(4)]
        fg = np.array([_gpu_run(kn, 100 + s, warm, ns) for s in range(8)])
        fo = np.array([j.result() for j in jobs])
    print(f"\nKn {kn}: steps {warm}..{warm + ns}, 8 FP32 GPU seeds, 4 FP64 oracle seeds")
    print(f"{'field':>9} {'FP64 mean':>12} {'FP32-FP64':>12} {'SE':>10} {'max|z| cells':>13}")
    for name, col in FIELDS:
        a, b = fg[:, :, col], fo[:, :, col]
        dm = a.mean(1).mean() - b.mean(1).mean()
        se = np.sqrt(a.mean(1).var(ddof=1) / len(a) + b.mean(1).var(ddof=1) / len(b))
        if name == "rho":
            # the total mass is the same in every run
            assert abs(dm) < 1e-9
            z = assert_within_3se(a, b, what=f"Kn {kn} {name} profile", window=9)
        else:
            assert_within_3se(a.mean(1), b.mean(1), what=f"Kn {kn} {name} domain mean")
            z = assert_within_3se(a, b, what=f"Kn {kn} {name} profile", window=9)
        print(f"{name:>9} {b.mean():12.5g} {dm:12.3e} {se:10.2e} {z.max():13.2f}")
