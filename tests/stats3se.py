"""The "within 3 standard errors" comparisons of the statistical tests.

A standard error comes from the spread of independent replicas (different
seeds), never from batches of one run, whose correlation understates it.
With k replicas the estimated SE has k - 1 degrees of freedom, so the
difference over its SE follows a t distribution, not a normal one; the bound
is taken at the same two-sided 99.73 % level as 3 standard errors of a
normal variable (t_{0.99865, dof}: 3.64 for 14 degrees of freedom, 3.26
for 31, 3.0 for many).

Profiles (one value per cell) may pool the two samples' variance and
average it over a few neighbouring cells (pooled), keeping the degrees of
freedom of a single cell.

Where many values are compared at once (cells, rings, regions), chance alone
puts some outside the bound: p = 0.27 % each.  The number allowed outside is
the smallest k that independent comparisons exceed with probability below
1 %, i.e. 0 for up to 3 values, 1 for up to 55, 2 for up to 162.  No
value may lie beyond 5 of its standard errors, or, where few replicas give
the t variable a heavier tail than that, beyond the t point that any of the
n values exceeds with probability below 1 % (ALPHA / n each, Bonferroni,
valid however the values are correlated): 6.8 SE for 200 cells at 10
degrees of freedom, 5 SE at 31 degrees of freedom and more.

Neighbouring cells of a profile are not independent: a fluctuation of the
flow spans many cells (10 to 85 of the 200 of the 1D Couette flow sampled
over 2 000 steps), so values beyond the bound come in runs.  Profiles therefore count runs, not cells: the
correlation length l (cells) of the replicas' deviations along the profile
is measured (1 + twice the sum of the lag correlations while they exceed
0.05), outside values closer than l cells form one run, a run counts once
per l cells it spans, and the number of runs allowed is that of n / l
independent regions, each outside with probability at most min(0.5, l p)
(for uncorrelated cells, l = 1: the rule above).
"""
from __future__ import annotations

import math

import numpy as np

P_OUT = 0.0027      # two-sided tail beyond 3 standard errors of a normal variable
ALPHA = 0.01        # false-alarm probability of a whole comparison
HARD = 5.0          # no value beyond this many standard errors (hard_bound)


def hard_bound(dof, n: int):
    """The bound no value may exceed: HARD, or the two-sided t point at
    level ALPHA / n where the t variable's tail is heavier."""
    from scipy import stats
    return np.maximum(HARD, stats.t.ppf(1.0 - ALPHA / (2.0 * n), np.maximum(dof, 1.0)))


def t_bound(dof: float) -> float:
    """Two-sided 99.73 % point of Student's t with dof degrees of freedom."""
    from scipy import stats
    return float(stats.t.ppf(1.0 - P_OUT / 2.0, max(dof, 1.0)))


def allowed_outside(n: int, p: float = P_OUT) -> int:
    """Smallest k with P(Binomial(n, p) > k) < ALPHA."""
    k, cdf = 0, 0.0
    while True:
        cdf += math.comb(n, k) * p ** k * (1.0 - p) ** (n - k)
        if 1.0 - cdf < ALPHA or k >= n:
            return k
        k += 1


def corr_length(a: np.ndarray, b: np.ndarray, max_lag: int = 64) -> float:
    """Correlation length (cells) of profiles a, b (replicas x cells): 1 +
    twice the sum of the lag-k correlations of the replicas' deviations from
    their group means (each cell's deviations scaled by their spread), while
    they exceed 0.05."""
    dev = np.concatenate([a - a.mean(0), b - b.mean(0)], axis=0)
    sd = np.sqrt((dev ** 2).mean(0))
    dev = dev / np.where(sd > 0, sd, 1.0)
    n = dev.shape[1]
    c0 = np.mean(dev ** 2)
    if not c0 > 0:
        return 1.0
    tot = 0.0
    for k in range(1, min(max_lag, n // 4)):
        r = float(np.mean(dev[:, :-k] * dev[:, k:]) / c0)
        if r < 0.05:
            break
        tot += r
    return 1.0 + 2.0 * tot


def count_runs(idx: np.ndarray, ell: float) -> int:
    """Runs among the sorted cell indices idx: indices closer than ell cells
    form one run, and a run counts once per ell cells it spans."""
    out = 0
    for run in np.split(idx, np.nonzero(np.diff(idx) >= ell)[0] + 1):
        if run.size:
            out += int(math.ceil((run[-1] - run[0] + 1) / ell))
    return out


def pooled(a: np.ndarray, b: np.ndarray, window: int):
    """Difference of the replica means of profiles a and b (replicas x
    cells), its standard error and degrees of freedom, with the two-sample
    pooled variance of each cell averaged over `window` neighbouring cells
    (the variance of a cell mean varies smoothly along a profile; a 4-seed
    variance alone has 3 degrees of freedom and a heavy tail).  The degrees
    of freedom are those of one cell, na + nb - 2, as if the window added
    nothing (neighbouring cells are correlated)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    na, nb = a.shape[0], b.shape[0]
    s2 = ((na - 1) * a.var(0, ddof=1) + (nb - 1) * b.var(0, ddof=1)) / (na + nb - 2)
    h = window // 2
    s2 = np.convolve(np.pad(s2, h, mode="edge"), np.ones(window) / window, mode="valid")
    return a.mean(0) - b.mean(0), np.sqrt(s2 * (1.0 / na + 1.0 / nb)), np.full(s2.shape, na + nb - 2.0)


def welch(a: np.ndarray, b: np.ndarray | None = None):
    """Difference of the replica means of a and b (axis 0; b None: a's mean
    against 0), its standard error and the Welch degrees of freedom."""
    a = np.asarray(a, dtype=np.float64)
    va = a.var(0, ddof=1) / a.shape[0]
    if b is None:
        return a.mean(0), np.sqrt(va), np.full(np.shape(va), a.shape[0] - 1.0)
    b = np.asarray(b, dtype=np.float64)
    vb = b.var(0, ddof=1) / b.shape[0]
    dof = (va + vb) ** 2 / (va ** 2 / (a.shape[0] - 1) + vb ** 2 / (b.shape[0] - 1) + 1e-300)
    return a.mean(0) - b.mean(0), np.sqrt(va + vb), dof


def assert_within_3se(a, b=None, what: str = "", floor: float = 0.0, window: int = 0):
    """Replicas a against replicas b (or against 0): every compared value
    within the 3-SE bound, up to allowed_outside(n) of them, and none beyond
    hard_bound standard errors.  floor: an absolute SE floor for values whose
    spread is exactly zero (e.g. a conserved total).  window > 1 (profiles
    against profiles): the pooled variance averaged over that many
    neighbouring cells (pooled), and outside cells counted as runs over
    the profile's correlation length (count_runs)."""
    profile = window > 1 and b is not None
    d, se, dof = pooled(a, b, window) if profile else welch(a, b)
    d, se, dof = np.atleast_1d(d), np.atleast_1d(se) + floor, np.atleast_1d(dof)
    z = np.abs(d) / np.where(se > 0, se, 1e-300)
    thr = np.array([t_bound(v) for v in dof])
    idx = np.nonzero(z > thr)[0]
    if profile:
        ell = corr_length(np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64))
        out, unit = count_runs(idx, ell), f"runs (correlation length {ell:.1f} cells) of {z.size} cells"
        k = allowed_outside(max(1, int(round(z.size / ell))), min(0.5, P_OUT * ell))
    else:
        out, unit = idx.size, f"of {z.size}"
        k = allowed_outside(z.size)
    assert out <= k and np.all(z <= np.maximum(hard_bound(dof, z.size), thr)), (
        f"{what}: {out} {unit} beyond 3 SE (allowed {k}); largest |diff|/SE "
        f"{np.sort(z)[-3:]} at {np.argsort(z)[-3:]}, diff {d[np.argsort(z)[-3:]]}, SE {se[np.argsort(z)[-3:]]}")
    return z
