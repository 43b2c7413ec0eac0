"""CPU checks of the 3-standard-error comparison used by the statistical
GPU tests: its false-alarm rate on replicas with no difference, and that a
difference of 8 standard errors in one of five values fails it (one value
of five may lie outside 3 standard errors, none beyond 5)."""
import numpy as np
import pytest

from stats3se import allowed_outside, assert_within_3se, corr_length, count_runs, hard_bound, t_bound


def test_bounds():
    assert allowed_outside(1) == 0 and allowed_outside(3) == 0 and allowed_outside(4) == 1
    assert allowed_outside(100) == 2
    assert abs(t_bound(1e7) - 3.0) < 1e-3 and 3.6 < t_bound(14) < 3.7


def test_false_alarm_rate_and_power():
    rng = np.random.default_rng(0)
    fails = 0
    for _ in range(400):
        a = rng.standard_normal((12, 100))
        b = rng.standard_normal((12, 100)) * 1.5 + 2.0
        try:
            assert_within_3se(a, b - 2.0, what="null")
        except AssertionError:
            fails += 1
    assert fails <= 12  # 1 % expected
    a = rng.standard_normal((32, 5))
    a[:, 2] += 8.0 / np.sqrt(32)  # 8 x its standard error
    with pytest.raises(AssertionError):
        assert_within_3se(a, what="shifted")


def test_pooled_profile_false_alarm_rate():
    rng = np.random.default_rng(1)
    x = np.linspace(0, 1, 200)
    sd = 0.5 + x  # a spread that varies smoothly along the profile
    fails = 0
    for _ in range(300):
        a = rng.standard_normal((8, 200)) * sd
        b = rng.standard_normal((4, 200)) * sd + 3.0
        try:
            assert_within_3se(a, b - 3.0, what="null", window=9)
        except AssertionError:
            fails += 1
    assert fails <= 9  # 1 % expected


def _smooth_noise(rng, shape, sig):
    """Unit-variance normal noise correlated along axis 1 by a Gaussian kernel
    of sig cells (autocorrelation exp(-k^2 / (4 sig^2)), correlation length
    2 sig sqrt(pi))."""
    r = int(4 * sig)
    k = np.arange(-r, r + 1)
    w = np.exp(-0.5 * (k / sig) ** 2)
    w /= np.sqrt((w ** 2).sum())
    e = rng.standard_normal((shape[0], shape[1] + 2 * r))
    return np.array([np.convolve(row, w, mode="valid") for row in e])


def test_correlation_length_and_runs():
    rng = np.random.default_rng(2)
    a, b = rng.standard_normal((8, 200)), rng.standard_normal((4, 200))
    assert corr_length(a, b) < 1.3
    # 2 sig sqrt(pi) = 10.6 for sig = 3, less the lags cut off below 0.05
    ell = corr_length(_smooth_noise(rng, (8, 200), 3.0), _smooth_noise(rng, (4, 200), 3.0))
    assert 8.0 < ell < 13.0
    assert count_runs(np.array([3, 5, 40]), 10.0) == 2
    assert count_runs(np.arange(80), 10.0) == 8  # a long run counts per 10 cells
    assert count_runs(np.array([0, 1, 2]), 1.0) == 3  # uncorrelated: every cell
    assert count_runs(np.array([], dtype=np.int64), 5.0) == 0


def test_correlated_profile_false_alarm_rate_and_power():
    """Profiles whose cells are correlated over ~20 cells (sampled DSMC
    profiles are, over 10 to 85 cells): outside cells come in runs,
    and the run count keeps the false-alarm rate near 1 %, where counting
    cells raised it to ~3.5 %.  A shift of 4.5 standard errors over 60
    cells still fails, and so does one of 8 over 3 cells."""
    rng = np.random.default_rng(3)
    x = np.linspace(0, 1, 200)
    sd = 0.5 + x
    fails = 0
    for _ in range(300):
        a = _smooth_noise(rng, (8, 200), 6.0) * sd
        b = _smooth_noise(rng, (4, 200), 6.0) * sd
        try:
            assert_within_3se(a, b, what="null", window=9)
        except AssertionError:
            fails += 1
    assert fails <= 9  # 1 % expected
    se = sd * np.sqrt(1.0 / 8 + 1.0 / 4)
    for lo, hi, shift in ((70, 130, 4.5), (100, 103, 8.0)):
        a = _smooth_noise(rng, (8, 200), 3.0) * sd
        b = _smooth_noise(rng, (4, 200), 3.0) * sd
        a[:, lo:hi] += shift * se[lo:hi]
        with pytest.raises(AssertionError):
            assert_within_3se(a, b, what="shifted", window=9)


def test_hard_bound():
    """5 SE wherever the t variable's tail is no heavier; with 10 degrees of
    freedom over 200 cells the point that any cell passes with probability
    1 % (Bonferroni)."""
    assert hard_bound(1e7, 200) == 5.0 and hard_bound(31, 5) == 5.0
    assert 6.7 < hard_bound(10, 200) < 6.8
    from scipy import stats
    assert abs(200 * 2 * stats.t.sf(hard_bound(10, 200), 10) - 0.01) < 1e-9
