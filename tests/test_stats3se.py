"""CPU checks of the 3-standard-error comparison used by the statistical
GPU tests: its false-alarm rate on replicas with no difference, and that a
difference of 8 standard errors in one of five values fails it (one value
of five may lie outside 3 standard errors, none beyond 5)."""
import numpy as np
import pytest

from stats3se import allowed_outside, assert_within_3se, t_bound


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
