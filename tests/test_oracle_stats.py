"""Pins of the oracle's integrated autocorrelation time: an AR(1) process has the closed
form tau_int = (1 + r)/(1 - r), and an iid series has tau_int = 1."""
import numpy as np

from oracle import stats


def _ar1(r, n, seed):
    rng = np.random.default_rng(seed)
    x = np.empty(n)
    x[0] = rng.normal() / np.sqrt(1 - r * r)
    eps = rng.normal(size=n)
    for t in range(1, n):
        x[t] = r * x[t - 1] + eps[t]
    return x


def test_ar1_closed_form():
    r = 0.8
    tau = stats.tau_int(_ar1(r, 100_000, 0))
    assert abs(tau - (1 + r) / (1 - r)) / 9.0 < 0.1


def test_iid_is_one():
    x = np.random.default_rng(1).normal(size=50_000)
    assert abs(stats.tau_int(x) - 1.0) < 0.1


def test_ess_sums_chains():
    x = np.random.default_rng(2).normal(size=(3, 20_000))
    assert abs(stats.ess(x) / 60_000 - 1.0) < 0.15
