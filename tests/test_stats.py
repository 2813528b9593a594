"""The error-bar and autocorrelation helpers against AR(1) closed forms."""
import numpy as np

from oracle.closed_forms import ar1_tau_int
from paper_2402_06415_gb300 import stats


def _ar1(rho, n, seed):
    rng = np.random.default_rng(seed)
    e = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = e[0] / np.sqrt(1 - rho * rho)
    for i in range(1, n):
        x[i] = rho * x[i - 1] + e[i]
    return x * np.sqrt(1 - rho * rho)  # unit variance


def test_tau_int_ar1():
    for rho in (0.0, 0.5, 0.9):
        taus = [stats.tau_int(_ar1(rho, 200000, s)) for s in range(3)]
        want = ar1_tau_int(rho)
        assert abs(np.mean(taus) - want) < 0.08 * want + 0.02, (rho, taus, want)


def test_blocking_error_ar1():
    rho = 0.8
    n = 200000
    x = _ar1(rho, n, 7)
    want = np.sqrt(2 * ar1_tau_int(rho) / n)  # unit variance
    got = stats.blocking_error(x)
    assert 0.8 * want < got < 1.25 * want, (got, want)


def test_independent_samples_per_second():
    x = _ar1(0.0, 100000, 1)
    v = stats.independent_samples_per_second(x, seconds=10.0, chains=2)
    assert abs(v - 100000 / 10 / 1.0 * 2) < 0.1 * v


def test_tau_int_chains_ar1():
    """Pooled over 32 short AR(1) chains (each 40 tau long) the estimate agrees
    with the closed form within its jackknife error (and 10 %)."""
    rho = 0.95
    want = ar1_tau_int(rho)  # 19.5
    X = np.stack([_ar1(rho, 800, 100 + s) for s in range(32)], axis=1)
    tau, err = stats.tau_int_chains(X)
    assert err > 0
    assert abs(tau - want) < max(3 * err, 0.1 * want), (tau, err, want)
