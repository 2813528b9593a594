"""Time-series statistics for Monte Carlo observables.

Host-side analysis (numpy); no part of the sweep itself.

* Blocking (binning) errors, Flyvbjerg & Petersen, J. Chem. Phys. 91, 461
  (1989): repeatedly average neighbouring pairs; the naive standard error of
  the blocked series rises to a plateau at the true standard error of the mean.
* Integrated autocorrelation time with Sokal's automatic window (Madras &
  Sokal, J. Stat. Phys. 50, 109 (1988)): tau(W) = 1/2 + sum_{t=1..W} rho(t),
  with the smallest W such that W >= c tau(W).
* Independent samples per second = (samples per second) / (2 tau_int).

The paper's own measurement protocol (Supplementary, Eq. S2 and the text
around it) averages the energy over the MC steps after a discarded warm-up
and over ten seeds; these helpers give the error bars of such averages.
"""
from __future__ import annotations

import numpy as np


def blocking_error(x, min_blocks: int = 32) -> float:
    """Standard error of the mean of a correlated series (plateau estimate:
    the largest naive error over blocking levels that keep >= min_blocks)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    if n < 2:
        return float("nan")
    best = x.std(ddof=1) / np.sqrt(n)
    while x.size >= 2 * min_blocks:
        m = x.size // 2
        x = 0.5 * (x[: 2 * m : 2] + x[1 : 2 * m : 2])
        err = x.std(ddof=1) / np.sqrt(x.size)
        best = max(best, err)
    return float(best)


def autocorrelation(x) -> np.ndarray:
    """Normalised autocorrelation function rho(t), t = 0 .. n-1 (FFT)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    y = x - x.mean()
    f = np.fft.rfft(y, 2 * n)
    acf = np.fft.irfft(f * np.conj(f))[:n]
    if acf[0] == 0.0:
        out = np.zeros(n)
        out[0] = 1.0
        return out
    return acf / acf[0]


def tau_int(x, c: float = 5.0) -> float:
    """Integrated autocorrelation time with Sokal's automatic window."""
    rho = autocorrelation(x)
    n = rho.size
    tau = 0.5
    for W in range(1, n):
        tau += rho[W]
        if W >= c * tau:
            return float(max(tau, 0.5))
    return float(max(tau, 0.5))


def _pooled_acf(X, mean):
    """Autocovariance averaged over the columns of X (steps x chains), about
    a common mean, normalised to rho(0) = 1."""
    n = X.shape[0]
    Y = X - mean
    f = np.fft.rfft(Y, 2 * n, axis=0)
    acov = np.fft.irfft(f * np.conj(f), axis=0)[:n].sum(axis=1)
    if acov[0] == 0.0:
        out = np.zeros(n)
        out[0] = 1.0
        return out
    return acov / acov[0]


def _sokal(rho, c):
    tau = 0.5
    for W in range(1, rho.size):
        tau += rho[W]
        if W >= c * tau:
            return float(max(tau, 0.5))
    return float(max(tau, 0.5))


def tau_int_chains(X, c: float = 5.0, groups: int = 8):
    """tau_int of an observable recorded by many independent chains of the
    same process: X (steps x chains).  The autocorrelation is pooled over the
    chains (deviations from the grand mean) before Sokal's automatic window;
    the error is a jackknife over `groups` groups of chains.  Returns
    (tau, error)."""
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    tau = _sokal(_pooled_acf(X, X.mean()), c)
    g = min(groups, X.shape[1])
    if g < 2:
        return tau, float("nan")
    parts = np.array_split(np.arange(X.shape[1]), g)
    jk = []
    for p in parts:
        keep = np.setdiff1d(np.arange(X.shape[1]), p)
        Xk = X[:, keep]
        jk.append(_sokal(_pooled_acf(Xk, Xk.mean()), c))
    jk = np.asarray(jk)
    err = float(np.sqrt((g - 1) / g * ((jk - jk.mean()) ** 2).sum()))
    return tau, err


def mean_and_error(x, discard: int = 0):
    x = np.asarray(x, dtype=np.float64)[discard:]
    return float(x.mean()), blocking_error(x)


def combine_runs(means, errors):
    """Mean of independent runs and its standard error (from the run means)."""
    m = np.asarray(means, dtype=np.float64)
    e = np.asarray(errors, dtype=np.float64)
    if m.size == 1:
        return float(m[0]), float(e[0])
    # Two estimates of the error: spread of the run means and propagated
    # within-run errors; the larger one is reported.
    spread = m.std(ddof=1) / np.sqrt(m.size)
    prop = np.sqrt((e ** 2).sum()) / m.size
    return float(m.mean()), float(max(spread, prop))


def independent_samples_per_second(x, seconds: float, chains: int = 1) -> float:
    """(records per second) / (2 tau_int) x chains."""
    x = np.asarray(x)
    if seconds <= 0:
        return float("nan")
    return float(x.size / seconds / (2.0 * tau_int(x)) * chains)
