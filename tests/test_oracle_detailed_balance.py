"""Exact transition-kernel checks of the oracle's Metropolis decision (CPU).

The flip probability of a site is taken from the oracle's own code: its
antiparallel-neighbour count and the exact number of 32-bit uniforms its
decision accepts (found by bisection on the decision).  The stationary weight
is the plain Boltzmann factor from ``oracle.exact`` (an independent energy).

* 3 x 3 periodic lattice (not bipartite, so no checkerboard): every
  single-site kernel satisfies detailed balance, and the sequential sweep over
  the 9 sites leaves the Boltzmann distribution invariant.
* 4 x 4 periodic lattice: each checkerboard half sweep (all sites of one colour
  at once) satisfies detailed balance exactly, up to the 2^-32 quantisation of
  the thresholds, and leaves the Boltzmann distribution invariant.
"""
import numpy as np
import pytest

from oracle import exact

BETAS = [0.3, 0.4406867935097715, 0.6]


def _flip_prob(orc, beta, S):
    t4, t8 = orc.threshold(beta, 4), orc.threshold(beta, 8)
    table = np.array([orc.accept_count(n, t4, t8) for n in range(5)], dtype=np.float64) / 2 ** 32
    return table[orc.n_anti_all(S)], (t4, t8)


def _rtol(t4, t8, nfactors):
    # each factor carries relative quantisation error < 1/T
    return 4.0 * nfactors / min(t4, t8)


@pytest.mark.parametrize("beta", BETAS)
def test_single_site_detailed_balance_3x3(orc, beta):
    L = 3
    S = exact.all_configs(L)
    pi = exact.boltzmann(L, beta)
    A, (t4, t8) = _flip_prob(orc, beta, S)  # (512, 3, 3)
    n = S.shape[0]
    idx = np.arange(n)
    for site in range(L * L):
        y, x = divmod(site, L)
        j = idx ^ (1 << site)  # configuration with this site flipped
        lhs = pi * A[:, y, x]
        rhs = pi[j] * A[j, y, x]
        np.testing.assert_allclose(lhs, rhs, rtol=_rtol(t4, t8, 1), atol=0)


@pytest.mark.parametrize("beta", BETAS)
def test_sequential_sweep_stationary_3x3(orc, beta):
    L = 3
    S = exact.all_configs(L)
    pi = exact.boltzmann(L, beta)
    A, (t4, t8) = _flip_prob(orc, beta, S)
    n = S.shape[0]
    idx = np.arange(n)
    P = np.eye(n)
    for site in range(L * L):
        y, x = divmod(site, L)
        Pi = np.zeros((n, n))
        Pi[idx, idx] = 1 - A[:, y, x]
        Pi[idx, idx ^ (1 << site)] = A[:, y, x]
        P = P @ Pi
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(pi @ P, pi, rtol=_rtol(t4, t8, 9), atol=1e-300)


@pytest.mark.parametrize("beta", BETAS)
@pytest.mark.parametrize("colour", [0, 1])
def test_half_sweep_detailed_balance_4x4(orc, beta, colour):
    L = 4
    S = exact.all_configs(L)
    pi = exact.boltzmann(L, beta)
    A, (t4, t8) = _flip_prob(orc, beta, S)  # (65536, 4, 4)
    sites = [(y, x) for y in range(L) for x in range(L) if (x + y) % 2 == colour]
    bits = np.array([1 << (y * L + x) for (y, x) in sites], dtype=np.int64)
    a = np.stack([A[:, y, x] for (y, x) in sites], axis=1)  # (65536, 8)
    n = S.shape[0]
    idx = np.arange(n, dtype=np.int64)
    stat = np.zeros(n)
    rtol = _rtol(t4, t8, 2 * len(sites))
    for F in range(1 << len(sites)):
        f = ((F >> np.arange(len(sites))) & 1).astype(bool)
        mask = int(bits[f].sum())
        j = idx ^ mask
        pxy = np.prod(np.where(f[None, :], a, 1 - a), axis=1)
        pyx = np.prod(np.where(f[None, :], a[j], 1 - a[j]), axis=1)
        lhs = pi * pxy
        rhs = pi[j] * pyx
        np.testing.assert_allclose(lhs, rhs, rtol=rtol, atol=1e-300)
        np.add.at(stat, j, lhs)
    np.testing.assert_allclose(stat, pi, rtol=rtol, atol=1e-300)


def test_wrong_kernel_breaks_detailed_balance(orc):
    """A Metropolis kernel with exp(-2 beta dE) instead of exp(-beta dE) fails
    the same check, so the check has teeth."""
    L, beta = 3, 0.4
    S = exact.all_configs(L)
    pi = exact.boltzmann(L, beta)
    t4, t8 = orc.threshold(2 * beta, 4), orc.threshold(2 * beta, 8)
    table = np.array([orc.accept_count(n, t4, t8) for n in range(5)], dtype=np.float64) / 2 ** 32
    A = table[orc.n_anti_all(S)]
    idx = np.arange(S.shape[0])
    j = idx ^ 1
    assert not np.allclose(pi * A[:, 0, 0], pi[j] * A[j, 0, 0], rtol=1e-6)
