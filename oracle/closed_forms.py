"""Closed forms of the 2D square-lattice Ising model (J = 1, h = 0).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  These are textbook exact
results; they pin the oracle chain where the paper (arXiv 2402.06415, which
reports only the XY model and, for Ising, timings) prints no Ising values.

* beta_c = ln(1 + sqrt 2) / 2                      (Kramers-Wannier 1941)
* Onsager (1944) internal energy per site of the infinite lattice:
      u = -coth(2K) [1 + (2/pi) (2 tanh^2(2K) - 1) K1(k)],
      k = 2 sinh(2K) / cosh^2(2K),  K1 = complete elliptic integral, 1st kind
* Yang (1952) spontaneous magnetisation: m = (1 - sinh(2K)^-4)^(1/8), K > K_c
* Kaufman (1949) partition function of the finite m x n torus:
      Z = 1/2 (2 sinh 2K)^(mn/2) (Z1 + Z2 + Z3 + Z4)
      Z1 = prod_{k<n} 2 cosh(m g_{2k+1}/2),  Z2 = prod_{k<n} 2 sinh(m g_{2k+1}/2)
      Z3 = prod_{k<n} 2 cosh(m g_{2k}/2),    Z4 = prod_{k<n} 2 sinh(m g_{2k}/2)
      cosh g_l = cosh(2K) coth(2K) - cos(pi l / n)  (g_l > 0, l >= 1)
      g_0 = 2K + ln tanh K  (signed: negative below T_c)
  and the finite-lattice energy per site e = -(1/N) d ln Z / d beta.
"""
from __future__ import annotations

import math

import mpmath
import numpy as np
from scipy import special

BETA_C = math.log(1.0 + math.sqrt(2.0)) / 2.0


def onsager_energy(beta: float) -> float:
    """Infinite-lattice internal energy per site (two bonds per site)."""
    K = float(beta)
    if abs(K - BETA_C) < 1e-12:
        return -math.sqrt(2.0)
    k = 2.0 * math.sinh(2 * K) / math.cosh(2 * K) ** 2
    K1 = special.ellipk(k * k)
    return -(1.0 / math.tanh(2 * K)) * (1.0 + (2.0 / math.pi) * (2.0 * math.tanh(2 * K) ** 2 - 1.0) * K1)


def yang_magnetisation(beta: float) -> float:
    """Spontaneous magnetisation per site; 0 at and above T_c."""
    K = float(beta)
    if K <= BETA_C:
        return 0.0
    return (1.0 - math.sinh(2 * K) ** -4) ** 0.125


def _kaufman_lnZ(m: int, n: int, beta):
    K = mpmath.mpf(beta)
    c2 = mpmath.cosh(2 * K)
    cth = mpmath.coth(2 * K)

    def gamma(l):
        if l == 0:
            return 2 * K + mpmath.log(mpmath.tanh(K))
        return mpmath.acosh(c2 * cth - mpmath.cos(mpmath.pi * l / n))

    g = [gamma(l) for l in range(2 * n)]
    Z1 = mpmath.mpf(1)
    Z2 = mpmath.mpf(1)
    Z3 = mpmath.mpf(1)
    Z4 = mpmath.mpf(1)
    for k in range(n):
        Z1 *= 2 * mpmath.cosh(m * g[2 * k + 1] / 2)
        Z2 *= 2 * mpmath.sinh(m * g[2 * k + 1] / 2)
        Z3 *= 2 * mpmath.cosh(m * g[2 * k] / 2)
        Z4 *= 2 * mpmath.sinh(m * g[2 * k] / 2)
    pref = mpmath.mpf(1) / 2 * (2 * mpmath.sinh(2 * K)) ** (mpmath.mpf(m * n) / 2)
    return mpmath.log(pref * (Z1 + Z2 + Z3 + Z4))


def kaufman_lnZ(L: int, beta: float, dps: int = 60) -> float:
    """ln Z of the L x L periodic lattice (Kaufman)."""
    with mpmath.workdps(dps):
        return float(_kaufman_lnZ(L, L, beta))


def kaufman_energy(L: int, beta: float, dps: int = 60) -> float:
    """Exact internal energy per site of the L x L periodic lattice."""
    with mpmath.workdps(dps):
        d = mpmath.diff(lambda b: _kaufman_lnZ(L, L, b), mpmath.mpf(beta))
        return float(-d / (L * L))


def thresholds_exact(beta: float, dE: int) -> int:
    """floor(exp(-beta dE) 2^32) in 60-digit arithmetic."""
    with mpmath.workdps(60):
        return int(mpmath.floor(mpmath.exp(-mpmath.mpf(beta) * dE) * mpmath.mpf(2) ** 32))


def ar1_tau_int(rho: float) -> float:
    """Integrated autocorrelation time of an AR(1) series (closed form)."""
    return 0.5 * (1.0 + rho) / (1.0 - rho)


__all__ = ["BETA_C", "onsager_energy", "yang_magnetisation", "kaufman_lnZ",
           "kaufman_energy", "thresholds_exact", "ar1_tau_int"]

_ = np  # numpy kept for callers that pass arrays of beta
