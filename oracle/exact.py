"""Brute-force enumeration and exact transition kernels on tiny lattices.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  Everything here is the plain
definition: the Boltzmann weight exp(-beta E) summed over every configuration,
with E = -sum_{x,y} s(x,y)[s(x+1,y) + s(x,y+1)] on the periodic lattice.
"""
from __future__ import annotations

import numpy as np


def all_configs(L: int) -> np.ndarray:
    """All 2^(L*L) configurations as int8 +-1 arrays of shape (2^N, L, L);
    configuration index k has site (x, y) = +1 iff bit (y*L + x) of k is set."""
    N = L * L
    if N > 20:
        raise ValueError("too many states for brute force")
    k = np.arange(1 << N, dtype=np.int64)[:, None]
    bits = (k >> np.arange(N, dtype=np.int64)[None, :]) & 1
    return (2 * bits - 1).astype(np.int8).reshape(-1, L, L)


def energy(s: np.ndarray) -> np.ndarray:
    """E for one configuration (L, L) or a stack (..., L, L)."""
    s = s.astype(np.int64)
    return -(s * (np.roll(s, -1, axis=-1) + np.roll(s, -1, axis=-2))).sum(axis=(-1, -2))


def magnetisation(s: np.ndarray) -> np.ndarray:
    return s.astype(np.int64).sum(axis=(-1, -2))


def averages(L: int, beta: float) -> dict:
    """Exact <E>, <E^2>, <M^2>, <|M|>, ln Z by enumeration."""
    S = all_configs(L)
    E = energy(S).astype(np.float64)
    M = magnetisation(S).astype(np.float64)
    a = -beta * E
    w = np.exp(a - a.max())
    Z = w.sum()
    return {
        "E": float((w * E).sum() / Z),
        "E2": float((w * E * E).sum() / Z),
        "M2": float((w * M * M).sum() / Z),
        "absM": float((w * np.abs(M)).sum() / Z),
        "lnZ": float(np.log(Z) + a.max()),
    }


def boltzmann(L: int, beta: float) -> np.ndarray:
    """Normalised Boltzmann distribution over the configurations of all_configs(L)."""
    E = energy(all_configs(L)).astype(np.float64)
    a = -beta * E
    w = np.exp(a - a.max())
    return w / w.sum()
