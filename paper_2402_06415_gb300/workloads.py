"""Seeded synthetic workloads (inputs only; none of the method's arithmetic).

These are the lattice sizes, temperatures and seeds of the configurations the
benchmarks and tests run.  Both the CUDA path and the CPU oracle receive their
inputs from here; nothing here computes a sweep.
"""
from __future__ import annotations

import numpy as np

BETA_C = 0.4406868

# single lattice, 1 bit per spin
PLAIN_L = 16384
PLAIN_BETAS = (0.40, 0.4406868, 0.50)

# batched ladders with parallel tempering
BATCH_L_CHOICES = (16, 24, 32, 48, 64, 96, 128)
BATCH_N_LADDERS = 64
BATCH_N_BETA = 64
BATCH_BETA_RANGE = (0.35, 0.50)
BATCH_PT_EVERY = 10


def batch_ladder_sizes(n_ladders: int = BATCH_N_LADDERS, seed: int = 6) -> list[int]:
    """Lattice size of each ladder, drawn uniformly from BATCH_L_CHOICES."""
    rng = np.random.default_rng(seed)
    return [int(BATCH_L_CHOICES[i]) for i in rng.integers(0, len(BATCH_L_CHOICES), n_ladders)]


def batch_betas(n_beta: int = BATCH_N_BETA, lo: float = BATCH_BETA_RANGE[0],
                hi: float = BATCH_BETA_RANGE[1]) -> np.ndarray:
    """Evenly spaced ascending temperature slots."""
    return np.linspace(lo, hi, n_beta)


def random_spins(L: int, seed: int) -> np.ndarray:
    """Independent +-1 spins from numpy's generator (for layout round trips)."""
    rng = np.random.default_rng(seed)
    return np.where(rng.random((L, L)) < 0.5, 1, -1).astype(np.int8)
