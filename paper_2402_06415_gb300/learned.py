"""Host driver of the learned block proposal: training data, training loop,
evaluation.  All arithmetic (sweeps, network forward/backward, Adam, block
Metropolis-Hastings) runs in libising.so; this module only moves data.

Training data: equilibrium configurations of the plain sweep at beta, cut into
(block+2)^2 windows at random positions (ring + interior).  Loss: maximum
likelihood of the interior given the ring edges (binary cross-entropy of the
per-site logits); for the staged proposal, of every network stage's sites given
the ring and the sites drawn before that stage.
"""
from __future__ import annotations

import time

import numpy as np

from . import _binding as B


def extract_windows(spins: np.ndarray, n: int, block: int, rng) -> np.ndarray:
    """n windows of (block+2)^2 int8 spins at random positions (periodic)."""
    L = spins.shape[0]
    F = block + 2
    ys = rng.integers(0, L, n)
    xs = rng.integers(0, L, n)
    ar = np.arange(F)
    rows = (ys[:, None] + ar[None, :]) % L  # (n, F)
    cols = (xs[:, None] + ar[None, :]) % L
    return spins[rows[:, :, None], cols[:, None, :]].astype(np.int8)


def generate_windows(Ls, beta: float, n_per_L: int, block: int, seed: int, thermalise: int = 2000,
                     thin: int = 50, per_config: int = 64, stream=None) -> np.ndarray:
    """Windows from plain-sweep configurations at beta for each L in Ls."""
    rng = np.random.default_rng(seed)
    out = []
    for k, L in enumerate(Ls):
        with B.Lattice(L, beta, B.ISING_LAYOUT_BITS, stream=stream, seed=seed * 100 + k) as lat:
            lat.sweep(thermalise, 0)
            got = 0
            while got < n_per_L:
                lat.sweep(thin, 0)
                m = min(per_config, n_per_L - got)
                out.append(extract_windows(lat.spins(), m, block, rng))
                got += m
    return np.concatenate(out)


class Trainer:
    """FP32 master weights + Adam on the GPU (ising_nn_*)."""

    def __init__(self, block: int = 16, seed: int = 0, params: dict | None = None, stream=None,
                 proposal: int = B.ISING_PROPOSAL_ONESHOT, precision: int = B.ISING_NN_TRAIN_FP32):
        self.block = block
        self.proposal = proposal
        self.h = B.ising_nn_create(block, B.NN_CHANNELS, stream)
        if proposal != B.ISING_PROPOSAL_ONESHOT:
            B.ising_nn_set_proposal(self.h, proposal)
        if precision != B.ISING_NN_TRAIN_FP32:
            B.ising_nn_set_train_precision(self.h, precision)
        if params is None:
            params = init_params(seed)
        B.ising_nn_set_params(self.h, B.nn_flatten(params))

    def close(self):
        if getattr(self, "h", None):
            B.ising_nn_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> dict:
        return B.nn_unflatten(B.ising_nn_get_params(self.h))

    def blob(self) -> np.ndarray:
        return B.ising_nn_export(self.h)

    def fit(self, windows: np.ndarray, epochs: int = 4, batch: int = 512, lr: float = 2e-3,
            seed: int = 0, verbose: bool = False) -> list[float]:
        """Minibatch Adam over device-resident windows; returns the loss per step."""
        import torch

        dev = torch.from_numpy(np.ascontiguousarray(windows)).cuda()
        rng = np.random.default_rng(seed)
        losses = []
        n = len(windows)
        t0 = time.time()
        for ep in range(epochs):
            order = torch.from_numpy(rng.permutation(n)).cuda()
            shuffled = dev[order].contiguous()
            for s in range(0, n - batch + 1, batch):
                chunk = shuffled[s:s + batch]
                losses.append(B.ising_nn_train_step(self.h, chunk, batch, lr))
            if verbose:
                print("epoch %d loss %.4f (%.1fs)" % (ep, np.mean(losses[-(n // batch):]),
                                                      time.time() - t0), flush=True)
        return losses


def init_params(seed: int = 0, scale: float = 1.0) -> dict:
    """He-style random initialisation (float32), the network's starting point."""
    rng = np.random.default_rng(seed)
    C = B.NN_CHANNELS
    return {
        "W1": (rng.standard_normal((C, 2, 3, 3)) * np.sqrt(2.0 / 18) * scale).astype(np.float32),
        "b1": np.zeros(C, np.float32),
        "W2": (rng.standard_normal((C, C, 3, 3)) * np.sqrt(2.0 / (9 * C)) * scale).astype(np.float32),
        "b2": np.zeros(C, np.float32),
        "W3": (rng.standard_normal((1, C, 3, 3)) * np.sqrt(1.0 / (9 * C)) * scale).astype(np.float32),
        "b3": np.zeros(1, np.float32),
    }
