"""Launch-shape autotuner for the packed sweep kernels.

Searches the kernel choice and its shape (sweeps per launch k, number of row
strips, words per tile row) for one lattice size on the current GPU, timing
each candidate with CUDA events on the lattice's stream after a warm-up.  The
choice never changes results (every configuration is bit-identical), only
speed.  Results are cached as JSON keyed by (GPU name, SM count, L, layout) in
``$ISING_TUNE_CACHE`` or ``~/.cache/ising_gb300/tune.json``.
"""
from __future__ import annotations

import json
import os
import time

from . import _binding as B

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "ising_gb300", "tune.json")


def _cache_path() -> str:
    return os.environ.get("ISING_TUNE_CACHE", DEFAULT_CACHE)


def _key(L: int, layout: int) -> str:
    import torch

    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s|%d|L=%d|layout=%d" % (p.name, p.multi_processor_count, L, layout)


def candidates(L: int, sms: int = 152) -> list[dict]:
    """Tiled configurations worth timing for an L x L packed lattice."""
    out = [{"kernel": B.ISING_KERNEL_HALF, "k": 1, "tile_rows": 1, "tile_words": 4}]
    Wc = (L // 2 + 31) // 32
    if L % 256 != 0:
        return out
    for tw in (32, 64, 16, 8):
        if Wc % tw:
            continue
        n_tx = Wc // tw
        for k in (1, 2, 3, 4):
            # strip counts that give whole waves of resident CTAs (2-6 per SM)
            rows_opts = set()
            for per_sm in (2, 3, 4, 5, 6):
                for waves in (1, 2, 3, 4):
                    n_ty = (sms * per_sm * waves + n_tx - 1) // n_tx
                    if 4 * k <= L and 8 <= L // max(n_ty, 1) <= 256:
                        rows_opts.add(n_ty)
            for n_ty in sorted(rows_opts):
                out.append({"kernel": B.ISING_KERNEL_TILED, "k": k, "tile_rows": n_ty,
                            "tile_words": tw})
    return out


def time_config(lat, cfg: dict, sweeps: int, reps: int = 3, stream=None) -> float:
    """Spin-flip attempts per ns of one configuration (best of reps)."""
    import torch

    lat.set_kernel(cfg["kernel"], cfg["k"], cfg["tile_rows"], cfg["tile_words"])
    st = stream or torch.cuda.current_stream()
    lat.sweep(max(cfg["k"], 2), 0)  # warm-up (kernel load, attribute setup)
    best = 0.0
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        lat.sweep(sweeps, 0)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = max(best, lat.L * lat.L * sweeps / (ms * 1e6))
    return best


def tune(L: int, beta: float = 0.4406868, sweeps: int = 24, reps: int = 3,
         cands: list[dict] | None = None, use_cache: bool = True, verbose: bool = False) -> dict:
    """Best configuration for an L x L packed lattice; returns
    {"config": {...}, "flips_per_ns": v, "table": [...]}."""
    import torch

    key = _key(L, B.ISING_LAYOUT_BITS)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return cache[key]
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    cands = cands if cands is not None else candidates(L, sms)
    table = []
    t0 = time.time()
    with B.Lattice(L, beta, B.ISING_LAYOUT_BITS, stream=torch.cuda.current_stream(),
                   seed=1) as lat:
        for cfg in cands:
            try:
                v = time_config(lat, cfg, sweeps, reps)
            except B.IsingError as e:
                if verbose:
                    print("skip", cfg, e)
                continue
            table.append({**cfg, "flips_per_ns": v})
            if verbose:
                print(cfg, "%.1f" % v, flush=True)
    table.sort(key=lambda r: -r["flips_per_ns"])
    best = {k: table[0][k] for k in ("kernel", "k", "tile_rows", "tile_words")}
    res = {"config": best, "flips_per_ns": table[0]["flips_per_ns"], "table": table,
           "seconds": time.time() - t0}
    if use_cache:
        cache[key] = res
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    return res


def tune_batch(Ls, betas, pt_every: int, sweeps: int = 100, reps: int = 2,
               cands: list[tuple[int, int]] | None = None, use_cache: bool = True,
               verbose: bool = False) -> dict:
    """Work decomposition (words per item, threads per CTA) of the batched
    persistent kernel; cached like tune()."""
    import numpy as np
    import torch

    key = "batch|%s|%d|nL=%d|Lsum=%d|nb=%d|pt=%d" % (
        torch.cuda.get_device_properties(torch.cuda.current_device()).name,
        torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count,
        len(Ls), int(np.sum(np.asarray(Ls) ** 2)), len(betas), pt_every)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return cache[key]
    cands = cands or [(w, t) for w in (64, 128, 256, 512, 1024) for t in (32, 64, 128, 256)]
    table = []
    st = torch.cuda.current_stream()
    with B.Batch(Ls, betas, pt_every, stream=st, seed=1) as b:
        for (w, t) in cands:
            try:
                B.ising_batch_set_kernel(b.h, w, t, 0)
            except B.IsingError:
                continue
            b.run(pt_every)  # warm-up
            best = 0.0
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                b.run(sweeps)
                e1.record(st)
                e1.synchronize()
                sites = sum(L * L for L in Ls) * len(betas)
                best = max(best, sites * sweeps / (e0.elapsed_time(e1) * 1e6))
            table.append({"words_per_item": w, "threads": t, "flips_per_ns": best})
            if verbose:
                print(table[-1], flush=True)
    table.sort(key=lambda r: -r["flips_per_ns"])
    res = {"config": {"words_per_item": table[0]["words_per_item"], "threads": table[0]["threads"]},
           "flips_per_ns": table[0]["flips_per_ns"], "table": table}
    if use_cache:
        cache[key] = res
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    return res
