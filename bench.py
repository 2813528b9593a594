#!/usr/bin/env python3
"""Benchmark: checkerboard Metropolis sweep of the 2D Ising model on GB300.

Workload: one L = 16384 periodic lattice, 1 bit per spin (32 MiB packed),
seeded random start, beta cycling through {0.40, 0.4406868, 0.50}; one step =
1000 full sweeps at one beta (records E/M every 10 sweeps).  Metric: spin-flip
attempts per ns (L^2 x sweeps / device time).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own replica (independent lattice,
replica id = rank): replicas only, no collective on the data path; value is
the sum of all ranks' flips over the slowest rank's time ("scaling": "weak").
--impl reference times the CPU oracle (rank 0 only) on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "spin-flips/ns & indep. samples/s at β_c (learned vs plain, same GB300)"
UNIT = "spin-flip attempts/ns"
L_BENCH = 16384
SWEEPS_PER_STEP = 1000
MEASURE_EVERY = 10
BETAS = [0.40, 0.4406868, 0.50]
SEED = 1
PROPOSALS = {"oneshot": 0, "staged": 1}  # ISING_PROPOSAL_ONESHOT / _STAGED
NN_ENGINES = {"mma_sync": 0, "tcgen05": 1}  # ISING_NN_ENGINE_MMA_SYNC / _TCGEN05
TRAIN_PRECISIONS = {"fp32": 0, "bf16_tc": 1}  # ISING_NN_TRAIN_FP32 / _BF16_TC

# Tiled-kernel launch shape for L = 16384 (sweeps per launch, row strips,
# words per tile row): the best shape of an autotuning sweep on GB300, used when
# the autotuner is switched off.
BENCH_KERNEL = {"kernel": 2, "k": 2, "tile_rows": 228, "tile_words": 64}


def configure_kernel(lat, tune: bool = False) -> dict:
    """Apply the benchmark's kernel configuration to a Lattice (L = 16384):
    the autotuner's choice among the warp-per-row tiled shapes when tune is
    set (cached per GPU), else BENCH_KERNEL (or ISING_BENCH_KERNEL=k,rows,words)."""
    cfg = dict(BENCH_KERNEL)
    env = os.environ.get("ISING_BENCH_KERNEL")
    if env:
        k, tr, tw = (int(v) for v in env.split(","))
        cfg.update(k=k, tile_rows=tr, tile_words=tw)
    elif tune:
        from paper_2402_06415_gb300 import autotune

        cands = [c for c in autotune.candidates(lat.L) if c["tile_words"] in (32, 64)]
        cfg = dict(autotune.tune(lat.L, cands=cands)["config"])
    lat.set_kernel(cfg["kernel"], cfg["k"], cfg["tile_rows"], cfg["tile_words"])
    return cfg


# ---------------------------------------------------------------------------
# clocks sampling (nvidia-smi) during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0,
            "_source": "fallback"}


# ---------------------------------------------------------------------------
# roofline model of the dominant kernel
# ---------------------------------------------------------------------------
# DRAM bytes (read + write) per launch of the sweep kernel from one ncu capture
# of the current kernel, by launch shape (sweeps per launch, row strips, words
# per tile row); profiles/k_tiled32_bits_L16384.md has the commands.  A shape
# without a capture of the current kernel reports null.  (The captures there
# predate the 1536-entry queue: 33.8 MB read + 0.3-0.6 MB written per launch for
# every shape, the lattice read once; the queue lives in shared memory.)
NCU_TRAFFIC = {}


def tiled32_ctas_per_sm(L: int, k: int, n_ty: int, tile_words: int) -> int:
    """Register-budget variant the library launches for a tiled shape: 3 when
    three CTAs' shared memory fits an SM (228 KiB; dynamic tile + the static queue
    of 1536 entries and sums + 1 KiB reserved per CTA), else 2 (the variant with up
    to 128 registers)."""
    ty_max = -(-L // n_ty)
    per_cta = 2 * (ty_max + 4 * k) * (tile_words + 8) * 4 + (12 * 1536 + 16 + 16 * k) + 1024
    return 3 if 3 * per_cta <= 228 * 1024 else 2


# Algorithmic work of the bit-sliced, lazily evaluated acceptance test per
# 32-site word, by the pipe it issues to.  ALU pipe (three-input logic, shifts):
# neighbour classes as two half adders (half sums, carries, ge2 and the class
# mask: 7), funnel shift 1, update 1 = 9; per Philox4x32-10 block 10 rounds x 2
# three-input XORs = 20, plus 4 planes x 3 logic ops (the lane's threshold bit,
# the borrow of u - T as a majority function, the equality chain) and 1 to merge
# the block's verdict into (acc, D) = 13; E[blocks] = 1.95 for independent
# words: 9 + 1.95 x 33 = 73.35.  FMA pipe: per block 10 rounds x 2 wide integer
# multiplies = 20, i.e. 39 per word.  Both pipes take 64 lanes per SM per
# clock, so the ALU pipe binds: per site 73.35 / 32 lane-ops.
ALU_OPS_PER_WORD = 9.0 + 1.95 * 33.0
FMA_OPS_PER_WORD = 1.95 * 20.0
ALU_OPS_PER_SITE = ALU_OPS_PER_WORD / 32.0
ALU_LANES_PER_SM = 64
N_SM = 152


def alu_peak_gops(peaks: dict, sm_mhz: float | None) -> float:
    """ALU-pipe lane-operations per second: 152 SMs x 64 lanes x SM clock."""
    mhz = sm_mhz or peaks.get("sm_max_mhz", 2070.0)
    return N_SM * ALU_LANES_PER_SM * mhz * 1e6 / 1e9


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part", "hardware")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sample(L: int, beta: float, n_sweeps: int = 1):
    """Time the single-threaded oracle on n_sweeps of an L x L lattice."""
    import oracle

    oracle.build()
    s = oracle.init(L, SEED)
    t0 = time.perf_counter()
    oracle.sweep(s, beta, SEED, n_sweeps, measure_every=MEASURE_EVERY)
    dt = time.perf_counter() - t0
    return L * L * n_sweeps / (dt * 1e9), dt


def oracle_sample_omp(L: int, beta: float, n_sweeps: int = 1):
    """Time the OpenMP build of the oracle sweep (all host cores)."""
    import oracle

    oracle.build()
    s = oracle.init(L, SEED)
    t0 = time.perf_counter()
    oracle.sweep_omp(s, beta, SEED, n_sweeps, measure_every=MEASURE_EVERY)
    dt = time.perf_counter() - t0
    return L * L * n_sweeps / (dt * 1e9), dt, oracle.omp_threads()


# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_value(local_ms: float, flips_per_rank: float, dist=None, device=None):
    """Whole-job throughput over ranks that each run their own replica: the
    slowest rank's time bounds the job; value = all ranks' flips / that time.
    Returns (value in flips/ns, max time in ms)."""
    ws = 1
    t_max = float(local_ms)
    if dist is not None and dist.is_initialized():
        import torch

        ws = dist.get_world_size()
        t = torch.tensor([t_max], dtype=torch.float64, device=device or "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    return flips_per_rank * ws / (t_max * 1e6), t_max


def replica_of_rank(rank: int) -> int:
    """Replica id (Philox stream) of the lattice a rank runs."""
    return rank


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    L = 8192
    times, vals = [], []
    for i in range(args.warmup + args.steps):
        v, dt = oracle_sample(L, BETAS[i % 3], 1)
        if i >= args.warmup:
            vals.append(v)
            times.append(dt)
    value = L * L * len(times) / (sum(times) * 1e9)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "2D Ising L=16384 checkerboard Metropolis (reference arm: "
                               "oracle on L=8192, 1 sweep per step)",
                   "L": L, "betas": BETAS, "sweeps_per_step": 1},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "1 sweep of an 8192^2 lattice per step, seed 1",
                         "cpu": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    import paper_2402_06415_gb300 as ising

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.current_stream()
    L = L_BENCH
    lat = ising.Lattice(L, BETAS[0], ising.ISING_LAYOUT_BITS, stream=stream)
    ising.ising_set_replica(lat.ctx, replica_of_rank(rank))
    cfg = configure_kernel(lat, tune=not args.no_tune)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def one_step(i, timed_events):
        lat.seed(SEED + 1000 * i)
        ising.ising_set_beta(lat.ctx, BETAS[i % 3])
        flush.zero_()  # L2 flush between steps (256 MiB > 129 MB L2)
        if timed_events:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.sweep(SWEEPS_PER_STEP, MEASURE_EVERY)
            e1.record(stream)
            return e0, e1
        lat.sweep(SWEEPS_PER_STEP, MEASURE_EVERY)
        return None

    for i in range(args.warmup):
        one_step(i, False)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    launches0 = ising.ising_launch_count(lat.ctx)
    # the headline: one event pair per step, nothing recorded between launches
    evs = [one_step(args.warmup + i, True) for i in range(args.steps)]
    torch.cuda.synchronize()
    barrier()
    launches = ising.ising_launch_count(lat.ctx) - launches0
    step_ms = [a.elapsed_time(b) for (a, b) in evs]
    # per-launch duration of the sweep kernel for the roofline: a separate,
    # shorter pass with an event pair around every launch on the lattice's
    # stream (the events add a little to each launch, so this errs slow)
    ising.ising_set_timing(lat.ctx, True)
    for i in range(max(1, min(2, args.steps))):
        one_step(args.warmup + args.steps + i, False)
    torch.cuda.synchronize()
    kern_ms, kern_launches = ising.ising_kernel_time(lat.ctx)
    ising.ising_set_timing(lat.ctx, False)
    clk = clocks.stop()
    flips_rank = float(L) * L * SWEEPS_PER_STEP * args.steps
    value, total_ms = job_value(sum(step_ms), flips_rank, dist, "cuda")
    flips = flips_rank * ws
    # sanity: the chain is alive (records present, energies in range)
    E, M = lat.series(SWEEPS_PER_STEP // MEASURE_EVERY)
    assert np.all(np.abs(E) <= 2 * L * L) and len(E) == SWEEPS_PER_STEP // MEASURE_EVERY

    # ---- end to end through the public API with host buffers -------------
    Wc = ising.ising_words_per_row(L)
    host_in = torch.empty((2, L, Wc), dtype=torch.int32, pin_memory=True)
    host_out = torch.empty((2, L, Wc), dtype=torch.int32, pin_memory=True)
    lat.seed(SEED)
    ising.ising_get_bits(lat.ctx, L, host_in.numpy().view(np.uint32))
    n_rec = SWEEPS_PER_STEP // MEASURE_EVERY
    Eh = np.zeros(n_rec, dtype=np.int64)
    Mh = np.zeros(n_rec, dtype=np.int64)
    e2e_times = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        ising.ising_set_key(lat.ctx, SEED + i)
        ising.ising_set_sweep_counter(lat.ctx, 0)
        ising.ising_set_beta(lat.ctx, BETAS[i % 3])
        lat.set_bits(host_in.numpy().view(np.uint32))           # H2D 32 MiB
        lat.sweep(SWEEPS_PER_STEP, MEASURE_EVERY)
        ising.lib().ising_series(lat.ctx, ising._binding._ptr(Eh), ising._binding._ptr(Mh), n_rec)
        ising.ising_get_bits(lat.ctx, L, host_out.numpy().view(np.uint32))  # D2H 32 MiB
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_times.append(t1 - t0)
    e2e_value, _ = job_value(1e3 * sum(e2e_times), flips_rank, dist, "cuda")
    h2d = 2 * L * Wc * 4
    d2h = 2 * L * Wc * 4 + n_rec * 16

    # ---- roofline of the dominant kernel (live CUDA-event timing) --------
    peaks = measured_peaks()
    per_launch_ms = kern_ms / max(kern_launches, 1)
    sites_per_launch = float(L) * L * cfg["k"]
    alu_gops = ALU_OPS_PER_SITE * sites_per_launch / (per_launch_ms * 1e6)
    peak = alu_peak_gops(peaks, clk.get("sm_mhz"))
    hbm_gbs = 0.25 * sites_per_launch / (per_launch_ms * 1e6)
    roofline = {
        "bound": "alu", "achieved": alu_gops, "peak": peak, "unit": "Gop/s",
        "frac": alu_gops / peak,
        "traffic": NCU_TRAFFIC.get((cfg["k"], cfg["tile_rows"], cfg["tile_words"])),
        "kernel": ("k_tiled32_bits<%d,%d,%d>" % (cfg["k"], cfg["tile_words"] // 32,
                                                 tiled32_ctas_per_sm(L, cfg["k"], cfg["tile_rows"],
                                                                     cfg["tile_words"]))
                   if cfg["tile_words"] in (32, 64) else "k_tiled_bits<%d>" % cfg["k"]),
        "peak_source": "ALU pipe (the binding pipe of the algorithmic mix: 73.35 ALU-pipe and "
                       "39 FMA-pipe lane-ops per 32-site word, both pipes 64 lanes/SM/clock): "
                       "152 SMs x 64 lanes x median SM clock under load",
        "alu_ceiling_flips_per_ns": 32.0 * peak / ALU_OPS_PER_WORD,
        "per_launch_ms": per_launch_ms, "launches": kern_launches,
        "hbm_packed_accounting": {"achieved_gbs": hbm_gbs,
                                  "frac_of_measured": hbm_gbs / peaks.get("hbm_gbs", 6800.0),
                                  "bytes_per_site_sweep": 0.25,
                                  "ceiling_frac_at_full_alu": 0.25 * 32.0 * peak / ALU_OPS_PER_WORD
                                  / peaks.get("hbm_gbs", 6800.0),
                                  "note": "60 % of the HBM roof is unreachable under "
                                          "Philox4x32-10: at 100 % of the ALU-pipe roof the sweep "
                                          "moves only this fraction of the packed-byte HBM roof"},
    }

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "2D Ising L=16384 packed (1 bit/spin), checkerboard Metropolis, "
                               "1000 sweeps per step, beta cycling 0.40/0.4406868/0.50",
                   "L": L, "betas": BETAS, "sweeps_per_step": SWEEPS_PER_STEP,
                   "measure_every": MEASURE_EVERY, "kernel": cfg,
                   "l2": "flushed between steps (256 MiB write); the 32 MiB lattice stays "
                         "L2-resident within a step", "parallelism": "replicas%d" % ws},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "clocks": clk,
    }
    if rank == 0 and not args.no_indep:
        line["indep_samples"] = measure_indep_samples(args, stream)
    if rank == 0 and not args.no_cpu_baseline:
        v, dt = oracle_sample(L, BETAS[1], 2)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "2 sweeps of the 16384^2 lattice at beta 0.4406868 "
                                          "(%.1f s)" % dt, "cpu": cpu_model(),
                                "nproc": os.cpu_count()}
        v, dt, thr = oracle_sample_omp(L, BETAS[1], 4)
        line["cpu_baseline_multicore"] = {
            "value": v, "unit": UNIT, "cores": thr, "kind": "oracle_openmp",
            "sample": "4 sweeps of the 16384^2 lattice at beta 0.4406868, rows of a colour "
                      "over %d OpenMP threads (%.1f s); timing only, same result as the "
                      "single-threaded oracle" % (thr, dt),
            "cpu": cpu_model(), "nproc": os.cpu_count()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    lat.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def measure_indep_samples(args, stream):
    """Independent samples per second at beta_c on L = 256 for the plain
    Metropolis chain, the learned chain (1 sweep + 1 staged 16x16 block pass per
    step) and Swendsen-Wang steps.

    tau_int (|M| and E) comes from many chains run together (one batch per
    method: `indep_chains` plain chains, `indep_learned_chains` learned chains,
    all started from plain-sweep equilibrium), pooled autocorrelation with
    Sokal's window and jackknife errors over groups of chains
    (stats.tau_int_chains); Swendsen-Wang from single chains (its tau is a few
    steps).  Speed in two regimes: one chain alone on the GPU (launch- and
    latency-bound: steps/s of one lattice) and the batch (throughput: steps/s
    of every chain of the batch together).  Independent samples/s = chains x
    steps/s / (2 tau_int)."""
    import numpy as np
    import torch

    import paper_2402_06415_gb300 as ising
    from paper_2402_06415_gb300 import learned, stats

    beta, L, block = 0.4406868, 256, 16
    t_all = time.perf_counter()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3

    t0 = time.perf_counter()
    wins = learned.generate_windows([64, 128, 256], beta, args.indep_train_windows // 3, block, seed=7,
                                    thermalise=2000, thin=20, per_config=64, stream=stream)
    with learned.Trainer(block, seed=8, proposal=PROPOSALS["staged"],
                         precision=TRAIN_PRECISIONS[args.train_precision]) as tr:
        losses = tr.fit(wins, epochs=args.indep_train_epochs, batch=512, lr=2e-3, seed=9)
        blob = tr.blob()
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0

    def batch_chains(mode, n_ch, n_steps, seed):
        with ising.Batch([L] * n_ch, [beta], 1, stream=stream, seed=seed) as b:
            ising.ising_batch_set_series(b.h, n_steps)
            b.run(args.indep_thermalise)  # plain-sweep equilibrium for every method
            if mode == "learned":
                ising.ising_batch_nn_load(b.h, blob)
                ising.ising_batch_set_proposal(b.h, PROPOSALS["staged"])

                def go():
                    for _ in range(n_steps):
                        b.run(1)
                        ising.ising_batch_block_pass(b.h, 1, block)
            else:
                def go():
                    b.run(n_steps)
            secs = timed(go)
            st, _ = ising.ising_batch_status(b.h)
            E, M, _ = ising.ising_batch_series(b.h, n_steps, n_ch)
            acc = ising.ising_batch_block_stats(b.h) if mode == "learned" else (0, 0)
        assert st == 0, "batch status %d" % st
        return E.astype(np.float64), np.abs(M).astype(np.float64), secs, acc

    out = {"L": L, "beta": beta, "block": block}
    for mode, n_ch, n_steps in (("plain", args.indep_chains, args.indep_plain_sweeps),
                                ("learned", args.indep_learned_chains, args.indep_learned_steps)):
        E, M, secs, acc = batch_chains(mode, n_ch, n_steps, 11)
        tm, dtm = stats.tau_int_chains(M)
        te, dte = stats.tau_int_chains(E)
        out[mode] = {"chains": n_ch, "steps_per_chain": n_steps,
                     "tau_int_absM": tm, "tau_int_absM_err": dtm, "tau_int_E": te, "tau_int_E_err": dte,
                     "run_over_tau_absM": n_steps / tm, "run_over_tau_E": n_steps / te,
                     "batch_steps_per_s_per_chain": n_steps / secs,
                     "batch_indep_absM_per_s": n_ch * n_steps / secs / (2 * tm),
                     "batch_indep_E_per_s": n_ch * n_steps / secs / (2 * te),
                     "mean_absm": float(M.mean() / (L * L)), "mean_e": float(E.mean() / (L * L))}
        if mode == "learned":
            out[mode]["block_acceptance"] = acc[1] / max(acc[0], 1)
    # one chain alone on the GPU
    with ising.Lattice(L, beta, ising.ISING_LAYOUT_BITS, stream=stream, seed=21) as lat:
        lat.sweep(2000, 0)
        n = args.indep_single_steps
        secs = timed(lambda: ising.ising_sweep(lat.ctx, 10 * n, 1))
        out["plain"]["single_steps_per_s"] = 10 * n / secs
        ising.ising_nn_load(lat.ctx, blob)
        ising.ising_set_proposal(lat.ctx, PROPOSALS["staged"])
        secs = timed(lambda: ising.ising_sweep_blocks(lat.ctx, n, 1, block, 1))
        out["learned"]["single_steps_per_s"] = n / secs
        secs = timed(lambda: ising.ising_sw_step(lat.ctx, 5 * n, 1))
        out["sw"] = {"single_steps_per_s": 5 * n / secs}
    Ms, Es = [], []
    for c in range(8):
        with ising.Lattice(L, beta, ising.ISING_LAYOUT_BITS, stream=stream, seed=40 + c) as lat:
            ising.ising_sw_step(lat.ctx, 200, 0)
            ising.ising_sw_step(lat.ctx, 4000, 1)
            E, M = lat.series(4000)
            Ms.append(np.abs(M).astype(np.float64))
            Es.append(E.astype(np.float64))
    tm, dtm = stats.tau_int_chains(np.stack(Ms, 1))
    te, dte = stats.tau_int_chains(np.stack(Es, 1))
    out["sw"].update({"chains": 8, "steps_per_chain": 4000, "tau_int_absM": tm, "tau_int_absM_err": dtm,
                      "tau_int_E": te, "tau_int_E_err": dte})
    for m in ("plain", "learned", "sw"):
        o = out[m]
        o["single_indep_absM_per_s"] = o["single_steps_per_s"] / (2 * o["tau_int_absM"])
        o["single_indep_E_per_s"] = o["single_steps_per_s"] / (2 * o["tau_int_E"])

    def ratio(a, b, key, err_a, err_b):
        r = a[key] / b[key]
        return r, r * float(np.hypot(err_a, err_b))

    pl, le = out["plain"], out["learned"]
    gains = {}
    for obs in ("absM", "E"):
        rel_l = le["tau_int_%s_err" % obs] / le["tau_int_%s" % obs]
        rel_p = pl["tau_int_%s_err" % obs] / pl["tau_int_%s" % obs]
        for reg in ("single", "batch"):
            r, dr = ratio(le, pl, "%s_indep_%s_per_s" % (reg, obs), rel_l, rel_p)
            gains["learned_over_plain_%s_%s" % (reg, obs)] = [r, dr]
    out["gain"] = gains
    out["train"] = {"windows": int(len(wins)), "epochs": args.indep_train_epochs,
                    "kernel": args.train_precision,
                    "loss_first": float(np.mean(losses[:5])), "loss_last": float(np.mean(losses[-5:])),
                    "seconds": t_train}
    out["seconds"] = time.perf_counter() - t_all
    out["note"] = ("tau_int in steps (plain: sweeps; learned: sweep + staged block pass; sw: "
                   "Swendsen-Wang steps); gains are independent samples/s of the learned chain over "
                   "the plain chain, [value, 1-sigma] from the tau errors; 'single' = one chain alone on "
                   "the GPU, 'batch' = the chains of one batch together")
    return out


def run_batch(args):
    """4096 replicas (64 ladders x 64 betas in [0.35, 0.50], sizes drawn from
    {16, ..., 128}), exchanges every 10 sweeps; one step = one graph replay of
    a persistent launch covering all sweeps of the step."""
    import numpy as np
    import torch

    import paper_2402_06415_gb300 as ising
    from paper_2402_06415_gb300 import workloads

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    Ls = workloads.batch_ladder_sizes()
    betas = workloads.batch_betas()
    pt = workloads.BATCH_PT_EVERY
    sweeps = args.sweeps
    stream = torch.cuda.current_stream()
    b = ising.Batch(Ls, betas, pt, stream=stream, seed=SEED)
    if args.batch_kernel:
        wpi, thr = (int(v) for v in args.batch_kernel.split(","))
    elif not args.no_tune:
        from paper_2402_06415_gb300 import autotune

        best = autotune.tune_batch(Ls, betas, pt)["config"]
        wpi, thr = best["words_per_item"], best["threads"]
    else:
        wpi, thr = 512, 256
    ising.ising_batch_set_kernel(b.h, wpi, thr, 0)
    ising.ising_batch_capture(b.h, sweeps)
    for _ in range(args.warmup):
        b.run(sweeps)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run(sweeps)
        e1.record(stream)
        times.append((e0, e1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    st, sw = ising.ising_batch_status(b.h)
    ms = sum(a.elapsed_time(c) for a, c in times)
    sites = sum(L * L for L in Ls) * len(betas)
    value = sites * sweeps * args.steps / (ms * 1e6)
    acc, att = b.swap_counts()
    rate = (acc[:, :-1].sum(0) / np.maximum(att[:, :-1].sum(0), 1)).tolist()
    info = ising.ising_batch_info(b.h)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "batched: 4096 replicas (64 ladders x 64 betas in [0.35,0.50]), "
                               "L per ladder from {16..128}, PT every 10 sweeps, one persistent "
                               "launch per step replayed from a CUDA graph",
                   "sweeps_per_step": sweeps, "replica_sites": sites, "items": info["items"],
                   "grid": info["grid"], "status": st, "device_sweeps": sw,
                   "words_per_item": wpi, "threads": thr},
        "pt_accept_rate_by_pair": [round(x, 4) for x in rate],
        "gpu_launches": args.steps, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    b.close()
    return 0


def run_learned(args):
    """Learned 16x16 block proposal at beta_c on L = 256 against the plain sweep:
    train the CNN on plain-sweep windows (L in {64, 128, 256}), then run chains of
    (1 sweep + 1 block pass) and of plain sweeps; report acceptance, tau_int of
    |M| and E, and independent samples per second of each."""
    import numpy as np
    import torch

    import paper_2402_06415_gb300 as ising
    from paper_2402_06415_gb300 import learned, stats

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    beta, L, block = 0.4406868, 256, 16
    t0 = time.perf_counter()
    wins = learned.generate_windows([64, 128, 256], beta, args.train_windows // 3, block, seed=7,
                                    thermalise=2000, thin=20, per_config=64)
    t_data = time.perf_counter() - t0
    kind = PROPOSALS[args.proposal]
    t0 = time.perf_counter()
    with learned.Trainer(block, seed=8, proposal=kind,
                         precision=TRAIN_PRECISIONS[args.train_precision]) as tr:
        losses = tr.fit(wins, epochs=args.train_epochs, batch=512, lr=2e-3, seed=9)
        blob = tr.blob()
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    n = args.chain_sweeps
    res = {}
    stream = torch.cuda.current_stream()
    for mode in ("plain", "learned"):
        taus_m, taus_e, ms_tot, acc = [], [], 0.0, [0, 0]
        for c in range(args.chains):
            with ising.Lattice(L, beta, ising.ISING_LAYOUT_BITS, stream=stream,
                               seed=100 + c) as lat:
                ising.ising_nn_load(lat.ctx, blob)
                ising.ising_set_proposal(lat.ctx, kind)
                every = 1 if mode == "learned" else 0
                ising.ising_sweep_blocks(lat.ctx, args.thermalise, 0, block, every)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ising.ising_sweep_blocks(lat.ctx, n, 1, block, every)
                e1.record(stream)
                e1.synchronize()
                ms_tot += e0.elapsed_time(e1)
                E, M = lat.series(n)
                taus_m.append(stats.tau_int(np.abs(M).astype(float)))
                taus_e.append(stats.tau_int(E.astype(float)))
                p_, a_ = ising.ising_block_stats(lat.ctx)
                acc[0] += p_
                acc[1] += a_
        sweeps_per_s = args.chains * n / (ms_tot / 1e3)
        tm, te = float(np.mean(taus_m)), float(np.mean(taus_e))
        res[mode] = {"sweeps_per_s": sweeps_per_s, "tau_int_absM": tm, "tau_int_E": te,
                     "indep_samples_per_s_absM": sweeps_per_s / (2 * tm),
                     "indep_samples_per_s_E": sweeps_per_s / (2 * te),
                     "block_acceptance": (acc[1] / acc[0]) if acc[0] else None,
                     "run_over_tau_absM": n / tm}
    # acceptance of networks trained per block size (same data recipe, smaller set)
    scan = []
    for Bs in args.scan_blocks:
        if Bs == block:
            bl, tr_loss = blob, float(np.mean(losses[-5:]))
        else:
            w_s = learned.generate_windows([64, 128, 256], beta, 10000, Bs, seed=11, thermalise=2000,
                                           thin=20, per_config=64)
            with learned.Trainer(Bs, seed=12, proposal=kind) as tr2:
                ls = tr2.fit(w_s, epochs=3, batch=512, lr=2e-3, seed=13)
                bl, tr_loss = tr2.blob(), float(np.mean(ls[-5:]))
        with ising.Lattice(L, beta, ising.ISING_LAYOUT_BITS, stream=stream, seed=300) as lat:
            ising.ising_nn_load(lat.ctx, bl)
            ising.ising_set_proposal(lat.ctx, kind)
            ising.ising_sweep(lat.ctx, args.thermalise, 0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ising.ising_sweep_blocks(lat.ctx, args.scan_sweeps, 0, Bs, 1)
            e1.record(stream)
            e1.synchronize()
            p_, a_ = ising.ising_block_stats(lat.ctx)
        scan.append({"block": Bs, "train_loss_per_site": tr_loss / (Bs * Bs),
                     "acceptance": a_ / max(p_, 1), "proposed": p_,
                     "sweeps_per_s": args.scan_sweeps / (e0.elapsed_time(e1) / 1e3)})
    gain_m = res["learned"]["indep_samples_per_s_absM"] / res["plain"]["indep_samples_per_s_absM"]
    gain_e = res["learned"]["indep_samples_per_s_E"] / res["plain"]["indep_samples_per_s_E"]
    line = {
        "metric": METRIC, "value": res["learned"]["indep_samples_per_s_absM"],
        "unit": "independent |M| samples/s (learned chain, L=256, beta_c)", "n_gpus": 1,
        "steps": args.chains, "warmup": args.thermalise, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "learned 16x16 block proposal (%s), L=256 at beta_c, 1 block pass "
                               "per sweep, vs plain sweep on the same GPU" % args.proposal,
                   "proposal": args.proposal,
                   "train_windows": int(len(wins)), "train_epochs": args.train_epochs,
                   "chain_sweeps": n, "chains": args.chains},
        "plain": res["plain"], "learned": res["learned"], "acceptance_by_block": scan,
        "gain_indep_samples_absM": gain_m, "gain_indep_samples_E": gain_e,
        "train": {"loss_first": float(np.mean(losses[:5])), "loss_last": float(np.mean(losses[-5:])),
                  "data_s": t_data, "train_s": t_train, "steps": len(losses),
                  "kernel": args.train_precision},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_batch_learned(args):
    """1024 replicas at L = 512 (32 ladders x 32 betas in [0.42, 0.46]): block
    passes (16 x 16) every 5 sweeps on every replica plus exchanges every 10,
    against the same batch without block passes; a bounded number of sweeps."""
    import numpy as np
    import torch

    import paper_2402_06415_gb300 as ising
    from paper_2402_06415_gb300 import learned, workloads

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    Ls = [512] * 32
    betas = workloads.batch_betas(32, 0.42, 0.46)
    block, every, pt = 16, 5, 10
    wins = learned.generate_windows([64, 128, 256], 0.4406868, 30000, block, seed=7,
                                    thermalise=2000, thin=20, per_config=64)
    kind = PROPOSALS[args.proposal]
    with learned.Trainer(block, seed=8, proposal=kind,
                         precision=TRAIN_PRECISIONS[args.train_precision]) as tr:
        tr.fit(wins, epochs=3, batch=512, lr=2e-3, seed=9)
        blob = tr.blob()
    stream = torch.cuda.current_stream()
    out = {}
    n = args.sweeps
    for mode in ("plain", "learned"):
        with ising.Batch(Ls, betas, pt, stream=stream, seed=SEED) as b:
            ising.ising_batch_nn_load(b.h, blob)
            ising.ising_batch_set_proposal(b.h, kind)
            b.run(20)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(n // every):
                b.run(every)
                if mode == "learned":
                    ising.ising_batch_block_pass(b.h, 1, block)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            st, sw = ising.ising_batch_status(b.h)
            p_, a_ = ising.ising_batch_block_stats(b.h)
            acc, att = b.swap_counts()
        sites = 512 * 512 * 1024
        out[mode] = {"ms": ms, "sweeps": (n // every) * every,
                     "flips_per_ns": sites * (n // every) * every / (ms * 1e6),
                     "block_acceptance": (a_ / p_) if p_ else None, "squares_proposed": p_,
                     "pt_accept": float(acc[:, :-1].sum() / max(att[:, :-1].sum(), 1)),
                     "status": st}
    line = {"metric": METRIC, "value": out["learned"]["flips_per_ns"], "unit": UNIT,
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic", "dtype": "bf16",
            "config": {"workload": "batched + learned: 1024 replicas L=512, 32 betas in "
                                   "[0.42,0.46], 16x16 block pass every 5 sweeps, PT every 10",
                       "sweeps": n},
            "plain": out["plain"], "learned": out["learned"],
            "cost_ratio_per_sweep": out["learned"]["ms"] / out["plain"]["ms"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_xy(args):
    """The paper's own MC experiment on the XY model (Results C, Fig. 4a): time
    per MC step at T = 0.85 for L = 8 .. 128 over 10^4 steps, in FP64 (the
    paper's precision) and FP32, next to the CPU oracle (1 core, FP64); plus
    site-update throughput on a large lattice."""
    import numpy as np
    import torch

    import oracle
    import paper_2402_06415_gb300 as ising

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    beta = 1.0 / 0.85
    stream = torch.cuda.current_stream()
    rows = []
    for L in (8, 16, 32, 64, 128):
        row = {"L": L}
        for prec in (64, 32):
            with ising.XY(L, beta, prec, stream=stream, seed=1) as x:
                x.sweep(200)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                x.sweep(args.xy_steps)
                e1.record(stream)
                e1.synchronize()
                row["gpu_us_per_step_fp%d" % prec] = 1e3 * e0.elapsed_time(e1) / args.xy_steps
                if prec == 64:
                    x.sweep(1, 1)
                    E, _, _ = x.series(1)
                    row["energy_per_site_fp64"] = float(E[-1]) / (L * L)
        u = oracle.xy_init(L, 1)
        n_cpu = max(20, 20000 // L)
        t0 = time.perf_counter()
        oracle.xy_sweep(u, beta, 1, n_cpu, record=False)
        row["cpu_us_per_step_fp64"] = 1e6 * (time.perf_counter() - t0) / n_cpu
        rows.append(row)
    thr = {}
    for prec in (64, 32):
        with ising.XY(4096, beta, prec, stream=stream, seed=2) as x:
            x.sweep(5)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x.sweep(50)
            e1.record(stream)
            e1.synchronize()
            thr["fp%d" % prec] = 4096 * 4096 * 50 / (e0.elapsed_time(e1) * 1e6)
    line = {"metric": "XY-model MC time per step (the paper's Fig. 4a experiment)",
            "value": thr["fp64"], "unit": "site updates/ns (L=4096, FP64)", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic", "dtype": "f64",
            "config": {"workload": "2D XY model, checkerboard Metropolis, T=0.85, 10^4 steps "
                                   "per size", "steps": args.xy_steps},
            "per_size": rows, "throughput_L4096": thr,
            "paper_context": "FPGA (XC7K325T, pipelined, FP64): 42.36 us per step at L=32 "
                             "(Tab. S3); 16.5x a Xeon Gold 6230 core at L=128"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_sw(args):
    """Cluster steps (Swendsen-Wang, Wolff) against single-site Metropolis at
    beta_c: independent |M| and E samples per second at L = 128 and 256 (tau_int
    from the recorded series; the cluster methods alone at L = 1024), plus the
    time of one cluster step at L = 4096 and 16384 (Wolff also at beta = 0.3,
    where its clusters are small and growth from the seed finds them)."""
    import numpy as np
    import torch

    import paper_2402_06415_gb300 as ising
    from paper_2402_06415_gb300 import stats

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    beta = 0.4406868
    stream = torch.cuda.current_stream()

    def chain(L, mode, n, therm):
        with ising.Lattice(L, beta, ising.ISING_LAYOUT_BITS, stream=stream, seed=500 + L) as lat:
            step = {"metropolis": lat.sweep, "sw": lat.sw_step, "wolff": lat.wolff_step}[mode]
            # Wolff from a hot start flips tiny clusters for a long time: bring the
            # lattice to equilibrium with Swendsen-Wang steps first
            (lat.sw_step if mode == "wolff" else step)(therm)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(n, 1)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            E, M = lat.series(n)
            extra = {}
            if mode == "wolff":
                w = lat.wolff_stats()
                extra = {"mean_cluster_fraction": w["flipped"] / (n * L * L),
                         "steps_grown": w["grown"], "steps_labelled": w["labelled"]}
        tm = stats.tau_int(np.abs(M).astype(float))
        te = stats.tau_int(E.astype(float))
        per_s = n / (ms / 1e3)
        return {"steps": n, "steps_per_s": per_s, "tau_int_absM": tm, "tau_int_E": te,
                "indep_samples_per_s_absM": per_s / (2 * tm),
                "indep_samples_per_s_E": per_s / (2 * te), "run_over_tau_absM": n / tm,
                "energy_per_site": float(np.mean(E)) / (L * L), **extra}

    rows = []
    for L in (128, 256):
        met = chain(L, "metropolis", args.chain_sweeps, args.thermalise)
        sw = chain(L, "sw", args.sw_steps, 200)
        wo = chain(L, "wolff", args.sw_steps, 200)
        rows.append({"L": L, "metropolis": met, "sw": sw, "wolff": wo,
                     "gain_indep_samples_absM": sw["indep_samples_per_s_absM"]
                     / met["indep_samples_per_s_absM"],
                     "wolff_gain_indep_samples_absM": wo["indep_samples_per_s_absM"]
                     / met["indep_samples_per_s_absM"]})
    # Metropolis needs runs of ~10^3 tau_int(|M|) ~ L^2.2 sweeps beyond L = 256
    rows.append({"L": 1024, "sw": chain(1024, "sw", args.sw_steps, 200),
                 "wolff": chain(1024, "wolff", args.sw_steps, 200)})
    thr = {}

    def step_time(L, b, mode, n):
        with ising.Lattice(L, b, ising.ISING_LAYOUT_BITS, stream=stream, seed=9) as lat:
            step = lat.sw_step if mode == "sw" else lat.wolff_step
            lat.sw_step(30)  # equilibrium clusters (a hot start has tiny ones)
            step(3)
            f0 = lat.wolff_stats()["flipped"] if mode == "wolff" else 0
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(n)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            r = {"ms_per_step": ms / n, "site_updates_per_ns": L * L * n / (ms * 1e6)}
            if mode == "wolff":
                w = lat.wolff_stats()
                r.update({"sites_flipped_per_ns": (w["flipped"] - f0) / (ms * 1e6),
                          "mean_cluster_fraction": (w["flipped"] - f0) / (n * L * L),
                          "steps_grown": w["grown"], "steps_labelled": w["labelled"]})
            return r

    for L in (4096, 16384):
        thr["L%d" % L] = step_time(L, beta, "sw", 10)
        thr["wolff_L%d" % L] = step_time(L, beta, "wolff", 10)
        thr["wolff_beta0.3_L%d" % L] = step_time(L, 0.3, "wolff", 200)
    line = {"metric": "independent samples/s at beta_c, cluster steps vs Metropolis",
            "value": rows[1]["sw"]["indep_samples_per_s_absM"],
            "unit": "independent |M| samples/s (SW, L=256, beta_c)", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic", "dtype": "u32",
            "config": {"workload": "2D Ising at beta_c: Swendsen-Wang and Wolff cluster steps vs "
                                   "checkerboard Metropolis sweeps, L in {128, 256} (cluster steps "
                                   "also 1024)",
                       "sw_steps": args.sw_steps, "metropolis_sweeps": args.chain_sweeps},
            "per_size": rows, "sw_throughput": thr}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_sw_step(args):
    """Time of one Swendsen-Wang step on one lattice at beta_c (default L = 16384):
    30 untimed steps bring the clusters to equilibrium size, then W warm-up and K
    timed steps, one CUDA-event pair around the K steps."""
    import torch

    import paper_2402_06415_gb300 as ising

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    L, beta = args.sw_L, 0.4406868
    with ising.Lattice(L, beta, ising.ISING_LAYOUT_BITS, stream=stream, seed=3) as lat:
        lat.sw_step(30 + args.warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.sw_step(args.steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
    line = {"metric": "Swendsen-Wang step time", "value": ms, "unit": "ms/step", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "data": "synthetic", "dtype": "u32",
            "config": {"workload": "one Swendsen-Wang step of the %d^2 Ising lattice at beta_c" % L},
            "site_updates_per_ns": L * L / (ms * 1e6)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_staged_pass(args):
    """Time of one staged 16x16 block pass (both square colours) on one lattice
    at beta_c (default L = 256) with a randomly initialised network: W warm-up and
    K timed passes, one CUDA-event pair around the K passes; --nn-engine picks the
    engine of the second convolution."""
    import torch

    import paper_2402_06415_gb300 as ising
    from paper_2402_06415_gb300 import learned

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    L, beta, block = args.pass_L, 0.4406868, 16
    engine = NN_ENGINES[args.nn_engine]
    with learned.Trainer(block, seed=1, proposal=PROPOSALS["staged"]) as tr:
        blob = tr.blob()
    with ising.Lattice(L, beta, ising.ISING_LAYOUT_BITS, stream=stream, seed=3) as lat:
        ising.ising_nn_load(lat.ctx, blob)
        ising.ising_set_proposal(lat.ctx, PROPOSALS["staged"])
        ising.ising_set_nn_engine(lat.ctx, engine)
        lat.sweep(50, 0)
        ising.ising_block_pass(lat.ctx, args.warmup, block)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ising.ising_block_pass(lat.ctx, args.steps, block)
        e1.record(stream)
        e1.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / args.steps
        prop, acc = ising.ising_block_stats(lat.ctx)
    line = {"metric": "staged block pass time", "value": us, "unit": "us/pass", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "data": "synthetic (random-init network)", "dtype": "f16/f32",
            "config": {"workload": "staged 16x16 block pass, both square colours, %d^2 lattice at "
                                   "beta_c" % L, "engine": args.nn_engine},
            "squares_per_pass": (L // block) ** 2, "acceptance": acc / max(prop, 1)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_train(args):
    """Training throughput of the staged 16 x 16 proposal's network: K timed
    train steps (minibatch of 512 windows x 8 network stages, then Adam) after W
    warm-up steps, with each training kernel (FP32 CUDA cores / BF16 tensor
    cores).  Algorithmic FLOPs per sample: the three 32 -> 32 contractions
    (forward, input gradient, weight gradient) 3 x 2 x 324 x 288 x 32, plus
    layers 1 and 3 (forward and gradients) 2 x 324 x 32 x 18 x 2 + 3 x 2 x 324 x 32 x 9."""
    import numpy as np
    import torch

    import paper_2402_06415_gb300 as ising
    from paper_2402_06415_gb300 import learned

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    block, batch = 16, 512
    wins = learned.generate_windows([64, 128], 0.4406868, 2048, block, seed=7, thermalise=500, thin=20,
                                    per_config=64, stream=stream)
    flop = 3 * 2 * 324 * 288 * 32 + 2 * 324 * 32 * 18 * 2 + 3 * 2 * 324 * 32 * 9
    res = {}
    for name in args.train_kernels:
        with learned.Trainer(block, seed=8, proposal=PROPOSALS["staged"],
                             precision=TRAIN_PRECISIONS[name]) as tr:
            d = torch.from_numpy(np.ascontiguousarray(wins[:batch])).cuda()
            n_net = 8
            for _ in range(args.warmup):
                ising.ising_nn_train_step(tr.h, d, batch, 1e-4)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                ising.ising_nn_train_step(tr.h, d, batch, 1e-4)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
        samples = batch * n_net
        res[name] = {"ms_per_step": ms, "samples_per_s": samples / (ms / 1e3),
                     "tflops": samples * flop / (ms / 1e3) / 1e12}
    line = {"metric": "CNN training throughput (staged 16x16 proposal)",
            "value": res[args.train_kernels[-1]]["samples_per_s"], "unit": "samples/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "data": "synthetic (plain-sweep windows at beta_c)", "dtype": "bf16/f32",
            "config": {"workload": "train steps of 512 windows x 8 network stages (16x16 staged proposal)",
                       "flop_per_sample": flop},
            "kernels": res}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_xy_step(args):
    """Time per sweep of the XY model (T = 0.85) on one L x L lattice in one
    precision (--xy-L, --xy-precision), one launch per half sweep: W warm-up
    sweeps (2 W launches of k_xy_half) then K timed sweeps with one CUDA-event
    pair."""
    import torch

    import paper_2402_06415_gb300 as ising

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    L, beta, prec = args.xy_L, 1.0 / 0.85, args.xy_precision
    with ising.XY(L, beta, prec, stream=stream, seed=2) as x:
        x.set_mode(1)
        x.sweep(args.warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x.sweep(args.steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
    line = {"metric": "XY sweep time", "value": ms * 1e3, "unit": "us/sweep", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "data": "synthetic", "dtype": "f%d" % prec,
            "config": {"workload": "XY model at T = 0.85 on a %d^2 lattice, FP%d, one launch per half sweep"
                                   % (L, prec)},
            "site_updates_per_ns": L * L / (ms * 1e6)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_quad(args):
    """The paper's quadripartition workloads (Fig. 5b/5d) for the Ising model:
    time per sweep on the square-octagon lattice (J1 = J2 = 1) and on the square
    lattice with J2 = 0 and with next-nearest neighbours (J2 = 0.5), N = 16 ..
    4096 sites, next to the CPU oracle; plus site-update throughput at 8192^2
    cells (2.7e8 sites)."""
    import numpy as np
    import torch

    import oracle
    import paper_2402_06415_gb300 as ising

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    beta = 0.4406868
    stream = torch.cuda.current_stream()
    models = [("square_octagon", ising.ISING_QUAD_SQOCT, 1.0, 1.0),
              ("square_nn", ising.ISING_QUAD_SQUARE, 1.0, 0.0),
              ("square_nn_nnn", ising.ISING_QUAD_SQUARE, 1.0, 0.5)]
    per_size, thr = [], {}
    launches = 0
    for name, lat, J1, J2 in models:
        for Lc in (2, 4, 6, 8, 16, 32):
            with ising.Quad(lat, Lc, beta, J1, J2, stream=stream, seed=1) as x:
                x.sweep(200)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                x.sweep(args.quad_sweeps)
                e1.record(stream)
                e1.synchronize()
                us = 1e3 * e0.elapsed_time(e1) / args.quad_sweeps
            s = oracle.quad_init(Lc, 1)
            n_cpu = max(20, 40000 // (4 * Lc * Lc))
            t0 = time.perf_counter()
            oracle.quad_sweep(lat, s, beta, J1, J2, 1, n_cpu, measure_every=n_cpu)
            cpu_us = 1e6 * (time.perf_counter() - t0) / n_cpu
            per_size.append({"lattice": name, "N": 4 * Lc * Lc, "gpu_us_per_sweep": us,
                             "oracle_us_per_sweep": cpu_us})
        Lc = 8192
        with ising.Quad(lat, Lc, beta, J1, J2, stream=stream, seed=2) as x:
            x.sweep(3)
            c0 = x.launch_count()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x.sweep(20)
            e1.record(stream)
            e1.synchronize()
            launches += x.launch_count() - c0
            ms = e0.elapsed_time(e1)
        thr[name] = {"ms_per_sweep": ms / 20, "site_updates_per_ns": 4 * Lc * Lc * 20 / (ms * 1e6)}
    line = {"metric": "quadripartite Ising sweeps (the paper's Fig. 5b/5d workloads)",
            "value": thr["square_octagon"]["site_updates_per_ns"],
            "unit": "site updates/ns (square-octagon, 8192^2 cells, beta=0.4406868)", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic", "dtype": "u32",
            "config": {"workload": "Ising on square-octagon and square (NN, NN+NNN) lattices, "
                                   "four-sublattice Metropolis sweep",
                       "small_sweeps": args.quad_sweeps, "beta": beta},
            "gpu_launches": launches, "per_size": per_size, "throughput_8192": thr}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_xy_precision(args):
    """The paper's operand-precision trial (Tab. S3) on the GPU: the XY model at
    T = 0.85 with spin angles in FP64, FP32 and fixed point with 16, 12 and 8
    fractional bits (the paper's (32,16), (24,12), (16,8)), full-width random
    words; the fixed-point types twice, with the acceptance probability at full
    width and truncated to the angle's type.  Time per MC step at L = 32 over
    10^4 steps (the paper's setting); internal energy per spin on a 1024^2
    lattice from an ordered start (below the BKT temperature), blocking errors,
    and its bias against FP64."""
    import numpy as np
    import torch

    import paper_2402_06415_gb300 as ising
    from paper_2402_06415_gb300 import stats

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    beta = 1.0 / 0.85
    stream = torch.cuda.current_stream()
    variants = [("(64, floating)", "fp", 64, False), ("(32, floating)", "fp", 32, False)]
    for qp in (False, True):
        variants += [("(32, 16)", "fix", 16, qp), ("(24, 12)", "fix", 12, qp), ("(16, 8)", "fix", 8, qp)]

    def make(kind, bits, qp, L, seed):
        if kind == "fp":
            return ising.XY(L, beta, bits, stream=stream, seed=seed)
        return ising.XYFix(L, beta, bits, stream=stream, seed=seed, quantise_p=qp)

    def timed(x, n):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x.sweep(n)
        e1.record(stream)
        e1.synchronize()
        return 1e3 * e0.elapsed_time(e1) / n

    rows = []
    Lb = args.precision_L
    for i, (name, kind, bits, qp) in enumerate(variants):
        with make(kind, bits, qp, 32, 11) as x:
            x.sweep(2000)
            us32 = timed(x, args.xy_steps)
        with make(kind, bits, qp, Lb, 100 + i) as x:
            if kind == "fp":
                u = np.zeros((Lb, Lb, 2))
                u[..., 0] = 1.0
                x.set_spins(u)
            else:
                x.set_angles(np.zeros((Lb, Lb), dtype=np.int32))
            x.sweep(2000)
            us_b = timed(x, 200)
            x.sweep(args.precision_sweeps, 1)
            if kind == "fp":
                E, _, _ = x.series(args.precision_sweeps)
            else:
                E2, _, _ = x.series(args.precision_sweeps)
                E = -E2.astype(np.float64) / 2.0 ** (2 * bits)
        e = E / (Lb * Lb)
        m, err = stats.mean_and_error(e)
        rows.append({"type": name, "probability": "truncated to the type" if qp else "32-bit",
                     "gpu_us_per_step_L32": us32,
                     "site_updates_per_ns_L%d" % Lb: Lb * Lb / (us_b * 1e3),
                     "energy_per_spin": m, "error": err, "tau_int_E": stats.tau_int(e)})
    ref, ref_err = rows[0]["energy_per_spin"], rows[0]["error"]
    for r in rows[1:]:
        d = r["energy_per_spin"] - ref
        r["bias_vs_fp64"] = d
        r["bias_sigma"] = d / float(np.hypot(r["error"], ref_err))
        r["bias_relative"] = d / abs(ref)
    line = {"metric": "XY operand-precision trial (the paper's Tab. S3 setting)",
            "value": rows[4]["gpu_us_per_step_L32"], "unit": "us per MC step, (16, 8) fixed point, L=32",
            "n_gpus": 1, "higher_is_better": False, "data": "synthetic", "dtype": "i32",
            "config": {"workload": "2D XY model T=0.85: angles in FP64 / FP32 / fixed point F=16,12,8, "
                                   "32-bit random words; timing at L=32, energy bias at L=%d" % Lb,
                       "timed_steps_L32": args.xy_steps, "chain_sweeps": args.precision_sweeps,
                       "thermalise": 2000, "start": "ordered"},
            "variants": rows,
            "paper_context": "FPGA at L=32: 42.36 / 42.29 / 41.82 / 41.75 / 41.68 us per step for "
                             "(64,fl) / (32,fl) / (32,16) / (24,12) / (16,8) (Tab. S3)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    global SWEEPS_PER_STEP
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="use the fixed kernel shape instead of the autotuner's choice")
    ap.add_argument("--no-indep", action="store_true",
                    help="skip the independent-samples comparison at beta_c (plain / learned / SW)")
    ap.add_argument("--indep-chains", type=int, default=64)
    ap.add_argument("--indep-plain-sweeps", type=int, default=200000)
    ap.add_argument("--indep-learned-chains", type=int, default=32)
    ap.add_argument("--indep-learned-steps", type=int, default=12000)
    ap.add_argument("--indep-single-steps", type=int, default=2000)
    ap.add_argument("--indep-thermalise", type=int, default=20000)
    ap.add_argument("--indep-train-windows", type=int, default=60000)
    ap.add_argument("--indep-train-epochs", type=int, default=3)
    ap.add_argument("--train-windows", type=int, default=100000)
    ap.add_argument("--proposal", choices=sorted(PROPOSALS), default="staged",
                    help="learned block proposal family (learned workloads)")
    ap.add_argument("--train-epochs", type=int, default=4)
    ap.add_argument("--chain-sweeps", type=int, default=60000)
    ap.add_argument("--chains", type=int, default=2)
    ap.add_argument("--thermalise", type=int, default=5000)
    ap.add_argument("--scan-blocks", type=int, nargs="*", default=[2, 4, 8, 16])
    ap.add_argument("--scan-sweeps", type=int, default=3000)
    ap.add_argument("--xy-steps", type=int, default=10000)
    ap.add_argument("--sw-steps", type=int, default=20000)
    ap.add_argument("--quad-sweeps", type=int, default=2000)
    ap.add_argument("--precision-sweeps", type=int, default=20000)
    ap.add_argument("--precision-L", type=int, default=1024)
    ap.add_argument("--sw-L", type=int, default=16384, help="lattice size of --workload sw_step")
    ap.add_argument("--xy-L", type=int, default=4096, help="lattice size of --workload xy_step")
    ap.add_argument("--xy-precision", type=int, choices=[32, 64], default=32,
                    help="precision of --workload xy_step")
    ap.add_argument("--pass-L", type=int, default=256, help="lattice size of --workload staged_pass")
    ap.add_argument("--train-precision", choices=sorted(TRAIN_PRECISIONS), default="bf16_tc",
                    help="training kernel of the learned workloads")
    ap.add_argument("--train-kernels", nargs="*", choices=sorted(TRAIN_PRECISIONS),
                    default=["fp32", "bf16_tc"], help="kernels timed by --workload train")
    ap.add_argument("--nn-engine", choices=sorted(NN_ENGINES), default="mma_sync",
                    help="engine of the staged proposal's second convolution (staged_pass)")
    ap.add_argument("--workload", choices=["plain", "batch", "learned", "batch_learned", "xy", "sw", "quad",
                                           "xy_precision", "sw_step", "staged_pass", "train", "xy_step"],
                    default="plain",
                    help="plain: one L=16384 lattice (default); batch: 4096 replicas with "
                         "parallel tempering")
    ap.add_argument("--batch-kernel", default="",
                    help="batch work decomposition 'words_per_item,threads'")
    ap.add_argument("--sweeps", type=int, default=SWEEPS_PER_STEP,
                    help="sweeps per step (default 1000; smaller only for profiling runs)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    SWEEPS_PER_STEP = args.sweeps
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "batch_learned":
        return run_batch_learned(args)
    if args.workload == "xy":
        return run_xy(args)
    if args.workload == "sw":
        return run_sw(args)
    if args.workload == "quad":
        return run_quad(args)
    if args.workload == "xy_precision":
        return run_xy_precision(args)
    if args.workload == "sw_step":
        return run_sw_step(args)
    if args.workload == "staged_pass":
        return run_staged_pass(args)
    if args.workload == "train":
        return run_train(args)
    if args.workload == "xy_step":
        return run_xy_step(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
