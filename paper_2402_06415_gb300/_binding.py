"""ctypes binding of libising.so: the C-ABI of include/ising.h, same names.

Argument marshalling only: every step of the sweep runs in the CUDA library.
There is no CPU fallback; if libising.so is missing or cannot be loaded every
call raises.  Functions return None on success and raise :class:`IsingError`
(with the library's message) on a non-zero status.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libising.so")

ISING_OK = 0
ISING_EINVAL = -1
ISING_ENOMEM = -2
ISING_ECUDA = -3
ISING_ETIMEOUT = -4
ISING_EINTERNAL = -5

ISING_LAYOUT_I8 = 0
ISING_LAYOUT_BITS = 1
ISING_CLUSTER_AUTO = 0
ISING_CLUSTER_KERNELS = 1
ISING_CLUSTER_PERSISTENT = 2
ISING_CLUSTER_GRAPH = 3

ISING_PROPOSAL_ONESHOT = 0
ISING_PROPOSAL_STAGED = 1
ISING_NN_ENGINE_MMA_SYNC = 0
ISING_NN_ENGINE_TCGEN05 = 1
ISING_NN_TRAIN_FP32 = 0
ISING_NN_TRAIN_BF16_TC = 1

ISING_KERNEL_AUTO = 0
ISING_KERNEL_HALF = 1
ISING_KERNEL_TILED = 2
ISING_KERNEL_RESIDENT = 3

_STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT",
                 -5: "EINTERNAL"}


class IsingError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s (%d): %s" % (_STATUS_NAMES.get(status, "?"), status, message))
        self.status = status
        self.message = message


# (name, restype, argtypes) of every exported entry point of include/ising.h
_p = ctypes.c_void_p
_i = ctypes.c_int
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_i64 = ctypes.c_int64
_d = ctypes.c_double
_PROTOS = [
    ("ising_create", _i, [ctypes.POINTER(_p), _i, _d, _i, _p]),
    ("ising_seed", _i, [_p, _u64]),
    ("ising_set_key", _i, [_p, _u64]),
    ("ising_set_replica", _i, [_p, _u32]),
    ("ising_set_beta", _i, [_p, _d]),
    ("ising_set_sweep_counter", _i, [_p, _i64]),
    ("ising_get_state", _i, [_p, _p, _p, _p]),
    ("ising_sweep", _i, [_p, _i, _i]),
    ("ising_measure", _i, [_p, _p, _p]),
    ("ising_series_count", _i, [_p, _p]),
    ("ising_series", _i, [_p, _p, _p, _i]),
    ("ising_get_spins", _i, [_p, _p]),
    ("ising_set_spins", _i, [_p, _p]),
    ("ising_get_bits", _i, [_p, _p]),
    ("ising_set_bits", _i, [_p, _p]),
    ("ising_get_spins_device", _i, [_p, _p]),
    ("ising_set_spins_device", _i, [_p, _p]),
    ("ising_get_bits_device", _i, [_p, _p]),
    ("ising_set_bits_device", _i, [_p, _p]),
    ("ising_words_per_row", _i, [_i]),
    ("ising_set_kernel", _i, [_p, _i, _i, _i, _i, _i, _i]),
    ("ising_get_kernel", _i, [_p, _p, _p, _p, _p, _p, _p]),
    ("ising_thresholds", _i, [_d, _p, _p]),
    ("ising_set_timing", _i, [_p, _i]),
    ("ising_kernel_time", _i, [_p, _p, _p]),
    ("ising_launch_count", _i, [_p, _p]),
    ("ising_sweep_bits_noalloc", _i, [_p, _p, _i, _d, _u64, _u32, _i64, _i, _i, _p, _p, _i, _p]),
    ("ising_batch_create", _i, [ctypes.POINTER(_p), _i, _p, _i, _p, _i, _p]),
    ("ising_batch_seed", _i, [_p, _u64]),
    ("ising_batch_set_kernel", _i, [_p, _i, _i, _i]),
    ("ising_batch_set_series", _i, [_p, _i]),
    ("ising_batch_run", _i, [_p, _i]),
    ("ising_batch_capture", _i, [_p, _i]),
    ("ising_batch_status", _i, [_p, _p, _p]),
    ("ising_batch_state", _i, [_p, _p, _p, _p]),
    ("ising_batch_swap_counts", _i, [_p, _p, _p]),
    ("ising_batch_series", _i, [_p, _i, _p, _p, _p]),
    ("ising_batch_get_spins", _i, [_p, _i, _i, _p]),
    ("ising_batch_info", _i, [_p, _p, _p, _p]),
    ("ising_batch_nn_load", _i, [_p, _p, ctypes.c_size_t]),
    ("ising_batch_block_pass", _i, [_p, _i, _i]),
    ("ising_batch_block_stats", _i, [_p, _p, _p]),
    ("ising_batch_destroy", _i, [_p]),
    ("ising_selftest_wait", _i, [_d, _p]),
    ("ising_nn_load", _i, [_p, _p, ctypes.c_size_t]),
    ("ising_block_pass", _i, [_p, _i, _i]),
    ("ising_block_stats", _i, [_p, _p, _p]),
    ("ising_sweep_blocks", _i, [_p, _i, _i, _i, _i]),
    ("ising_sw_step", _i, [_p, _i, _i]),
    ("ising_wolff_step", _i, [_p, _i, _i]),
    ("ising_cluster_set_mode", _i, [_p, _i]),
    ("ising_wolff_set_limits", _i, [_p, _i, _i]),
    ("ising_wolff_stats", _i, [_p, _p, _p, _p, _p]),
    ("ising_nn_param_count", _i, []),
    ("ising_nn_create", _i, [ctypes.POINTER(_p), _i, _i, _p]),
    ("ising_nn_set_params", _i, [_p, _p, _i]),
    ("ising_nn_get_params", _i, [_p, _p, _i]),
    ("ising_nn_export", _i, [_p, _p, ctypes.c_size_t]),
    ("ising_nn_logits", _i, [_p, _p, _i, _p]),
    ("ising_nn_loss_grad", _i, [_p, _p, _i, _p, _p]),
    ("ising_nn_train_step", _i, [_p, _p, _i, ctypes.c_float, _p]),
    ("ising_nn_destroy", _i, [_p]),
    ("ising_nn_apply_grads", _i, [_p, _p, _i, ctypes.c_float]),
    ("ising_set_proposal", _i, [_p, _i]),
    ("ising_batch_set_proposal", _i, [_p, _i]),
    ("ising_nn_set_proposal", _i, [_p, _i]),
    ("ising_set_nn_engine", _i, [_p, _i]),
    ("ising_batch_set_nn_engine", _i, [_p, _i]),
    ("ising_nn_set_engine", _i, [_p, _i]),
    ("ising_nn_set_train_precision", _i, [_p, _i]),
    ("ising_proposal_schedule", _i, [_i, _i, _p, _p, _i, ctypes.POINTER(_i)]),
    ("ising_nn_stage_logits", _i, [_p, _p, _i, _i, ctypes.c_double, _p]),
    ("ising_nn_log_q", _i, [_p, _p, _i, ctypes.c_double, _p]),
    ("ising_xy_create", _i, [ctypes.POINTER(_p), _i, _d, _i, _p]),
    ("ising_xy_seed", _i, [_p, _u64]),
    ("ising_xy_sweep", _i, [_p, _i, _i]),
    ("ising_xy_series", _i, [_p, _p, _p, _p, _i]),
    ("ising_xy_get_spins", _i, [_p, _p]),
    ("ising_xy_set_spins", _i, [_p, _p]),
    ("ising_xy_accepted", _i, [_p, _p]),
    ("ising_xy_destroy", _i, [_p]),
    ("ising_xy_set_mode", _i, [_p, _i]),
    ("ising_xy_launch_count", _i, [_p, _p]),
    ("ising_selftest_grid_barrier", _i, [_d, _p]),
    ("ising_xyfix_set_mode", _i, [_p, _i]),
    ("ising_xyfix_create", _i, [ctypes.POINTER(_p), _i, _d, _i, _i, _p]),
    ("ising_xyfix_seed", _i, [_p, _u64]),
    ("ising_xyfix_sweep", _i, [_p, _i, _i]),
    ("ising_xyfix_series", _i, [_p, _p, _p, _p, _i]),
    ("ising_xyfix_get_angles", _i, [_p, _p]),
    ("ising_xyfix_set_angles", _i, [_p, _p]),
    ("ising_xyfix_info", _i, [_p, _p, _p, _p]),
    ("ising_xyfix_destroy", _i, [_p]),
    ("ising_quad_create", _i, [ctypes.POINTER(_p), _i, _i, _d, _d, _d, _p]),
    ("ising_quad_seed", _i, [_p, _u64]),
    ("ising_quad_set_replica", _i, [_p, ctypes.c_uint32]),
    ("ising_quad_sweep", _i, [_p, _i, _i]),
    ("ising_quad_series", _i, [_p, _p, _p, _p, _i]),
    ("ising_quad_get_spins", _i, [_p, _p]),
    ("ising_quad_set_spins", _i, [_p, _p]),
    ("ising_quad_launch_count", _i, [_p, _p]),
    ("ising_quad_destroy", _i, [_p]),
    ("ising_destroy", _i, [_p]),
    ("ising_last_error", ctypes.c_char_p, []),
]

EXPORTED = [name for (name, _, _) in _PROTOS]

_lib = None


def lib() -> ctypes.CDLL:
    """Load libising.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            from . import build as _build

            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libising.so is missing; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _PROTOS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int) -> None:
    if status != ISING_OK:
        raise IsingError(status, lib().ising_last_error().decode("utf-8", "replace"))


def _ptr(a) -> ctypes.c_void_p:
    """Host numpy array (C-contiguous) or torch tensor -> raw pointer."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if hasattr(a, "is_contiguous") and not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError("expected a numpy array or a torch tensor")


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(int(stream.cuda_stream))


# ---------------------------------------------------------------------------
# entry points (same names as the C-ABI)
# ---------------------------------------------------------------------------

def ising_create(L: int, beta: float, layout: int = ISING_LAYOUT_BITS, stream=None) -> int:
    out = ctypes.c_void_p()
    _check(lib().ising_create(ctypes.byref(out), int(L), float(beta), int(layout),
                              _stream_ptr(stream)))
    return out.value


def ising_seed(ctx: int, seed: int) -> None:
    _check(lib().ising_seed(ctx, int(seed)))


def ising_set_key(ctx: int, seed: int) -> None:
    _check(lib().ising_set_key(ctx, int(seed)))


def ising_set_replica(ctx: int, replica: int) -> None:
    _check(lib().ising_set_replica(ctx, int(replica)))


def ising_set_beta(ctx: int, beta: float) -> None:
    _check(lib().ising_set_beta(ctx, float(beta)))


def ising_set_sweep_counter(ctx: int, t: int) -> None:
    _check(lib().ising_set_sweep_counter(ctx, int(t)))


def ising_get_state(ctx: int):
    seed, rep, sw = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_int64()
    _check(lib().ising_get_state(ctx, ctypes.byref(seed), ctypes.byref(rep), ctypes.byref(sw)))
    return int(seed.value), int(rep.value), int(sw.value)


def ising_sweep(ctx: int, n_sweeps: int, measure_every: int = 0) -> None:
    _check(lib().ising_sweep(ctx, int(n_sweeps), int(measure_every)))


def ising_measure(ctx: int):
    E, M = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().ising_measure(ctx, ctypes.byref(E), ctypes.byref(M)))
    return int(E.value), int(M.value)


def ising_series_count(ctx: int) -> int:
    n = ctypes.c_int64()
    _check(lib().ising_series_count(ctx, ctypes.byref(n)))
    return int(n.value)


def ising_series(ctx: int, n: int | None = None):
    if n is None:
        n = min(ising_series_count(ctx), 65536)
    E = np.zeros(max(n, 1), dtype=np.int64)
    M = np.zeros(max(n, 1), dtype=np.int64)
    _check(lib().ising_series(ctx, _ptr(E), _ptr(M), int(n)))
    return E[:n], M[:n]


def ising_get_spins(ctx: int, L: int, out: np.ndarray | None = None) -> np.ndarray:
    if out is None:
        out = np.empty((L, L), dtype=np.int8)
    _check(lib().ising_get_spins(ctx, _ptr(out)))
    return out


def ising_set_spins(ctx: int, spins: np.ndarray) -> None:
    s = np.ascontiguousarray(spins, dtype=np.int8)
    _check(lib().ising_set_spins(ctx, _ptr(s)))


def ising_words_per_row(L: int) -> int:
    return int(lib().ising_words_per_row(int(L)))


def ising_get_bits(ctx: int, L: int, out: np.ndarray | None = None) -> np.ndarray:
    if out is None:
        out = np.empty((2, L, ising_words_per_row(L)), dtype=np.uint32)
    _check(lib().ising_get_bits(ctx, _ptr(out)))
    return out


def ising_set_bits(ctx: int, words: np.ndarray) -> None:
    w = np.ascontiguousarray(words, dtype=np.uint32)
    _check(lib().ising_set_bits(ctx, _ptr(w)))


def ising_get_spins_device(ctx: int, dev_out) -> None:
    _check(lib().ising_get_spins_device(ctx, _ptr(dev_out)))


def ising_set_spins_device(ctx: int, dev_in) -> None:
    _check(lib().ising_set_spins_device(ctx, _ptr(dev_in)))


def ising_get_bits_device(ctx: int, dev_out) -> None:
    _check(lib().ising_get_bits_device(ctx, _ptr(dev_out)))


def ising_set_bits_device(ctx: int, dev_in) -> None:
    _check(lib().ising_set_bits_device(ctx, _ptr(dev_in)))


def ising_set_kernel(ctx: int, kernel: int, sweeps_per_launch: int = 1, tile_rows: int = 1,
                     tile_words: int = 4, grid: int = 0, block: int = 0) -> None:
    _check(lib().ising_set_kernel(ctx, int(kernel), int(sweeps_per_launch), int(tile_rows),
                                  int(tile_words), int(grid), int(block)))


def ising_get_kernel(ctx: int) -> dict:
    v = [ctypes.c_int() for _ in range(6)]
    _check(lib().ising_get_kernel(ctx, *[ctypes.byref(x) for x in v]))
    keys = ["kernel", "sweeps_per_launch", "tile_rows", "tile_words", "grid", "block"]
    return {k: int(x.value) for k, x in zip(keys, v)}


def ising_thresholds(beta: float):
    t4, t8 = ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().ising_thresholds(float(beta), ctypes.byref(t4), ctypes.byref(t8)))
    return int(t4.value), int(t8.value)


def ising_set_timing(ctx: int, enable: bool) -> None:
    _check(lib().ising_set_timing(ctx, 1 if enable else 0))


def ising_kernel_time(ctx: int):
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(lib().ising_kernel_time(ctx, ctypes.byref(ms), ctypes.byref(n)))
    return float(ms.value), int(n.value)


def ising_launch_count(ctx: int) -> int:
    n = ctypes.c_int64()
    _check(lib().ising_launch_count(ctx, ctypes.byref(n)))
    return int(n.value)


def ising_sweep_bits_noalloc(dev_in, dev_out, L: int, beta: float, seed: int, replica: int,
                             sweep0: int, n_sweeps: int, measure_every: int = 0, dev_E=None,
                             dev_M=None, sweeps_per_launch: int = 2, stream=None) -> None:
    """Allocation-free sweep on caller-owned device buffers (see include/ising.h)."""
    E = _ptr(dev_E) if dev_E is not None else ctypes.c_void_p(0)
    M = _ptr(dev_M) if dev_M is not None else ctypes.c_void_p(0)
    _check(lib().ising_sweep_bits_noalloc(_ptr(dev_in), _ptr(dev_out), int(L), float(beta),
                                          int(seed), int(replica), int(sweep0), int(n_sweeps),
                                          int(measure_every), E, M, int(sweeps_per_launch),
                                          _stream_ptr(stream)))


def ising_destroy(ctx: int) -> None:
    _check(lib().ising_destroy(ctx))


def ising_last_error() -> str:
    return lib().ising_last_error().decode("utf-8", "replace")


class Lattice:
    """Owning wrapper around one ising_ctx (closes it on exit / deletion)."""

    def __init__(self, L: int, beta: float, layout: int = ISING_LAYOUT_BITS, stream=None,
                 seed: int | None = None, replica: int = 0):
        self.L = int(L)
        self.layout = layout
        self.ctx = ising_create(L, beta, layout, stream)
        if replica:
            ising_set_replica(self.ctx, replica)
        if seed is not None:
            ising_seed(self.ctx, seed)

    def close(self):
        if getattr(self, "ctx", None):
            ising_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def seed(self, seed: int):
        ising_seed(self.ctx, seed)

    def sweep(self, n: int, measure_every: int = 0):
        ising_sweep(self.ctx, n, measure_every)

    def sw_step(self, n: int, measure_every: int = 0):
        """n Swendsen-Wang cluster steps (packed layout only)."""
        ising_sw_step(self.ctx, n, measure_every)

    def wolff_step(self, n: int, measure_every: int = 0):
        """n Wolff single-cluster steps (packed layout only)."""
        ising_wolff_step(self.ctx, n, measure_every)

    def cluster_set_mode(self, mode: int):
        """ISING_CLUSTER_AUTO / _KERNELS / _PERSISTENT / _GRAPH for sw_step and wolff_step."""
        _check(lib().ising_cluster_set_mode(self.ctx, int(mode)))

    def wolff_set_limits(self, max_sites: int, max_levels: int = 0):
        ising_wolff_set_limits(self.ctx, max_sites, max_levels)

    def wolff_stats(self) -> dict:
        return ising_wolff_stats(self.ctx)

    def measure(self):
        return ising_measure(self.ctx)

    def series(self, n=None):
        return ising_series(self.ctx, n)

    def spins(self) -> np.ndarray:
        return ising_get_spins(self.ctx, self.L)

    def set_spins(self, s):
        ising_set_spins(self.ctx, s)

    def bits(self) -> np.ndarray:
        return ising_get_bits(self.ctx, self.L)

    def set_bits(self, w):
        ising_set_bits(self.ctx, w)

    def set_kernel(self, *a, **k):
        ising_set_kernel(self.ctx, *a, **k)

    def kernel(self) -> dict:
        return ising_get_kernel(self.ctx)


# ---------------------------------------------------------------------------
# batched replicas with parallel tempering
# ---------------------------------------------------------------------------

def ising_batch_create(Ls, betas, pt_every: int, stream=None) -> int:
    Lh = np.ascontiguousarray(Ls, dtype=np.int32)
    bh = np.ascontiguousarray(betas, dtype=np.float64)
    out = ctypes.c_void_p()
    _check(lib().ising_batch_create(ctypes.byref(out), len(Lh), _ptr(Lh), len(bh), _ptr(bh),
                                    int(pt_every), _stream_ptr(stream)))
    return out.value


def ising_batch_seed(b: int, seed: int) -> None:
    _check(lib().ising_batch_seed(b, int(seed)))


def ising_batch_set_kernel(b: int, words_per_item: int = 512, threads: int = 256,
                           grid: int = 0) -> None:
    _check(lib().ising_batch_set_kernel(b, int(words_per_item), int(threads), int(grid)))


def ising_batch_set_series(b: int, capacity: int) -> None:
    _check(lib().ising_batch_set_series(b, int(capacity)))


def ising_batch_run(b: int, n_sweeps: int) -> None:
    _check(lib().ising_batch_run(b, int(n_sweeps)))


def ising_batch_capture(b: int, n_sweeps: int) -> None:
    _check(lib().ising_batch_capture(b, int(n_sweeps)))


def ising_batch_status(b: int):
    st, sw = ctypes.c_int(), ctypes.c_int64()
    _check(lib().ising_batch_status(b, ctypes.byref(st), ctypes.byref(sw)))
    return int(st.value), int(sw.value)


def ising_batch_state(b: int, n_rep: int):
    perm = np.zeros(n_rep, dtype=np.int32)
    E = np.zeros(n_rep, dtype=np.int64)
    M = np.zeros(n_rep, dtype=np.int64)
    _check(lib().ising_batch_state(b, _ptr(perm), _ptr(E), _ptr(M)))
    return perm, E, M


def ising_batch_swap_counts(b: int, n_rep: int):
    acc = np.zeros(n_rep, dtype=np.int64)
    att = np.zeros(n_rep, dtype=np.int64)
    _check(lib().ising_batch_swap_counts(b, _ptr(acc), _ptr(att)))
    return acc, att


def ising_batch_series(b: int, n_steps: int, n_rep: int):
    E = np.zeros((max(n_steps, 1), n_rep), dtype=np.int32)
    M = np.zeros((max(n_steps, 1), n_rep), dtype=np.int32)
    S = np.zeros((max(n_steps, 1), n_rep), dtype=np.int16)
    _check(lib().ising_batch_series(b, int(n_steps), _ptr(E), _ptr(M), _ptr(S)))
    return E[:n_steps], M[:n_steps], S[:n_steps]


def ising_batch_get_spins(b: int, ladder: int, replica: int, L: int) -> np.ndarray:
    out = np.empty((L, L), dtype=np.int8)
    _check(lib().ising_batch_get_spins(b, int(ladder), int(replica), _ptr(out)))
    return out


def ising_batch_info(b: int):
    n, g, sw = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    _check(lib().ising_batch_info(b, ctypes.byref(n), ctypes.byref(g), ctypes.byref(sw)))
    return {"items": int(n.value), "grid": int(g.value), "sweep": int(sw.value)}


def ising_batch_nn_load(b: int, blob: np.ndarray) -> None:
    v = np.ascontiguousarray(blob)
    _check(lib().ising_batch_nn_load(b, _ptr(v), v.nbytes))


def ising_batch_block_pass(b: int, n_passes: int, block: int = 16) -> None:
    _check(lib().ising_batch_block_pass(b, int(n_passes), int(block)))


def ising_batch_block_stats(b: int):
    p, a = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().ising_batch_block_stats(b, ctypes.byref(p), ctypes.byref(a)))
    return int(p.value), int(a.value)


def ising_selftest_wait(timeout_s: float) -> int:
    """Runs the bounded-wait self test; raises IsingError(ETIMEOUT) as designed."""
    st = ctypes.c_int()
    _check(lib().ising_selftest_wait(float(timeout_s), ctypes.byref(st)))
    return int(st.value)


def ising_batch_destroy(b: int) -> None:
    _check(lib().ising_batch_destroy(b))


class Batch:
    """Owning wrapper of an ising_batch."""

    def __init__(self, Ls, betas, pt_every: int, stream=None, seed: int | None = None):
        self.Ls = [int(x) for x in Ls]
        self.betas = np.asarray(betas, dtype=np.float64)
        self.n_beta = len(self.betas)
        self.n_rep = len(self.Ls) * self.n_beta
        self.h = ising_batch_create(self.Ls, self.betas, pt_every, stream)
        if seed is not None:
            ising_batch_seed(self.h, seed)

    def close(self):
        if getattr(self, "h", None):
            ising_batch_destroy(self.h)
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

    def run(self, n):
        ising_batch_run(self.h, n)

    def state(self):
        p, E, M = ising_batch_state(self.h, self.n_rep)
        nl = len(self.Ls)
        return p.reshape(nl, self.n_beta), E.reshape(nl, self.n_beta), M.reshape(nl, self.n_beta)

    def swap_counts(self):
        a, t = ising_batch_swap_counts(self.h, self.n_rep)
        nl = len(self.Ls)
        return a.reshape(nl, self.n_beta), t.reshape(nl, self.n_beta)

    def spins(self, ladder, replica):
        return ising_batch_get_spins(self.h, ladder, replica, self.Ls[ladder])


# ---------------------------------------------------------------------------
# learned block proposal
# ---------------------------------------------------------------------------
NN_CHANNELS = 32
NN_SHAPES = [("W1", (32, 2, 3, 3)), ("b1", (32,)), ("W2", (32, 32, 3, 3)), ("b2", (32,)),
             ("W3", (1, 32, 3, 3)), ("b3", (1,))]


def nn_flatten(params: dict) -> np.ndarray:
    """Parameter dict (W1, b1, W2, b2, W3, b3) -> flat float32 vector (C-ABI order)."""
    return np.concatenate([np.asarray(params[k], dtype=np.float32).reshape(-1)
                           for k, _ in NN_SHAPES]).astype(np.float32)


def nn_unflatten(v) -> dict:
    out, o = {}, 0
    for k, shp in NN_SHAPES:
        n = int(np.prod(shp))
        out[k] = np.asarray(v[o:o + n]).reshape(shp)
        o += n
    return out


def ising_nn_load(ctx: int, blob: np.ndarray) -> None:
    b = np.ascontiguousarray(blob)
    _check(lib().ising_nn_load(ctx, _ptr(b), b.nbytes))


def ising_block_pass(ctx: int, n_passes: int, block: int = 16) -> None:
    _check(lib().ising_block_pass(ctx, int(n_passes), int(block)))


def ising_sweep_blocks(ctx: int, n_sweeps: int, measure_every: int = 0, block: int = 16,
                       block_every: int = 1) -> None:
    _check(lib().ising_sweep_blocks(ctx, int(n_sweeps), int(measure_every), int(block),
                                    int(block_every)))


def ising_sw_step(ctx: int, n_steps: int, measure_every: int = 0) -> None:
    _check(lib().ising_sw_step(ctx, int(n_steps), int(measure_every)))


def ising_wolff_step(ctx: int, n_steps: int, measure_every: int = 0) -> None:
    _check(lib().ising_wolff_step(ctx, int(n_steps), int(measure_every)))


def ising_wolff_set_limits(ctx: int, max_sites: int, max_levels: int = 0) -> None:
    _check(lib().ising_wolff_set_limits(ctx, int(max_sites), int(max_levels)))


def ising_wolff_stats(ctx: int) -> dict:
    v = [ctypes.c_int64() for _ in range(4)]
    _check(lib().ising_wolff_stats(ctx, *(ctypes.byref(x) for x in v)))
    return dict(zip(("last_size", "flipped", "grown", "labelled"), (int(x.value) for x in v)))


def ising_block_stats(ctx: int):
    p, a = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().ising_block_stats(ctx, ctypes.byref(p), ctypes.byref(a)))
    return int(p.value), int(a.value)


def ising_nn_param_count() -> int:
    return int(lib().ising_nn_param_count())


def ising_nn_create(block: int = 16, channels: int = NN_CHANNELS, stream=None) -> int:
    out = ctypes.c_void_p()
    _check(lib().ising_nn_create(ctypes.byref(out), int(block), int(channels), _stream_ptr(stream)))
    return out.value


def ising_nn_set_params(nn: int, flat: np.ndarray) -> None:
    v = np.ascontiguousarray(flat, dtype=np.float32)
    _check(lib().ising_nn_set_params(nn, _ptr(v), v.size))


def ising_nn_get_params(nn: int) -> np.ndarray:
    v = np.zeros(ising_nn_param_count(), dtype=np.float32)
    _check(lib().ising_nn_get_params(nn, _ptr(v), v.size))
    return v


def ising_nn_export(nn: int) -> np.ndarray:
    blob = np.zeros(ising_nn_param_count(), dtype=np.uint16)
    _check(lib().ising_nn_export(nn, _ptr(blob), blob.nbytes))
    return blob


def ising_nn_logits(nn: int, dev_windows, count: int, dev_logits) -> None:
    _check(lib().ising_nn_logits(nn, _ptr(dev_windows), int(count), _ptr(dev_logits)))


def ising_nn_loss_grad(nn: int, dev_windows, count: int, want_grads: bool = True):
    loss = ctypes.c_float()
    g = np.zeros(ising_nn_param_count(), dtype=np.float32) if want_grads else None
    _check(lib().ising_nn_loss_grad(nn, _ptr(dev_windows), int(count), ctypes.byref(loss),
                                    _ptr(g) if g is not None else ctypes.c_void_p(0)))
    return float(loss.value), g


def ising_nn_train_step(nn: int, dev_windows, count: int, lr: float) -> float:
    loss = ctypes.c_float()
    _check(lib().ising_nn_train_step(nn, _ptr(dev_windows), int(count), float(lr),
                                     ctypes.byref(loss)))
    return float(loss.value)


def ising_nn_destroy(nn: int) -> None:
    _check(lib().ising_nn_destroy(nn))


def ising_nn_apply_grads(nn: int, grads: np.ndarray, lr: float) -> None:
    g = np.ascontiguousarray(grads, dtype=np.float32)
    _check(lib().ising_nn_apply_grads(nn, _ptr(g), g.size, float(lr)))


def ising_set_proposal(ctx: int, kind: int) -> None:
    _check(lib().ising_set_proposal(ctx, int(kind)))


def ising_batch_set_proposal(b: int, kind: int) -> None:
    _check(lib().ising_batch_set_proposal(b, int(kind)))


def ising_nn_set_proposal(nn: int, kind: int) -> None:
    _check(lib().ising_nn_set_proposal(nn, int(kind)))


def ising_set_nn_engine(ctx: int, engine: int) -> None:
    _check(lib().ising_set_nn_engine(ctx, int(engine)))


def ising_batch_set_nn_engine(b: int, engine: int) -> None:
    _check(lib().ising_batch_set_nn_engine(b, int(engine)))


def ising_nn_set_engine(nn: int, engine: int) -> None:
    _check(lib().ising_nn_set_engine(nn, int(engine)))


def ising_nn_set_train_precision(nn: int, precision: int) -> None:
    _check(lib().ising_nn_set_train_precision(nn, int(precision)))


def ising_proposal_schedule(block: int, kind: int = ISING_PROPOSAL_STAGED):
    """(stage_of_site (block, block) uint8, stage_exact (n_stages,) uint8)."""
    so = np.zeros(block * block, dtype=np.uint8)
    ex = np.zeros(64, dtype=np.uint8)
    n = ctypes.c_int()
    _check(lib().ising_proposal_schedule(int(block), int(kind), _ptr(so), _ptr(ex), ex.size,
                                         ctypes.byref(n)))
    return so.reshape(block, block), ex[:n.value].copy()


def ising_nn_stage_logits(nn: int, dev_windows, count: int, stage: int, beta: float,
                          dev_logits) -> None:
    _check(lib().ising_nn_stage_logits(nn, _ptr(dev_windows), int(count), int(stage), float(beta),
                                       _ptr(dev_logits)))


def ising_nn_log_q(nn: int, dev_windows, count: int, beta: float, dev_log_q) -> None:
    _check(lib().ising_nn_log_q(nn, _ptr(dev_windows), int(count), float(beta), _ptr(dev_log_q)))


# ---------------------------------------------------------------------------
# 2D XY model
# ---------------------------------------------------------------------------

class XY:
    """Owning wrapper of an ising_xy context (unit-vector spins)."""

    def __init__(self, L: int, beta: float, precision: int = 64, stream=None, seed=None):
        self.L = int(L)
        out = ctypes.c_void_p()
        _check(lib().ising_xy_create(ctypes.byref(out), self.L, float(beta), int(precision),
                                     _stream_ptr(stream)))
        self.h = out.value
        if seed is not None:
            self.seed(seed)

    def close(self):
        if getattr(self, "h", None):
            _check(lib().ising_xy_destroy(self.h))
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

    def seed(self, seed: int):
        _check(lib().ising_xy_seed(self.h, int(seed)))

    def sweep(self, n: int, measure_every: int = 0):
        _check(lib().ising_xy_sweep(self.h, int(n), int(measure_every)))

    def series(self, n: int):
        E, Mx, My = (np.zeros(max(n, 1)) for _ in range(3))
        _check(lib().ising_xy_series(self.h, _ptr(E), _ptr(Mx), _ptr(My), int(n)))
        return E[:n], Mx[:n], My[:n]

    def spins(self) -> np.ndarray:
        u = np.zeros((self.L, self.L, 2))
        _check(lib().ising_xy_get_spins(self.h, _ptr(u)))
        return u

    def set_spins(self, u: np.ndarray):
        v = np.ascontiguousarray(u, dtype=np.float64)
        _check(lib().ising_xy_set_spins(self.h, _ptr(v)))

    def accepted(self) -> int:
        a = ctypes.c_int64()
        _check(lib().ising_xy_accepted(self.h, ctypes.byref(a)))
        return int(a.value)

    def set_mode(self, mode: int):
        """0 automatic, 1 one launch per half sweep, 2 persistent kernel."""
        _check(lib().ising_xy_set_mode(self.h, int(mode)))

    def launch_count(self) -> int:
        c = ctypes.c_int64()
        _check(lib().ising_xy_launch_count(self.h, ctypes.byref(c)))
        return int(c.value)


def ising_selftest_grid_barrier(timeout_s: float) -> int:
    """1 if the persistent kernels' grid barrier timed out as designed."""
    st = ctypes.c_int()
    _check(lib().ising_selftest_grid_barrier(float(timeout_s), ctypes.byref(st)))
    return int(st.value)


# ---------------------------------------------------------------------------
# fixed-point XY model (operand-precision study)
# ---------------------------------------------------------------------------

ISING_XYFIX_QUANTISE_P = 1


class XYFix:
    """Owning wrapper of an ising_xyfix context (angles with F fractional bits)."""

    def __init__(self, L: int, beta: float, frac_bits: int, stream=None, seed=None,
                 quantise_p: bool = False):
        self.L = int(L)
        self.F = int(frac_bits)
        out = ctypes.c_void_p()
        _check(lib().ising_xyfix_create(ctypes.byref(out), self.L, float(beta), self.F,
                                        ISING_XYFIX_QUANTISE_P if quantise_p else 0,
                                        _stream_ptr(stream)))
        self.h = out.value
        if seed is not None:
            self.seed(seed)

    def close(self):
        if getattr(self, "h", None):
            _check(lib().ising_xyfix_destroy(self.h))
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

    def seed(self, seed: int):
        _check(lib().ising_xyfix_seed(self.h, int(seed)))

    def sweep(self, n: int, measure_every: int = 0):
        _check(lib().ising_xyfix_sweep(self.h, int(n), int(measure_every)))

    def series(self, n: int):
        """(E2, Mx, My) integers of the last n records: energy = -E2 2^-2F."""
        E2, Mx, My = (np.zeros(max(n, 1), dtype=np.int64) for _ in range(3))
        _check(lib().ising_xyfix_series(self.h, _ptr(E2), _ptr(Mx), _ptr(My), int(n)))
        return E2[:n], Mx[:n], My[:n]

    def angles(self) -> np.ndarray:
        k = np.zeros((self.L, self.L), dtype=np.int32)
        _check(lib().ising_xyfix_get_angles(self.h, _ptr(k)))
        return k

    def set_angles(self, k: np.ndarray):
        v = np.ascontiguousarray(k, dtype=np.int32)
        if v.shape != (self.L, self.L):
            raise ValueError("angles must have shape (L, L)")
        _check(lib().ising_xyfix_set_angles(self.h, _ptr(v)))

    def set_mode(self, mode: int):
        """0 automatic, 1 one launch per half sweep, 2 persistent kernel."""
        _check(lib().ising_xyfix_set_mode(self.h, int(mode)))

    def info(self):
        K, a, n = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().ising_xyfix_info(self.h, ctypes.byref(K), ctypes.byref(a), ctypes.byref(n)))
        return {"K": int(K.value), "accepted": int(a.value), "launches": int(n.value)}


# ---------------------------------------------------------------------------
# four-sublattice lattices (square NN + NNN, square-octagon)
# ---------------------------------------------------------------------------

ISING_QUAD_SQUARE = 0
ISING_QUAD_SQOCT = 1


class Quad:
    """Owning wrapper of an ising_quad context; spins as s[q][Y][X]."""

    def __init__(self, lattice: int, Lc: int, beta: float, J1: float = 1.0, J2: float = 0.0,
                 stream=None, seed=None, replica: int = 0):
        self.Lc = int(Lc)
        self.lattice = int(lattice)
        self.J1, self.J2 = float(J1), float(J2)
        out = ctypes.c_void_p()
        _check(lib().ising_quad_create(ctypes.byref(out), self.lattice, self.Lc, float(beta),
                                       self.J1, self.J2, _stream_ptr(stream)))
        self.h = out.value
        if replica:
            _check(lib().ising_quad_set_replica(self.h, int(replica)))
        if seed is not None:
            self.seed(seed)

    def close(self):
        if getattr(self, "h", None):
            _check(lib().ising_quad_destroy(self.h))
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

    def seed(self, seed: int):
        _check(lib().ising_quad_seed(self.h, int(seed)))

    def sweep(self, n: int, measure_every: int = 0):
        _check(lib().ising_quad_sweep(self.h, int(n), int(measure_every)))

    def series(self, n: int):
        """(B1, B2, M) of the last n records; energy = -J1 B1 - J2 B2."""
        B1, B2, M = (np.zeros(max(n, 1), dtype=np.int64) for _ in range(3))
        _check(lib().ising_quad_series(self.h, _ptr(B1), _ptr(B2), _ptr(M), int(n)))
        return B1[:n], B2[:n], M[:n]

    def spins(self) -> np.ndarray:
        s = np.zeros((4, self.Lc, self.Lc), dtype=np.int8)
        _check(lib().ising_quad_get_spins(self.h, _ptr(s)))
        return s

    def set_spins(self, s: np.ndarray):
        v = np.ascontiguousarray(s, dtype=np.int8)
        if v.shape != (4, self.Lc, self.Lc):
            raise ValueError("spins must have shape (4, Lc, Lc)")
        _check(lib().ising_quad_set_spins(self.h, _ptr(v)))

    def launch_count(self) -> int:
        c = ctypes.c_int64()
        _check(lib().ising_quad_launch_count(self.h, ctypes.byref(c)))
        return int(c.value)
