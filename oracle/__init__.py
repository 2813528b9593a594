"""CPU oracle for the checkerboard Metropolis sweep of the 2D Ising model.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package.  The
product path (``paper_2402_06415_gb300``) never imports it; the two share no
code.  What the oracle computes, and which passage of arXiv 2402.06415 each
part follows, is stated in ``ising_oracle.c`` (sweep, Philox, counter map,
Swendsen-Wang), ``xy_oracle.c`` (XY model), ``xyfix_oracle.c`` (fixed-point XY
for the precision study), ``quad_oracle.c`` (four-sublattice lattices),
``closed_forms.py`` (Onsager / Yang / Kaufman) and ``exact.py`` (brute force).

The C part is compiled by :func:`build` (plain gcc, no CUDA) into
``liboracle.so`` next to this file and called through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ising_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "xy_oracle.c"), os.path.join(_HERE, "quad_oracle.c"),
         os.path.join(_HERE, "xyfix_oracle.c"), os.path.join(_HERE, "ising_oracle_omp.c")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

TAG_INIT = 1
TAG_MET = 2
TAG_PT = 3

BETA_C = float(np.log(1.0 + np.sqrt(2.0)) / 2.0)


def build(force: bool = False) -> str:
    """Compile ``ising_oracle.c`` with gcc into ``liboracle.so``."""
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, *_SRCS, "-lm"]
    # OpenMP only spreads the timing build's rows (ising_oracle_omp.c) over
    # threads; without it that file compiles serially.
    r = subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        u32, i32, u64, i64, dbl = (ctypes.c_uint32, ctypes.c_int, ctypes.c_uint64,
                                   ctypes.c_int64, ctypes.c_double)
        p = ctypes.c_void_p
        L.orc_philox4x32_10.argtypes = [p, p, p]
        L.orc_philox4x32_10.restype = None
        L.orc_words_per_row.argtypes = [i32]
        L.orc_words_per_row.restype = i32
        L.orc_threshold.argtypes = [dbl, i32]
        L.orc_threshold.restype = u32
        L.orc_decide.argtypes = [i32, u32, u32, u32]
        L.orc_decide.restype = i32
        L.orc_met_planes.argtypes = [u64, u32, u32, i32, u32, p]
        L.orc_met_planes.restype = None
        L.orc_assemble_u.argtypes = [p, i32]
        L.orc_assemble_u.restype = u32
        L.orc_site_uniform.argtypes = [i32, u64, u32, u32, i32, i32]
        L.orc_site_uniform.restype = u32
        L.orc_n_anti.argtypes = [i32, p, i32, i32]
        L.orc_n_anti.restype = i32
        L.orc_energy_mag.argtypes = [i32, p, p, p]
        L.orc_energy_mag.restype = None
        L.orc_init.argtypes = [i32, u64, u32, p]
        L.orc_init.restype = None
        L.orc_half_sweep.argtypes = [i32, u32, u32, u64, u32, u32, i32, p]
        L.orc_half_sweep.restype = None
        L.orc_sweep.argtypes = [i32, dbl, u64, u32, u32, i32, i32, p, p, p]
        L.orc_sweep.restype = i32
        L.orc_sweep_omp.argtypes = [i32, dbl, u64, u32, u32, i32, i32, p, p, p]
        L.orc_sweep_omp.restype = i32
        L.orc_omp_threads.argtypes = []
        L.orc_omp_threads.restype = i32
        L.orc_accept_count.argtypes = [i32, u32, u32]
        L.orc_accept_count.restype = u64
        L.orc_n_anti_all.argtypes = [i32, i32, p, p]
        L.orc_n_anti_all.restype = None
        L.orc_pt_step.argtypes = [i32, p, u64, u32, u32, p, p, p, p]
        L.orc_pt_step.restype = None
        L.orc_sw_threshold.argtypes = [dbl]
        L.orc_sw_threshold.restype = u32
        L.orc_sw_step.argtypes = [i32, dbl, u64, u32, u32, p, p]
        L.orc_sw_step.restype = i64
        L.orc_wolff_seed_site.argtypes = [i32, u64, u32, u32]
        L.orc_wolff_seed_site.restype = u32
        L.orc_wolff_step.argtypes = [i32, dbl, u64, u32, u32, p, p, p]
        L.orc_wolff_step.restype = i64
        L.orc_quad_neighbours.argtypes = [i32, i32, i32, i32, i32, p]
        L.orc_quad_neighbours.restype = i32
        L.orc_quad_threshold.argtypes = [i32, dbl, dbl, dbl, i32, i32, p]
        L.orc_quad_threshold.restype = u32
        L.orc_quad_init.argtypes = [i32, u64, u32, p]
        L.orc_quad_init.restype = None
        L.orc_quad_uniform.argtypes = [i32, u64, u32, u32, i32, i32, i32]
        L.orc_quad_uniform.restype = u32
        L.orc_quad_anti.argtypes = [i32, i32, p, i32, i32, i32, p, p]
        L.orc_quad_anti.restype = None
        L.orc_quad_observables.argtypes = [i32, i32, p, p, p, p]
        L.orc_quad_observables.restype = None
        L.orc_quad_quarter.argtypes = [i32, i32, dbl, dbl, dbl, u64, u32, u32, i32, p]
        L.orc_quad_quarter.restype = None
        L.orc_quad_sweep.argtypes = [i32, i32, dbl, dbl, dbl, u64, u32, u32, i32, i32, p, p, p, p]
        L.orc_quad_sweep.restype = i32
        L.orc_xyfix_K.argtypes = [i32]
        L.orc_xyfix_K.restype = ctypes.c_int32
        L.orc_xyfix_trig.argtypes = [i32, ctypes.c_int32, p, p]
        L.orc_xyfix_trig.restype = None
        L.orc_xyfix_accept.argtypes = [i32, dbl, ctypes.c_int32, i32]
        L.orc_xyfix_accept.restype = u32
        L.orc_xyfix_dE.argtypes = [i32, ctypes.c_int32, ctypes.c_int32, i64, i64]
        L.orc_xyfix_dE.restype = i64
        L.orc_xyfix_init.argtypes = [i32, i32, u64, u32, p]
        L.orc_xyfix_init.restype = None
        L.orc_xyfix_sweep.argtypes = [i32, i32, i32, dbl, u64, u32, u32, p]
        L.orc_xyfix_sweep.restype = i64
        L.orc_xyfix_observables.argtypes = [i32, i32, p, p, p, p]
        L.orc_xyfix_observables.restype = None
        L.orc_xy_sincos_d.argtypes = [dbl, p, p]
        L.orc_xy_sincos_d.restype = None
        L.orc_xy_exp_d.argtypes = [dbl]
        L.orc_xy_exp_d.restype = dbl
        L.orc_xy_sincos_f.argtypes = [ctypes.c_float, p, p]
        L.orc_xy_sincos_f.restype = None
        L.orc_xy_exp_f.argtypes = [ctypes.c_float]
        L.orc_xy_exp_f.restype = ctypes.c_float
        L.orc_xy_init_d.argtypes = [i32, u64, u32, p]
        L.orc_xy_init_d.restype = None
        L.orc_xy_init_f.argtypes = [i32, u64, u32, p]
        L.orc_xy_init_f.restype = None
        L.orc_xy_sweep_d.argtypes = [i32, dbl, u64, u32, u32, p]
        L.orc_xy_sweep_d.restype = i64
        L.orc_xy_sweep_f.argtypes = [i32, ctypes.c_float, u64, u32, u32, p]
        L.orc_xy_sweep_f.restype = i64
        L.orc_xy_observables_d.argtypes = [i32, p, p, p, p]
        L.orc_xy_observables_d.restype = None
        L.orc_xy_observables_f.argtypes = [i32, p, p, p, p]
        L.orc_xy_observables_f.restype = None
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


# ---------------------------------------------------------------------------
# numpy-facing wrappers
# ---------------------------------------------------------------------------

def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for counter ``ctr`` (4 x u32) and ``key`` (2 x u32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def threshold(beta: float, dE: int) -> int:
    """floor(exp(-beta dE) 2^32) as used by the acceptance test."""
    return int(lib().orc_threshold(float(beta), int(dE)))


def decide(n_anti: int, u: int, thr4: int, thr8: int) -> bool:
    return bool(lib().orc_decide(int(n_anti), int(u), int(thr4), int(thr8)))


def accept_count(n_anti: int, thr4: int, thr8: int) -> int:
    """Exact count of 32-bit uniforms for which the decision flips."""
    return int(lib().orc_accept_count(int(n_anti), int(thr4), int(thr8)))


def met_planes(seed: int, replica: int, sweep: int, colour: int, group: int) -> np.ndarray:
    out = np.zeros(32, dtype=np.uint32)
    lib().orc_met_planes(seed, replica, sweep, colour, group, _ptr(out))
    return out


def assemble_u(planes: np.ndarray, lane: int) -> int:
    P = np.ascontiguousarray(planes, dtype=np.uint32)
    return int(lib().orc_assemble_u(_ptr(P), int(lane)))


def site_uniform(L: int, seed: int, replica: int, sweep: int, x: int, y: int) -> int:
    return int(lib().orc_site_uniform(L, seed, replica, sweep, x, y))


def n_anti(s: np.ndarray, x: int, y: int) -> int:
    s = np.ascontiguousarray(s, dtype=np.int8)
    return int(lib().orc_n_anti(s.shape[0], _ptr(s), x, y))


def n_anti_all(S: np.ndarray) -> np.ndarray:
    """n_anti of every site for a stack of configurations (n, L, L)."""
    S = np.ascontiguousarray(S, dtype=np.int8)
    if S.ndim == 2:
        S = S[None]
    out = np.zeros(S.shape, dtype=np.int32)
    lib().orc_n_anti_all(S.shape[1], S.shape[0], _ptr(S), _ptr(out))
    return out


def energy_mag(s: np.ndarray):
    s = np.ascontiguousarray(s, dtype=np.int8)
    E = ctypes.c_int64()
    M = ctypes.c_int64()
    lib().orc_energy_mag(s.shape[0], _ptr(s), ctypes.byref(E), ctypes.byref(M))
    return int(E.value), int(M.value)


def init(L: int, seed: int, replica: int = 0) -> np.ndarray:
    """Seeded random start, int8 +-1, row-major [y][x]."""
    s = np.zeros((L, L), dtype=np.int8)
    lib().orc_init(L, seed, replica, _ptr(s))
    return s


def half_sweep(s: np.ndarray, beta: float, seed: int, replica: int, sweep: int,
               colour: int) -> None:
    """In-place colour-``colour`` half sweep with the uniforms of ``sweep``."""
    assert s.dtype == np.int8 and s.flags["C_CONTIGUOUS"]
    lib().orc_half_sweep(s.shape[0], threshold(beta, 4), threshold(beta, 8), seed,
                         replica, sweep, colour, _ptr(s))


def sweep(s: np.ndarray, beta: float, seed: int, n_sweeps: int, t0: int = 0,
          replica: int = 0, measure_every: int = 1):
    """Run ``n_sweeps`` sweeps in place; returns the (E, M) records as int64
    arrays (one record after each sweep t with (t+1) % measure_every == 0)."""
    assert s.dtype == np.int8 and s.flags["C_CONTIGUOUS"] and s.shape[0] == s.shape[1]
    L = s.shape[0]
    n_rec = sum(1 for t in range(t0, t0 + n_sweeps) if (t + 1) % measure_every == 0)
    E = np.zeros(max(n_rec, 1), dtype=np.int64)
    M = np.zeros(max(n_rec, 1), dtype=np.int64)
    got = lib().orc_sweep(L, float(beta), seed, replica, t0, n_sweeps, measure_every,
                          _ptr(s), _ptr(E), _ptr(M))
    if got < 0:
        raise ValueError("oracle sweep rejected its arguments")
    assert got == n_rec
    return E[:n_rec], M[:n_rec]


def sweep_omp(s: np.ndarray, beta: float, seed: int, n_sweeps: int, t0: int = 0,
              replica: int = 0, measure_every: int = 1):
    """:func:`sweep` with the rows of each colour spread over OpenMP threads
    (timing build of the same steps; equal to :func:`sweep` bit for bit)."""
    assert s.dtype == np.int8 and s.flags["C_CONTIGUOUS"] and s.shape[0] == s.shape[1]
    L = s.shape[0]
    n_rec = sum(1 for t in range(t0, t0 + n_sweeps) if (t + 1) % measure_every == 0)
    E = np.zeros(max(n_rec, 1), dtype=np.int64)
    M = np.zeros(max(n_rec, 1), dtype=np.int64)
    got = lib().orc_sweep_omp(L, float(beta), seed, replica, t0, n_sweeps, measure_every,
                              _ptr(s), _ptr(E), _ptr(M))
    if got < 0:
        raise ValueError("oracle sweep rejected its arguments")
    assert got == n_rec
    return E[:n_rec], M[:n_rec]


def omp_threads() -> int:
    """Threads the OpenMP timing sweep uses (1 without OpenMP)."""
    return int(lib().orc_omp_threads())


# ---------------------------------------------------------------------------
# Parallel-tempering ladders (replica exchange between adjacent betas)
# ---------------------------------------------------------------------------

def pt_step(betas, seed: int, ladder: int, n_step: int, E, perm, accepts=None, attempts=None):
    """One exchange step of one ladder, in place on perm (and the counters)."""
    b = np.ascontiguousarray(betas, dtype=np.float64)
    Ea = np.ascontiguousarray(E, dtype=np.int64)
    assert perm.dtype == np.int32 and perm.flags["C_CONTIGUOUS"]
    acc = accepts if accepts is not None else np.zeros(len(b), dtype=np.int64)
    att = attempts if attempts is not None else np.zeros(len(b), dtype=np.int64)
    lib().orc_pt_step(len(b), _ptr(b), seed, ladder, n_step, _ptr(Ea), _ptr(perm), _ptr(acc),
                      _ptr(att))


def run_ladders(Ls, betas, seed: int, n_sweeps: int, pt_every: int, ladder_ids=None,
                record=False):
    """Serial reference of the batched run: ladder l has len(betas) replicas of
    size Ls[l] x Ls[l]; replica i of ladder id l has Philox replica id
    l * len(betas) + i and starts from the seeded random start.  Every sweep t
    runs each replica at the beta of its current slot; after sweeps t with
    (t + 1) % pt_every == 0 every ladder does exchange step (t + 1) / pt_every - 1.
    Returns (spins, perm, E, M, accepts, attempts[, series]) with E, M of the last
    sweep; series (record=True) lists (E, M, slot) arrays at every exchange step."""
    nb = len(betas)
    ids = list(ladder_ids) if ladder_ids is not None else list(range(len(Ls)))
    nl = len(Ls)
    spins = [[init(Ls[k], seed, ids[k] * nb + i) for i in range(nb)] for k in range(nl)]
    perm = np.tile(np.arange(nb, dtype=np.int32), (nl, 1))
    acc = np.zeros((nl, nb), dtype=np.int64)
    att = np.zeros((nl, nb), dtype=np.int64)
    E = np.zeros((nl, nb), dtype=np.int64)
    M = np.zeros((nl, nb), dtype=np.int64)
    series = []
    t = 0
    while t < n_sweeps:
        n = min(pt_every - (t % pt_every), n_sweeps - t)
        slots = np.zeros((nl, nb), dtype=np.int32)
        for k in range(nl):
            slot_of = np.empty(nb, dtype=np.int32)
            slot_of[perm[k]] = np.arange(nb, dtype=np.int32)
            slots[k] = slot_of
            for i in range(nb):
                e, m = sweep(spins[k][i], betas[slot_of[i]], seed, n, t0=t,
                             replica=ids[k] * nb + i, measure_every=1)
                E[k, i], M[k, i] = e[-1], m[-1]
        t += n
        if t % pt_every == 0:
            if record:
                series.append((E.copy(), M.copy(), slots.copy()))
            for k in range(nl):
                row = np.ascontiguousarray(perm[k])
                pt_step(betas, seed, ids[k], t // pt_every - 1, E[k], row, acc[k], att[k])
                perm[k] = row
    if record:
        return spins, perm, E, M, acc, att, series
    return spins, perm, E, M, acc, att


# ---------------------------------------------------------------------------
# 2D XY model (the paper's Monte Carlo workload)
# ---------------------------------------------------------------------------

def xy_sincos(x: float, precision: int = 64):
    s, c = (ctypes.c_double(), ctypes.c_double()) if precision == 64 else (ctypes.c_float(), ctypes.c_float())
    f = lib().orc_xy_sincos_d if precision == 64 else lib().orc_xy_sincos_f
    f(x, ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def xy_exp(x: float, precision: int = 64) -> float:
    return (lib().orc_xy_exp_d if precision == 64 else lib().orc_xy_exp_f)(x)


def xy_init(L: int, seed: int, replica: int = 0, precision: int = 64) -> np.ndarray:
    """Seeded random start: unit vectors (cos, sin) as an (L, L, 2) array."""
    dt = np.float64 if precision == 64 else np.float32
    u = np.zeros((L, L, 2), dtype=dt)
    (lib().orc_xy_init_d if precision == 64 else lib().orc_xy_init_f)(L, seed, replica, _ptr(u))
    return u


def xy_observables(u: np.ndarray):
    """(E, Mx, My) in double: E = -sum_x u_x . (u_{x+e1} + u_{x+e2})."""
    E, Mx, My = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    f = lib().orc_xy_observables_d if u.dtype == np.float64 else lib().orc_xy_observables_f
    f(u.shape[0], _ptr(u), ctypes.byref(E), ctypes.byref(Mx), ctypes.byref(My))
    return E.value, Mx.value, My.value


def xy_sweep(u: np.ndarray, beta: float, seed: int, n_sweeps: int, t0: int = 0, replica: int = 0,
             record: bool = True):
    """n_sweeps sweeps in place; returns (accepted per sweep, E per sweep)."""
    L = u.shape[0]
    f = lib().orc_xy_sweep_d if u.dtype == np.float64 else lib().orc_xy_sweep_f
    acc = np.zeros(n_sweeps, dtype=np.int64)
    E = np.zeros(n_sweeps)
    for k in range(n_sweeps):
        acc[k] = f(L, beta, seed, replica, t0 + k, _ptr(u))
        if record:
            E[k] = xy_observables(u)[0]
    return acc, E


# ---------------------------------------------------------------------------
# Swendsen-Wang cluster update
# ---------------------------------------------------------------------------

def sw_threshold(beta: float) -> int:
    return int(lib().orc_sw_threshold(float(beta)))


def sw_steps(s: np.ndarray, beta: float, seed: int, n_steps: int, step0: int = 0,
             replica: int = 0):
    """n Swendsen-Wang steps in place; returns (E, M, clusters) after each step."""
    assert s.dtype == np.int8 and s.flags["C_CONTIGUOUS"]
    L = s.shape[0]
    parent = np.zeros(L * L, dtype=np.uint32)
    E = np.zeros(n_steps, dtype=np.int64)
    M = np.zeros(n_steps, dtype=np.int64)
    C = np.zeros(n_steps, dtype=np.int64)
    for k in range(n_steps):
        C[k] = lib().orc_sw_step(L, float(beta), seed, replica, step0 + k, _ptr(s), _ptr(parent))
        E[k], M[k] = energy_mag(s)
    return E, M, C


def wolff_seed_site(L: int, seed: int, step: int, replica: int = 0) -> int:
    return int(lib().orc_wolff_seed_site(L, seed, replica, step))


def wolff_steps(s: np.ndarray, beta: float, seed: int, n_steps: int, step0: int = 0,
                replica: int = 0):
    """n Wolff steps in place; returns (E, M, cluster size) after each step."""
    assert s.dtype == np.int8 and s.flags["C_CONTIGUOUS"]
    L = s.shape[0]
    stack = np.zeros(L * L, dtype=np.uint32)
    mark = np.zeros(L * L, dtype=np.uint8)
    E = np.zeros(n_steps, dtype=np.int64)
    M = np.zeros(n_steps, dtype=np.int64)
    C = np.zeros(n_steps, dtype=np.int64)
    for k in range(n_steps):
        C[k] = lib().orc_wolff_step(L, float(beta), seed, replica, step0 + k, _ptr(s), _ptr(stack),
                                    _ptr(mark))
        E[k], M[k] = energy_mag(s)
    return E, M, C


# ---------------------------------------------------------------------------
# four-sublattice lattices: square NN (+ NNN) and square-octagon
# ---------------------------------------------------------------------------

QUAD_SQUARE = 0
QUAD_SQOCT = 1


def quad_neighbours(lattice: int, Lc: int, q: int, X: int, Y: int):
    """[(q', X', Y', type)] of site (q, X, Y); type 1 = J1 bond, 2 = J2 bond."""
    out = np.zeros(32, dtype=np.int32)
    n = lib().orc_quad_neighbours(lattice, Lc, q, X, Y, _ptr(out))
    return [tuple(int(v) for v in out[4 * k:4 * k + 4]) for k in range(n)]


def quad_threshold(lattice: int, beta: float, J1: float, J2: float, a1: int, a2: int):
    """(threshold, always) of the class with a1 / a2 antiparallel J1 / J2 neighbours."""
    al = ctypes.c_int()
    t = lib().orc_quad_threshold(lattice, float(beta), float(J1), float(J2), a1, a2,
                                 ctypes.byref(al))
    return int(t), bool(al.value)


def quad_init(Lc: int, seed: int, replica: int = 0) -> np.ndarray:
    """Seeded random start, int8 +-1 as s[q][Y][X]."""
    s = np.zeros((4, Lc, Lc), dtype=np.int8)
    lib().orc_quad_init(Lc, seed, replica, _ptr(s))
    return s


def quad_uniform(Lc: int, seed: int, replica: int, t: int, q: int, X: int, Y: int) -> int:
    return int(lib().orc_quad_uniform(Lc, seed, replica, t, q, X, Y))


def quad_anti(lattice: int, s: np.ndarray, q: int, X: int, Y: int):
    a1, a2 = ctypes.c_int(), ctypes.c_int()
    lib().orc_quad_anti(lattice, s.shape[1], _ptr(s), q, X, Y, ctypes.byref(a1), ctypes.byref(a2))
    return a1.value, a2.value


def quad_observables(lattice: int, s: np.ndarray):
    """(B1, B2, M): J1-bond sum, J2-bond sum of s s', magnetisation."""
    b1, b2, m = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    lib().orc_quad_observables(lattice, s.shape[1], _ptr(s), ctypes.byref(b1), ctypes.byref(b2),
                               ctypes.byref(m))
    return int(b1.value), int(b2.value), int(m.value)


def quad_quarter(lattice: int, s: np.ndarray, beta: float, J1: float, J2: float, seed: int,
                 t: int, q: int, replica: int = 0) -> None:
    lib().orc_quad_quarter(lattice, s.shape[1], float(beta), float(J1), float(J2), seed, replica,
                           t, q, _ptr(s))


def quad_sweep(lattice: int, s: np.ndarray, beta: float, J1: float, J2: float, seed: int,
               n_sweeps: int, t0: int = 0, replica: int = 0, measure_every: int = 1):
    """n sweeps in place (sublattices 0..3); returns (B1, B2, M) records as int64
    arrays.  Energy: E = -J1 B1 - J2 B2."""
    assert s.dtype == np.int8 and s.flags["C_CONTIGUOUS"] and s.shape[0] == 4
    Lc = s.shape[1]
    n_rec = sum(1 for t in range(t0, t0 + n_sweeps) if (t + 1) % measure_every == 0)
    B1 = np.zeros(max(n_rec, 1), dtype=np.int64)
    B2 = np.zeros(max(n_rec, 1), dtype=np.int64)
    M = np.zeros(max(n_rec, 1), dtype=np.int64)
    got = lib().orc_quad_sweep(lattice, Lc, float(beta), float(J1), float(J2), seed, replica, t0,
                               n_sweeps, measure_every, _ptr(s), _ptr(B1), _ptr(B2), _ptr(M))
    if got < 0:
        raise ValueError("bad arguments")
    return B1[:got], B2[:got], M[:got]


def quad_square_image(s: np.ndarray) -> np.ndarray:
    """s[q][Y][X] of the SQUARE lattice as the L x L image, site (2X + i, 2Y + j)."""
    Lc = s.shape[1]
    img = np.zeros((2 * Lc, 2 * Lc), dtype=s.dtype)
    for q in range(4):
        img[(q >> 1)::2, (q & 1)::2] = s[q]
    return img


# ---------------------------------------------------------------------------
# fixed-point XY model (operand-precision study)
# ---------------------------------------------------------------------------

def xyfix_K(F: int) -> int:
    """Number of grid angles k 2^-F in [0, 2 pi)."""
    return int(lib().orc_xyfix_K(F))


def xyfix_trig(F: int, k: int):
    c, s = ctypes.c_int32(), ctypes.c_int32()
    lib().orc_xyfix_trig(F, k, ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


def xyfix_accept(F: int, beta: float, e: int, qp: bool = False) -> int:
    """Threshold for dE = e 2^-F; qp: the probability truncated to F bits first."""
    return int(lib().orc_xyfix_accept(F, float(beta), int(e), int(bool(qp))))


def xyfix_dE(F: int, k: int, k2: int, hx: int, hy: int) -> int:
    return int(lib().orc_xyfix_dE(F, k, k2, hx, hy))


def xyfix_init(L: int, F: int, seed: int, replica: int = 0) -> np.ndarray:
    """Seeded random start: angle indices k as an (L, L) int32 array."""
    k = np.zeros((L, L), dtype=np.int32)
    lib().orc_xyfix_init(L, F, seed, replica, _ptr(k))
    return k


def xyfix_observables(k: np.ndarray, F: int):
    """(E2, Mx, My) integers: energy = -E2 2^-2F, magnetisation (Mx, My) 2^-F."""
    e, mx, my = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    lib().orc_xyfix_observables(k.shape[0], F, _ptr(k), ctypes.byref(e), ctypes.byref(mx),
                                ctypes.byref(my))
    return int(e.value), int(mx.value), int(my.value)


def xyfix_sweep(k: np.ndarray, F: int, beta: float, seed: int, n_sweeps: int, t0: int = 0,
                replica: int = 0, record: bool = True, qp: bool = False):
    """n sweeps in place; returns (accepted per sweep, E2 per sweep).  qp: the
    acceptance probability is truncated to F fractional bits."""
    assert k.dtype == np.int32 and k.flags["C_CONTIGUOUS"]
    L = k.shape[0]
    acc = np.zeros(n_sweeps, dtype=np.int64)
    E2 = np.zeros(n_sweeps, dtype=np.int64)
    for i in range(n_sweeps):
        acc[i] = lib().orc_xyfix_sweep(L, F, int(bool(qp)), float(beta), seed, replica, t0 + i, _ptr(k))
        if record:
            E2[i] = xyfix_observables(k, F)[0]
    return acc, E2
