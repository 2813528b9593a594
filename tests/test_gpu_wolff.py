"""Wolff single-cluster step on the GPU against the CPU oracle.

A step is fixed by (seed, step, replica, spins): the seed site and the bonds
come from the counter-based generator and the flipped cluster is the seed's
connected component, so both ways the GPU finds it (bounded growth from the
seed in one CTA, or connected components of the whole lattice) must give the
oracle's configuration bit for bit, and the same cluster size.  The limits
parametrise which way runs: growth only, labelling only, and a mix in which
growth gives up part way; each also as one CUDA graph per step (growth sets
the condition of an IF node that holds the labelling kernels).
"""
import numpy as np
import pytest

import oracle
import paper_2402_06415_gb300 as ising

pytestmark = pytest.mark.gpu

BETA_C = 0.5 * np.log(1.0 + np.sqrt(2.0))

KERNELS, PERSISTENT = ising.ISING_CLUSTER_KERNELS, ising.ISING_CLUSTER_PERSISTENT
GRAPH = ising.ISING_CLUSTER_GRAPH
# (mode, (max_sites, max_levels)): the persistent kernel; the kernel path with the
# default bounds, never growing, growing with generous bounds, tiny bounds; the
# graph path with the default bounds, never growing, tiny bounds
LIMITS = {"persistent": (PERSISTENT, None), "default": (KERNELS, None), "label": (KERNELS, (0, 0)),
          "grow": (KERNELS, (16384, 100000)), "tiny": (KERNELS, (64, 3)),
          "graph": (GRAPH, None), "graph_label": (GRAPH, (0, 0)), "graph_tiny": (GRAPH, (64, 3))}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()
    ising.lib()


def _run(L, beta, seed, n, limits, replica=0):
    s = oracle.init(L, seed, replica=replica)
    sizes = []
    with ising.Lattice(L, beta, seed=seed, replica=replica) as lat:
        lat.set_spins(s)
        mode, lim = LIMITS[limits]
        lat.cluster_set_mode(mode)
        if lim is not None:
            lat.wolff_set_limits(*lim)
        for _ in range(n):
            lat.wolff_step(1, 1)
            sizes.append(lat.wolff_stats()["last_size"])
        got = lat.spins()
        E, M = lat.series(n)
        st = lat.wolff_stats()
    E_ref, M_ref, C_ref = oracle.wolff_steps(s, beta, seed, n, replica=replica)
    assert np.array_equal(got, s)
    assert np.array_equal(E, E_ref) and np.array_equal(M, M_ref)
    assert sizes == list(C_ref)
    assert st["grown"] + st["labelled"] == n
    assert st["flipped"] == int(C_ref.sum())
    return st


@pytest.mark.parametrize("limits", list(LIMITS))
@pytest.mark.parametrize("L", [4, 6, 62, 64, 130, 256])
@pytest.mark.parametrize("beta", [1e-9, 0.3, BETA_C, 0.7, 50.0])
def test_wolff_bit_exact(L, beta, limits):
    st = _run(L, beta, 0xF00D0000 + L, 8, limits, replica=1)
    if limits in ("label", "persistent", "graph_label"):
        assert st["grown"] == 0
    if limits == "grow" and L * L <= 16384 // 4:
        assert st["labelled"] == 0


@pytest.mark.parametrize("limits", ["default", "label", "tiny", "persistent", "graph", "graph_tiny"])
@pytest.mark.parametrize("L,beta", [(2048, BETA_C), (2560, 0.3), (2048, 0.7)])
def test_wolff_tiled_labelling_bit_exact(L, beta, limits):
    """Lattices of >= 2048 sites a side that are multiples of the 128 x 64 tile
    label through the shared-memory tiles."""
    _run(L, beta, 60 + L, 4, limits)


@pytest.mark.parametrize("limits", ["default", "graph"])
def test_wolff_growth_used_away_from_criticality(limits):
    """At beta = 0.3 clusters are small: on the kernel and graph paths every
    step finishes by growth."""
    st = _run(1024, 0.3, 9, 40, limits)
    assert st["labelled"] == 0 and st["grown"] == 40


@pytest.mark.parametrize("L,beta", [(1024, 0.3), (2048, BETA_C)])
def test_wolff_graph_unrolled_steps(L, beta):
    """Without records the graph path runs eight steps per launch (here 2 x 8
    plus a remainder of 3): the same chain as the oracle's, bit for bit."""
    seed, n = 41, 19
    s = oracle.init(L, seed)
    with ising.Lattice(L, beta, seed=seed) as lat:
        lat.set_spins(s)
        lat.cluster_set_mode(GRAPH)
        lat.wolff_step(n, 0)
        got = lat.spins()
        st = lat.wolff_stats()
    _, _, C_ref = oracle.wolff_steps(s, beta, seed, n)
    assert np.array_equal(got, s)
    assert st["grown"] + st["labelled"] == n and st["flipped"] == int(C_ref.sum())


def test_wolff_graph_rebuilt_when_arguments_change():
    """Graph steps, sweeps (which move the lattice to the other buffer), a new
    beta and new limits in between: the graph follows, and the step counter it
    keeps on the device continues the host's, bit for bit."""
    L, seed = 1024, 77
    s = oracle.init(L, seed)
    with ising.Lattice(L, 0.3, seed=seed) as lat:
        lat.set_spins(s)
        lat.cluster_set_mode(GRAPH)
        lat.wolff_step(3)
        lat.sweep(3)
        lat.wolff_step(2)
        ising.ising_set_beta(lat.ctx, BETA_C)
        lat.wolff_step(2)
        lat.wolff_set_limits(64, 3)
        lat.wolff_step(2)
        got = lat.spins()
        st = lat.wolff_stats()
    t = s.copy()
    oracle.wolff_steps(t, 0.3, seed, 3)
    oracle.sweep(t, 0.3, seed, 3)
    oracle.wolff_steps(t, 0.3, seed, 2, step0=3)
    oracle.wolff_steps(t, BETA_C, seed, 2, step0=5)
    oracle.wolff_steps(t, BETA_C, seed, 2, step0=7)
    assert np.array_equal(got, t)
    assert st["grown"] + st["labelled"] == 9


def test_wolff_counter_and_seed_reset():
    L, beta, seed = 96, BETA_C, 5
    s = oracle.init(L, seed)
    with ising.Lattice(L, beta, seed=seed) as lat:
        lat.wolff_step(3)
        lat.sweep(2)
        lat.wolff_step(2)
        got = lat.spins()
        lat.seed(seed)  # back to the start: fresh spins and step counter
        assert lat.wolff_stats()["flipped"] == 0
        lat.wolff_step(3)
        again = lat.spins()
    t = s.copy()
    oracle.wolff_steps(t, beta, seed, 3)
    ref3 = t.copy()
    oracle.sweep(t, beta, seed, 2)
    oracle.wolff_steps(t, beta, seed, 2, step0=3)
    assert np.array_equal(got, t)
    assert np.array_equal(again, ref3)


@pytest.mark.parametrize("L", [6, 64, 200])
def test_wolff_paths_interleaved_and_sparse_records(L):
    """Persistent and kernel steps in turn (one step counter), records every
    third step starting mid-run: the series holds the oracle's E, M at steps
    t with (t + 1) % 3 == 0."""
    beta, seed = BETA_C, 31 + L
    s = oracle.init(L, seed)
    with ising.Lattice(L, beta, seed=seed) as lat:
        for k, (mode, n) in enumerate([(PERSISTENT, 4), (KERNELS, 3), (GRAPH, 2), (PERSISTENT, 5),
                                       (KERNELS, 1), (GRAPH, 2), (PERSISTENT, 3)]):
            lat.cluster_set_mode(mode)
            lat.wolff_step(n, 3)
        got = lat.spins()
        E, M = lat.series(20 // 3)
    E_ref, M_ref, _ = oracle.wolff_steps(s, beta, seed, 20)
    assert np.array_equal(got, s)
    idx = [t for t in range(20) if (t + 1) % 3 == 0]
    assert np.array_equal(E, E_ref[idx]) and np.array_equal(M, M_ref[idx])


def test_wolff_large_lattice_steps():
    """A 4096^2 lattice (16.8 M sites) at beta_c: eight steps bit for bit."""
    L, seed, n = 4096, 8, 8
    s = oracle.init(L, seed)
    with ising.Lattice(L, BETA_C, seed=seed) as lat:
        lat.wolff_step(n, 1)
        got = lat.spins()
        E, M = lat.series(n)
    E_ref, M_ref, _ = oracle.wolff_steps(s, BETA_C, seed, n)
    assert np.array_equal(got, s)
    assert np.array_equal(E, E_ref) and np.array_equal(M, M_ref)


def test_wolff_rejects_bad_arguments():
    with ising.Lattice(16, 0.4) as lat:
        with pytest.raises(ising.IsingError):
            lat.wolff_set_limits(16385)
        with pytest.raises(ising.IsingError):
            lat.wolff_set_limits(-1)
        with pytest.raises(ising.IsingError):
            lat.wolff_step(-1)
        with pytest.raises(ising.IsingError):
            lat.cluster_set_mode(4)
    with ising.Lattice(16, 0.4, ising.ISING_LAYOUT_I8) as lat:
        with pytest.raises(ising.IsingError):
            lat.wolff_step(1)
