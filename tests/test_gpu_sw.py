"""Swendsen-Wang cluster step on the GPU against the CPU oracle.

The cluster step is fixed by (seed, step, replica, spins): the bonds and the
cluster flips come from the counter-based generator and each cluster is keyed
by its smallest site, so the GPU's lock-free union-find must give the oracle's
configuration bit for bit, whatever order its threads link in.
"""
import numpy as np
import pytest

import oracle
import paper_2402_06415_gb300 as ising

pytestmark = pytest.mark.gpu

BETA_C = 0.5 * np.log(1.0 + np.sqrt(2.0))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()
    ising.lib()


@pytest.mark.parametrize("mode", [ising.ISING_CLUSTER_KERNELS, ising.ISING_CLUSTER_PERSISTENT])
@pytest.mark.parametrize("L", [4, 6, 62, 64, 128, 130, 256, 384])
@pytest.mark.parametrize("beta", [1e-9, 0.3, BETA_C, 0.7, 50.0])
def test_sw_bit_exact(L, beta, mode):
    seed, n = 0xBEEF0000 + L, 6
    s = oracle.init(L, seed)
    with ising.Lattice(L, beta, seed=seed) as lat:
        lat.set_spins(s)
        lat.cluster_set_mode(mode)
        lat.sw_step(n, 1)
        got = lat.spins()
        E, M = lat.series(n)
    E_ref, M_ref, _ = oracle.sw_steps(s, beta, seed, n)
    assert np.array_equal(got, s)
    assert np.array_equal(E, E_ref) and np.array_equal(M, M_ref)


def test_sw_after_metropolis_and_replica():
    """Metropolis sweeps then cluster steps (separate counters), replica 3."""
    L, beta, seed = 96, BETA_C, 77
    s = oracle.init(L, seed, replica=3)
    with ising.Lattice(L, beta, seed=seed, replica=3) as lat:
        lat.set_spins(s)
        lat.sweep(4)
        lat.sw_step(5)
        lat.sweep(2)
        lat.sw_step(1)
        got = lat.spins()
    oracle.sweep(s, beta, seed, 4, replica=3)
    oracle.sw_steps(s, beta, seed, 5, replica=3)
    oracle.sweep(s, beta, seed, 2, t0=4, replica=3)
    oracle.sw_steps(s, beta, seed, 1, step0=5, replica=3)
    assert np.array_equal(got, s)


@pytest.mark.parametrize("L", [10, 96, 1000])
def test_sw_persistent_sparse_records_and_resume(L):
    """Persistent and kernel calls in turn on one step counter; records every
    fourth step, starting mid-run."""
    beta, seed = BETA_C, 70 + L
    s = oracle.init(L, seed)
    with ising.Lattice(L, beta, seed=seed) as lat:
        for mode, n in [(ising.ISING_CLUSTER_PERSISTENT, 5), (ising.ISING_CLUSTER_KERNELS, 2),
                        (ising.ISING_CLUSTER_PERSISTENT, 11)]:
            lat.cluster_set_mode(mode)
            lat.sw_step(n, 4)
        got = lat.spins()
        E, M = lat.series(18 // 4)
    E_ref, M_ref, _ = oracle.sw_steps(s, beta, seed, 18)
    assert np.array_equal(got, s)
    idx = [t for t in range(18) if (t + 1) % 4 == 0]
    assert np.array_equal(E, E_ref[idx]) and np.array_equal(M, M_ref[idx])


@pytest.mark.parametrize("L,beta", [(2048, BETA_C), (2560, 0.3), (2048, 0.7)])
def test_sw_tiled_labelling_bit_exact(L, beta):
    """Lattices of >= 2048 sites a side that are multiples of the 128 x 64 tile
    take the shared-memory labelling path."""
    seed = 40 + L
    s = oracle.init(L, seed)
    with ising.Lattice(L, beta, seed=seed) as lat:
        lat.set_spins(s)
        lat.sw_step(2, 1)
        got = lat.spins()
        E, M = lat.series(2)
    E_ref, M_ref, _ = oracle.sw_steps(s, beta, seed, 2)
    assert np.array_equal(got, s)
    assert np.array_equal(E, E_ref) and np.array_equal(M, M_ref)


@pytest.mark.parametrize("pattern", ["stripes", "stripes_noise"])
def test_sw_tiled_union_list_overflow(pattern):
    """Vertical stripes at large beta: every vertical bond is active and no
    horizontal one, so each tile has ~8000 vertical bonds that need a union, more
    than its union list holds; the tile kernel then unites by a scan.  One step
    (the stripes themselves) and a few more from the noisier start."""
    L, beta, seed = 2048, 50.0, 77
    s = np.empty((L, L), dtype=np.int8)
    s[:, 0::2] = 1
    s[:, 1::2] = -1
    n = 1
    if pattern == "stripes_noise":
        flip = np.random.default_rng(78).random((L, L)) < 0.02
        s[flip] *= -1
        n = 3
    with ising.Lattice(L, beta, seed=seed) as lat:
        lat.set_spins(s)
        lat.sw_step(n, 1)
        got = lat.spins()
        E, M = lat.series(n)
    E_ref, M_ref, _ = oracle.sw_steps(s, beta, seed, n)
    assert np.array_equal(got, s)
    assert np.array_equal(E, E_ref) and np.array_equal(M, M_ref)


def test_sw_large_lattice_one_step():
    """A 4096^2 lattice (16.8 M sites, clusters spanning many CTAs) at beta_c."""
    L, seed = 4096, 5
    s = oracle.init(L, seed)
    with ising.Lattice(L, BETA_C, seed=seed) as lat:
        lat.set_spins(s)
        lat.sw_step(2)
        got = lat.spins()
    oracle.sw_steps(s, BETA_C, seed, 2)
    assert np.array_equal(got, s)


def test_sw_step_counter_resets_on_seed():
    L, beta, seed = 64, 0.44, 21
    with ising.Lattice(L, beta, seed=seed) as lat:
        lat.sw_step(3)
        lat.seed(seed)            # back to the seeded start, step counter 0
        s = lat.spins()
        lat.sw_step(2)
        got = lat.spins()
    oracle.sw_steps(s, beta, seed, 2)
    assert np.array_equal(got, s)


def test_sw_rejects_byte_layout():
    with ising.Lattice(8, 0.4, layout=ising.ISING_LAYOUT_I8) as lat:
        with pytest.raises(ising.IsingError):
            lat.sw_step(1)
