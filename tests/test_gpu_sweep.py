"""Parity of the CUDA sweep (through the C-ABI) with the CPU oracle.

Bit-exact: spins after n sweeps and the full E/M record series, for every
kernel (half-sweep, shared-memory tiled with k sweeps per launch, resident
int8, global int8), both layouts, ragged word tails (L/2 not a multiple of 32),
several betas and seeds, and the full-size L = 16384 lattice on its first five
sweeps.
"""
import numpy as np
import pytest

import oracle
import paper_2402_06415_gb300 as ising

pytestmark = pytest.mark.gpu

BETA_C = 0.4406868
BITS, I8 = ising.ISING_LAYOUT_BITS, ising.ISING_LAYOUT_I8
HALF, TILED, RES = ising.ISING_KERNEL_HALF, ising.ISING_KERNEL_TILED, ising.ISING_KERNEL_RESIDENT


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ising.lib()


def _oracle_run(L, beta, seed, n, replica=0, measure_every=1):
    s = oracle.init(L, seed, replica)
    E, M = oracle.sweep(s, beta, seed, n, replica=replica, measure_every=measure_every)
    return s, E, M


def _gpu_run(L, beta, seed, n, layout, kernel=None, kargs=(), replica=0, measure_every=1):
    with ising.Lattice(L, beta, layout) as lat:
        if replica:
            ising.ising_set_replica(lat.ctx, replica)
        if kernel is not None:
            lat.set_kernel(kernel, *kargs)
        lat.seed(seed)
        lat.sweep(n, measure_every)
        E, M = lat.series()
        return lat.spins(), E, M


@pytest.mark.parametrize("L", [4, 6, 8, 16, 30, 64, 66, 100, 128, 130, 256])
@pytest.mark.parametrize("layout", [BITS, I8])
def test_random_start_bit_exact(L, layout):
    with ising.Lattice(L, 0.4, layout, seed=123) as lat:
        got = lat.spins()
        E, M = lat.measure()
    ref = oracle.init(L, 123)
    assert np.array_equal(got, ref)
    assert (E, M) == oracle.energy_mag(ref)


CASES = [
    # (layout, kernel, kernel args, L)
    (BITS, HALF, (), 4),
    (BITS, HALF, (), 6),
    (BITS, HALF, (), 16),
    (BITS, HALF, (), 30),
    (BITS, HALF, (), 64),
    (BITS, HALF, (), 66),
    (BITS, HALF, (), 100),
    (BITS, HALF, (), 130),
    (BITS, HALF, (), 512),
    (BITS, TILED, (1, 4, 4), 256),
    (BITS, TILED, (2, 4, 4), 256),
    (BITS, TILED, (3, 3, 4), 256),
    (BITS, TILED, (4, 2, 4), 512),
    (BITS, TILED, (8, 7, 8), 512),
    (BITS, TILED, (2, 16, 16), 1024),
    (BITS, TILED, (5, 5, 4), 1024),
    (BITS, TILED, (1, 19, 32), 2048),
    (BITS, TILED, (2, 7, 32), 2048),
    (BITS, TILED, (3, 20, 32), 2048),
    (BITS, TILED, (8, 9, 32), 2048),
    (I8, RES, (), 4),
    (I8, RES, (), 10),
    (I8, RES, (), 64),
    (I8, RES, (), 66),
    (I8, RES, (), 128),
    (I8, HALF, (), 8),
    (I8, HALF, (), 66),
    (I8, HALF, (), 512),
]


@pytest.mark.parametrize("layout,kernel,kargs,L", CASES)
@pytest.mark.parametrize("beta", [0.3, BETA_C, 0.6])
def test_sweeps_bit_exact(layout, kernel, kargs, L, beta):
    n = 9
    seed = 1000 + L
    ref, E_ref, M_ref = _oracle_run(L, beta, seed, n)
    got, E, M = _gpu_run(L, beta, seed, n, layout, kernel, kargs)
    assert np.array_equal(got, ref)
    assert np.array_equal(E, E_ref) and np.array_equal(M, M_ref)


@pytest.mark.parametrize("kargs", [(2, 37, 64), (1, 152, 32), (4, 64, 32), (2, 16, 64), (4, 19, 32)])
def test_tiled32_L4096(kargs):
    """Warp-per-row tiled kernel with its compaction queue, 64- and 32-word tiles;
    (2, 16, 64) (256-row strips, ~1700 undecided words per half sweep against 1536
    entries) overflows the queue, so the in-place path runs too.  Tiles too tall for
    three CTAs' shared memory per SM ((2, 37, 64), (2, 16, 64), and (4, 19, 32):
    216-row strips of 32 words, K = 4) run the variant compiled for two CTAs per
    SM with the larger register budget; the others the three-CTA variant."""
    L, beta, seed, n = 4096, BETA_C, 31, 7
    ref, E_ref, M_ref = _oracle_run(L, beta, seed, n)
    got, E, M = _gpu_run(L, beta, seed, n, BITS, TILED, kargs)
    assert np.array_equal(got, ref)
    assert np.array_equal(E, E_ref) and np.array_equal(M, M_ref)


@pytest.mark.parametrize("layout", [BITS, I8])
def test_cfg_L64_long_chain_bit_exact(layout):
    """The L = 64 workload: 2000 sweeps with a record every sweep."""
    L, n = 64, 2000
    for beta, seed in [(0.30, 1), (BETA_C, 2), (0.60, 3)]:
        ref, E_ref, M_ref = _oracle_run(L, beta, seed, n)
        got, E, M = _gpu_run(L, beta, seed, n, layout)
        assert np.array_equal(got, ref)
        assert np.array_equal(E, E_ref) and np.array_equal(M, M_ref)


def test_replica_id_and_measure_every():
    L, beta, seed = 128, 0.45, 5
    ref, E_ref, M_ref = _oracle_run(L, beta, seed, 12, replica=3, measure_every=4)
    for layout, kernel, kargs in [(BITS, HALF, ()), (BITS, None, ()), (I8, RES, ()), (I8, HALF, ())]:
        got, E, M = _gpu_run(L, beta, seed, 12, layout, kernel, kargs, replica=3, measure_every=4)
        assert np.array_equal(got, ref)
        assert np.array_equal(E, E_ref) and np.array_equal(M, M_ref)


def test_tiled32_queue_overflow_ordered_start():
    """An ordered start at beta = 0.6: every site is tested against T8 and stays
    so (few flips), and a tested site is still undecided after 8 planes with
    probability 2^-8, so ~12 % of words (1 - (255/256)^32) are queued, ~2000 per
    half sweep of a 256 x 66-word tile at L = 4096 against a queue of 1536: the
    in-place finishing path runs in every half sweep."""
    L, beta, seed, n = 4096, 0.6, 5, 3
    start = np.ones((L, L), dtype=np.int8)
    ref = start.copy()
    E_ref, M_ref = oracle.sweep(ref, beta, seed, n)
    with ising.Lattice(L, beta, BITS) as lat:
        lat.set_kernel(TILED, 2, 16, 64)
        lat.set_spins(start)
        ising.ising_set_key(lat.ctx, seed)
        lat.sweep(n, 1)
        got = lat.spins()
        E, M = lat.series()
    assert np.array_equal(got, ref)
    assert np.array_equal(E, E_ref) and np.array_equal(M, M_ref)


@pytest.mark.parametrize("layout,kernel,kargs,L", [(BITS, TILED, (4, 4, 4), 256),
                                                   (BITS, HALF, (), 66), (I8, RES, (), 66)])
def test_resume_matches_single_run(layout, kernel, kargs, L):
    beta, seed = BETA_C, 77
    full, E_full, M_full = _gpu_run(L, beta, seed, 13, layout, kernel, kargs)
    with ising.Lattice(L, beta, layout) as lat:
        lat.set_kernel(kernel, *kargs)
        lat.seed(seed)
        lat.sweep(5, 1)
        saved = lat.spins()
    with ising.Lattice(L, beta, layout) as lat:
        lat.set_kernel(kernel, *kargs)
        lat.set_spins(saved)
        ising.ising_set_key(lat.ctx, seed)
        ising.ising_set_sweep_counter(lat.ctx, 5)
        lat.sweep(8, 1)
        got = lat.spins()
        E, M = lat.series()
    assert np.array_equal(got, full)
    assert np.array_equal(E, E_full[5:]) and np.array_equal(M, M_full[5:])


def test_layouts_agree_and_roundtrip():
    L, beta, seed = 130, 0.44, 9
    a, Ea, Ma = _gpu_run(L, beta, seed, 20, BITS, HALF)
    b, Eb, Mb = _gpu_run(L, beta, seed, 20, I8, RES)
    assert np.array_equal(a, b) and np.array_equal(Ea, Eb) and np.array_equal(Ma, Mb)
    rng = np.random.default_rng(1)
    s = np.where(rng.random((L, L)) < 0.5, 1, -1).astype(np.int8)
    for layout in (BITS, I8):
        with ising.Lattice(L, beta, layout) as lat:
            lat.set_spins(s)
            assert np.array_equal(lat.spins(), s)
            w = lat.bits()
            assert lat.measure() == oracle.energy_mag(s)
        with ising.Lattice(L, beta, 1 - layout) as lat2:
            lat2.set_bits(w)
            assert np.array_equal(lat2.spins(), s)


def test_device_buffers_roundtrip():
    import torch

    L = 256
    with ising.Lattice(L, 0.5, BITS, seed=3) as lat:
        d = torch.empty((L, L), dtype=torch.int8, device="cuda")
        ising.ising_get_spins_device(lat.ctx, d)
        torch.cuda.synchronize()
        host = lat.spins()
        assert np.array_equal(d.cpu().numpy(), host)
        words = torch.empty((2, L, ising.ising_words_per_row(L)), dtype=torch.int32, device="cuda")
        ising.ising_get_bits_device(lat.ctx, words)
        torch.cuda.synchronize()
        assert np.array_equal(words.cpu().numpy().view(np.uint32), lat.bits())
        flipped = -d
        ising.ising_set_spins_device(lat.ctx, flipped)
        torch.cuda.synchronize()
        assert np.array_equal(lat.spins(), -host)


def test_stream_is_borrowed():
    import torch

    s = torch.cuda.Stream()
    L, beta, seed = 256, BETA_C, 4
    ref, E_ref, M_ref = _oracle_run(L, beta, seed, 6)
    with ising.Lattice(L, beta, BITS, stream=s, seed=seed) as lat:
        lat.sweep(6, 1)
        assert np.array_equal(lat.spins(), ref)
        E, M = lat.series()
        assert np.array_equal(E, E_ref)


def test_set_spins_validates():
    with ising.Lattice(8, 0.4, BITS) as lat:
        bad = np.ones((8, 8), dtype=np.int8)
        bad[3, 3] = 0
        with pytest.raises(ising.IsingError) as e:
            lat.set_spins(bad)
        assert e.value.status == ising.ISING_EINVAL


def test_kernel_config_validation():
    with ising.Lattice(130, 0.4, BITS) as lat:
        with pytest.raises(ising.IsingError):
            lat.set_kernel(TILED, 2, 2, 4)  # L % 256 != 0
        with pytest.raises(ising.IsingError):
            lat.set_kernel(RES)
    with ising.Lattice(512, 0.4, BITS) as lat:
        with pytest.raises(ising.IsingError):
            lat.set_kernel(TILED, 9, 4, 4)
        with pytest.raises(ising.IsingError):
            lat.set_kernel(TILED, 2, 4, 6)
        lat.set_kernel(TILED, 3, 5, 8)
        assert lat.kernel()["sweeps_per_launch"] == 3


def test_injected_failures_leave_no_leak(monkeypatch):
    import torch

    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("ISING_FAULT", "alloc")
    with pytest.raises(ising.IsingError) as e:
        ising.ising_create(1024, 0.4, BITS)
    assert e.value.status == ising.ISING_ENOMEM
    monkeypatch.setenv("ISING_FAULT", "launch")
    with ising.Lattice(256, 0.4, BITS) as lat:
        with pytest.raises(ising.IsingError) as e:
            lat.sweep(3, 1)
        assert e.value.status == ising.ISING_ECUDA
    monkeypatch.setenv("ISING_FAULT", "copy")
    with ising.Lattice(256, 0.4, BITS) as lat:
        with pytest.raises(ising.IsingError):
            lat.spins()
    monkeypatch.delenv("ISING_FAULT")
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < 8 << 20


def test_full_size_L16384_first_sweeps():
    """The L = 16384 workload (packed, the bench's kernel) on its first five
    sweeps at beta_c: spins and E/M records bit-exact against the oracle."""
    L, beta, seed, n = 16384, BETA_C, 1, 5
    ref, E_ref, M_ref = _oracle_run(L, beta, seed, n)
    import bench

    with ising.Lattice(L, beta, BITS) as lat:
        bench.configure_kernel(lat)
        lat.seed(seed)
        lat.sweep(n, 1)
        E, M = lat.series()
        got = lat.spins()
    assert np.array_equal(E, E_ref) and np.array_equal(M, M_ref)
    assert np.array_equal(got, ref)


def test_bounded_wait_times_out_and_context_survives():
    """A device wait on a flag nothing sets gives up after its budget and
    reports ETIMEOUT; the context keeps working afterwards."""
    import time

    t0 = time.perf_counter()
    with pytest.raises(ising.IsingError) as e:
        ising.ising_selftest_wait(0.2)
    dt = time.perf_counter() - t0
    assert e.value.status == ising.ISING_ETIMEOUT
    assert 0.05 < dt < 5.0
    ref, E_ref, _ = _oracle_run(64, BETA_C, 3, 4)
    got, E, _ = _gpu_run(64, BETA_C, 3, 4, BITS, HALF)
    assert np.array_equal(got, ref) and np.array_equal(E, E_ref)
