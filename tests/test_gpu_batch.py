"""Batched replicas with parallel tempering on the GPU against the oracle.

Per replica bit-exact spins, E and M; identical slot permutations and exchange
counts; independent of the work decomposition; CUDA-graph replay continues
the chain; recorded series match the oracle's exchange-step records.
"""
import numpy as np
import pytest

import oracle
import paper_2402_06415_gb300 as ising
from paper_2402_06415_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ising.lib()


def _compare(b, ref, Ls, ladder_rows=None):
    spins, perm, E, M, acc, att = ref[:6]
    p, Eg, Mg = b.state()
    ag, tg = b.swap_counts()
    rows = ladder_rows if ladder_rows is not None else range(len(Ls))
    for k, l in enumerate(rows):
        assert np.array_equal(p[l], perm[k]), l
        assert np.array_equal(Eg[l], E[k]) and np.array_equal(Mg[l], M[k]), l
        assert np.array_equal(ag[l][:-1], acc[k][:-1]) and np.array_equal(tg[l][:-1], att[k][:-1])
        for i in range(len(b.betas)):
            assert np.array_equal(b.spins(l, i), spins[k][i]), (l, i)


SMALL_LS = [16, 24, 6, 32, 66]
SMALL_BETAS = np.linspace(0.35, 0.5, 8)


@pytest.mark.parametrize("kernel", [(512, 256), (16, 128), (4096, 256), (64, 256), (64, 32), (256, 64)])
def test_batch_bit_exact_small(kernel):
    seed, n, pt = 11, 23, 5
    ref = oracle.run_ladders(SMALL_LS, SMALL_BETAS, seed, n, pt)
    with ising.Batch(SMALL_LS, SMALL_BETAS, pt) as b:
        ising.ising_batch_set_kernel(b.h, *kernel)
        ising.ising_batch_seed(b.h, seed)
        b.run(n)
        assert ising.ising_batch_status(b.h) == (0, n)
        _compare(b, ref, SMALL_LS)


def test_batch_runs_in_pieces_and_graph_replay():
    seed, pt = 12, 4
    ref = oracle.run_ladders(SMALL_LS, SMALL_BETAS, seed, 36, pt)
    with ising.Batch(SMALL_LS, SMALL_BETAS, pt, seed=seed) as b:
        b.run(3)
        b.run(9)  # crosses exchange steps mid-call
        ising.ising_batch_capture(b.h, 8)
        for _ in range(3):
            b.run(8)  # graph replay: the device sweep counter advances
        assert ising.ising_batch_status(b.h) == (0, 36)
        _compare(b, ref, SMALL_LS)


def test_batch_series_matches_oracle_records():
    seed, pt, n = 13, 3, 15
    ref = oracle.run_ladders(SMALL_LS, SMALL_BETAS, seed, n, pt, record=True)
    series = ref[6]
    with ising.Batch(SMALL_LS, SMALL_BETAS, pt) as b:
        ising.ising_batch_set_series(b.h, 16)
        ising.ising_batch_seed(b.h, seed)
        b.run(n)
        E, M, S = ising.ising_batch_series(b.h, len(series), b.n_rep)
    for k, (Er, Mr, Sr) in enumerate(series):
        assert np.array_equal(E[k], Er.ravel()) and np.array_equal(M[k], Mr.ravel())
        assert np.array_equal(S[k], Sr.ravel())


def test_batch_workload_sample_ladders():
    """The 64 x 64 ladder workload (sizes 16..128), 20 sweeps with exchanges
    every 10; three ladders checked against the oracle."""
    Ls = workloads.batch_ladder_sizes()
    betas = workloads.batch_betas()
    seed, n, pt = 3, 20, workloads.BATCH_PT_EVERY
    pick = [0, Ls.index(128), Ls.index(24)]
    ref = oracle.run_ladders([Ls[l] for l in pick], betas, seed, n, pt, ladder_ids=pick)
    with ising.Batch(Ls, betas, pt, seed=seed) as b:
        b.run(n)
        assert ising.ising_batch_status(b.h)[0] == 0
        _compare(b, ref, [Ls[l] for l in pick], ladder_rows=pick)


def test_batch_argument_checks():
    with pytest.raises(ising.IsingError):
        ising.Batch([16, 5], SMALL_BETAS, 5)
    with pytest.raises(ising.IsingError):
        ising.Batch([16], SMALL_BETAS[::-1], 5)
    with pytest.raises(ising.IsingError):
        ising.Batch([16], SMALL_BETAS, 0)
