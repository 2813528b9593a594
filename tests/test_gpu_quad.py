"""Four-sublattice Ising sweeps (square NN + NNN, square-octagon) on the GPU
against the CPU oracle: spins and the (B1, B2, M) series bit-exact; at the
benchmark size (8192^2 cells, 2.7e8 sites) sampled sites of one sweep are
recomputed one by one from the states before and after it."""
import numpy as np
import pytest

import oracle
import paper_2402_06415_gb300 as ising

pytestmark = pytest.mark.gpu

SQ, OCT = ising.ISING_QUAD_SQUARE, ising.ISING_QUAD_SQOCT


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()
    ising.lib()


CASES = [(SQ, 1.0, 0.0), (SQ, 1.0, 0.5), (SQ, 1.0, -0.5), (SQ, 0.75, 1.25), (SQ, 1.0, 0.3141592653589793),
         (OCT, 1.0, 1.0), (OCT, 1.0, 0.5), (OCT, -1.0, 1.0)]


@pytest.mark.parametrize("lattice,J1,J2", CASES)
@pytest.mark.parametrize("Lc", [2, 3, 5, 32, 33, 70, 128, 256, 300])
@pytest.mark.parametrize("beta", [0.2, 0.4406868, 0.9])
def test_quad_bit_exact(lattice, J1, J2, Lc, beta):
    seed, n = 0xC0FFEE00 + Lc, 5
    s = oracle.quad_init(Lc, seed)
    with ising.Quad(lattice, Lc, beta, J1, J2, seed=seed) as x:
        assert np.array_equal(x.spins(), s)
        x.sweep(n, 1)
        got = x.spins()
        B1, B2, M = x.series(n)
    R1, R2, RM = oracle.quad_sweep(lattice, s, beta, J1, J2, seed, n)
    assert np.array_equal(got, s)
    assert np.array_equal(B1, R1) and np.array_equal(B2, R2) and np.array_equal(M, RM)


def test_quad_replica_resume_and_set_spins():
    Lc, beta, seed = 40, 0.5, 3
    s = oracle.quad_init(Lc, seed, replica=2)
    with ising.Quad(OCT, Lc, beta, 1.0, 1.0, seed=seed, replica=2) as x:
        assert np.array_equal(x.spins(), s)
        x.sweep(3)
        x.sweep(4, 2)
        got = x.spins()
        B1, B2, M = x.series(2)
    R1, R2, RM = oracle.quad_sweep(OCT, s, beta, 1.0, 1.0, seed, 7, replica=2, measure_every=2)
    assert np.array_equal(got, s)
    assert np.array_equal(B1, R1[-2:]) and np.array_equal(M, RM[-2:])
    rng = np.random.default_rng(5)
    mine = rng.choice(np.array([-1, 1], dtype=np.int8), size=(4, Lc, Lc))
    with ising.Quad(SQ, Lc, beta, 1.0, 0.5, seed=seed) as x:
        x.set_spins(mine)
        assert np.array_equal(x.spins(), mine)
        x.sweep(2)
        got = x.spins()
    oracle.quad_sweep(SQ, mine, beta, 1.0, 0.5, seed, 2)
    assert np.array_equal(got, mine)


def test_quad_large_one_sweep():
    """2048^2 cells (16.8 M sites): full bit-exact comparison of one sweep."""
    Lc, beta, seed = 2048, 0.4406868, 17
    with ising.Quad(SQ, Lc, beta, 1.0, 0.0, seed=seed) as x:
        s = x.spins()
        x.sweep(1)
        got = x.spins()
    assert np.array_equal(s, oracle.quad_init(Lc, seed))
    oracle.quad_sweep(SQ, s, beta, 1.0, 0.0, seed, 1)
    assert np.array_equal(got, s)


@pytest.mark.parametrize("lattice,J1,J2", [(SQ, 1.0, 0.0), (OCT, 1.0, 1.0)])
def test_quad_benchmark_size_sampled(lattice, J1, J2):
    """8192^2 cells: each sampled site of sublattice q must follow from the
    final spins of sublattices < q and the initial spins of sublattices > q."""
    Lc, beta, seed, t = 8192, 0.4406868, 1, 0
    with ising.Quad(lattice, Lc, beta, J1, J2, seed=seed) as x:
        x.sweep(1)
        before = x.spins()
        x.sweep(1)
        after = x.spins()
    rng = np.random.default_rng(7)
    z = {SQ: (4, 4), OCT: (2, 1)}[lattice]
    table = {(a1, a2): oracle.quad_threshold(lattice, beta, J1, J2, a1, a2)
             for a1 in range(z[0] + 1) for a2 in range(z[1] + 1)}
    t = 1
    checked = 0
    for q in range(4):
        view = before.copy()
        view[:q] = after[:q]
        for _ in range(300):
            X, Y = (int(v) for v in rng.integers(0, Lc, 2))
            a1, a2 = oracle.quad_anti(lattice, view, q, X, Y)
            thr, always = table[(a1, a2)]
            flip = always or oracle.quad_uniform(Lc, seed, 0, t, q, X, Y) < thr
            want = -before[q, Y, X] if flip else before[q, Y, X]
            assert after[q, Y, X] == want, (q, X, Y)
            checked += 1
    assert checked == 1200


def test_quad_rejects_bad_arguments():
    with pytest.raises(ising.IsingError):
        ising.Quad(SQ, 1, 0.5)
    with pytest.raises(ising.IsingError):
        ising.Quad(7, 8, 0.5)
    with pytest.raises(ising.IsingError):
        ising.Quad(OCT, 8, -1.0)
    with ising.Quad(SQ, 4, 0.5) as x:
        with pytest.raises(ising.IsingError):
            x.set_spins(np.zeros((4, 4, 4), dtype=np.int8))
