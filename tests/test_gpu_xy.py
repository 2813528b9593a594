"""XY-model sweep on the GPU against the CPU oracle.

Spins (unit vectors) bit-exact after n sweeps in double and single precision
(both sides use the same published recipe for sin/cos/exp with explicit FMAs),
the same number of accepted updates, and the energy / magnetisation records
equal to the oracle's up to summation order (1e-12 relative in double).
"""
import numpy as np
import pytest

import oracle
import paper_2402_06415_gb300 as ising

pytestmark = pytest.mark.gpu

T_PAPER = 0.85


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ising.lib()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("L", [2, 4, 6, 16, 64, 130])
@pytest.mark.parametrize("beta", [0.3, 1.0 / T_PAPER, 3.0, 25.0])
def test_xy_bit_exact(precision, L, beta):
    # beta = 25 drives -beta dE below -80 (the branch of the acceptance test that
    # needs no exponential at all) as well as through the hardware-exp band
    seed, n = 100 + L, 7
    u = oracle.xy_init(L, seed, precision=precision)
    start = u.astype(np.float64).copy()
    acc, E_ref = oracle.xy_sweep(u, beta, seed, n)
    with ising.XY(L, beta, precision, seed=seed) as x:
        assert np.array_equal(x.spins(), start)
        x.sweep(n, 1)
        got = x.spins()
        E, Mx, My = x.series(n)
        assert x.accepted() == int(acc.sum())
    assert np.array_equal(got, u.astype(np.float64))
    np.testing.assert_allclose(E, E_ref, rtol=1e-12 if precision == 64 else 1e-9, atol=1e-9)
    _, mx, my = oracle.xy_observables(u)
    assert abs(Mx[-1] - mx) < 1e-9 * L * L and abs(My[-1] - my) < 1e-9 * L * L


def test_xy_paper_size_long_chain():
    """The paper's L = 32 at T = 0.85: 2000 sweeps, double precision."""
    L, beta, seed, n = 32, 1.0 / T_PAPER, 9, 2000
    u = oracle.xy_init(L, seed)
    _, E_ref = oracle.xy_sweep(u, beta, seed, n)
    with ising.XY(L, beta, 64, seed=seed) as x:
        x.sweep(n, 1)
        assert np.array_equal(x.spins(), u)
        E, _, _ = x.series(n)
    np.testing.assert_allclose(E, E_ref, rtol=1e-12, atol=1e-9)


def test_xy_set_spins_roundtrip_and_resume():
    L, beta, seed = 16, 1.0, 4
    with ising.XY(L, beta, 64, seed=seed) as x:
        x.sweep(5)
        mid = x.spins()
    u = mid.copy()
    oracle.xy_sweep(u, beta, seed, 3, t0=5, record=False)
    with ising.XY(L, beta, 64, seed=seed) as x:
        x.set_spins(mid)
        assert np.array_equal(x.spins(), mid)
    # resuming needs the sweep counter: a fresh context at t = 0 differs
    with ising.XY(L, beta, 64, seed=seed) as x:
        x.sweep(8)
        assert np.array_equal(x.spins(), u)


def test_xy_rejects_bad_arguments():
    with pytest.raises(ising.IsingError):
        ising.XY(5, 1.0)
    with pytest.raises(ising.IsingError):
        ising.XY(8, 1.0, precision=16)
    with pytest.raises(ising.IsingError):
        ising.XY(8, -1.0)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("L", [4, 32, 64, 130, 512])
def test_xy_kernel_modes_bit_exact(precision, mode, L):
    """One launch per half sweep (mode 1) and the persistent cooperative kernel
    (mode 2) give the oracle's spins, acceptances and records."""
    beta, seed, n = 1.0 / T_PAPER, 31 + L, 9
    u = oracle.xy_init(L, seed, precision=precision)
    acc, E_ref = oracle.xy_sweep(u, beta, seed, n)
    with ising.XY(L, beta, precision, seed=seed) as x:
        x.set_mode(mode)
        x.sweep(4, 2)
        x.sweep(5, 1)
        got = x.spins()
        E, _, _ = x.series(5)
        assert x.accepted() == int(acc.sum())
        launches = x.launch_count()
    assert np.array_equal(got, u.astype(np.float64))
    np.testing.assert_allclose(E, E_ref[4:], rtol=1e-12 if precision == 64 else 1e-9, atol=1e-9)
    assert launches == (2 if mode == 2 else 2 * n + 2 + 5)


def test_grid_barrier_times_out_and_context_survives():
    assert ising.ising_selftest_grid_barrier(0.05) == 1
    with ising.XY(16, 1.0, 32, seed=1) as x:
        x.sweep(3)
        assert x.spins().shape == (16, 16, 2)
