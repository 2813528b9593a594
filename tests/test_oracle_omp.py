"""The OpenMP timing build of the oracle sweep gives the single-threaded
oracle's result bit for bit (it only spreads the rows of one colour over
threads; every uniform is a function of seed, sweep and site)."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("L", [4, 6, 64, 66, 130, 512])
def test_omp_sweep_equals_serial(L):
    a = oracle.init(L, 11)
    b = a.copy()
    Ea, Ma = oracle.sweep(a, 0.4406868, 11, 9, t0=3, replica=2, measure_every=2)
    Eb, Mb = oracle.sweep_omp(b, 0.4406868, 11, 9, t0=3, replica=2, measure_every=2)
    assert np.array_equal(a, b)
    assert np.array_equal(Ea, Eb) and np.array_equal(Ma, Mb)


def test_omp_threads_reported():
    assert oracle.omp_threads() >= 1
