"""Pins of the fixed-point XY oracle used for the operand-precision study (CPU).

* Angle grid and trig tables against the mathematics: K = round(2 pi 2^F)
  angles, every table entry within half a unit in the last place (2^-F-1) of
  the true cos / sin, exact at 0 and quarter turns.
* Acceptance thresholds: 60-digit floor(exp(-beta dE 2^-F) 2^32), and with
  the probability truncated to F bits, floor(exp(-beta dE 2^-F) 2^F) 2^(32-F).
* The fixed-point energy change against the exact energy change of the grid
  angles (computed from cos of angle differences, Eq. S1 with its sign
  corrected), within the error bound of the table and product rounding.
* Chains: the 2 x 2 torus' exact <E> (1-D Bessel integral) within 3 sigma for
  F = 12 and 16; high-temperature series for F = 16; random start uniform on
  the grid.
"""
import math

import mpmath
import numpy as np
import pytest
from scipy import integrate, special

import oracle
from paper_2402_06415_gb300 import stats


@pytest.mark.parametrize("F", [8, 12, 16])
def test_grid_and_tables(orc, F):
    K = oracle.xyfix_K(F)
    assert K == round(2 * math.pi * 2 ** F)
    assert abs(K / 2 ** F - 2 * math.pi) <= 2 ** -F
    assert oracle.xyfix_trig(F, 0) == (2 ** F, 0)
    rng = np.random.default_rng(F)
    for k in list(rng.integers(0, K, 300)) + [K - 1, K // 2]:
        c, s = oracle.xyfix_trig(F, int(k))
        a = mpmath.mpf(int(k)) / 2 ** F
        assert abs(c - mpmath.cos(a) * 2 ** F) <= 0.5 + 1e-9
        assert abs(s - mpmath.sin(a) * 2 ** F) <= 0.5 + 1e-9


@pytest.mark.parametrize("F", [8, 12, 16])
@pytest.mark.parametrize("beta", [0.5, 1 / 0.85, 3.0])
def test_acceptance_table_closed_form(orc, F, beta):
    mpmath.mp.dps = 60
    rng = np.random.default_rng(F + 1)
    for e in [1, 2, 2 ** F, 8 * 2 ** F] + list(rng.integers(1, 9 * 2 ** F, 50)):
        want = int(mpmath.floor(mpmath.exp(-mpmath.mpf(beta) * mpmath.mpf(int(e)) / 2 ** F) * 2 ** 32))
        assert oracle.xyfix_accept(F, beta, int(e)) == min(want, 2 ** 32 - 1)
        p = mpmath.exp(-mpmath.mpf(beta) * mpmath.mpf(int(e)) / 2 ** F)
        want_q = int(mpmath.floor(p * 2 ** F)) * 2 ** (32 - F)
        assert oracle.xyfix_accept(F, beta, int(e), qp=True) == min(want_q, 2 ** 32 - 1)


@pytest.mark.parametrize("F", [8, 12, 16])
def test_energy_change_within_rounding_bound(orc, F):
    K = oracle.xyfix_K(F)
    rng = np.random.default_rng(2 * F)
    worst = 0.0
    for _ in range(2000):
        k, k2 = (int(v) for v in rng.integers(0, K, 2))
        nb = [int(v) for v in rng.integers(0, K, 4)]
        hx = sum(oracle.xyfix_trig(F, n)[0] for n in nb)
        hy = sum(oracle.xyfix_trig(F, n)[1] for n in nb)
        got = oracle.xyfix_dE(F, k, k2, hx, hy) / 2 ** F
        th, th2 = k / 2 ** F, k2 / 2 ** F
        exact = -sum(math.cos(th2 - n / 2 ** F) - math.cos(th - n / 2 ** F) for n in nb)
        worst = max(worst, abs(got - exact))
    # table rounding (2^-F-1 per entry) through |du| <= 2, |h| <= 4, plus the final rounding
    assert worst <= 12 * 2 ** -F, worst
    assert worst > 0


def _exact_E_2x2(beta):
    def lnZ(b):
        val, _ = integrate.quad(lambda p: special.i0(4 * b * abs(math.cos(p / 2))) ** 2,
                                0, 2 * math.pi, epsabs=1e-13, epsrel=1e-13, limit=200)
        return math.log(val)
    h = 1e-5
    return -(lnZ(beta + h) - lnZ(beta - h)) / (2 * h)


@pytest.mark.parametrize("F", [12, 16])
@pytest.mark.parametrize("beta", [0.5, 1.0 / 0.85])
def test_chain_matches_exact_2x2(orc, F, beta):
    k = oracle.xyfix_init(2, F, 5)
    _, E2 = oracle.xyfix_sweep(k, F, beta, 5, 40000)
    E = -E2[500:] / 2.0 ** (2 * F)
    e, de = stats.mean_and_error(E)
    want = _exact_E_2x2(beta)
    assert abs(e - want) < 3 * de, (e, de, want)
    assert de < 0.02 * abs(want)


def test_high_temperature_series(orc):
    F, beta, L = 16, 0.05, 16
    k = oracle.xyfix_init(L, F, 7)
    _, E2 = oracle.xyfix_sweep(k, F, beta, 7, 3000)
    e, de = stats.mean_and_error(-E2[200:] / 2.0 ** (2 * F) / (L * L))
    want = -2 * special.i1(beta) / special.i0(beta)
    assert abs(e - want) < 3 * de + 1e-4, (e, de, want)


@pytest.mark.parametrize("F", [8, 16])
def test_random_start_uniform_on_grid(orc, F):
    K = oracle.xyfix_K(F)
    k = oracle.xyfix_init(64, F, 3)
    assert k.min() >= 0 and k.max() < K
    th = k / 2 ** F
    assert abs(np.cos(th).mean()) < 4 / 64 and abs(np.sin(th).mean()) < 4 / 64
    assert abs(k.mean() / K - 0.5) < 0.02
