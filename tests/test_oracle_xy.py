"""Pins for the XY-model oracle (CPU only).

* Its own sin / cos / exp (Taylor polynomials with explicit FMAs) agree with the
  C library to ~1 ulp in double and to float rounding in single precision.
* Random start: unit vectors with uniform angles.
* Chain vs exact results: the 2 x 2 periodic lattice (every neighbour pair joined
  by two bonds) has Z = (2 pi)^3 int_0^2pi I0(4 b |cos(phi/2)|)^2 dphi, so <E> is a
  1-D integral; high temperature: u = -2 I1(b)/I0(b) + O(b^4) (smallest closed
  loop = plaquette); low temperature: u = -2 + T/2 + O(T^2) (one quadratic mode
  per site).
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle
from paper_2402_06415_gb300 import stats


def test_double_math_matches_libm():
    rng = np.random.default_rng(0)
    for x in np.concatenate([rng.uniform(-2 * np.pi, 2 * np.pi, 2000), [0.0, np.pi / 4, np.pi]]):
        s, c = oracle.xy_sincos(float(x))
        assert abs(s - math.sin(x)) <= 2 * np.spacing(1.0) and abs(c - math.cos(x)) <= 2 * np.spacing(1.0)
    for x in rng.uniform(-60, 0, 2000):
        assert abs(oracle.xy_exp(float(x)) / math.exp(x) - 1) < 4e-16


def test_float_math_matches_libm():
    rng = np.random.default_rng(1)
    for x in rng.uniform(-2 * np.pi, 2 * np.pi, 2000).astype(np.float32):
        s, c = oracle.xy_sincos(float(x), 32)
        assert abs(s - math.sin(float(x))) < 3e-7 and abs(c - math.cos(float(x))) < 3e-7
    for x in rng.uniform(-60, 0, 2000).astype(np.float32):
        assert abs(oracle.xy_exp(float(x), 32) / math.exp(float(x)) - 1) < 4e-7


@pytest.mark.parametrize("precision", [64, 32])
def test_random_start(precision):
    u = oracle.xy_init(64, 3, precision=precision)
    assert np.allclose(np.hypot(u[..., 0], u[..., 1]), 1.0, atol=1e-6)
    th = np.arctan2(u[..., 1], u[..., 0])
    assert abs(np.cos(th).mean()) < 4 / 64 and abs(np.sin(th).mean()) < 4 / 64
    assert abs((np.cos(th) ** 2).mean() - 0.5) < 0.03


def _exact_E_2x2(beta):
    def lnZ(b):
        val, _ = integrate.quad(lambda p: special.i0(4 * b * abs(math.cos(p / 2))) ** 2,
                                0, 2 * math.pi, epsabs=1e-13, epsrel=1e-13, limit=200)
        return math.log(val)
    h = 1e-5
    return -(lnZ(beta + h) - lnZ(beta - h)) / (2 * h)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("beta", [0.5, 1.0 / 0.85])
def test_chain_matches_exact_2x2(precision, beta):
    u = oracle.xy_init(2, 5, precision=precision)
    _, E = oracle.xy_sweep(u, beta, 5, 40000)
    e, de = stats.mean_and_error(E[500:])
    want = _exact_E_2x2(beta)
    assert abs(e - want) < 3 * de, (e, de, want)
    assert de < 0.02 * abs(want)


def test_high_temperature_series():
    beta, L = 0.05, 16
    u = oracle.xy_init(L, 7)
    _, E = oracle.xy_sweep(u, beta, 7, 3000)
    e, de = stats.mean_and_error(E[200:] / (L * L))
    want = -2 * special.i1(beta) / special.i0(beta)
    assert abs(e - want) < 3 * de + 1e-4, (e, de, want)
    assert de < 0.003


def test_low_temperature_spin_waves():
    beta, L = 20.0, 16
    u = np.zeros((L, L, 2))
    u[..., 0] = 1.0
    _, E = oracle.xy_sweep(u, beta, 9, 3000)
    e, de = stats.mean_and_error(E[1000:] / (L * L))
    want = -2 + 0.5 / beta
    assert abs(e - want) < 3 * de + 3e-4, (e, de, want)
