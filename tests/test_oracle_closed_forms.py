"""Pins for the closed forms and the brute-force enumeration (CPU only).

Brute force (the plain Boltzmann sum) and Kaufman's finite-torus partition
function are independent routes to the same numbers; Onsager's energy and
Yang's magnetisation are checked at their textbook special values and limits.
"""
import math

import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import exact


@pytest.mark.parametrize("beta", [0.1, 0.3, cf.BETA_C, 0.6, 1.2])
def test_kaufman_equals_brute_force_4x4(beta):
    a = exact.averages(4, beta)
    assert abs(cf.kaufman_lnZ(4, beta) - a["lnZ"]) < 1e-10
    assert abs(cf.kaufman_energy(4, beta) * 16 - a["E"]) < 1e-8


def test_brute_force_small_limits():
    # beta -> 0: <E> = 0, <M^2> = N
    a = exact.averages(4, 1e-9)
    assert abs(a["E"]) < 1e-6 and abs(a["M2"] - 16) < 1e-6
    # beta large: ground states only, E = -2N, M^2 = N^2
    a = exact.averages(4, 8.0)
    assert abs(a["E"] + 32) < 1e-6 and abs(a["M2"] - 256) < 1e-6
    # 2x2 periodic lattice: every bond appears twice; Z = 2 e^{8b} + 12 + 2 e^{-8b}
    b = 0.37
    Z = 2 * math.exp(8 * b) + 12 + 2 * math.exp(-8 * b)
    assert abs(exact.averages(2, b)["lnZ"] - math.log(Z)) < 1e-12


def test_beta_c():
    assert abs(cf.BETA_C - 0.44068679350977147) < 1e-15
    assert abs(math.sinh(2 * cf.BETA_C) - 1.0) < 1e-14


def test_onsager_special_values():
    assert cf.onsager_energy(cf.BETA_C) == -math.sqrt(2.0)
    for d in (1e-4, -1e-4):
        assert abs(cf.onsager_energy(cf.BETA_C + d) + math.sqrt(2)) < 5e-3
    # high temperature: ln Z / N = ln 2 + 2 ln cosh b + t^4 + 2 t^6 + ...
    # (t = tanh b; smallest closed graph = one plaquette), so
    # u = -2t - (4t^3 + 12t^5)(1 - t^2) + O(t^7)
    b = 0.01
    t = math.tanh(b)
    assert abs(cf.onsager_energy(b) - (-2 * t - (4 * t ** 3 + 12 * t ** 5) * (1 - t * t))) < 1e-9
    # low temperature: u -> -2 + 8 e^{-8b} + ...
    b = 2.0
    assert abs(cf.onsager_energy(b) - (-2 + 8 * math.exp(-8 * b))) < 1e-8


def test_kaufman_approaches_onsager():
    for beta in (0.3, 0.6):
        assert abs(cf.kaufman_energy(64, beta) - cf.onsager_energy(beta)) < 1e-9
    # at beta_c the finite-size shift is real and negative
    e64 = cf.kaufman_energy(64, cf.BETA_C)
    assert -1.43 < e64 < -1.42


def test_yang_magnetisation():
    assert cf.yang_magnetisation(cf.BETA_C) == 0.0
    assert cf.yang_magnetisation(cf.BETA_C + 1e-6) < 0.3
    # low-temperature series m = 1 - 2u^2 - 8u^3 - 34u^4 - ..., u = e^{-4b}
    b = 1.0
    u = math.exp(-4 * b)
    series = 1 - 2 * u ** 2 - 8 * u ** 3 - 34 * u ** 4 - 152 * u ** 5
    assert abs(cf.yang_magnetisation(b) - series) < 1e-7


def test_enumeration_matches_definition_4x4():
    """E of a few hand-made states."""
    up = np.ones((4, 4), dtype=np.int8)
    assert exact.energy(up) == -32
    cb = np.fromfunction(lambda y, x: 1 - 2 * ((x + y) % 2), (4, 4)).astype(np.int8)
    assert exact.energy(cb) == 32
    stripe = np.ones((4, 4), dtype=np.int8)
    stripe[:, :2] = -1  # two vertical domain walls x 4 rows = 8 broken bonds
    assert exact.energy(stripe) == -32 + 2 * 8
