"""<|M|> at finite L: a pin that no closed form gives.

Row-to-row transfer matrix of the periodic L x L Ising model with the
magnetisation tracked as a polynomial index: exact Z(M) for L = 6 (2^36
configurations) in a few thousand small matrix products.  The transfer matrix is
itself pinned (against brute-force enumeration at L = 4 and against Kaufman's
closed-form energy at L = 6); the oracle's Metropolis chain on 6 x 6 must then
reproduce <|M|>, <M^2> and <E> within 3 sigma at beta in {0.3, beta_c, 0.6}.
"""
import math

import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import exact
from paper_2402_06415_gb300 import stats


def _rows(L):
    r = np.arange(2 ** L)
    s = 1 - 2 * ((r[:, None] >> np.arange(L)) & 1)        # spins of row r, [2^L, L]
    m = s.sum(axis=1)
    eh = -(s * np.roll(s, -1, axis=1)).sum(axis=1)        # horizontal bonds of a row
    ev = -(s @ s.T)                                        # vertical bonds between rows
    return s, m, eh, ev


def transfer_matrix_ZM(L, beta):
    """Z(M) for M = -L^2 .. L^2 (index M + L^2), and Z(M) weighted by the
    energy, by summing over the first row and closing the torus."""
    _, m, eh, ev = _rows(L)
    n, NM = 2 ** L, 2 * L * L + 1
    W = np.exp(-beta * (ev + eh[None, :]))                 # row r -> row r' (incl. r' bonds)
    ZM = np.zeros(NM)
    for r0 in range(n):
        v = np.zeros((n, NM))
        v[r0, m[r0] + L * L] = math.exp(-beta * eh[r0])
        for _ in range(L - 1):
            u = W.T @ v                                    # [r', M]
            out = np.zeros_like(u)
            for rp in range(n):                            # add row r' magnetisation
                out[rp] = np.roll(u[rp], m[rp])
            v = out
        ZM += (v * np.exp(-beta * ev[:, r0])[:, None]).sum(axis=0)
    return ZM


def tm_averages(L, beta, h=1e-5):
    ZM = transfer_matrix_ZM(L, beta)
    M = np.arange(-L * L, L * L + 1)
    Z = ZM.sum()
    lnZ = lambda b: math.log(transfer_matrix_ZM(L, b).sum())
    E = -(lnZ(beta + h) - lnZ(beta - h)) / (2 * h)
    return {"absM": float((np.abs(M) * ZM).sum() / Z), "M2": float((M ** 2 * ZM).sum() / Z), "E": E}


@pytest.mark.parametrize("beta", [0.3, cf.BETA_C, 0.6])
def test_transfer_matrix_matches_enumeration_4x4(beta):
    ex = exact.averages(4, beta)
    tm = tm_averages(4, beta)
    assert abs(tm["M2"] - ex["M2"]) < 1e-9 * ex["M2"]
    assert abs(tm["E"] - ex["E"]) < 1e-6 * abs(ex["E"])


@pytest.mark.parametrize("beta", [0.3, cf.BETA_C, 0.6])
def test_transfer_matrix_matches_kaufman_6x6(beta):
    tm = tm_averages(6, beta)
    assert abs(tm["E"] / 36 - cf.kaufman_energy(6, beta)) < 1e-6


@pytest.mark.parametrize("beta", [0.3, cf.BETA_C, 0.6])
def test_chain_abs_magnetisation_6x6(orc, beta):
    want = tm_averages(6, beta)
    am, ae, mm, me, em, ee = [], [], [], [], [], []
    for seed in range(1, 5):
        s = orc.init(6, seed)
        E, M = orc.sweep(s, beta, seed, 40000)
        E, M = E[500:].astype(float), M[500:].astype(float)
        a, b = stats.mean_and_error(np.abs(M)); am.append(a); ae.append(b)
        a, b = stats.mean_and_error(M ** 2); mm.append(a); me.append(b)
        a, b = stats.mean_and_error(E); em.append(a); ee.append(b)
    absM, d_absM = stats.combine_runs(am, ae)
    M2, d_M2 = stats.combine_runs(mm, me)
    Em, d_E = stats.combine_runs(em, ee)
    assert abs(absM - want["absM"]) < 3 * d_absM, (absM, d_absM, want["absM"])
    assert abs(M2 - want["M2"]) < 3 * d_M2, (M2, d_M2, want["M2"])
    assert abs(Em - want["E"]) < 3 * d_E, (Em, d_E, want["E"])
    assert d_absM < 0.03 * want["absM"]
