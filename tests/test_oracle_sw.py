"""Pins of the oracle's Swendsen-Wang cluster step (CPU).

The cluster step (Swendsen & Wang 1987) is the cluster-update direction the
paper points to beyond its single-site Monte Carlo.  Pins:

* One step re-derived independently: bonds drawn from the published Philox
  counter map, clusters from scipy's connected components (not a union-find),
  the minimum site of each component as its key, and the flipped configuration
  compared with the oracle's, site by site.
* Special cases: beta = 0 activates no bond (every site its own cluster);
  very large beta on an ordered lattice activates every bond (one cluster).
* 4 x 4 lattice: <E> and <M^2> of the chain agree with exact enumeration.
* 64 x 64 lattice: energy per site vs Onsager at beta = 0.6 and vs Kaufman's
  finite-lattice value at beta_c.
"""
import math

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

from oracle import closed_forms as cf
from oracle import exact
from paper_2402_06415_gb300 import stats

TAG_BOND, TAG_FLIP = 10, 11


def _block(orc, seed, g, step, tag, replica=0):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    return orc.philox([g, step, replica, tag << 16], key)


def _reference_step(orc, s, beta, seed, step):
    L = s.shape[0]
    N = L * L
    thr = math.floor((1.0 - math.exp(-2.0 * beta)) * 2 ** 32)
    rows, cols = [], []
    for y in range(L):
        for x in range(L):
            a = y * L + x
            for d in range(2):
                xn, yn = ((x + 1) % L, y) if d == 0 else (x, (y + 1) % L)
                if s[y, x] != s[yn, xn]:
                    continue
                b = 2 * a + d
                if _block(orc, seed, b >> 2, step, TAG_BOND)[b & 3] < thr:
                    rows.append(a)
                    cols.append(yn * L + xn)
    g = coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(N, N))
    nc, lab = connected_components(g, directed=False)
    out = s.copy().reshape(-1)
    for c in range(nc):
        sites = np.flatnonzero(lab == c)
        m = int(sites.min())
        if _block(orc, seed, m >> 2, step, TAG_FLIP)[m & 3] >> 31:
            out[sites] = -out[sites]
    return out.reshape(L, L), nc


@pytest.mark.parametrize("L,beta", [(2, 0.5), (4, 0.44), (6, 0.3), (8, cf.BETA_C), (10, 0.8)])
def test_step_matches_connected_components(orc, L, beta):
    seed = 0x1234_0000_0000 + L
    s = orc.init(L, seed)
    for step in range(3):
        want, nc = _reference_step(orc, s, beta, seed, step)
        got = s.copy()
        _, _, C = orc.sw_steps(got, beta, seed, 1, step0=step)
        assert np.array_equal(got, want), step
        assert C[0] == nc
        s = got


def test_threshold_closed_form(orc):
    for beta in [0.0, 0.1, cf.BETA_C, 1.0, 5.0]:
        want = min(math.floor((1.0 - math.exp(-2.0 * beta)) * 2 ** 32), 2 ** 32 - 1)
        assert orc.sw_threshold(beta) == want
    assert orc.sw_threshold(0.0) == 0
    assert orc.sw_threshold(50.0) == 2 ** 32 - 1


def test_beta_zero_every_site_alone(orc):
    L = 8
    s = orc.init(L, 3)
    _, _, C = orc.sw_steps(s, 0.0, 3, 4)
    assert (C == L * L).all()


def test_large_beta_one_cluster(orc):
    L = 8
    s = np.ones((L, L), dtype=np.int8)
    E, M, C = orc.sw_steps(s, 50.0, 5, 6)
    assert (C == 1).all()
    assert (np.abs(M) == L * L).all() and (E == -2 * L * L).all()


@pytest.mark.parametrize("beta", [0.3, cf.BETA_C, 0.6])
def test_chain_matches_enumeration_4x4(orc, beta):
    ex = exact.averages(4, beta)
    Em, Ee, Mm, Me = [], [], [], []
    for seed in range(1, 5):
        s = orc.init(4, seed)
        E, M, _ = orc.sw_steps(s, beta, seed, 15000)
        m, e = stats.mean_and_error(E[100:].astype(np.float64))
        Em.append(m); Ee.append(e)
        m, e = stats.mean_and_error(M[100:].astype(np.float64) ** 2)
        Mm.append(m); Me.append(e)
    E_mean, E_err = stats.combine_runs(Em, Ee)
    M_mean, M_err = stats.combine_runs(Mm, Me)
    assert abs(E_mean - ex["E"]) < 3 * E_err, (E_mean, E_err, ex["E"])
    assert abs(M_mean - ex["M2"]) < 3 * M_err, (M_mean, M_err, ex["M2"])
    assert E_err < 0.03 * abs(ex["E"]) and M_err < 0.03 * ex["M2"]


def test_chain_onsager_low_T(orc):
    L, beta = 64, 0.6
    s = np.ones((L, L), dtype=np.int8)
    E, _, _ = orc.sw_steps(s, beta, 11, 1500)
    e, de = stats.mean_and_error(E[100:] / (L * L))
    assert abs(e - cf.onsager_energy(beta)) < 3 * de + 1e-6, (e, de)
    assert de < 1e-3


def test_chain_kaufman_critical(orc):
    L, beta = 64, cf.BETA_C
    em, ee = [], []
    for seed in (21, 22, 23):
        s = orc.init(L, seed)
        E, _, _ = orc.sw_steps(s, beta, seed, 2500)
        a, b = stats.mean_and_error(E[100:] / (L * L))
        em.append(a); ee.append(b)
    e, de = stats.combine_runs(em, ee)
    want = cf.kaufman_energy(L, beta)
    assert abs(e - want) < 3 * de, (e, de, want)
    assert de < 3e-3
