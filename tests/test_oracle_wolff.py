"""Pins of the oracle's Wolff single-cluster step (CPU).

The single-cluster update (Wolff 1989) is the second cluster method next to
Swendsen-Wang, on the same bonds: a bond between equal spins is active with
probability 1 - exp(-2 beta), and the connected cluster of active bonds that
holds a randomly drawn seed site is flipped.  Pins:

* One step re-derived independently: the seed site and the bonds drawn from
  the published Philox counter map, the seed's cluster from scipy's connected
  components over all active bonds of the lattice (not grown from the seed),
  the flipped configuration compared site by site.
* Seed site: m = floor(u N / 2^32) from word 0 of the seed block, uniform over
  the lattice in a chi-square test.
* Special cases: beta = 0 activates no bond (the cluster is the seed alone);
  very large beta on an ordered lattice flips the whole lattice.
* 4 x 4 lattice: <E> and <M^2> of the chain agree with exact enumeration, and
  so does the improved estimator <|C|> = <M^2> / N (the mean size of the
  flipped cluster), a relation of the cluster algorithm itself.
* 64 x 64 lattice at beta_c: energy per site vs Kaufman's finite-lattice value.
"""
import math

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components
from scipy.stats import chi2

from oracle import closed_forms as cf
from oracle import exact
from paper_2402_06415_gb300 import stats

TAG_SEED, TAG_BOND = 16, 17


def _block(orc, seed, g, step, tag, replica=0):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    return orc.philox([g, step, replica, tag << 16], key)


def _reference_step(orc, s, beta, seed, step, replica=0):
    L = s.shape[0]
    N = L * L
    thr = math.floor((1.0 - math.exp(-2.0 * beta)) * 2 ** 32)
    m = (int(_block(orc, seed, 0, step, TAG_SEED, replica)[0]) * N) >> 32
    rows, cols = [], []
    for y in range(L):
        for x in range(L):
            a = y * L + x
            for d in range(2):
                xn, yn = ((x + 1) % L, y) if d == 0 else (x, (y + 1) % L)
                if s[y, x] != s[yn, xn]:
                    continue
                b = 2 * a + d
                if _block(orc, seed, b >> 2, step, TAG_BOND, replica)[b & 3] < thr:
                    rows.append(a)
                    cols.append(yn * L + xn)
    g = coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(N, N))
    _, lab = connected_components(g, directed=False)
    sites = np.flatnonzero(lab == lab[m])
    out = s.copy().reshape(-1)
    out[sites] = -out[sites]
    return out.reshape(L, L), m, len(sites)


@pytest.mark.parametrize("L,beta", [(2, 0.5), (3, 0.7), (4, 0.44), (6, 0.3), (8, cf.BETA_C),
                                    (10, 0.8), (13, 0.6)])
def test_step_matches_connected_components(orc, L, beta):
    seed = 0x5678_0000_0000 + L
    s = orc.init(L, seed)
    for step in range(6):
        want, m, size = _reference_step(orc, s, beta, seed, step, replica=1)
        assert orc.wolff_seed_site(L, seed, step, replica=1) == m
        got = s.copy()
        _, _, C = orc.wolff_steps(got, beta, seed, 1, step0=step, replica=1)
        assert np.array_equal(got, want), step
        assert C[0] == size
        s = got


def test_seed_site_uniform(orc):
    L, n = 5, 25000
    counts = np.zeros(L * L)
    for t in range(n):
        counts[orc.wolff_seed_site(L, 99, t)] += 1
    stat = ((counts - n / (L * L)) ** 2 / (n / (L * L))).sum()
    assert stat < chi2.ppf(0.999, L * L - 1), stat
    assert orc.wolff_seed_site(1, 99, 0) == 0


def test_beta_zero_single_site(orc):
    L = 8
    s = orc.init(L, 3)
    before = s.copy()
    _, _, C = orc.wolff_steps(s, 0.0, 3, 5)
    assert (C == 1).all()
    assert (before != s).sum() % 2 == 1


def test_large_beta_flips_everything(orc):
    L = 8
    s = np.ones((L, L), dtype=np.int8)
    E, M, C = orc.wolff_steps(s, 50.0, 5, 3)
    assert (C == L * L).all()
    assert list(M) == [-L * L, L * L, -L * L] and (E == -2 * L * L).all()


@pytest.mark.parametrize("beta", [0.3, cf.BETA_C, 0.6])
def test_chain_matches_enumeration_4x4(orc, beta):
    ex = exact.averages(4, beta)
    Em, Ee, Mm, Me, Cm, Ce = [], [], [], [], [], []
    for seed in range(1, 5):
        s = orc.init(4, seed)
        E, M, C = orc.wolff_steps(s, beta, seed, 20000)
        for arr, mm, ee in ((E[100:], Em, Ee), (M[100:] ** 2, Mm, Me), (C[100:], Cm, Ce)):
            m, e = stats.mean_and_error(arr.astype(np.float64))
            mm.append(m); ee.append(e)
    E_mean, E_err = stats.combine_runs(Em, Ee)
    M_mean, M_err = stats.combine_runs(Mm, Me)
    C_mean, C_err = stats.combine_runs(Cm, Ce)
    assert abs(E_mean - ex["E"]) < 3 * E_err, (E_mean, E_err, ex["E"])
    assert abs(M_mean - ex["M2"]) < 3 * M_err, (M_mean, M_err, ex["M2"])
    assert abs(C_mean - ex["M2"] / 16) < 3 * C_err, (C_mean, C_err, ex["M2"] / 16)
    assert E_err < 0.03 * abs(ex["E"]) and M_err < 0.03 * ex["M2"]


def test_chain_kaufman_critical(orc):
    L, beta = 64, cf.BETA_C
    em, ee = [], []
    for seed in (31, 32, 33):
        s = orc.init(L, seed)
        E, _, C = orc.wolff_steps(s, beta, seed, 6000)
        a, b = stats.mean_and_error(E[300:] / (L * L))
        em.append(a); ee.append(b)
    e, de = stats.combine_runs(em, ee)
    want = cf.kaufman_energy(L, beta)
    assert abs(e - want) < 3 * de, (e, de, want)
    assert de < 4e-3
