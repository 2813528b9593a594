"""Pins for the oracle's parallel-tempering ladder (CPU).

Exchange between adjacent temperatures leaves the product of Boltzmann
distributions invariant, so every temperature slot of a ladder must sample its
own Boltzmann distribution: on 4 x 4 lattices the per-slot <E> and <M^2>
agree with exact enumeration within 3 sigma, and the exchange acceptance rate
of each adjacent pair agrees with its exact expectation
sum_{x,y} pi_a(x) pi_b(y) min(1, exp[(b_a - b_b)(E_x - E_y)]).  A reversed
sign in the exchange rule fails both.
"""
import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2402_06415_gb300 import stats

BETAS = np.array([0.30, 0.38, 0.46, 0.54])


def _energy_hist(L, beta):
    S = exact.all_configs(L)
    E = exact.energy(S)
    p = exact.boltzmann(L, beta)
    vals = np.unique(E)
    return vals, np.array([p[E == v].sum() for v in vals])


def _exact_swap_rate(L, ba, bb):
    ea, pa = _energy_hist(L, ba)
    eb, pb = _energy_hist(L, bb)
    d = (ba - bb) * (ea[:, None] - eb[None, :])
    return float((pa[:, None] * pb[None, :] * np.minimum(1.0, np.exp(d))).sum())


def _run(betas, seed, n_sweeps, sign=+1):
    """Ladder of 4x4 replicas, exchange after every sweep; returns per-slot series."""
    L, nb = 4, len(betas)
    spins = [oracle.init(L, seed, i) for i in range(nb)]
    perm = np.arange(nb, dtype=np.int32)
    acc = np.zeros(nb, dtype=np.int64)
    att = np.zeros(nb, dtype=np.int64)
    Es = np.zeros((n_sweeps, nb))
    M2 = np.zeros((n_sweeps, nb))
    E = np.zeros(nb, dtype=np.int64)
    for t in range(n_sweeps):
        slot_of = np.empty(nb, dtype=np.int32)
        slot_of[perm] = np.arange(nb)
        for i in range(nb):
            e, m = oracle.sweep(spins[i], betas[slot_of[i]], seed, 1, t0=t, replica=i)
            E[i] = e[-1]
            Es[t, slot_of[i]] = e[-1]
            M2[t, slot_of[i]] = float(m[-1]) ** 2
        oracle.pt_step(betas[::sign] if sign < 0 else betas, seed, 0, t, E, perm, acc, att)
    return Es, M2, acc, att


def test_pt_slots_sample_their_boltzmann_distribution():
    Es, M2, acc, att = _run(BETAS, 17, 30000)
    for k, b in enumerate(BETAS):
        ex = exact.averages(4, b)
        e, de = stats.mean_and_error(Es[500:, k])
        m, dm = stats.mean_and_error(M2[500:, k])
        assert abs(e - ex["E"]) < 3 * de, (b, e, de, ex["E"])
        assert abs(m - ex["M2"]) < 3 * dm, (b, m, dm, ex["M2"])
    for a in range(len(BETAS) - 1):
        want = _exact_swap_rate(4, BETAS[a], BETAS[a + 1])
        n = att[a]
        got = acc[a] / n
        sd = np.sqrt(want * (1 - want) / n) * 3  # exchanges are correlated: 3x binomial
        assert abs(got - want) < 3 * sd, (a, got, want, sd)


def test_reversed_exchange_sign_is_detected():
    """Exchanging with the beta order reversed in the rule drives low-energy
    states to the hot end: the hottest slot's <E> moves far from exact."""
    Es, _, _, _ = _run(BETAS, 18, 6000, sign=-1)
    ex = exact.averages(4, BETAS[0])
    e, de = stats.mean_and_error(Es[500:, 0])
    assert abs(e - ex["E"]) > 5 * de


def test_pt_step_pairs_and_counters():
    nb = 6
    perm = np.arange(nb, dtype=np.int32)
    acc = np.zeros(nb, dtype=np.int64)
    att = np.zeros(nb, dtype=np.int64)
    # colder slots hold higher energies: d = (b_a - b_b)(E_a - E_b) >= 0 for
    # every adjacent pair, so every attempted exchange is accepted
    E = np.array([-60, -50, -40, -30, -20, -10], dtype=np.int64)
    oracle.pt_step(np.linspace(0.3, 0.5, nb), 1, 0, 0, E, perm, acc, att)
    # even step: pairs (0,1),(2,3),(4,5)
    assert perm.tolist() == [1, 0, 3, 2, 5, 4]
    assert att.tolist() == [1, 0, 1, 0, 1, 0] and acc.tolist() == [1, 0, 1, 0, 1, 0]
    oracle.pt_step(np.linspace(0.3, 0.5, nb), 1, 0, 1, E, perm, acc, att)
    # odd step: pairs (1,2),(3,4) only
    assert att.tolist() == [1, 1, 1, 1, 1, 0]


@pytest.mark.parametrize("seed", [1, 2])
def test_run_ladders_matches_manual_loop(seed):
    betas = np.linspace(0.35, 0.5, 4)
    sp, perm, E, M, acc, att = oracle.run_ladders([8, 6], betas, seed, 25, 5)
    # both ladders replayed by hand with the beta of each replica's slot per round
    sp0 = [oracle.init(8, seed, i) for i in range(4)]
    sp1 = [oracle.init(6, seed, 4 + i) for i in range(4)]
    P = [np.arange(4, dtype=np.int32), np.arange(4, dtype=np.int32)]
    for rnd in range(5):
        for l, spl in enumerate((sp0, sp1)):
            slot_of = np.empty(4, dtype=np.int32)
            slot_of[P[l]] = np.arange(4)
            El = np.zeros(4, dtype=np.int64)
            for i in range(4):
                e, _ = oracle.sweep(spl[i], betas[slot_of[i]], seed, 5, t0=5 * rnd,
                                    replica=4 * l + i)
                El[i] = e[-1]
            oracle.pt_step(betas, seed, l, rnd, El, P[l])
    assert np.array_equal(sp[1][0], sp1[0]) and np.array_equal(P[1], perm[1])
    assert np.array_equal(P[0], perm[0])
