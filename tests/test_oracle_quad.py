"""Pins of the four-sublattice (quadripartite) Ising oracle (CPU).

* Lattice structure against independent constructions: the square lattice's
  NN / NNN pairs from array rolls on the L x L grid; the square-octagon lattice
  from geometry (regular truncated square tiling, every edge of length a: two
  sites bond iff their minimum-image distance is a).  No site has a neighbour
  in its own sublattice.
* Bond sums against the same independent bond lists.
* Thresholds: 60-digit floor(exp(-beta dE) 2^32) of every class.
* Site uniforms re-assembled from the published counter map.
* Chains vs exact enumeration (2^16 states): the plain square lattice (J2 = 0,
  must reproduce the ordinary 4 x 4 Ising averages although the update order
  differs), the NN + NNN square lattice (J2 = 0.5 and -0.5) and the
  square-octagon lattice (N = 16).
* L = 64 plain square lattice vs Onsager at beta = 0.3.
"""
import math

import mpmath
import numpy as np
import pytest

import oracle
from oracle import closed_forms as cf
from oracle import exact
from paper_2402_06415_gb300 import stats

SQ, OCT = oracle.QUAD_SQUARE, oracle.QUAD_SQOCT


def _sid(Lc, q, X, Y):
    return (q * Lc + Y) * Lc + X


def _square_bonds(Lc):
    """[(a, b, type)] each bond once, from the L x L grid (site ids as s[q][Y][X])."""
    L = 2 * Lc
    ids = np.zeros((L, L), dtype=np.int64)        # [y][x]
    for y in range(L):
        for x in range(L):
            ids[y, x] = _sid(Lc, (x & 1) + 2 * (y & 1), x >> 1, y >> 1)
    out = []
    for dx, dy, t in [(1, 0, 1), (0, 1, 1), (1, 1, 2), (1, -1, 2)]:
        nb = np.roll(np.roll(ids, -dy, axis=0), -dx, axis=1)   # nb[y, x] = ids[y + dy, x + dx]
        out += [(int(a), int(b), t) for a, b in zip(ids.ravel(), nb.ravel())]
    return out


def _octagon_bonds(Lc):
    """Bonds of the 4.8.8 lattice from geometry (edge length 1)."""
    c = 1.0 + math.sqrt(2.0)                # cell spacing
    h = 1.0 / math.sqrt(2.0)                # centre-to-vertex distance
    offs = {0: (0.0, h), 1: (h, 0.0), 2: (0.0, -h), 3: (-h, 0.0)}   # A top, B right, C bottom, D left
    pos, cell = {}, {}
    for q in range(4):
        for Y in range(Lc):
            for X in range(Lc):
                i = _sid(Lc, q, X, Y)
                pos[i] = (X * c + offs[q][0], Y * c + offs[q][1])
                cell[i] = (X, Y)
    box = Lc * c
    out = []
    keys = sorted(pos)
    for ia, a in enumerate(keys):
        for b in keys[ia + 1:]:
            dx = pos[a][0] - pos[b][0]
            dy = pos[a][1] - pos[b][1]
            dx -= box * round(dx / box)
            dy -= box * round(dy / box)
            if abs(math.hypot(dx, dy) - 1.0) < 1e-9:
                out.append((a, b, 1 if cell[a] == cell[b] else 2))
    return out


def _oracle_pairs(lattice, Lc):
    got = []
    for q in range(4):
        for Y in range(Lc):
            for X in range(Lc):
                for (q2, X2, Y2, t) in oracle.quad_neighbours(lattice, Lc, q, X, Y):
                    got.append((_sid(Lc, q, X, Y), _sid(Lc, q2, X2, Y2), t))
    return got


@pytest.mark.parametrize("lattice,Lc", [(SQ, 2), (SQ, 3), (SQ, 5), (OCT, 2), (OCT, 3), (OCT, 4)])
def test_structure_matches_independent_construction(orc, lattice, Lc):
    bonds = _square_bonds(Lc) if lattice == SQ else _octagon_bonds(Lc)
    want = sorted([(a, b, t) for a, b, t in bonds] + [(b, a, t) for a, b, t in bonds])
    got = sorted(_oracle_pairs(lattice, Lc))
    assert got == want
    N = 4 * Lc * Lc
    for a, b, _ in got:
        assert a // (Lc * Lc) != b // (Lc * Lc)          # no neighbour in the own sublattice
    deg = np.bincount([a for a, _, _ in got], minlength=N)
    assert (deg == (8 if lattice == SQ else 3)).all()


@pytest.mark.parametrize("lattice,Lc", [(SQ, 3), (OCT, 3)])
def test_bond_sums_match_bond_list(orc, lattice, Lc):
    bonds = _square_bonds(Lc) if lattice == SQ else _octagon_bonds(Lc)
    rng = np.random.default_rng(3)
    for _ in range(5):
        s = rng.choice(np.array([-1, 1], dtype=np.int8), size=(4, Lc, Lc))
        f = s.ravel().astype(np.int64)
        b1 = sum(f[a] * f[b] for a, b, t in bonds if t == 1)
        b2 = sum(f[a] * f[b] for a, b, t in bonds if t == 2)
        assert oracle.quad_observables(lattice, s) == (b1, b2, int(f.sum()))


@pytest.mark.parametrize("lattice", [SQ, OCT])
@pytest.mark.parametrize("beta,J1,J2", [(0.44, 1.0, 0.0), (0.3, 1.0, 0.5), (0.7, 1.0, -0.5),
                                        (0.2, 0.75, 1.25)])
def test_thresholds_closed_form(orc, lattice, beta, J1, J2):
    z1, z2 = (4, 4) if lattice == SQ else (2, 1)
    mpmath.mp.dps = 60
    for a1 in range(z1 + 1):
        for a2 in range(z2 + 1):
            t, always = oracle.quad_threshold(lattice, beta, J1, J2, a1, a2)
            dE = 2 * mpmath.mpf(J1) * (z1 - 2 * a1) + 2 * mpmath.mpf(J2) * (z2 - 2 * a2)
            if dE <= 0:
                assert always
                continue
            assert not always
            assert t == int(mpmath.floor(mpmath.exp(-mpmath.mpf(beta) * dE) * 2 ** 32))


def test_uniform_from_counter_map(orc):
    Lc, seed, r, t = 70, 0x1_0000_0005, 2, 9
    key = [seed & 0xFFFFFFFF, seed >> 32]
    Wq = (Lc + 31) // 32
    for (q, X, Y) in [(0, 0, 0), (3, 69, 69), (2, 33, 5), (1, 64, 40)]:
        g = Y * Wq + (X >> 5)
        planes = []
        for b in range(8):
            planes += list(oracle.philox([g, t, r, (13 << 16) | (q << 8) | b], key))
        u = sum(((int(planes[k]) >> (X & 31)) & 1) << (31 - k) for k in range(32))
        assert oracle.quad_uniform(Lc, seed, r, t, q, X, Y) == u


def test_random_start_balanced(orc):
    s = oracle.quad_init(64, 11)
    assert abs(int(s.astype(np.int64).sum())) < 4 * math.sqrt(s.size)
    assert not np.array_equal(s, oracle.quad_init(64, 12))
    assert not np.array_equal(s, oracle.quad_init(64, 11, replica=1))


def _enumerate(bonds, N, beta, J1, J2):
    st = np.arange(2 ** N, dtype=np.int64)
    spins = 1 - 2 * ((st[:, None] >> np.arange(N)) & 1).astype(np.int64)
    E = np.zeros(2 ** N)
    for a, b, t in bonds:
        E -= (J1 if t == 1 else J2) * spins[:, a] * spins[:, b]
    M2 = spins.sum(axis=1).astype(np.float64) ** 2
    w = np.exp(-beta * (E - E.min()))
    Z = w.sum()
    return float((w * E).sum() / Z), float((w * M2).sum() / Z)


def _chain(lattice, Lc, beta, J1, J2, n, seeds):
    em, ee, mm, me = [], [], [], []
    for seed in seeds:
        s = oracle.quad_init(Lc, seed)
        B1, B2, M = oracle.quad_sweep(lattice, s, beta, J1, J2, seed, n)
        E = -J1 * B1[200:] - J2 * B2[200:]
        a, b = stats.mean_and_error(E)
        em.append(a); ee.append(b)
        a, b = stats.mean_and_error(M[200:].astype(np.float64) ** 2)
        mm.append(a); me.append(b)
    return stats.combine_runs(em, ee), stats.combine_runs(mm, me)


@pytest.mark.parametrize("beta", [0.3, cf.BETA_C, 0.6])
def test_plain_square_chain_matches_ising_4x4(orc, beta):
    (E, dE), (M2, dM2) = _chain(SQ, 2, beta, 1.0, 0.0, 30000, range(1, 5))
    ex = exact.averages(4, beta)
    assert abs(E - ex["E"]) < 3 * dE, (E, dE, ex["E"])
    assert abs(M2 - ex["M2"]) < 3 * dM2, (M2, dM2, ex["M2"])
    assert dE < 0.05 * abs(ex["E"])


@pytest.mark.parametrize("beta,J2", [(0.3, 0.5), (0.4, -0.5)])
def test_nnn_square_chain_matches_enumeration(orc, beta, J2):
    want_E, want_M2 = _enumerate(_square_bonds(2), 16, beta, 1.0, J2)
    (E, dE), (M2, dM2) = _chain(SQ, 2, beta, 1.0, J2, 30000, range(1, 5))
    assert abs(E - want_E) < 3 * dE, (E, dE, want_E)
    assert abs(M2 - want_M2) < 3 * dM2, (M2, dM2, want_M2)
    assert dE < 0.05 * abs(want_E)


@pytest.mark.parametrize("beta,J1,J2", [(0.5, 1.0, 1.0), (0.9, 1.0, 1.0), (0.6, 1.0, 0.5)])
def test_octagon_chain_matches_enumeration(orc, beta, J1, J2):
    want_E, want_M2 = _enumerate(_octagon_bonds(2), 16, beta, J1, J2)
    (E, dE), (M2, dM2) = _chain(OCT, 2, beta, J1, J2, 30000, range(1, 5))
    assert abs(E - want_E) < 3 * dE, (E, dE, want_E)
    assert abs(M2 - want_M2) < 3 * dM2, (M2, dM2, want_M2)
    assert dE < 0.05 * abs(want_E)


def test_plain_square_onsager_L64(orc):
    beta, Lc = 0.3, 32
    em, ee = [], []
    for seed in (1, 2):
        s = oracle.quad_init(Lc, seed)
        B1, _, _ = oracle.quad_sweep(SQ, s, beta, 1.0, 0.0, seed, 1500)
        a, b = stats.mean_and_error(-B1[150:] / (4 * Lc * Lc))
        em.append(a); ee.append(b)
    e, de = stats.combine_runs(em, ee)
    assert abs(e - cf.onsager_energy(beta)) < 3 * de, (e, de)
    assert de < 2e-3
