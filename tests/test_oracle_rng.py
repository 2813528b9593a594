"""Pins for the oracle's random numbers (CPU only).

* Philox4x32-10 block function against cuRAND's own implementation of the same
  generator (the cuRAND header evaluated on the host, an independent code base).
* The site uniforms assembled from the plane words: uniform, independent
  across the 32 lanes of a group and across sweeps / colours / replicas (a
  transposed or dropped index in the assembly makes lanes equal or correlated).
* The seeded random start: independent +-1 with probability 1/2.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_host(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available to build the cuRAND host checker")
    exe = str(tmp_path_factory.mktemp("curand") / "curand_philox_host")
    subprocess.run([nvcc, "-O1", "-o", exe, os.path.join(HERE, "curand_philox_host.cu")],
                   check=True)
    return exe


def test_philox_matches_curand(orc, curand_host):
    rng = np.random.default_rng(12345)
    rows = [[0, 0, 0, 0, 0, 0], [0xFFFFFFFF] * 6, [1, 2, 3, 4, 5, 6]]
    rows += rng.integers(0, 2 ** 32, size=(400, 6), dtype=np.uint64).tolist()
    inp = "\n".join(" ".join(str(int(v)) for v in r) for r in rows) + "\n"
    out = subprocess.run([curand_host], input=inp, capture_output=True, text=True,
                         check=True).stdout.split("\n")
    for r, line in zip(rows, out):
        want = [int(v) for v in line.split()]
        got = orc.philox(r[:4], r[4:]).tolist()
        assert got == want, (r, got, want)


def test_threshold_closed_form(orc):
    from oracle.closed_forms import thresholds_exact

    for beta in [0.05, 0.3, 0.35, 0.40, 0.4406868, orc.BETA_C, 0.5, 0.6, 1.0, 3.0]:
        for dE in (4, 8):
            assert orc.threshold(beta, dE) == thresholds_exact(beta, dE), (beta, dE)
    # beta_c: exp(-4 beta_c) = 3 - 2 sqrt 2 exactly (sinh 2K_c = 1)
    t4 = orc.threshold(orc.BETA_C, 4)
    assert abs(t4 / 2 ** 32 - (3 - 2 * np.sqrt(2))) < 2 ** -31


def test_decision_acceptance_counts(orc):
    """The flip decision accepts exactly T uniforms for dE = 4, 8 (strict
    p < P) and all of them for dE <= 0."""
    for beta in [0.3, orc.BETA_C, 0.6]:
        t4, t8 = orc.threshold(beta, 4), orc.threshold(beta, 8)
        assert orc.accept_count(1, t4, t8) == t4
        assert orc.accept_count(0, t4, t8) == t8
        for n in (2, 3, 4):
            assert orc.accept_count(n, t4, t8) == 2 ** 32
        # strictness: u == T does not flip, u == T-1 does
        assert not orc.decide(1, t4, t4, t8) and orc.decide(1, t4 - 1, t4, t8)


def _group_uniforms(orc, seed, replica, sweep, colour, group):
    P = orc.met_planes(seed, replica, sweep, colour, group)
    return np.array([orc.assemble_u(P, lane) for lane in range(32)], dtype=np.float64)


def test_site_uniforms_uniform_and_independent(orc):
    us = []
    for g in range(400):
        us.append(_group_uniforms(orc, 7, 0, 3, g & 1, g))
    U = np.array(us) / 2 ** 32  # (400, 32)
    # uniform on [0, 1): mean 1/2, variance 1/12, KS-like decile check
    assert abs(U.mean() - 0.5) < 4 * np.sqrt(1 / 12 / U.size)
    assert abs(U.var() - 1 / 12) < 0.01
    hist = np.histogram(U.ravel(), bins=10, range=(0, 1))[0]
    chi2 = ((hist - U.size / 10) ** 2 / (U.size / 10)).sum()
    assert chi2 < 35.0  # 9 dof, p ~ 1e-4
    # lanes independent: no pair of lanes equal, correlation matrix ~ identity
    C = np.corrcoef(U.T)
    off = C[~np.eye(32, dtype=bool)]
    assert np.abs(off).max() < 0.25  # 400 samples: sd of r ~ 0.05
    assert np.abs(off).mean() < 0.06


def test_site_uniform_streams_differ(orc):
    base = _group_uniforms(orc, 7, 0, 3, 0, 5)
    for args in [(8, 0, 3, 0, 5), (7, 1, 3, 0, 5), (7, 0, 4, 0, 5), (7, 0, 3, 1, 5),
                 (7, 0, 3, 0, 6)]:
        other = _group_uniforms(orc, *args)
        assert not np.any(other == base), args


def test_site_uniform_matches_group_lane(orc):
    """site_uniform(x, y) picks group y*Wc + (x>>1)//32 and lane (x>>1) % 32."""
    L = 200  # 100 colour sites per row -> 4 words, the last one partial
    Wc = orc.lib().orc_words_per_row(L)
    assert Wc == 4
    for (x, y) in [(0, 0), (1, 0), (63, 5), (64, 5), (199, 199), (130, 17)]:
        j = x >> 1
        c = (x + y) & 1
        P = orc.met_planes(11, 2, 9, c, y * Wc + j // 32)
        assert orc.site_uniform(L, 11, 2, 9, x, y) == orc.assemble_u(P, j % 32)


def test_random_start_fair_and_seeded(orc):
    s = orc.init(128, seed=42)
    assert set(np.unique(s).tolist()) == {-1, 1}
    p = (s == 1).mean()
    assert abs(p - 0.5) < 4 * 0.5 / 128
    # neighbouring sites uncorrelated
    r = (s[:, :-1].astype(float) * s[:, 1:]).mean()
    assert abs(r) < 4 / 128
    assert np.array_equal(s, orc.init(128, seed=42))
    assert not np.array_equal(s, orc.init(128, seed=43))
    assert not np.array_equal(s, orc.init(128, seed=42, replica=1))
