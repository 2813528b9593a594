"""Pins for the CPU reference of the learned block proposal (CPU only).

* The convolution equals scipy's correlate2d summed over channels.
* Backward gradients equal central finite differences (tiny network).
* bf16 rounding equals torch's float -> bfloat16 conversion.
* The quantised proposal density sums to one over all interior configurations.
* The block energy change equals the difference of full-lattice energies.
* The block Metropolis-Hastings kernel satisfies detailed balance exactly on a
  4 x 4 lattice with a 2 x 2 block (enumeration), for a random network, and a
  chain of block moves alone (random offsets, two square colours) reproduces
  the exact <E> within 3 sigma.
"""
import itertools

import numpy as np
import pytest
from scipy import signal

from oracle import cnn, exact


def test_conv_matches_scipy():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 6, 6))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    got = cnn.conv3x3(x, W, b)
    for n in range(2):
        for o in range(4):
            want = b[o] + sum(signal.correlate2d(x[n, c], W[o, c], mode="same") for c in range(3))
            np.testing.assert_allclose(got[n, o], want, rtol=1e-12, atol=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    p = cnn.init_params(C=3, seed=2)
    for k in p:
        p[k] = p[k] + 0.1 * rng.standard_normal(p[k].shape)  # avoid exact ReLU kinks at 0
    B = 2
    spins = np.where(rng.random((8, 8)) < 0.5, 1, -1).astype(np.int8)
    frs, ints = zip(*[cnn.frame(spins, ox, oy, B) for (ox, oy) in [(0, 0), (3, 1), (5, 6)]])
    frs, ints = np.stack(frs), np.stack(ints)
    _, g = cnn.loss_and_grads(p, frs, ints)
    eps = 1e-6
    for k in p:
        flat = p[k].ravel()
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _ = cnn.loss_and_grads(p, frs, ints)
            flat[idx] = old - eps
            lm, _ = cnn.loss_and_grads(p, frs, ints)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[k].ravel()[idx]) < 1e-6 * max(1.0, abs(fd)), (k, idx, fd)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    a = np.concatenate([rng.standard_normal(1000) * 10.0 ** rng.integers(-6, 6, 1000),
                        [0.0, 1.0, -1.0, 1.00390625, 1.0078125, 3.0e-39]])
    want = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(cnn.bf16_round(a), want)


def test_frame_layout():
    L, B = 8, 4
    s = np.arange(L * L).reshape(L, L) % 3 - 1
    s = np.where(s == 0, 1, s).astype(np.int8)
    fr, interior = cnn.frame(s, 6, 5, B)
    assert fr.shape == (2, 6, 6) and interior.shape == (4, 4)
    assert fr[1].sum() == 4 * B and fr[1][0, 0] == fr[1][0, -1] == fr[1][-1, 0] == fr[1][-1, -1] == 0
    assert np.all(fr[0][1:-1, 1:-1] == 0)
    assert fr[0][0, 1] == s[4, 6] and fr[0][1, 0] == s[5, 5] and fr[0][-1, 2] == s[(5 + B) % L, 7]
    assert np.array_equal(interior, s[np.ix_(np.arange(5, 9) % L, np.arange(6, 10) % L)])


def test_proposal_density_normalised():
    rng = np.random.default_rng(4)
    P = cnn.quantise(rng.standard_normal((2, 2)) * 3)
    tot = 0.0
    for bits in itertools.product([-1, 1], repeat=4):
        tot += np.exp(cnn.log_q(P, np.array(bits).reshape(2, 2)))
    assert abs(tot - 1.0) < 1e-12
    assert np.all(P >= 1) and np.all(P <= 2 ** 32 - 1)
    assert cnn.quantise(np.array([-1e9, 1e9])).tolist() == [1, 2 ** 32 - 1]


def test_block_energy_change_is_full_energy_difference():
    rng = np.random.default_rng(5)
    L, B = 8, 4
    for _ in range(20):
        s = np.where(rng.random((L, L)) < 0.5, 1, -1).astype(np.int8)
        ox, oy = rng.integers(0, L, 2)
        new = np.where(rng.random((B, B)) < 0.5, 1, -1).astype(np.int8)
        t = s.copy()
        t[np.ix_(np.arange(oy, oy + B) % L, np.arange(ox, ox + B) % L)] = new
        assert cnn.block_energy_change(s, ox, oy, B, new) == exact.energy(t) - exact.energy(s)


def test_block_mh_detailed_balance_4x4():
    """T(x -> y) = q(y) min(1, pi(y) q(x) / (pi(x) q(y))) for y != x on the block;
    pi(x) T(x -> y) = pi(y) T(y -> x) for every pair, with the quantised q."""
    L, B, beta, ox, oy = 4, 2, 0.44, 1, 2
    p = cnn.init_params(C=4, seed=7, scale=3.0)
    rng = np.random.default_rng(8)
    states = exact.all_configs(L)
    pi = exact.boltzmann(L, beta)
    idx = {c.tobytes(): i for i, c in enumerate(states)}
    checked = 0
    for k in rng.choice(len(states), size=60, replace=False):
        x = states[k]
        fr, old = cnn.frame(x, ox, oy, B)
        P = cnn.quantise(cnn.forward(p, fr[None])[0])
        for bits in itertools.product([-1, 1], repeat=B * B):
            new = np.array(bits, dtype=np.int8).reshape(B, B)
            if np.array_equal(new, old):
                continue
            y = x.copy()
            y[np.ix_([oy, oy + 1], [ox, ox + 1])] = new
            j = idx[y.tobytes()]
            dE = cnn.block_energy_change(x, ox, oy, B, new)
            a_xy = min(1.0, np.exp(-beta * dE + cnn.log_q(P, old) - cnn.log_q(P, new)))
            a_yx = min(1.0, np.exp(beta * dE + cnn.log_q(P, new) - cnn.log_q(P, old)))
            lhs = pi[k] * np.exp(cnn.log_q(P, new)) * a_xy
            rhs = pi[j] * np.exp(cnn.log_q(P, old)) * a_yx  # same boundary: same P
            assert abs(lhs - rhs) <= 1e-12 * max(lhs, rhs, 1e-300)
            checked += 1
    assert checked > 500


def test_block_chain_matches_enumeration_4x4():
    from oracle import init as orc_init
    from paper_2402_06415_gb300 import stats

    L, B, beta = 4, 2, 0.44
    p = {k: cnn.bf16_round(v) for k, v in cnn.init_params(C=32, seed=9).items()}
    rng = np.random.default_rng(0)
    s = orc_init(L, 11)
    Es = []
    for _ in range(5000):
        ox, oy = rng.integers(0, B, 2)
        for col in (0, 1):
            for by in range(L // B):
                for bx in range(L // B):
                    if (bx + by) % 2 == col:
                        u = rng.integers(0, 2 ** 32, (B, B), dtype=np.uint64)
                        cnn.block_mh(s, (ox + bx * B) % L, (oy + by * B) % L, B, p, beta, u,
                                     rng.random())
        Es.append(exact.energy(s))
    e, de = stats.mean_and_error(Es[200:])
    want = exact.averages(L, beta)["E"]
    assert abs(e - want) < 3 * de, (e, de, want)
