"""Pins for the CPU reference of the staged block proposal and of Adam (CPU only).

* The schedule draws every interior site once; network stages hold only
  class-0 / class-1 sites; every exact stage is exactly drawable (each unknown
  neighbour of a stage site has all its other neighbours known, and sites of
  one stage neither touch nor share an unknown neighbour).
* The exact-stage log-odds equal the conditional probability obtained by
  summing the Boltzmann weight over every unknown site of the square
  (brute-force enumeration), and two sites of one exact stage are
  conditionally independent.
* The staged proposal density sums to one over all 2^16 interiors of a 4 x 4
  square, and the density reported by a draw equals the teacher-forced one.
* Staged block moves alone (random offsets, two square colours) reproduce the
  exact <E> of a 4 x 4 lattice (enumeration) and of an 8 x 8 lattice (Kaufman)
  within 3 sigma.
* Gradients of the masked (per-stage) loss equal central finite differences.
* Adam reproduces a two-step example worked out by hand from its definition.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import cnn, exact, staged
from oracle.closed_forms import kaufman_energy

NB = ((-1, 0), (1, 0), (0, -1), (0, 1))


@pytest.mark.parametrize("B", [2, 4, 6, 8, 16])
def test_schedule_is_a_valid_partition(B):
    st = staged.schedule(B)
    seen = np.zeros((B, B), dtype=int)
    known = staged.ring_mask(B)
    for kind, sites in st:
        assert sites
        for (i, j) in sites:
            seen[i, j] += 1
            if kind == "net":
                assert staged.site_class(B, i, j) in (0, 1)
        if kind == "exact":
            summed = set()
            sset = set(sites)
            for (i, j) in sites:
                for dy, dx in NB:
                    a, b = i + 1 + dy, j + 1 + dx
                    if known[a, b]:
                        continue
                    assert (a - 1, b - 1) not in sset          # no two stage sites touch
                    assert (a, b) not in summed                # no shared summed neighbour
                    summed.add((a, b))
                    for ey, ex in NB:
                        c, d = a + ey, b + ex
                        if (c, d) != (i + 1, j + 1):
                            assert known[c, d]
        for (i, j) in sites:
            known[i + 1, j + 1] = True
    assert np.all(seen == 1)


def test_site_class_geometry():
    B = 16
    cls = np.array([[staged.site_class(B, i, j) for j in range(B)] for i in range(B)])
    assert (cls == 3).sum() == B * B // 2 and (cls == 0).sum() == B * B // 4
    for i in range(B):
        for j in range(B):
            for dy, dx in NB:
                a, b = i + dy, j + dx
                if 0 <= a < B and 0 <= b < B:
                    assert (cls[i, j] == 3) != (cls[a, b] == 3)  # bipartite
    # a class-3 site never has two class-2 neighbours
    for i in range(B):
        for j in range(B):
            if cls[i, j] == 3:
                n2 = sum(1 for dy, dx in NB if 0 <= i + dy < B and 0 <= j + dx < B
                         and cls[i + dy, j + dx] == 2)
                assert n2 <= 1


def _block_energy(win, B):
    """-sum over bonds with at least one end in the interior (corners unused)."""
    F = B + 2
    e = 0.0
    for y in range(F):
        for x in range(F):
            for yy, xx in ((y, x + 1), (y + 1, x)):
                if yy >= F or xx >= F:
                    continue
                if (1 <= y <= B and 1 <= x <= B) or (1 <= yy <= B and 1 <= xx <= B):
                    e -= win[y, x] * win[yy, xx]
    return e


@pytest.mark.parametrize("beta", [0.3, 0.4406868, 0.7])
def test_exact_stage_matches_enumeration(beta):
    B = 4
    st = staged.schedule(B)
    rng = np.random.default_rng(int(beta * 1000))
    for trial in range(4):
        win = np.where(rng.random((B + 2, B + 2)) < 0.5, 1, -1).astype(np.int64)
        win[0, 0] = win[0, -1] = win[-1, 0] = win[-1, -1] = 0
        for k, (kind, sites) in enumerate(st):
            if kind != "exact":
                continue
            known = staged.known_before(B, st, k)
            unk = [(a - 1, b - 1) for a in range(1, B + 1) for b in range(1, B + 1) if not known[a, b]]
            # brute-force marginal of every unknown site, and joint of two stage sites
            Z = 0.0
            plus = {s: 0.0 for s in sites}
            pair = sites[:2] if len(sites) >= 2 else None
            pp = 0.0
            for bits in itertools.product([-1, 1], repeat=len(unk)):
                w = win.copy()
                for (i, j), v in zip(unk, bits):
                    w[i + 1, j + 1] = v
                wt = math.exp(-beta * _block_energy(w, B))
                Z += wt
                for (i, j) in sites:
                    if w[i + 1, j + 1] > 0:
                        plus[(i, j)] += wt
                if pair and w[pair[0][0] + 1, pair[0][1] + 1] > 0 and w[pair[1][0] + 1, pair[1][1] + 1] > 0:
                    pp += wt
            for (i, j) in sites:
                p_exact = 1.0 / (1.0 + math.exp(-staged.exact_logodds(win, known, beta, i, j)))
                assert abs(p_exact - plus[(i, j)] / Z) < 1e-12, (k, i, j)
            if pair:
                assert abs(pp / Z - plus[pair[0]] * plus[pair[1]] / Z ** 2) < 1e-12


def test_staged_density_normalised_and_draw_consistent():
    B, beta = 4, 0.4406868
    p = cnn.init_params(C=3, seed=5, scale=2.0)
    st = staged.schedule(B)
    rng = np.random.default_rng(6)
    win = np.where(rng.random((B + 2, B + 2)) < 0.5, 1, -1).astype(np.int64)
    allw = np.repeat(win[None], 2 ** (B * B), axis=0)
    allw[:, 1:-1, 1:-1] = np.array(list(itertools.product([-1, 1], repeat=B * B))).reshape(-1, B, B)
    lq = staged.log_q_many(p, allw, beta, B, st)
    assert abs(np.exp(lq).sum() - 1.0) < 1e-9
    for k in rng.choice(len(allw), 8, replace=False):  # the stack agrees with the site-by-site form
        assert abs(lq[k] - staged.log_q(p, allw[k], beta, B, st)) < 1e-9
    for _ in range(5):
        u = rng.integers(0, 2 ** 32, (B, B), dtype=np.uint64)
        new, lq = staged.propose(p, win, beta, B, u, st)
        w = win.copy()
        w[1:-1, 1:-1] = new
        assert abs(lq - staged.log_q(p, w, beta, B, st)) < 1e-9


def test_staged_draw_frequencies_2x2():
    """Empirical frequencies of 2 x 2 proposals equal exp(log q) (chi-square)."""
    B, beta = 2, 0.5
    p = cnn.init_params(C=3, seed=9, scale=2.0)
    st = staged.schedule(B)
    rng = np.random.default_rng(10)
    win = np.array([[0, 1, -1, 0], [1, 0, 0, 1], [-1, 0, 0, 1], [0, 1, 1, 0]], dtype=np.int64)
    n = 6000
    counts = {}
    for _ in range(n):
        u = rng.integers(0, 2 ** 32, (B, B), dtype=np.uint64)
        new, _ = staged.propose(p, win, beta, B, u, st)
        counts[new.tobytes()] = counts.get(new.tobytes(), 0) + 1
    chi2 = 0.0
    for bits in itertools.product([-1, 1], repeat=4):
        w = win.copy()
        w[1:-1, 1:-1] = np.array(bits).reshape(2, 2)
        e = n * math.exp(staged.log_q(p, w, beta, B, st))
        o = counts.get(np.array(bits, dtype=np.int8).reshape(2, 2).tobytes(), 0)
        chi2 += (o - e) ** 2 / e
    assert chi2 < 40.0  # 15 degrees of freedom: P(chi2 > 40) ~ 5e-4


def _block_chain(L, B, beta, p, n_pass, seed):
    from oracle import init as orc_init

    rng = np.random.default_rng(seed)
    s = orc_init(L, seed)
    st = staged.schedule(B)
    Es, acc, tot = [], 0, 0
    for _ in range(n_pass):
        ox, oy = rng.integers(0, B, 2)
        for col in (0, 1):
            for by in range(L // B):
                for bx in range(L // B):
                    if (bx + by) % 2 == col:
                        u = rng.integers(0, 2 ** 32, (B, B), dtype=np.uint64)
                        acc += staged.block_mh(s, (ox + bx * B) % L, (oy + by * B) % L, B, p, beta, u,
                                               rng.random(), st)
                        tot += 1
        Es.append(exact.energy(s))
    return np.array(Es, dtype=np.float64), acc / tot


def test_staged_block_chain_matches_enumeration_4x4():
    from paper_2402_06415_gb300 import stats

    L, B, beta = 4, 2, 0.44
    p = {k: cnn.bf16_round(v) for k, v in cnn.init_params(C=4, seed=12, scale=2.0).items()}
    Es, acc = _block_chain(L, B, beta, p, 4000, 13)
    e, de = stats.mean_and_error(Es[200:])
    want = exact.averages(L, beta)["E"]
    assert 0.05 < acc < 1.0
    assert abs(e - want) < 3 * de, (e, de, want)


def test_staged_block_chain_matches_kaufman_8x8():
    from paper_2402_06415_gb300 import stats

    L, B, beta = 8, 4, 0.4406868
    p = {k: cnn.bf16_round(v) for k, v in cnn.init_params(C=4, seed=14, scale=1.0).items()}
    Es, acc = _block_chain(L, B, beta, p, 1500, 15)
    e, de = stats.mean_and_error(Es[100:])
    want = kaufman_energy(L, beta) * L * L
    assert acc > 0.02
    assert abs(e - want) < 3 * de, (e, de, want)


def test_masked_gradients_match_finite_differences():
    rng = np.random.default_rng(16)
    p = cnn.init_params(C=3, seed=17)
    for k in p:
        p[k] = p[k] + 0.1 * rng.standard_normal(p[k].shape)
    B = 4
    wins = np.where(rng.random((3, B + 2, B + 2)) < 0.5, 1, -1).astype(np.int8)
    _, g = staged.staged_loss_and_grads(p, wins, B)
    eps = 1e-6
    for k in p:
        flat = p[k].ravel()
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _ = staged.staged_loss_and_grads(p, wins, B)
            flat[idx] = old - eps
            lm, _ = staged.staged_loss_and_grads(p, wins, B)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[k].ravel()[idx]) < 1e-6 * max(1.0, abs(fd)), (k, idx, fd)


def test_staged_loss_is_minus_net_log_q():
    """The training loss of one window is -sum over network stages of the log
    of its quantisation-free stage probabilities (teacher forcing)."""
    B, beta = 4, 0.4
    p = cnn.init_params(C=3, seed=18)
    st = staged.schedule(B)
    rng = np.random.default_rng(19)
    win = np.where(rng.random((B + 2, B + 2)) < 0.5, 1, -1).astype(np.int8)
    loss, _ = staged.staged_loss_and_grads(p, win[None], B, st)
    want = 0.0
    for k, (kind, sites) in enumerate(st):
        if kind != "net":
            continue
        lg = staged.stage_logits(p, win.astype(np.int64), beta, B, st, k)
        for (i, j) in sites:
            z = lg[i, j] * win[i + 1, j + 1]
            want += math.log1p(math.exp(-z))
    assert abs(loss - want) < 1e-10


def test_adam_two_steps_by_hand():
    """lr 0.1, b1 0.9, b2 0.999, eps 1e-8, p0 = 1, g1 = 0.5, g2 = -0.25.
    Step 1: m = 0.05, v = 2.5e-4, m^ = 0.5, v^ = 0.25, p1 = 1 - 0.1 * 0.5 / (0.5 + 1e-8).
    Step 2: m = 0.045 - 0.025 = 0.02, v = 2.4975e-4 + 6.25e-5 = 3.1225e-4,
            m^ = 0.02 / 0.19 = 0.105263, v^ = 3.1225e-4 / 1.999e-3 = 0.156203,
            p2 = p1 - 0.1 m^ / (sqrt(v^) + 1e-8) = 0.9 - 0.1 * 0.266334 = 0.873366."""
    p = {"w": np.array([1.0])}
    m = {"w": np.zeros(1)}
    v = {"w": np.zeros(1)}
    p, m, v = staged.adam_step(p, {"w": np.array([0.5])}, m, v, 1, 0.1)
    p1 = 1.0 - 0.1 * 0.5 / (0.5 + 1e-8)
    assert abs(m["w"][0] - 0.05) < 1e-15 and abs(v["w"][0] - 2.5e-4) < 1e-18
    assert abs(p["w"][0] - p1) < 1e-15
    p, m, v = staged.adam_step(p, {"w": np.array([-0.25])}, m, v, 2, 0.1)
    assert abs(m["w"][0] - 0.02) < 1e-15 and abs(v["w"][0] - 3.1225e-4) < 1e-17
    p2 = p1 - 0.1 * (0.02 / 0.19) / (math.sqrt(3.1225e-4 / 1.999e-3) + 1e-8)
    assert abs(p["w"][0] - p2) < 1e-14
    assert abs(p2 - 0.8733663) < 1e-7


def test_bf16_operand_objective_within_rounding_of_exact():
    """The BF16-operand objective (the tensor-core training path's rounding
    points) differs from the exact one and stays close to it: the loss to
    1e-3 relative, the layer-3 gradients (one rounded operand, h2) to 1e-2 of
    the tensor's largest element, the others to 0.15 of it.  The loose bound is
    not rounding noise: rounding W2 and h1 moves z2, which flips the ReLU mask
    of the odd position near zero, and each flip changes whole terms of the
    layer-2 and layer-1 gradients."""
    B = 4
    p = cnn.init_params(seed=3)
    rng = np.random.default_rng(4)
    wins = rng.choice(np.array([-1, 1], dtype=np.int8), size=(12, B + 2, B + 2))
    l0, g0 = staged.staged_loss_and_grads(p, wins, B)
    l1, g1 = staged.staged_loss_and_grads(p, wins, B, bf16_operands=True)
    assert l1 != l0 and abs(l1 - l0) < 1e-3 * abs(l0)
    for k in g0:
        assert not np.array_equal(g1[k], g0[k])
        d = np.abs(g1[k] - g0[k]).max() / np.abs(g0[k]).max()
        assert d < (1e-2 if k in ("W3", "b3") else 0.15), (k, d)
    # rounding is the identity on values that are already BF16: with every
    # rounded quantity exact (zero network), both objectives agree exactly
    z = {k: np.zeros_like(v) for k, v in p.items()}
    assert staged.staged_loss_and_grads(z, wins, B)[0] == staged.staged_loss_and_grads(z, wins, B, bf16_operands=True)[0]
