"""The two bit-sliced identities the packed sweep kernels use, checked against
their plain definitions on the CPU (no GPU, no oracle):

* neighbour classes from two half adders: with a_i = s xor n_i (antiparallel
  neighbour i), a pair's count a_1 + a_2 is the half sum h = n_1 xor n_2 (s
  cancels) plus twice the carry (s^n_1) & (s^n_2); "at least two antiparallel"
  (dE <= 0, always flips) is c_1 | c_2 | (h_1 & h_2), and h_1 | h_2 is 1 with
  exactly one antiparallel neighbour (test against T4) and 0 with none (T8);
* the acceptance test u < T over bit planes: the strict comparison of the top
  bits is the borrow out of the bit-sliced subtraction u - T, carried from the
  least significant plane up with one majority function per plane, and lanes
  whose top bits equal T's stay undecided.  Taken a block of planes at a time
  and merged into (accepted, undecided), this equals the most-significant-first
  test, and after all 32 planes it equals the integer comparison u < T.

The GPU tests compare the kernels that use these identities with the oracle bit
for bit; this file pins the identities themselves.
"""
import itertools

import numpy as np

M32 = 0xFFFFFFFF


def test_half_adder_classes_exhaustive():
    for s, m, n, x, y in itertools.product((0, 1), repeat=5):
        anti = (s ^ m) + (s ^ n) + (s ^ x) + (s ^ y)
        h1, h2 = m ^ n, x ^ y
        c1, c2 = (s ^ m) & (s ^ n), (s ^ x) & (s ^ y)
        ge2 = c1 | c2 | (h1 & h2)
        cls = h1 | h2
        assert ge2 == (anti >= 2)
        if anti == 1:
            assert cls == 1
        if anti == 0:
            assert cls == 0


def _planes_of(u):
    """Plane k of 32 lanes: bit i = bit (31 - k) of lane i's u."""
    return [sum(((int(u[i]) >> (31 - k)) & 1) << i for i in range(32)) for k in range(32)]


def _lane_mask(bits):
    return sum(int(b) << i for i, b in enumerate(bits))


def _borrow_blocks(planes, cls, D, t4, t8, n_planes, block):
    """Blocks of `block` planes, each compared as one borrow chain from its last
    plane up and merged into (acc, D)."""
    m4 = [M32 if (t4 >> (31 - k)) & 1 else 0 for k in range(32)]
    m8 = [M32 if (t8 >> (31 - k)) & 1 else 0 for k in range(32)]
    acc = 0
    for b0 in range(0, n_planes, block):
        bor, eq = 0, D
        for k in range(b0 + block - 1, b0 - 1, -1):
            tm = ((cls & m4[k]) | (~cls & m8[k])) & M32
            nu = ~planes[k] & M32
            bor = (nu & tm) | (nu & bor) | (tm & bor)
            eq &= ~(tm ^ planes[k]) & M32
        acc |= D & bor
        D = eq
    return acc, D


def test_borrow_chain_is_integer_compare():
    rng = np.random.default_rng(7)
    for trial in range(300):
        u = rng.integers(0, 2**32, 32, dtype=np.uint64)
        t4, t8 = (int(v) for v in rng.integers(0, 2**32, 2))
        cls_bits = rng.integers(0, 2, 32)
        if trial % 3 == 0:  # many lanes share the threshold's leading bits
            for i in range(32):
                t = t4 if cls_bits[i] else t8
                keep = int(rng.integers(0, 33))
                low = int(rng.integers(0, 2**32)) & ((1 << (32 - keep)) - 1) if keep < 32 else 0
                u[i] = (t & ~((1 << (32 - keep)) - 1) & M32) | low if keep > 0 else u[i]
        cls = _lane_mask(cls_bits)
        D = int(rng.integers(0, 2**32))
        planes = _planes_of(u)
        want = _lane_mask([(D >> i) & 1 and int(u[i]) < (t4 if cls_bits[i] else t8) for i in range(32)])
        for block in (4, 8):
            acc, rest = _borrow_blocks(planes, cls, D, t4, t8, 32, block)
            assert rest == _lane_mask([(D >> i) & 1 and int(u[i]) == (t4 if cls_bits[i] else t8)
                                       for i in range(32)])
            assert acc == want
        # the first 8 planes as one chain, then 4-plane blocks (the kernels' split)
        acc8, rest8 = _borrow_blocks(planes, cls, D, t4, t8, 8, 8)
        acc_rest, _ = _borrow_blocks(planes[8:] + [0] * 8, cls, rest8,
                                     (t4 << 8) & M32, (t8 << 8) & M32, 24, 4)
        assert acc8 | acc_rest == want


def test_borrow_chain_top_bits_only():
    """After n planes a lane is accepted iff its top n bits are below T's and
    undecided iff they are equal."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        u = rng.integers(0, 2**32, 32, dtype=np.uint64)
        t4, t8 = (int(v) for v in rng.integers(0, 2**32, 2))
        cls_bits = rng.integers(0, 2, 32)
        cls, D = _lane_mask(cls_bits), M32
        planes = _planes_of(u)
        for n in (4, 8, 12):
            acc, rest = _borrow_blocks(planes, cls, D, t4, t8, n, 4)
            top = [int(u[i]) >> (32 - n) for i in range(32)]
            tt = [(t4 if cls_bits[i] else t8) >> (32 - n) for i in range(32)]
            assert acc == _lane_mask([top[i] < tt[i] for i in range(32)])
            assert rest == _lane_mask([top[i] == tt[i] for i in range(32)])
