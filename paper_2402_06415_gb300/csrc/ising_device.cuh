// Device building blocks of the checkerboard Metropolis sweep (sm_103a).
//
// * Philox4x32-10 (Salmon et al., SC'11) keyed by the seed and addressed by
//   (group, sweep, replica, tag | colour | block): the paper's per-site random
//   draw (Supplementary, MC details, step 1) as a stateless counter-based
//   stream, so a site's random number depends only on (seed, sweep, site).
// * The bit-sliced neighbour classes of one 32-site word: the Ising form of the
//   local energy change (Eq. S1 analogue), dE = 8 - 4 n_anti.
// * The acceptance test "p < P(dE)" (step 3) against integer thresholds,
//   evaluated bit-serially from the most significant plane: exact, and
//   usually decided after a handful of planes.  (The tiled and batched
//   kernels compare the planes of a Philox block as one borrow chain, the
//   borrow of u - T carried up from the block's last plane, which gives the
//   same verdicts with one logic operation less per plane.)
//
// Spin words: bit i of word w of colour-row (y, c) is site j = 32 w + i of the
// L/2 colour-c sites of row y, at x = 2 j + ((y + c) & 1); bit = 1 means +1.
#pragma once
#include <cstdint>

#include "internal.h"

namespace ising {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

constexpr uint32_t kTagInit = 1;
constexpr uint32_t kTagMet = 2;
constexpr uint32_t kTagPT = 3;

// Philox4x32-10 block function.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x);
    const uint32_t lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z);
    const uint32_t lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ (k0 + r * kPhiloxW0), lo1, hi0 ^ c.w ^ (k1 + r * kPhiloxW1), lo0);
  }
  return c;
}

// Same block function with the ten round keys given (k0 + r W0, k1 + r W1).
__device__ __forceinline__ uint4 philox10_rk(uint4 c, const uint32_t (&rk0)[10],
                                             const uint32_t (&rk1)[10]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x);
    const uint32_t lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z);
    const uint32_t lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ rk0[r], lo1, hi0 ^ c.w ^ rk1[r], lo0);
  }
  return c;
}

__device__ __forceinline__ uint32_t ctr_w(uint32_t tag, uint32_t colour, uint32_t block) {
  return (tag << 16) | (colour << 8) | block;
}

// Neighbour classes of a word of colour-c spins s given the four neighbour
// words (other colour): ge2 = at least two antiparallel neighbours (dE <= 0,
// always flips), one = exactly one (dE = 4), zero = none (dE = 8).
struct Classes {
  uint32_t ge2, one, zero;
};

__device__ __forceinline__ Classes classify(uint32_t s, uint32_t n1, uint32_t n2, uint32_t n3,
                                            uint32_t n4) {
  const uint32_t a1 = s ^ n1, a2 = s ^ n2, a3 = s ^ n3, a4 = s ^ n4;
  Classes k;
  k.ge2 = (a1 & a2) | (a3 & a4) | ((a1 ^ a2) & (a3 ^ a4));
  k.zero = ~(a1 | a2 | a3 | a4);
  k.one = ~(k.ge2 | k.zero);
  return k;
}

// Neighbour classes of a word s in the form the plane test needs, with the
// four neighbours taken as two pairs (m, n) and (x, y): ge2 = at least two
// antiparallel neighbours (always flips), cls = 1 on lanes with exactly one
// and 0 on lanes with none (lanes of ge2 are never tested, so their cls is
// free).  Per pair the antiparallel count is a half sum plus a carry, where s
// cancels from the half sum (h = (s^m) ^ (s^n) = m ^ n), so a word pair that
// shares a neighbour pair computes h1 once.
struct HalfClasses {
  uint32_t ge2, cls;
};
__device__ __forceinline__ HalfClasses classify_hs(uint32_t s, uint32_t h1, uint32_t m, uint32_t n,
                                                   uint32_t x, uint32_t y) {
  const uint32_t c1 = (s ^ m) & (s ^ n);
  const uint32_t h2 = x ^ y;
  const uint32_t c2 = (s ^ x) & (s ^ y);
  return {c1 | c2 | (h1 & h2), h1 | h2};
}

// Bit-serial "u < T" for the undecided lanes D over the 4 planes of one Philox
// block (planes 4b .. 4b+3, plane 0 = most significant bit of u).  For lanes
// of class `one` T = t4, for class `zero` T = t8.  Lanes whose plane bit equals
// the threshold bit stay undecided; u_bit = 0 < T_bit = 1 accepts; the reverse
// rejects.  `acc` collects accepted lanes.
__device__ __forceinline__ void compare_block(uint4 r, int b, uint32_t t4, uint32_t t8,
                                              uint32_t one, uint32_t zero, uint32_t& D,
                                              uint32_t& acc) {
  const uint32_t p[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = 4 * b + q;                       // plane index
    const uint32_t m4 = 0u - ((t4 >> (31 - k)) & 1u);  // all-ones iff T4 bit set
    const uint32_t m8 = 0u - ((t8 >> (31 - k)) & 1u);
    // per-lane threshold bit: T4's for class `one`, T8's otherwise (lanes of
    // neither class are never in D); one three-input logic op
    const uint32_t tm = (one & m4) | (~one & m8);
    acc |= D & tm & ~p[q];
    D &= ~(tm ^ p[q]);
  }
}

// Flip mask for one word: always-flip lanes plus the lanes whose uniform falls
// below their threshold.  Planes are generated lazily, four per Philox block,
// until no lane of the warp is undecided.  All 32 lanes of the warp must call
// this together (warp vote); lanes with nothing to decide pass valid = 0.
__device__ __forceinline__ uint32_t flip_mask(const Classes& k, uint32_t valid, uint32_t g,
                                              uint32_t t, uint32_t rep, uint32_t colour,
                                              uint32_t key0, uint32_t key1, uint32_t t4,
                                              uint32_t t8) {
  const uint32_t one = k.one & valid;
  const uint32_t zero = k.zero & valid;
  uint32_t D = one | zero;
  uint32_t acc = 0;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    if (!__any_sync(0xffffffffu, D != 0u)) break;
    const uint4 r = philox10(make_uint4(g, t, rep, ctr_w(kTagMet, colour, b)), key0, key1);
    compare_block(r, b, t4, t8, one, zero, D, acc);
  }
  return (k.ge2 & valid) | acc;
}

// flip_mask with the ten Philox round keys given (as philox10_rk).
__device__ __forceinline__ uint32_t flip_mask_rk(const Classes& k, uint32_t valid, uint32_t g,
                                                 uint32_t t, uint32_t rep, uint32_t colour,
                                                 const uint32_t (&rk0)[10], const uint32_t (&rk1)[10],
                                                 uint32_t t4, uint32_t t8) {
  const uint32_t one = k.one & valid;
  const uint32_t zero = k.zero & valid;
  uint32_t D = one | zero;
  uint32_t acc = 0;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    if (!__any_sync(0xffffffffu, D != 0u)) break;
    const uint4 r = philox10_rk(make_uint4(g, t, rep, ctr_w(kTagMet, colour, b)), rk0, rk1);
    compare_block(r, b, t4, t8, one, zero, D, acc);
  }
  return (k.ge2 & valid) | acc;
}

// Valid-lane mask of word w when the colour row has n sites (n = L/2).
__device__ __forceinline__ uint32_t valid_mask(int w, int Wc, int n) {
  if (w < Wc - 1) return 0xffffffffu;
  const int nb = n - 32 * (Wc - 1);
  return nb >= 32 ? 0xffffffffu : ((1u << nb) - 1u);
}

// x-neighbour word of the other colour that is not at the same index:
// offset o = (y + c) & 1 of the updated colour; o = 0 -> index j-1, o = 1 -> j+1.
// `row` is the other colour's row (Wc words, unused lanes zero).
template <typename Row>
__device__ __forceinline__ uint32_t side_word(const Row& row, int w, int Wc, int n, int o) {
  const int nb = n - 32 * (Wc - 1);
  const uint32_t cur = row(w);
  if (o == 0) {
    const uint32_t carry = (w > 0) ? (row(w - 1) >> 31) : ((row(Wc - 1) >> (nb - 1)) & 1u);
    return (cur << 1) | carry;
  } else {
    if (w < Wc - 1) return (cur >> 1) | (row(w + 1) << 31);
    return (cur >> 1) | ((row(0) & 1u) << (nb - 1));
  }
}

// Spins while *word == value, for at most `limit` clock64 cycles.  Returns
// true when the word changed, false when the budget ran out (the caller then
// records an error status and returns instead of waiting forever).
__device__ __forceinline__ bool bounded_wait_while_eq(const volatile unsigned int* word,
                                                      unsigned int value, long long limit) {
  const long long start = clock64();
  while (*word == value) {
    if (clock64() - start > limit) return false;
    __nanosleep(128);
  }
  return true;
}

// Grid-wide barrier for persistent cooperative kernels (all CTAs co-resident):
// generation counter + arrival count in global memory, a tight bounded spin
// (clock64 budget `limit`).  On time-out it records 1 in ctl->status; every
// thread of the CTA gets the same answer (read once into shared memory).
// (GridCtl itself, a plain struct the host allocates, is in internal.h.)

__device__ __forceinline__ unsigned int atom_add_acq_rel_gpu(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Arrival is an acq_rel atomic (it publishes, cumulatively, every write the CTA
// made before the __syncthreads); waiting is an acquire load of the
// generation, so no separate fences are needed.
__device__ __forceinline__ bool grid_sync_bounded(GridCtl* ctl, long long limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g = ld_acquire_gpu(&ctl->gen);
    if (atom_add_acq_rel_gpu(&ctl->count, 1u) == gridDim.x - 1) {
      ctl->count = 0u;  // ordered before the release below; nobody arrives again until it
      atom_add_acq_rel_gpu(&ctl->gen, 1u);
    } else {
      const long long start = clock64();
      while (ld_acquire_gpu(&ctl->gen) == g) {
        if (clock64() - start > limit) {
          atomicExch(&ctl->status, 1);
          break;
        }
      }
    }
    s_ok = ld_acquire_gpu((const unsigned int*)&ctl->status) == 0u;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace ising
