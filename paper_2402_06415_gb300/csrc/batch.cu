// Batched replicas with parallel tempering: one persistent cooperative launch.
//
// n_ladders ladders, each of n_beta replicas of one lattice size L_l, run the
// checkerboard Metropolis sweep (arXiv 2402.06415, Results A / Supplementary
// MC steps 1-3) at the temperature of their current slot; after every
// pt_every sweeps each ladder exchanges configurations between adjacent
// temperature slots (replica exchange; not in the paper).  Replica i of
// ladder l has Philox replica id l * n_beta + i, so every replica's chain is
// exactly the single-lattice chain of that id with its beta changing between
// rounds.
//
// Work: a round (sweeps between two exchange steps) of a group of replicas of
// one ladder is an "item"; items are assigned to CTAs on the host (largest
// first, to the least loaded CTA).  A CTA loads an item's replicas into shared
// memory, runs the round there, measures E and M, and writes them back.  A
// grid-wide barrier (bounded spin; on timeout the kernel sets a status word
// and returns) separates rounds from exchange steps.  The sweep counter and
// the exchange-step counter live in device memory, so a CUDA graph that
// captured one launch continues the chain on every replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <queue>
#include <string>
#include <vector>

#include "internal.h"
#include "ising.h"
#include "ising_device.cuh"

namespace ising {
namespace {

constexpr int kMaxRepPerItem = 64;

struct BatchCounters {
  unsigned int bar_count;
  unsigned int bar_gen;
  int status;      // 0 ok, 1 barrier timeout, 2 internal (odd energy difference)
  unsigned int sweep;  // next sweep index
  long long launches;
};

struct BatchDev {
  uint32_t* spins;
  const long long* off;  // word offset of replica r
  const int* lad_L;      // L of ladder l
  const uint32_t* t4;    // thresholds per temperature slot
  const uint32_t* t8;
  const double* q;       // exp(-4 (beta[a+1] - beta[a])) per adjacent pair
  int* perm;             // [ladder][slot] -> replica index in the ladder
  int* slot_of;          // [ladder][replica] -> slot
  int* E;                // per replica, after its last round
  int* M;
  unsigned long long* acc;  // [ladder][slot a] accepted exchanges of pair (a, a+1)
  unsigned long long* att;
  int* ser_E;            // [cap][n_rep] energies at exchange steps (or null)
  int* ser_M;
  short* ser_slot;       // slot the replica sampled during that round
  int ser_cap;
  const int* item_ladder;
  const int* item_i0;
  const int* item_nr;
  const int* cta_first;  // CSR over CTAs
  const int* cta_items;
  BatchCounters* ctr;
  int n_ladders, n_beta, pt_every;
  uint32_t key0, key1;
  uint32_t rk0[10], rk1[10];  // Philox round keys of (key0, key1)
  long long spin_limit;  // clock64 cycles a barrier may wait
};

__device__ bool grid_barrier(const BatchDev& d) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = &d.ctr->bar_gen;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&d.ctr->bar_count, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(&d.ctr->bar_count, 0u);
      __threadfence();
      atomicAdd(&d.ctr->bar_gen, 1u);
    } else if (!bounded_wait_while_eq(gen, g, d.spin_limit)) {
      atomicExch(&d.ctr->status, 1);
    }
    __threadfence();
  }
  __syncthreads();
  return *((volatile int*)&d.ctr->status) == 0;
}


// Side word (the x-neighbours of the other colour, as side_word) and valid
// mask without branches: the 32 lanes of a warp hold words of several rows,
// so they disagree on the row parity and on first / last word, and a branch
// would run both ways.
__device__ __forceinline__ uint32_t side_word_bf(const uint32_t* rm, int w, int Wc, int n, int o) {
  const int nb = n - 32 * (Wc - 1);
  const uint32_t cur = rm[w];
  const uint32_t prevw = rm[w > 0 ? w - 1 : Wc - 1];
  const uint32_t nextw = rm[w < Wc - 1 ? w + 1 : 0];
  const uint32_t c0 = w > 0 ? (prevw >> 31) : ((prevw >> (nb - 1)) & 1u);
  const uint32_t c1 = w < Wc - 1 ? (nextw << 31) : ((nextw & 1u) << (nb - 1));
  return o == 0 ? ((cur << 1) | c0) : ((cur >> 1) | c1);
}
__device__ __forceinline__ uint32_t valid_mask_bf(int w, int Wc, int n) {
  const int nb = n - 32 * (Wc - 1);
  const uint32_t last = nb >= 32 ? 0xffffffffu : ((1u << (nb & 31)) - 1u);
  return w < Wc - 1 ? 0xffffffffu : last;
}
constexpr int kQueueCap = 512;  // undecided words per half sweep finished by whole warps

// Bit-plane compare of Philox blocks B0 .. B1-1 for the undecided lanes D of one
// word, with the replica's per-plane threshold masks tm[k] = (all ones iff bit
// 31 - k of t4, the same for t8) read from shared memory; cls marks the lanes
// that test against t4.  VOTE: stop once no lane of the warp is undecided
// (every lane of the warp must call it); without it every block is drawn.
template <int B0, int B1, bool VOTE>
__device__ __forceinline__ void planes_tab(uint32_t g, uint32_t t, uint32_t rep, uint32_t colour,
                                           const uint32_t (&rk0)[10], const uint32_t (&rk1)[10],
                                           const uint2* __restrict__ tm, uint32_t& D, uint32_t cls,
                                           uint32_t& acc) {
#pragma unroll
  for (int b = B0; b < B1; ++b) {
    if (VOTE && !__any_sync(0xffffffffu, D != 0u)) break;
    const uint4 r = philox10_rk(make_uint4(g, t, rep, ctr_w(kTagMet, colour, b)), rk0, rk1);
    const uint32_t p[4] = {r.x, r.y, r.z, r.w};
    // the block's 4 planes as one 4-bit comparison (borrow of u - T from the
    // block's last plane up, equality chain), then merged into (acc, D)
    uint32_t bor = 0u, eq = D;
#pragma unroll
    for (int q = 3; q >= 0; --q) {
      const uint2 m = tm[4 * b + q];
      const uint32_t tk = (cls & m.x) | (~cls & m.y);  // lane's threshold bit
      bor = (~p[q] & tk) | (~p[q] & bor) | (tk & bor);
      eq &= ~(tk ^ p[q]);
    }
    acc |= D & bor;
    D = eq;
  }
}

// Planes 0..7 (Philox blocks 0 and 1) of two independent words (two replicas'
// masks), all drawn, as one strict comparison of the top 8 bits: u_8 < T_8 is
// the borrow out of the bit-sliced subtraction u_8 - T_8, carried from plane 7
// up to plane 0 with one majority function per plane, borrow' = maj(~u_k, T_k,
// borrow); lanes whose 8 bits equal the threshold's stay undecided.  Same
// (acc, D) as planes_tab<0, 2, false> with one logic operation less per plane;
// block 1 is drawn first so that one block's planes are live at a time.
__device__ __forceinline__ void planes8_tab2(uint32_t ga, uint32_t gb, uint32_t t, uint32_t repa, uint32_t repb,
                                             uint32_t colour, const uint32_t (&rk0)[10], const uint32_t (&rk1)[10],
                                             const uint2* __restrict__ tma, const uint2* __restrict__ tmb,
                                             uint32_t& Da, uint32_t clsa, uint32_t& acca,
                                             uint32_t& Db, uint32_t clsb, uint32_t& accb) {
  uint32_t bora = 0u, borb = 0u, eqa = Da, eqb = Db;
#pragma unroll
  for (int b = 1; b >= 0; --b) {
    const uint32_t cw = ctr_w(kTagMet, colour, b);
    const uint4 ra = philox10_rk(make_uint4(ga, t, repa, cw), rk0, rk1);
    const uint4 rb = philox10_rk(make_uint4(gb, t, repb, cw), rk0, rk1);
    const uint32_t pa[4] = {ra.x, ra.y, ra.z, ra.w};
    const uint32_t pb[4] = {rb.x, rb.y, rb.z, rb.w};
#pragma unroll
    for (int q = 3; q >= 0; --q) {
      const uint2 ma = tma[4 * b + q], mb = tmb[4 * b + q];
      const uint32_t ta = (clsa & ma.x) | (~clsa & ma.y);
      const uint32_t tb = (clsb & mb.x) | (~clsb & mb.y);
      bora = (~pa[q] & ta) | (~pa[q] & bora) | (ta & bora);
      borb = (~pb[q] & tb) | (~pb[q] & borb) | (tb & borb);
      eqa &= ~(ta ^ pa[q]);
      eqb &= ~(tb ^ pb[q]);
    }
  }
  acca |= Da & bora;
  accb |= Db & borb;
  Da = eqa;
  Db = eqb;
}

// One round (ns sweeps from global sweep t0) of one item, in shared memory.
struct ItemSmem {
  uint2 tm[kMaxRepPerItem][32];  // per replica and plane: threshold masks (t4, t8)
  uint32_t q_idx[kQueueCap], q_d[kQueueCap], q_cls[kQueueCap];
  int q_n[2];
};

__device__ void run_item(const BatchDev& d, int item, uint32_t t0, int ns, bool record,
                         uint32_t step, uint32_t* sm, uint32_t* s_t4, uint32_t* s_t8,
                         unsigned int* s_anti, unsigned int* s_ones, ItemSmem& X) {
  const int l = d.item_ladder[item], i0 = d.item_i0[item], nr = d.item_nr[item];
  const int L = d.lad_L[l];
  const int Wc = (L / 2 + 31) / 32, n = L / 2;
  const int plane = L * Wc, per_rep = 2 * plane;
  const int r0 = l * d.n_beta + i0;
  const long long base = d.off[r0];
  const int total = nr * per_rep;
  for (int i = threadIdx.x; i < total; i += blockDim.x) sm[i] = d.spins[base + i];
  for (int qq = threadIdx.x; qq < nr; qq += blockDim.x) {
    // written by other CTAs' exchange steps: read through L2, not a stale L1 line
    const int slot = __ldcg(&d.slot_of[l * d.n_beta + i0 + qq]);
    s_t4[qq] = d.t4[slot];
    s_t8[qq] = d.t8[slot];
    s_anti[qq] = 0u;
    s_ones[qq] = 0u;
  }
  if (threadIdx.x < 2) X.q_n[threadIdx.x] = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < nr * 32; e += blockDim.x) {
    const int qq = e >> 5, k = e & 31;
    X.tm[qq][k] = make_uint2(0u - ((s_t4[qq] >> (31 - k)) & 1u), 0u - ((s_t8[qq] >> (31 - k)) & 1u));
  }
  __syncthreads();
  // Half sweeps in two phases, as in the single-lattice tiled kernel: phase 1
  // draws the first two Philox blocks (8 planes) of every word and queues the
  // words with lanes still undecided (~7 %); phase 2 finishes the queued words
  // with every lane of a warp on one of them, instead of each warp waiting for
  // its slowest word.  (Warp-owned replicas with only __syncwarp() between half
  // sweeps measured slower: too few resident warps per SM for this many
  // replicas.)
  const int lane = threadIdx.x & 31;
  const int words = nr * plane;
  const int half = plane / 2, pairs = nr * half;  // word pairs (rows 2 yy, 2 yy + 1)
  const FastDiv fplane = make_fastdiv((uint32_t)plane), fwc = make_fastdiv((uint32_t)Wc);
  const FastDiv fhalf = make_fastdiv((uint32_t)half);
  for (int s = 0; s < ns; ++s) {
    const uint32_t t = t0 + (uint32_t)s;
    for (int c = 0; c < 2; ++c) {
      const int cur = c;  // queue counter of this half sweep (the other is reset meanwhile)
      auto enq = [&](int idx, uint32_t D, uint32_t cls) {  // returns true if the queue was full
        if (D == 0u) return false;
        const int slot = atomicAdd(&X.q_n[cur], 1);
        if (slot < kQueueCap) {
          X.q_idx[slot] = (uint32_t)idx;
          X.q_d[slot] = D;
          X.q_cls[slot] = cls;
          return false;
        }
        return true;
      };
      // two vertically adjacent words of one replica per lane (rows 2 yy and
      // 2 yy + 1; L is even): they share the other colour's rows 2 yy, 2 yy + 1
      // as neighbours (and the half sum of that pair), the replica and the
      // index division, and their two Philox chains interleave; 80 registers
      // keep three CTAs of 256 threads per SM
      for (int p0 = threadIdx.x & ~31; p0 < pairs; p0 += blockDim.x) {
        const int p = p0 + lane;
        const bool act = p < pairs;
        const int qq = act ? (int)fdiv((uint32_t)p, fhalf) : 0;
        const int rem = act ? p - qq * half : 0;
        const int yy = (int)fdiv((uint32_t)rem, fwc), w = rem - yy * Wc;
        const int ya = 2 * yy;
        uint32_t* So = sm + qq * per_rep + c * plane;
        const uint32_t* Sn = sm + qq * per_rep + (1 - c) * plane;
        const uint32_t* rowa = Sn + ya * Wc;  // other colour, rows ya and ya + 1
        const uint32_t* rowb = rowa + Wc;
        const int pa = ya * Wc + w, pb = pa + Wc;
        const uint32_t sa = So[pa], sb = So[pb];
        const uint32_t u0 = Sn[(ya == 0 ? L - 1 : ya - 1) * Wc + w];
        const uint32_t m0 = rowa[w], m1 = rowb[w];
        const uint32_t d1 = Sn[(ya + 2 == L ? 0 : ya + 2) * Wc + w];
        // x-offset (y + c) & 1: c for the even row ya, the other for ya + 1
        const uint32_t side_a = side_word_bf(rowa, w, Wc, n, c);
        const uint32_t side_b = side_word_bf(rowb, w, Wc, n, c ^ 1);
        const uint32_t valid = act ? valid_mask_bf(w, Wc, n) : 0u;
        const uint32_t h01 = m0 ^ m1;
        const HalfClasses ka = classify_hs(sa, h01, m0, m1, u0, side_a);
        const HalfClasses kb = classify_hs(sb, h01, m0, m1, d1, side_b);
        uint32_t Da = ~ka.ge2 & valid, Db = ~kb.ge2 & valid, acca = 0, accb = 0;
        const uint32_t rep = (uint32_t)(r0 + qq);
        planes8_tab2((uint32_t)pa, (uint32_t)pb, t, rep, rep, (uint32_t)c, d.rk0, d.rk1, X.tm[qq], X.tm[qq],
                     Da, ka.cls, acca, Db, kb.cls, accb);
        if (act) {
          So[pa] = sa ^ ((ka.ge2 & valid) | acca);
          So[pb] = sb ^ ((kb.ge2 & valid) | accb);
        }
        const bool ovfa = enq(qq * plane + pa, Da, ka.cls);
        const bool ovfb = enq(qq * plane + pb, Db, kb.cls);
        if (__any_sync(0xffffffffu, ovfa || ovfb)) {  // queue full: finish in place
          uint32_t ea = ovfa ? Da : 0u, eb = ovfb ? Db : 0u, xa = 0, xb = 0;
          planes_tab<2, 8, true>((uint32_t)pa, t, rep, (uint32_t)c, d.rk0, d.rk1, X.tm[qq], ea, ka.cls, xa);
          planes_tab<2, 8, true>((uint32_t)pb, t, rep, (uint32_t)c, d.rk0, d.rk1, X.tm[qq], eb, kb.cls, xb);
          if (ovfa) So[pa] ^= xa;
          if (ovfb) So[pb] ^= xb;
        }
      }
      __syncthreads();
      const int nq = min(X.q_n[cur], kQueueCap);
      if (threadIdx.x == 0) X.q_n[cur ^ 1] = 0;
      for (int b0 = threadIdx.x & ~31; b0 < nq; b0 += blockDim.x) {
        const int e = b0 + lane;
        const bool act = e < nq;
        const int idx = act ? (int)X.q_idx[e] : 0;
        uint32_t D = act ? X.q_d[e] : 0u, acc = 0;
        const uint32_t cls = act ? X.q_cls[e] : 0u;
        const int qq = (int)fdiv((uint32_t)idx, fplane);
        const int rem = idx - qq * plane;
        const int y = (int)fdiv((uint32_t)rem, fwc), w = rem - y * Wc;
        planes_tab<2, 8, true>((uint32_t)(y * Wc + w), t, (uint32_t)(r0 + qq), (uint32_t)c, d.rk0, d.rk1,
                               X.tm[qq], D, cls, acc);
        if (act && acc) sm[qq * per_rep + c * plane + y * Wc + w] ^= acc;
      }
      __syncthreads();
    }
  }
  // observables of the new configurations: bonds of every colour-0 site
  for (int idx = threadIdx.x; idx < words; idx += blockDim.x) {
    const int qq = idx / plane, rem = idx - (idx / plane) * plane;
    const int y = rem / Wc, w = rem - (rem / Wc) * Wc;
    const uint32_t* P0 = sm + qq * per_rep;
    const uint32_t* P1 = P0 + plane;
    const uint32_t* rm = P1 + y * Wc;
    const uint32_t valid = valid_mask_bf(w, Wc, n);
    const uint32_t sv = P0[y * Wc + w];
    const uint32_t up = P1[(y == 0 ? L - 1 : y - 1) * Wc + w];
    const uint32_t dn = P1[(y == L - 1 ? 0 : y + 1) * Wc + w];
    const uint32_t mid = rm[w];
    const uint32_t side = side_word_bf(rm, w, Wc, n, y & 1);
    const unsigned int a = __popc((sv ^ up) & valid) + __popc((sv ^ dn) & valid) +
                           __popc((sv ^ mid) & valid) + __popc((sv ^ side) & valid);
    const unsigned int o = __popc(sv & valid) + __popc(mid & valid);
    atomicAdd(&s_anti[qq], a);
    atomicAdd(&s_ones[qq], o);
  }
  __syncthreads();
  const int N = L * L;
  for (int qq = threadIdx.x; qq < nr; qq += blockDim.x) {
    const int r = r0 + qq;
    const int e = 2 * (int)s_anti[qq] - 2 * N;
    const int m = 2 * (int)s_ones[qq] - N;
    d.E[r] = e;
    d.M[r] = m;
    if (record && d.ser_E) {
      const size_t row = (size_t)(step % (uint32_t)d.ser_cap) * (size_t)(d.n_ladders * d.n_beta);
      d.ser_E[row + r] = e;
      d.ser_M[row + r] = m;
      d.ser_slot[row + r] = (short)__ldcg(&d.slot_of[l * d.n_beta + i0 + qq]);
    }
  }
  for (int i = threadIdx.x; i < total; i += blockDim.x) d.spins[base + i] = sm[i];
  __syncthreads();
}

// Exchange step n_step of ladder l: pairs (a, a+1), a = n_step & 1, +2, ...
// Accept iff u < floor(min(1, exp[(b_a - b_{a+1})(E_a - E_{a+1})]) 2^32).  With
// ascending betas the exponent is >= 0 iff E_a <= E_{a+1}; otherwise it equals
// -4 m (b_{a+1} - b_a) with m = (E_a - E_{a+1}) / 4 (energy differences are
// multiples of 4 on an even periodic lattice), and exp of it is q_a^m, formed by
// repeated squaring: no transcendental function runs on the device.
__device__ void exchange_ladder(const BatchDev& d, int l, uint32_t n_step) {
  const int nb = d.n_beta;
  const int par = (int)(n_step & 1u);
  for (int p = threadIdx.x;; p += blockDim.x) {
    const int a = 2 * p + par;
    if (a + 1 >= nb) break;
    int* perm = d.perm + l * nb;
    // perm and E were written by other CTAs before the grid barrier: bypass L1
    const int ra = __ldcg(&perm[a]), rb = __ldcg(&perm[a + 1]);
    const int diff = __ldcg(&d.E[l * nb + ra]) - __ldcg(&d.E[l * nb + rb]);
    bool accept = true;
    if (diff > 0) {
      if (diff & 3) {
        atomicExch(&d.ctr->status, 2);
        accept = false;
      } else {
        unsigned int m = (unsigned int)(diff >> 2);
        double x = 1.0, b = d.q[a];
        while (m) {
          if (m & 1u) x = __dmul_rn(x, b);
          b = __dmul_rn(b, b);
          m >>= 1;
        }
        const double tf = floor(__dmul_rn(x, 4294967296.0));
        const unsigned long long thr = tf <= 0.0 ? 0ull : (unsigned long long)tf;
        const uint4 r = philox10(make_uint4((uint32_t)a, n_step, (uint32_t)l, ctr_w(kTagPT, 0, 0)),
                                 d.key0, d.key1);
        accept = (unsigned long long)r.x < thr;
      }
    }
    d.att[l * nb + a] += 1ull;
    if (accept) {
      perm[a] = rb;
      perm[a + 1] = ra;
      d.slot_of[l * nb + rb] = a;
      d.slot_of[l * nb + ra] = a + 1;
      d.acc[l * nb + a] += 1ull;
    }
  }
}

__global__ void __launch_bounds__(256, 3) k_batch(BatchDev d, int n_sweeps) {
  extern __shared__ uint32_t sm[];
  __shared__ uint32_t s_t4[kMaxRepPerItem], s_t8[kMaxRepPerItem];
  __shared__ unsigned int s_anti[kMaxRepPerItem], s_ones[kMaxRepPerItem];
  __shared__ ItemSmem X;
  if (*((volatile int*)&d.ctr->status) != 0) return;
  const uint32_t sweep0 = *((volatile unsigned int*)&d.ctr->sweep);
  const int j0 = d.cta_first[blockIdx.x], j1 = d.cta_first[blockIdx.x + 1];
  int done = 0;
  while (done < n_sweeps) {
    const uint32_t tg = sweep0 + (uint32_t)done;
    const int to_pt = d.pt_every - (int)(tg % (uint32_t)d.pt_every);
    const int ns = min(to_pt, n_sweeps - done);
    const bool at_pt = ns == to_pt;
    const uint32_t step = (tg + (uint32_t)ns) / (uint32_t)d.pt_every - 1u;
    for (int j = j0; j < j1; ++j)
      run_item(d, d.cta_items[j], tg, ns, at_pt, step, sm, s_t4, s_t8, s_anti, s_ones, X);
    done += ns;
    if (!grid_barrier(d)) return;
    if (at_pt) {
      for (int l = blockIdx.x; l < d.n_ladders; l += gridDim.x) exchange_ladder(d, l, step);
      if (!grid_barrier(d)) return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.ctr->sweep = sweep0 + (uint32_t)n_sweeps;
    d.ctr->launches += 1;
  }
}

// Waits on a word nothing writes, with the same bounded spin as the grid
// barrier; records 1 in *status when the budget runs out.
__global__ void k_wait_selftest(const unsigned int* never_set, long long limit, int* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    if (!bounded_wait_while_eq(never_set, 0u, limit)) *status = 1;
}

__global__ void k_batch_init(uint32_t* spins, const long long* off, const int* lad_L, int n_beta,
                             int n_rep, uint32_t key0, uint32_t key1) {
  // one thread per (replica, word); grid-stride over replicas, block-stride over words
  for (int r = blockIdx.x; r < n_rep; r += gridDim.x) {
    const int L = lad_L[r / n_beta];
    const int Wc = (L / 2 + 31) / 32, n = L / 2;
    const int plane = L * Wc;
    for (int i = threadIdx.x; i < 2 * plane; i += blockDim.x) {
      const int c = i / plane, rem = i - (i / plane) * plane;
      const int y = rem / Wc, w = rem - (rem / Wc) * Wc;
      const uint4 v = philox10(make_uint4((uint32_t)(y * Wc + w), 0u, (uint32_t)r,
                                          ctr_w(kTagInit, (uint32_t)c, 0)),
                               key0, key1);
      spins[off[r] + i] = v.x & valid_mask(w, Wc, n);
    }
  }
}

}  // namespace
}  // namespace ising

using namespace ising;

struct ising_batch {
  int n_ladders = 0, n_beta = 0, pt_every = 1, n_rep = 0;
  std::vector<int> L;
  std::vector<double> betas;
  std::vector<long long> off;
  long long total_words = 0;
  uint64_t seed = 0;
  int64_t sweep = 0;
  cudaStream_t stream = nullptr;
  int words_per_item = 512, threads = 256, grid = 0, grid_used = 0;
  size_t smem = 0;
  int ser_cap = 0;
  // device
  uint32_t* spins = nullptr;
  long long* d_off = nullptr;
  int* d_L = nullptr;
  uint32_t *d_t4 = nullptr, *d_t8 = nullptr;
  double* d_q = nullptr;
  int *d_perm = nullptr, *d_slot = nullptr, *d_E = nullptr, *d_M = nullptr;
  unsigned long long *d_acc = nullptr, *d_att = nullptr;
  int *d_serE = nullptr, *d_serM = nullptr;
  short* d_serS = nullptr;
  int *d_item_l = nullptr, *d_item_i0 = nullptr, *d_item_nr = nullptr;
  int *d_cta_first = nullptr, *d_cta_items = nullptr;
  BatchCounters* d_ctr = nullptr;
  int n_items = 0;
  // learned block proposal on every replica
  __nv_bfloat16 *nn_w = nullptr, *nn_w2t = nullptr;
  float* d_beta_slot = nullptr;
  long long* d_unit0 = nullptr;
  int unit_B = 0;
  long long unit_total = 0;
  unsigned long long* d_blk_stats = nullptr;
  int64_t block_passes = 0;
  int proposal = 0;                  // ISING_PROPOSAL_ONESHOT / _STAGED
  int nn_engine = 0;                 // ISING_NN_ENGINE_MMA_SYNC / _TCGEN05 (staged proposal)
  nnc::StagedPlan* plan = nullptr;   // device plan of the staged proposal
  int plan_B = 0;
  // captured graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_sweeps = -1;
};

namespace {

int bfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

#define BTRY(expr)                                                                       \
  do {                                                                                   \
    cudaError_t e__ = (expr);                                                            \
    if (e__ != cudaSuccess)                                                              \
      return bfail(ISING_ECUDA, "%s: %s", #expr, cudaGetErrorString(e__));               \
  } while (0)

template <typename T>
int balloc(T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T) > 0 ? count * sizeof(T) : 1);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return bfail(ISING_ENOMEM, "cudaMalloc(%zu): %s", count * sizeof(T), cudaGetErrorString(e));
  }
  return ISING_OK;
}

void bfree(ising_batch* b) {
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  void* ptrs[] = {b->spins, b->d_off, b->d_L, b->d_t4, b->d_t8, b->d_q, b->d_perm, b->d_slot,
                  b->d_E, b->d_M, b->d_acc, b->d_att, b->d_serE, b->d_serM, b->d_serS,
                  b->d_item_l, b->d_item_i0, b->d_item_nr, b->d_cta_first, b->d_cta_items,
                  b->d_ctr, b->nn_w, b->nn_w2t, b->d_beta_slot, b->d_unit0, b->d_blk_stats, b->plan};
  for (void* p : ptrs) cudaFree(p);
}

int words_per_replica(int L) { return 2 * L * ((L / 2 + 31) / 32); }

// Items and their assignment to CTAs (largest first to the least loaded CTA).
int plan_items(ising_batch* b) {
  std::vector<int> il, ii0, inr;
  std::vector<long long> cost;
  for (int l = 0; l < b->n_ladders; ++l) {
    const int per = words_per_replica(b->L[l]) / 2;  // words per colour plane
    int nr = std::max(1, b->words_per_item / std::max(per, 1));
    nr = std::min(nr, kMaxRepPerItem);
    for (int i0 = 0; i0 < b->n_beta; i0 += nr) {
      const int k = std::min(nr, b->n_beta - i0);
      il.push_back(l);
      ii0.push_back(i0);
      inr.push_back(k);
      cost.push_back((long long)k * per);
    }
  }
  b->n_items = (int)il.size();
  size_t max_words = 0;
  for (int j = 0; j < b->n_items; ++j)
    max_words = std::max(max_words, (size_t)inr[j] * words_per_replica(b->L[il[j]]));
  b->smem = max_words * sizeof(uint32_t);
  if (b->smem > 200 * 1024) return bfail(ISING_EINVAL, "an item needs %zu B of shared memory", b->smem);
  BTRY(cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
  int dev = 0, sms = 0, per_sm = 0;
  BTRY(cudaGetDevice(&dev));
  BTRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BTRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, b->threads, b->smem));
  if (per_sm < 1) return bfail(ISING_EINVAL, "kernel does not fit on an SM with this item size");
  int grid = per_sm * sms;
  if (b->grid > 0) grid = std::min(grid, b->grid);
  grid = std::max(1, std::min(grid, std::max(b->n_items, b->n_ladders)));
  b->grid_used = grid;
  std::vector<int> order(b->n_items);
  for (int j = 0; j < b->n_items; ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  using P = std::pair<long long, int>;
  std::priority_queue<P, std::vector<P>, std::greater<P>> pq;
  for (int c = 0; c < grid; ++c) pq.push({0, c});
  std::vector<std::vector<int>> per_cta(grid);
  for (int j : order) {
    P top = pq.top();
    pq.pop();
    per_cta[top.second].push_back(j);
    pq.push({top.first + cost[j], top.second});
  }
  std::vector<int> first(grid + 1, 0), items;
  for (int c = 0; c < grid; ++c) {
    first[c] = (int)items.size();
    items.insert(items.end(), per_cta[c].begin(), per_cta[c].end());
  }
  first[grid] = (int)items.size();
  cudaFree(b->d_item_l);
  cudaFree(b->d_item_i0);
  cudaFree(b->d_item_nr);
  cudaFree(b->d_cta_first);
  cudaFree(b->d_cta_items);
  b->d_item_l = b->d_item_i0 = b->d_item_nr = b->d_cta_first = b->d_cta_items = nullptr;
  if (int st = balloc(&b->d_item_l, il.size())) return st;
  if (int st = balloc(&b->d_item_i0, il.size())) return st;
  if (int st = balloc(&b->d_item_nr, il.size())) return st;
  if (int st = balloc(&b->d_cta_first, first.size())) return st;
  if (int st = balloc(&b->d_cta_items, items.size())) return st;
  BTRY(cudaMemcpy(b->d_item_l, il.data(), il.size() * 4, cudaMemcpyHostToDevice));
  BTRY(cudaMemcpy(b->d_item_i0, ii0.data(), ii0.size() * 4, cudaMemcpyHostToDevice));
  BTRY(cudaMemcpy(b->d_item_nr, inr.data(), inr.size() * 4, cudaMemcpyHostToDevice));
  BTRY(cudaMemcpy(b->d_cta_first, first.data(), first.size() * 4, cudaMemcpyHostToDevice));
  BTRY(cudaMemcpy(b->d_cta_items, items.data(), items.size() * 4, cudaMemcpyHostToDevice));
  return ISING_OK;
}

BatchDev dev_view(const ising_batch* b) {
  BatchDev d;
  d.spins = b->spins;
  d.off = b->d_off;
  d.lad_L = b->d_L;
  d.t4 = b->d_t4;
  d.t8 = b->d_t8;
  d.q = b->d_q;
  d.perm = b->d_perm;
  d.slot_of = b->d_slot;
  d.E = b->d_E;
  d.M = b->d_M;
  d.acc = b->d_acc;
  d.att = b->d_att;
  d.ser_E = b->d_serE;
  d.ser_M = b->d_serM;
  d.ser_slot = b->d_serS;
  d.ser_cap = b->ser_cap;
  d.item_ladder = b->d_item_l;
  d.item_i0 = b->d_item_i0;
  d.item_nr = b->d_item_nr;
  d.cta_first = b->d_cta_first;
  d.cta_items = b->d_cta_items;
  d.ctr = b->d_ctr;
  d.n_ladders = b->n_ladders;
  d.n_beta = b->n_beta;
  d.pt_every = b->pt_every;
  d.key0 = (uint32_t)(b->seed & 0xffffffffu);
  d.key1 = (uint32_t)(b->seed >> 32);
  {
    const RngParams rp = make_rng(b->seed, 0, 0, 0);
    for (int r = 0; r < 10; ++r) {
      d.rk0[r] = rp.rk0[r];
      d.rk1[r] = rp.rk1[r];
    }
  }
  d.spin_limit = 4000000000ll;  // ~2 s at 2 GHz
  return d;
}

cudaError_t launch_batch(ising_batch* b, int n_sweeps) {
  BatchDev d = dev_view(b);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->grid_used);
  cfg.blockDim = dim3(b->threads);
  cfg.dynamicSmemBytes = b->smem;
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch, d, n_sweeps);
}

int check_b(ising_batch* b) {
  if (!b) return bfail(ISING_EINVAL, "null batch");
  return ISING_OK;
}

}  // namespace

extern "C" {

int ising_batch_create(ising_batch** out, int n_ladders, const int* L, int n_beta,
                       const double* betas, int pt_every, void* stream) {
  if (!out) return bfail(ISING_EINVAL, "null output pointer");
  *out = nullptr;
  if (n_ladders < 1 || n_beta < 1 || !L || !betas)
    return bfail(ISING_EINVAL, "need n_ladders >= 1, n_beta >= 1 and non-null L, betas");
  if (n_beta > 4096 || n_ladders > (1 << 20)) return bfail(ISING_EINVAL, "too many replicas");
  if (pt_every < 1) return bfail(ISING_EINVAL, "pt_every must be >= 1");
  for (int l = 0; l < n_ladders; ++l)
    if (L[l] < 4 || L[l] > 1024 || (L[l] & 1))
      return bfail(ISING_EINVAL, "ladder %d: L must be even and in [4, 1024] (got %d)", l, L[l]);
  for (int a = 0; a < n_beta; ++a) {
    if (!std::isfinite(betas[a]) || betas[a] <= 0)
      return bfail(ISING_EINVAL, "betas must be finite and > 0");
    if (a > 0 && betas[a] < betas[a - 1]) return bfail(ISING_EINVAL, "betas must be ascending");
  }
  ising_batch* b = new (std::nothrow) ising_batch();
  if (!b) return bfail(ISING_ENOMEM, "host allocation failed");
  b->n_ladders = n_ladders;
  b->n_beta = n_beta;
  b->pt_every = pt_every;
  b->n_rep = n_ladders * n_beta;
  b->L.assign(L, L + n_ladders);
  b->betas.assign(betas, betas + n_beta);
  b->stream = (cudaStream_t)stream;
  b->off.resize(b->n_rep);
  long long o = 0;
  for (int r = 0; r < b->n_rep; ++r) {
    b->off[r] = o;
    o += words_per_replica(b->L[r / n_beta]);
  }
  b->total_words = o;
  std::vector<uint32_t> t4(n_beta), t8(n_beta);
  std::vector<double> q(std::max(n_beta - 1, 1), 1.0);
  for (int a = 0; a < n_beta; ++a) ising_thresholds(betas[a], &t4[a], &t8[a]);
  for (int a = 0; a + 1 < n_beta; ++a) q[a] = std::exp(-4.0 * (betas[a + 1] - betas[a]));
  int st = ISING_OK;
  auto A = [&](auto** p, size_t n) {
    if (!st) st = balloc(p, n);
  };
  A(&b->spins, (size_t)o);
  A(&b->d_off, (size_t)b->n_rep);
  A(&b->d_L, (size_t)n_ladders);
  A(&b->d_t4, (size_t)n_beta);
  A(&b->d_t8, (size_t)n_beta);
  A(&b->d_q, q.size());
  A(&b->d_perm, (size_t)b->n_rep);
  A(&b->d_slot, (size_t)b->n_rep);
  A(&b->d_E, (size_t)b->n_rep);
  A(&b->d_M, (size_t)b->n_rep);
  A(&b->d_acc, (size_t)b->n_rep);
  A(&b->d_att, (size_t)b->n_rep);
  A(&b->d_ctr, 1);
  if (!st) {
    cudaError_t e = cudaSuccess;
    e = cudaMemcpy(b->d_off, b->off.data(), b->off.size() * 8, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(b->d_L, L, (size_t)n_ladders * 4, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(b->d_t4, t4.data(), (size_t)n_beta * 4, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(b->d_t8, t8.data(), (size_t)n_beta * 4, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(b->d_q, q.data(), q.size() * 8, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemset(b->d_ctr, 0, sizeof(BatchCounters));
    if (e) st = bfail(ISING_ECUDA, "batch setup copy: %s", cudaGetErrorString(e));
  }
  if (!st) st = plan_items(b);
  if (st) {
    bfree(b);
    delete b;
    return st;
  }
  *out = b;
  return ising_batch_seed(b, 0);
}

int ising_batch_seed(ising_batch* b, uint64_t seed) {
  if (int st = check_b(b)) return st;
  b->seed = seed;
  b->sweep = 0;
  std::vector<int> perm(b->n_rep);
  for (int r = 0; r < b->n_rep; ++r) perm[r] = r % b->n_beta;
  BTRY(cudaMemcpyAsync(b->d_perm, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice, b->stream));
  BTRY(cudaMemcpyAsync(b->d_slot, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice, b->stream));
  BTRY(cudaMemsetAsync(b->d_acc, 0, (size_t)b->n_rep * 8, b->stream));
  BTRY(cudaMemsetAsync(b->d_att, 0, (size_t)b->n_rep * 8, b->stream));
  BTRY(cudaMemsetAsync(b->d_E, 0, (size_t)b->n_rep * 4, b->stream));
  BTRY(cudaMemsetAsync(b->d_M, 0, (size_t)b->n_rep * 4, b->stream));
  BTRY(cudaMemsetAsync(b->d_ctr, 0, sizeof(BatchCounters), b->stream));
  k_batch_init<<<std::min(b->n_rep, 152 * 16), 256, 0, b->stream>>>(
      b->spins, b->d_off, b->d_L, b->n_beta, b->n_rep, (uint32_t)(seed & 0xffffffffu),
      (uint32_t)(seed >> 32));
  BTRY(cudaGetLastError());
  BTRY(cudaStreamSynchronize(b->stream));
  set_last_error("");
  return ISING_OK;
}

int ising_batch_set_kernel(ising_batch* b, int words_per_item, int threads, int grid) {
  if (int st = check_b(b)) return st;
  if (words_per_item < 16 || words_per_item > 16384)
    return bfail(ISING_EINVAL, "words_per_item must be in [16, 16384]");
  if (threads != 0 && threads != 32 && threads != 64 && threads != 128 && threads != 256)
    return bfail(ISING_EINVAL, "threads must be 32, 64, 128 or 256");
  if (grid < 0) return bfail(ISING_EINVAL, "grid must be >= 0");
  BTRY(cudaStreamSynchronize(b->stream));
  b->words_per_item = words_per_item;
  b->threads = threads ? threads : 256;
  b->grid = grid;
  if (b->graph_exec) {
    cudaGraphExecDestroy(b->graph_exec);
    cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
    b->graph_sweeps = -1;
  }
  if (int st = plan_items(b)) return st;
  set_last_error("");
  return ISING_OK;
}

int ising_batch_set_series(ising_batch* b, int capacity) {
  if (int st = check_b(b)) return st;
  if (capacity < 0) return bfail(ISING_EINVAL, "capacity must be >= 0");
  BTRY(cudaStreamSynchronize(b->stream));
  cudaFree(b->d_serE);
  cudaFree(b->d_serM);
  cudaFree(b->d_serS);
  b->d_serE = b->d_serM = nullptr;
  b->d_serS = nullptr;
  b->ser_cap = 0;
  if (capacity > 0) {
    const size_t n = (size_t)capacity * b->n_rep;
    if (int st = balloc(&b->d_serE, n)) return st;
    if (int st = balloc(&b->d_serM, n)) return st;
    if (int st = balloc(&b->d_serS, n)) return st;
    b->ser_cap = capacity;
  }
  if (b->graph_exec) {  // the graph holds the old pointers
    cudaGraphExecDestroy(b->graph_exec);
    cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
    b->graph_sweeps = -1;
  }
  set_last_error("");
  return ISING_OK;
}

int ising_batch_run(ising_batch* b, int n_sweeps) {
  if (int st = check_b(b)) return st;
  NvtxRange nvtx("ising_batch_run");
  if (n_sweeps < 0) return bfail(ISING_EINVAL, "n_sweeps must be >= 0");
  if (b->sweep + n_sweeps >= ((int64_t)1 << 32)) return bfail(ISING_EINVAL, "sweep counter overflow");
  if (n_sweeps == 0) return ISING_OK;
  if (b->graph_exec && b->graph_sweeps == n_sweeps) {
    BTRY(cudaGraphLaunch(b->graph_exec, b->stream));
  } else {
    BTRY(launch_batch(b, n_sweeps));
  }
  b->sweep += n_sweeps;
  set_last_error("");
  return ISING_OK;
}

int ising_batch_capture(ising_batch* b, int n_sweeps) {
  if (int st = check_b(b)) return st;
  if (n_sweeps < 1) return bfail(ISING_EINVAL, "n_sweeps must be >= 1");
  BTRY(cudaStreamSynchronize(b->stream));
  if (b->graph_exec) {
    cudaGraphExecDestroy(b->graph_exec);
    cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
  }
  cudaStream_t cap;
  BTRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaStream_t saved = b->stream;
  b->stream = cap;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (!e) e = launch_batch(b, n_sweeps);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cap, &g);
  b->stream = saved;
  cudaStreamDestroy(cap);
  if (e || e2) {
    if (g) cudaGraphDestroy(g);
    return bfail(ISING_ECUDA, "graph capture: %s", cudaGetErrorString(e ? e : e2));
  }
  e = cudaGraphInstantiate(&b->graph_exec, g, 0);
  if (e) {
    cudaGraphDestroy(g);
    return bfail(ISING_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  b->graph = g;
  b->graph_sweeps = n_sweeps;
  set_last_error("");
  return ISING_OK;
}

int ising_batch_status(ising_batch* b, int* status, int64_t* sweep) {
  if (int st = check_b(b)) return st;
  BatchCounters h;
  BTRY(cudaMemcpyAsync(&h, b->d_ctr, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
  BTRY(cudaStreamSynchronize(b->stream));
  if (status) *status = h.status;
  if (sweep) *sweep = (int64_t)h.sweep;
  set_last_error("");
  if (h.status == 1) return bfail(ISING_ETIMEOUT, "grid barrier timed out");
  if (h.status == 2) return bfail(ISING_EINTERNAL, "odd energy difference in an exchange");
  return ISING_OK;
}

int ising_batch_state(ising_batch* b, int32_t* perm, int64_t* E, int64_t* M) {
  if (int st = ising_batch_status(b, nullptr, nullptr)) return st;
  std::vector<int> hp(b->n_rep), he(b->n_rep), hm(b->n_rep);
  BTRY(cudaMemcpy(hp.data(), b->d_perm, hp.size() * 4, cudaMemcpyDeviceToHost));
  BTRY(cudaMemcpy(he.data(), b->d_E, he.size() * 4, cudaMemcpyDeviceToHost));
  BTRY(cudaMemcpy(hm.data(), b->d_M, hm.size() * 4, cudaMemcpyDeviceToHost));
  for (int r = 0; r < b->n_rep; ++r) {
    if (perm) perm[r] = hp[r];
    if (E) E[r] = he[r];
    if (M) M[r] = hm[r];
  }
  return ISING_OK;
}

int ising_batch_swap_counts(ising_batch* b, int64_t* accepts, int64_t* attempts) {
  if (int st = ising_batch_status(b, nullptr, nullptr)) return st;
  std::vector<unsigned long long> ha(b->n_rep), ht(b->n_rep);
  BTRY(cudaMemcpy(ha.data(), b->d_acc, ha.size() * 8, cudaMemcpyDeviceToHost));
  BTRY(cudaMemcpy(ht.data(), b->d_att, ht.size() * 8, cudaMemcpyDeviceToHost));
  for (int r = 0; r < b->n_rep; ++r) {
    if (accepts) accepts[r] = (int64_t)ha[r];
    if (attempts) attempts[r] = (int64_t)ht[r];
  }
  return ISING_OK;
}

int ising_batch_series(ising_batch* b, int n_steps, int32_t* E, int32_t* M, int16_t* slot) {
  if (int st = ising_batch_status(b, nullptr, nullptr)) return st;
  const int64_t done = b->sweep / b->pt_every;
  if (n_steps < 0 || n_steps > b->ser_cap || n_steps > done)
    return bfail(ISING_EINVAL, "n_steps exceeds the recorded exchange steps");
  for (int k = 0; k < n_steps; ++k) {
    const int64_t step = done - n_steps + k;
    const size_t row = (size_t)(step % b->ser_cap) * b->n_rep;
    if (E) BTRY(cudaMemcpy(E + (size_t)k * b->n_rep, b->d_serE + row, b->n_rep * 4, cudaMemcpyDeviceToHost));
    if (M) BTRY(cudaMemcpy(M + (size_t)k * b->n_rep, b->d_serM + row, b->n_rep * 4, cudaMemcpyDeviceToHost));
    if (slot) BTRY(cudaMemcpy(slot + (size_t)k * b->n_rep, b->d_serS + row, b->n_rep * 2, cudaMemcpyDeviceToHost));
  }
  return ISING_OK;
}

int ising_batch_get_spins(ising_batch* b, int ladder, int replica, int8_t* host_out) {
  if (int st = check_b(b)) return st;
  if (ladder < 0 || ladder >= b->n_ladders || replica < 0 || replica >= b->n_beta || !host_out)
    return bfail(ISING_EINVAL, "bad ladder / replica / buffer");
  BTRY(cudaStreamSynchronize(b->stream));
  const int L = b->L[ladder], Wc = (L / 2 + 31) / 32;
  const int r = ladder * b->n_beta + replica;
  std::vector<uint32_t> w((size_t)2 * L * Wc);
  BTRY(cudaMemcpy(w.data(), b->spins + b->off[r], w.size() * 4, cudaMemcpyDeviceToHost));
  for (int y = 0; y < L; ++y)
    for (int x = 0; x < L; ++x) {
      const int c = (x + y) & 1, j = x >> 1;
      host_out[y * L + x] = ((w[(size_t)c * L * Wc + (size_t)y * Wc + (j >> 5)] >> (j & 31)) & 1u) ? 1 : -1;
    }
  set_last_error("");
  return ISING_OK;
}

int ising_batch_info(ising_batch* b, int* n_items, int* grid, int64_t* sweep) {
  if (int st = check_b(b)) return st;
  if (n_items) *n_items = b->n_items;
  if (grid) *grid = b->grid_used;
  if (sweep) *sweep = b->sweep;
  set_last_error("");
  return ISING_OK;
}

int ising_batch_nn_load(ising_batch* b, const void* bf16_weights, size_t bytes) {
  if (int st = check_b(b)) return st;
  if (!bf16_weights || bytes != nn_blob_bytes())
    return bfail(ISING_EINVAL, "weights blob must be %zu bytes of bf16", nn_blob_bytes());
  if (!b->nn_w) {
    cudaError_t e = nn_alloc_weights(&b->nn_w, &b->nn_w2t);
    if (!e) e = cudaMalloc((void**)&b->d_beta_slot, (size_t)b->n_beta * sizeof(float));
    if (!e) e = cudaMalloc((void**)&b->d_blk_stats, 3 * sizeof(unsigned long long));
    if (!e) e = cudaMemset(b->d_blk_stats, 0, 3 * sizeof(unsigned long long));
    if (!e) {
      std::vector<float> bf(b->betas.begin(), b->betas.end());
      e = cudaMemcpy(b->d_beta_slot, bf.data(), bf.size() * 4, cudaMemcpyHostToDevice);
    }
    if (e) {
      cudaGetLastError();
      return bfail(ISING_ENOMEM, "batch block-proposal buffers: %s", cudaGetErrorString(e));
    }
  }
  BTRY(nn_load_blob(b->nn_w, b->nn_w2t, bf16_weights, b->stream));
  set_last_error("");
  return ISING_OK;
}

int ising_batch_block_pass(ising_batch* b, int n_passes, int block) {
  if (int st = check_b(b)) return st;
  NvtxRange nvtx("ising_batch_block_pass");
  if (!b->nn_w) return bfail(ISING_EINVAL, "no network loaded (ising_batch_nn_load)");
  if (block != 2 && block != 4 && block != 8 && block != 16)
    return bfail(ISING_EINVAL, "block must be 2, 4, 8 or 16");
  for (int l = 0; l < b->n_ladders; ++l)
    if (b->L[l] % (2 * block) != 0)
      return bfail(ISING_EINVAL, "ladder %d: L = %d is not a multiple of 2 x block", l, b->L[l]);
  if (n_passes < 0) return bfail(ISING_EINVAL, "n_passes must be >= 0");
  if (b->unit_B != block) {
    std::vector<long long> u0(b->n_rep + 1, 0);
    for (int r = 0; r < b->n_rep; ++r) {
      const long long nbx = b->L[r / b->n_beta] / block;
      u0[r + 1] = u0[r] + nbx * nbx / 2;
    }
    cudaFree(b->d_unit0);
    b->d_unit0 = nullptr;
    if (int st = balloc(&b->d_unit0, u0.size())) return st;
    BTRY(cudaMemcpy(b->d_unit0, u0.data(), u0.size() * 8, cudaMemcpyHostToDevice));
    b->unit_B = block;
    b->unit_total = u0[b->n_rep];
  }
  if (b->proposal == ISING_PROPOSAL_STAGED && b->plan_B != block) {
    BTRY(nnc::nn_upload_plan(block, ISING_PROPOSAL_STAGED, &b->plan, nullptr, b->stream));
    b->plan_B = block;
  }
  const RngParams rng = make_rng(b->seed, 0, 0, 0);
  for (int k = 0; k < n_passes; ++k) {
    for (int col = 0; col < 2; ++col) {
      if (b->proposal == ISING_PROPOSAL_STAGED)
        BTRY(nn_batch_staged_block_pass(b->spins, b->d_off, b->d_L, b->d_slot, b->d_beta_slot,
                                        b->d_unit0, b->unit_total, b->n_rep, b->n_beta, b->plan, col,
                                        (uint32_t)b->block_passes, rng, b->nn_engine, b->nn_w,
                                        b->nn_w2t, b->d_blk_stats, b->stream));
      else
        BTRY(nn_batch_block_pass(b->spins, b->d_off, b->d_L, b->d_slot, b->d_beta_slot, b->d_unit0,
                                 b->unit_total, b->n_rep, b->n_beta, block, col,
                                 (uint32_t)b->block_passes, rng, b->nn_w, b->nn_w2t,
                                 b->d_blk_stats, b->stream));
    }
    ++b->block_passes;
  }
  set_last_error("");
  return ISING_OK;
}

int ising_batch_set_proposal(ising_batch* b, int kind) {
  if (int st = check_b(b)) return st;
  if (kind != ISING_PROPOSAL_ONESHOT && kind != ISING_PROPOSAL_STAGED)
    return bfail(ISING_EINVAL, "proposal kind must be ISING_PROPOSAL_ONESHOT or ISING_PROPOSAL_STAGED");
  b->proposal = kind;
  set_last_error("");
  return ISING_OK;
}

int ising_batch_set_nn_engine(ising_batch* b, int engine) {
  if (int st = check_b(b)) return st;
  if (engine != ISING_NN_ENGINE_MMA_SYNC && engine != ISING_NN_ENGINE_TCGEN05)
    return bfail(ISING_EINVAL, "engine must be ISING_NN_ENGINE_MMA_SYNC or ISING_NN_ENGINE_TCGEN05");
  b->nn_engine = engine;
  set_last_error("");
  return ISING_OK;
}

int ising_batch_block_stats(ising_batch* b, int64_t* proposed, int64_t* accepted) {
  if (int st = check_b(b)) return st;
  unsigned long long h[3] = {0, 0, 0};
  if (b->d_blk_stats) {
    BTRY(cudaMemcpyAsync(h, b->d_blk_stats, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
    BTRY(cudaStreamSynchronize(b->stream));
  }
  if (proposed) *proposed = (int64_t)h[0];
  if (accepted) *accepted = (int64_t)h[1];
  if (h[2]) return bfail(ISING_ETIMEOUT, "a block pass gave up waiting for its tensor-core work");
  set_last_error("");
  return ISING_OK;
}

int ising_selftest_wait(double timeout_s, int* device_status) {
  if (!(timeout_s > 0.0 && timeout_s <= 10.0)) return bfail(ISING_EINVAL, "timeout must be in (0, 10] s");
  int dev = 0, khz = 0;
  BTRY(cudaGetDevice(&dev));
  BTRY(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
  const long long limit = (long long)(timeout_s * (double)khz * 1000.0);
  unsigned int* flag = nullptr;
  int* st = nullptr;
  if (int e = balloc(&flag, 1)) return e;
  if (int e = balloc(&st, 1)) {
    cudaFree(flag);
    return e;
  }
  cudaError_t e = cudaMemset(flag, 0, sizeof(unsigned int));
  if (!e) e = cudaMemset(st, 0, sizeof(int));
  if (!e) {
    k_wait_selftest<<<1, 32>>>(flag, limit, st);
    e = cudaGetLastError();
  }
  int h = 0;
  if (!e) e = cudaMemcpy(&h, st, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(flag);
  cudaFree(st);
  if (e) return bfail(ISING_ECUDA, "self-test: %s", cudaGetErrorString(e));
  if (device_status) *device_status = h;
  if (h == 1) return bfail(ISING_ETIMEOUT, "bounded device wait ran out after %.3f s", timeout_s);
  set_last_error("");
  return ISING_OK;
}

int ising_batch_destroy(ising_batch* b) {
  if (!b) return ISING_OK;
  cudaStreamSynchronize(b->stream);
  bfree(b);
  delete b;
  set_last_error("");
  return ISING_OK;
}

}  // extern "C"
