// Temporally blocked (tiled) sweep kernels of the packed lattice and their
// per-K launchers.  Included by one translation unit per K (k_tiled_k<K>.cu),
// each instantiating only its own K so that the large unrolled kernels compile
// in parallel; everything here has internal linkage, and ISING_TILED_INSTANTIATE
// defines the external entry points of one K.
#pragma once
#include "internal.h"
#include "ising_device.cuh"

namespace ising {
namespace {

__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Adds (a, b) over the block to dst[0], dst[1] (one atomic pair per block).
// Every thread of the block must call it.
__device__ void block_add2(unsigned long long a, unsigned long long b, unsigned long long* dst) {
  __shared__ unsigned long long sh[2][32];
  __syncthreads();
  a = warp_sum_u64(a);
  b = warp_sum_u64(b);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh[0][warp] = a;
    sh[1][warp] = b;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    a = lane < nw ? sh[0][lane] : 0ull;
    b = lane < nw ? sh[1][lane] : 0ull;
    a = warp_sum_u64(a);
    b = warp_sum_u64(b);
    if (lane == 0) {
      if (a) atomicAdd(dst, a);
      if (b) atomicAdd(dst + 1, b);
    }
  }
}

// Temporal blocking: one CTA loads a tile of Ty rows x Tw words of both colour
// planes plus a halo of H = 2K rows above and below and one word left and right
// (read as 4-word, 16-byte aligned chunks), runs K full sweeps on it in shared
// memory, and stores the inner Ty x Tw words.  Each half sweep invalidates one
// more halo row on each side and one more halo bit, so after K sweeps exactly
// the inner region is correct (K <= 8 keeps the bit penetration inside the
// halo word).  Sites in the halo are updated with the same (sweep, site)
// random numbers as their owners, so the result is bit-identical to K plain
// sweeps.  Tiles are processed persistently: tile = blockIdx.x + i gridDim.x.
template <int K>
__global__ void __launch_bounds__(256) k_tiled_bits(const uint32_t* __restrict__ in,
                                                    uint32_t* __restrict__ out, int L, int Wc,
                                                    int n_ty, int Tw, uint32_t t0,
                                                    RngParams rng, RecordSlots slots,
                                                    unsigned long long* __restrict__ rec) {
  extern __shared__ uint4 smem4[];
  uint32_t* S = reinterpret_cast<uint32_t*>(smem4);
  constexpr int H = 2 * K;
  const int SP = Tw + 8;
  const int Ty_max = (L + n_ty - 1) / n_ty;
  const int SR = Ty_max + 2 * H;
  uint32_t* S0 = S;
  uint32_t* S1 = S + SR * SP;
  const int n_tx = Wc / Tw;
  const int n_tiles = n_ty * n_tx;
  const int lane = threadIdx.x & 31;
  unsigned long long acc_anti[K], acc_ones[K];
#pragma unroll
  for (int s = 0; s < K; ++s) acc_anti[s] = acc_ones[s] = 0ull;

  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int ty = tile / n_tx, tx = tile - (tile / n_tx) * n_tx;
    const int y0 = (int)((long long)ty * L / n_ty);
    const int y1 = (int)((long long)(ty + 1) * L / n_ty);
    const int Ty = y1 - y0;
    const int w0 = tx * Tw;
    const int rows = Ty + 2 * H;
    const int qrow = SP / 4;
    for (int i = threadIdx.x; i < 2 * rows * qrow; i += blockDim.x) {
      const int c = i / (rows * qrow);
      const int rem = i - c * rows * qrow;
      const int r = rem / qrow, q = rem - (rem / qrow) * qrow;
      const int gy = wrap(y0 - H + r, L);
      const int gw = wrap(w0 - 4 + 4 * q, Wc);
      const uint4 v =
          *reinterpret_cast<const uint4*>(in + (size_t)c * L * Wc + (size_t)gy * Wc + gw);
      reinterpret_cast<uint4*>(S + c * SR * SP + r * SP)[q] = v;
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2 * K; ++h) {
      const int c = h & 1;
      const int sw = h >> 1;
      const uint32_t t = t0 + (uint32_t)sw;
      const int r_lo = h + 1;
      const int ncols = Tw + 2;
      const int count = (rows - 2 * h - 2) * ncols;
      uint32_t* So = c ? S1 : S0;
      const uint32_t* Sn = c ? S0 : S1;
      for (int base = (threadIdx.x & ~31); base < count; base += blockDim.x) {
        const int idx = base + lane;
        const bool active = idx < count;
        int r = r_lo, col = 3;
        if (active) {
          r = r_lo + idx / ncols;
          col = 3 + (idx - (idx / ncols) * ncols);
        }
        const uint32_t s = So[r * SP + col];
        const uint32_t up = Sn[(r - 1) * SP + col];
        const uint32_t dn = Sn[(r + 1) * SP + col];
        const uint32_t mid = Sn[r * SP + col];
        const int o = (y0 + r + c) & 1;  // H is even
        const uint32_t side = o == 0 ? ((mid << 1) | (Sn[r * SP + col - 1] >> 31))
                                     : ((mid >> 1) | (Sn[r * SP + col + 1] << 31));
        const int gy = wrap(y0 - H + r, L);
        const int gw = wrap(w0 - 4 + col, Wc);
        const Classes k = classify(s, up, dn, mid, side);
        const uint32_t f = flip_mask(k, active ? 0xffffffffu : 0u, (uint32_t)gy * Wc + gw, t,
                                     rng.replica, c, rng.key0, rng.key1, rng.t4, rng.t8);
        const uint32_t ns = s ^ f;
        if (active) {
          So[r * SP + col] = ns;
          if (c == 1 && r >= H && r < H + Ty && col >= 4 && col < 4 + Tw) {
            acc_anti[sw] += __popc(ns ^ up) + __popc(ns ^ dn) + __popc(ns ^ mid) + __popc(ns ^ side);
            acc_ones[sw] += __popc(ns) + __popc(mid);
          }
        }
      }
      __syncthreads();
    }
    const int qin = Tw / 4;
    for (int i = threadIdx.x; i < 2 * Ty * qin; i += blockDim.x) {
      const int c = i / (Ty * qin);
      const int rem = i - c * Ty * qin;
      const int r = rem / qin, q = rem - (rem / qin) * qin;
      const uint4 v = reinterpret_cast<const uint4*>(S + c * SR * SP + (H + r) * SP + 4)[q];
      *reinterpret_cast<uint4*>(out + (size_t)c * L * Wc + (size_t)(y0 + r) * Wc + w0 + 4 * q) = v;
    }
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < K; ++s)
    if (slots.slot[s] >= 0) block_add2(acc_anti[s], acc_ones[s], rec + 2 * (size_t)slots.slot[s]);
}

// Planes of Philox blocks b = B0 .. B1-1 for the undecided lanes D of one
// word; cls marks the lanes that test against t4 (the others test against t8).
// Accepted lanes are added to acc.  Stops early once no lane of the warp is
// undecided (warp vote), so every lane of the warp must call it.
template <int B0, int B1>
__device__ __forceinline__ void lazy_planes(uint32_t g, uint32_t t, uint32_t rep, uint32_t colour,
                                            const RngParams& rng, uint32_t& D, uint32_t cls,
                                            uint32_t& acc) {
#pragma unroll
  for (int b = B0; b < B1; ++b) {
    if (!__any_sync(0xffffffffu, D != 0u)) break;
    const uint4 r = philox10_rk(make_uint4(g, t, rep, ctr_w(kTagMet, colour, b)), rng.rk0, rng.rk1);
    const uint32_t p[4] = {r.x, r.y, r.z, r.w};
    // the block's 4 planes as one 4-bit comparison (borrow of u - T from the
    // block's last plane up, equality chain), then merged into (acc, D)
    uint32_t bor = 0u, eq = D;
#pragma unroll
    for (int q = 3; q >= 0; --q) {
      const int k = 4 * b + q;
      const uint32_t m4 = rng.tm4[k], m8 = rng.tm8[k];
      const uint32_t tm = (cls & m4) | (~cls & m8);  // lane's threshold bit
      bor = (~p[q] & tm) | (~p[q] & bor) | (tm & bor);
      eq &= ~(tm ^ p[q]);
    }
    acc |= D & bor;
    D = eq;
  }
}

// lazy_planes for two independent words at once (one warp vote for both; two
// Philox chains in flight per thread).
template <int B0, int B1>
__device__ __forceinline__ void lazy_planes2(uint32_t ga, uint32_t gb, uint32_t t, uint32_t rep,
                                             uint32_t colour, const RngParams& rng, uint32_t& Da,
                                             uint32_t clsa, uint32_t& acca, uint32_t& Db,
                                             uint32_t clsb, uint32_t& accb) {
#pragma unroll
  for (int b = B0; b < B1; ++b) {
    if (!__any_sync(0xffffffffu, (Da | Db) != 0u)) break;
    const uint32_t cw = ctr_w(kTagMet, colour, b);
    const uint4 ra = philox10_rk(make_uint4(ga, t, rep, cw), rng.rk0, rng.rk1);
    const uint4 rb = philox10_rk(make_uint4(gb, t, rep, cw), rng.rk0, rng.rk1);
    const uint32_t pa[4] = {ra.x, ra.y, ra.z, ra.w};
    const uint32_t pb[4] = {rb.x, rb.y, rb.z, rb.w};
    uint32_t bora = 0u, borb = 0u, eqa = Da, eqb = Db;
#pragma unroll
    for (int q = 3; q >= 0; --q) {
      const int k = 4 * b + q;
      const uint32_t m4 = rng.tm4[k], m8 = rng.tm8[k];
      const uint32_t ta = (clsa & m4) | (~clsa & m8);
      const uint32_t tb = (clsb & m4) | (~clsb & m8);
      bora = (~pa[q] & ta) | (~pa[q] & bora) | (ta & bora);
      borb = (~pb[q] & tb) | (~pb[q] & borb) | (tb & borb);
      eqa &= ~(ta ^ pa[q]);
      eqb &= ~(tb ^ pb[q]);
    }
    acca |= Da & bora;
    accb |= Db & borb;
    Da = eqa;
    Db = eqb;
  }
}

// Planes 0..7 (Philox blocks 0 and 1) of one or two words, all evaluated, as
// one strict comparison of the top 8 bits: u_8 < T_8 is the borrow out of the
// bit-sliced subtraction u_8 - T_8, carried from plane 7 (the least
// significant of the eight) up to plane 0 with one majority function per
// plane, borrow' = maj(~u_k, T_k, borrow); lanes whose 8 bits equal the
// threshold's stay undecided.  Gives the same (acc, D) as the MSB-first test
// over the same planes with one logic operation less per plane.  Block 1 is
// drawn first, so only one block's planes are live at a time.
template <int NW>
__device__ __forceinline__ void planes8(const uint32_t (&g)[NW], uint32_t t, uint32_t rep,
                                        uint32_t colour, const RngParams& rng, uint32_t (&D)[NW],
                                        const uint32_t (&cls)[NW], uint32_t (&acc)[NW]) {
  uint32_t bor[NW], eq[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    bor[w] = 0u;
    eq[w] = D[w];
  }
#pragma unroll
  for (int b = 1; b >= 0; --b) {
    const uint32_t cw = ctr_w(kTagMet, colour, b);
    uint4 r[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) r[w] = philox10_rk(make_uint4(g[w], t, rep, cw), rng.rk0, rng.rk1);
#pragma unroll
    for (int q = 3; q >= 0; --q) {
      const int k = 4 * b + q;
      const uint32_t m4 = rng.tm4[k], m8 = rng.tm8[k];
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint32_t p = q == 0 ? r[w].x : q == 1 ? r[w].y : q == 2 ? r[w].z : r[w].w;
        const uint32_t tm = (cls[w] & m4) | (~cls[w] & m8);  // lane's threshold bit
        bor[w] = (~p & tm) | (~p & bor[w]) | (tm & bor[w]);
        eq[w] &= ~(tm ^ p);
      }
    }
  }
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    acc[w] |= D[w] & bor[w];
    D[w] = eq[w];
  }
}

// Tiled sweep with one warp per 32-word tile row segment.  Same tiling, halo
// and results as k_tiled_bits; differences are for speed only:
//  * the inner 32*TWW words of a row are updated by TWW warps (lane = word), the
//    two halo words per row by a separate short pass, so no integer division
//    or modulo runs per word;
//  * phase 1 evaluates the first two Philox blocks (8 planes) of every word as
//    one 8-bit comparison (planes8); words with lanes still undecided (about 1
//    in 10) go to a shared-memory
//    queue, and phase 2 finishes them with all lanes of a warp busy on queued
//    words, instead of every warp waiting for its slowest word;
//  * per-sweep observables are summed in shared memory, not registers.
//
// MINB is the number of CTAs per SM the register budget is sized for: 3 (80
// registers) for tiles that fit three CTAs' shared memory on an SM, 2 (up to
// 128 registers) for taller tiles, which fit only two.
template <int K, int TWW, int MINB>
__global__ void __launch_bounds__(256, MINB) k_tiled32_bits(const uint32_t* __restrict__ in,
                                                         uint32_t* __restrict__ out, int L, int Wc,
                                                         int n_ty, uint32_t t0, RngParams rng,
                                                         RecordSlots slots,
                                                         unsigned long long* __restrict__ rec) {
  constexpr int H = 2 * K;
  constexpr int TW = 32 * TWW;
  constexpr int SP = TW + 8;
  // queue capacity: about 1 word in 10 is still undecided after 8 planes (11 %
  // in an ordered lattice), ~500 words per half sweep of a 72 x 64-word tile
  // and ~800 of a 216 x 32-word tile; a full queue sends the rest to the slow
  // in-place path.  18 KB, so tiles of up to 200 KiB still fit an SM.
  constexpr int QCAP = 1536;
  extern __shared__ uint4 smem4[];
  __shared__ uint32_t q_pos[QCAP], q_d[QCAP], q_cls[QCAP];
  __shared__ int q_n[2];
  __shared__ unsigned long long s_anti[K], s_ones[K];
  uint32_t* S = reinterpret_cast<uint32_t*>(smem4);
  const int Ty_max = (L + n_ty - 1) / n_ty;
  const int SR = Ty_max + 2 * H;
  uint32_t* S0 = S;
  uint32_t* S1 = S + SR * SP;
  const int n_tx = Wc / TW;
  const int n_tiles = n_ty * n_tx;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  if (tid < K) {
    s_anti[tid] = 0ull;
    s_ones[tid] = 0ull;
  }

  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int ty = tile / n_tx, tx = tile - (tile / n_tx) * n_tx;
    const int y0 = (int)((long long)ty * L / n_ty);
    const int y1 = (int)((long long)(ty + 1) * L / n_ty);
    const int Ty = y1 - y0;
    const int w0 = tx * TW;
    const int rows = Ty + 2 * H;
    constexpr int QROW = SP / 4;
    const int per_colour = rows * QROW;
    for (int i = tid; i < 2 * per_colour; i += blockDim.x) {
      // no runtime division or modulo: one compare for the colour, constant
      // divisor for the row, conditional wraps (|y0 - H + r| < 2L, |w| < 2 Wc)
      const int c = i >= per_colour;
      const int rem = i - c * per_colour;
      const int r = rem / QROW, q = rem - (rem / QROW) * QROW;
      int gy = y0 - H + r;
      gy += gy < 0 ? L : 0;
      gy -= gy >= L ? L : 0;
      int gw = w0 - 4 + 4 * q;
      gw += gw < 0 ? Wc : 0;
      gw -= gw >= Wc ? Wc : 0;
      const uint4 v =
          *reinterpret_cast<const uint4*>(in + (size_t)c * L * Wc + (size_t)gy * Wc + gw);
      reinterpret_cast<uint4*>(S + c * SR * SP + r * SP)[q] = v;
    }
    if (tid == 0) q_n[0] = 0;
    __syncthreads();
    // global row of tile row r (no modulo: |y0 - H + r| < 2L since H <= 16 <= L)
    auto grow = [&](int r) {
      int gy = y0 - H + r;
      gy += gy < 0 ? L : 0;
      gy -= gy >= L ? L : 0;
      return gy;
    };
    auto gcol = [&](int col) {
      int gw = w0 - 4 + col;
      gw += gw < 0 ? Wc : 0;
      gw -= gw >= Wc ? Wc : 0;
      return gw;
    };
#pragma unroll
    for (int h = 0; h < 2 * K; ++h) {
      const int c = h & 1;
      const int sw = h >> 1;
      const uint32_t t = t0 + (uint32_t)sw;
      const int r_lo = h + 1;
      const int nrows = rows - 2 * h - 2;
      uint32_t* So = c ? S1 : S0;
      const uint32_t* Sn = c ? S0 : S1;
      int* qn = &q_n[h & 1];

      // ---- phase 1: classes, planes 0..7, write, queue the undecided ----
      auto phase1 = [&](int r, int col, bool active) {
        const uint32_t s = So[r * SP + col];
        const uint32_t up = Sn[(r - 1) * SP + col];
        const uint32_t dn = Sn[(r + 1) * SP + col];
        const uint32_t mid = Sn[r * SP + col];
        const int o = (y0 + r + c) & 1;
        const uint32_t side = o == 0 ? ((mid << 1) | (Sn[r * SP + col - 1] >> 31))
                                     : ((mid >> 1) | (Sn[r * SP + col + 1] << 31));
        const HalfClasses k = classify_hs(s, up ^ dn, up, dn, mid, side);
        const uint32_t valid = active ? 0xffffffffu : 0u;
        const uint32_t cls = k.cls;
        const uint32_t g = (uint32_t)grow(r) * (uint32_t)Wc + (uint32_t)gcol(col);
        uint32_t Dv[1] = {~k.ge2 & valid}, accv[1] = {0u};
        const uint32_t gv[1] = {g}, clsv[1] = {cls};
        planes8<1>(gv, t, rng.replica, c, rng, Dv, clsv, accv);
        const uint32_t D = Dv[0], acc = accv[0];
        bool ovf = false;
        if (active) {
          So[r * SP + col] = s ^ ((k.ge2 & valid) | acc);
          if (D != 0u) {
            const int slot = atomicAdd(qn, 1);
            if (slot < QCAP) {
              q_pos[slot] = ((uint32_t)r << 8) | (uint32_t)col;
              q_d[slot] = D;
              q_cls[slot] = cls;
            } else {
              ovf = true;
            }
          }
        }
        // queue full (not expected at these tile sizes): finish in place
        if (__any_sync(0xffffffffu, ovf)) {
          uint32_t e = ovf ? D : 0u, acc2 = 0;
          lazy_planes<2, 8>(g, t, rng.replica, c, rng, e, cls, acc2);
          if (ovf) So[r * SP + col] ^= acc2;
        }
      };
      // queue a word whose lanes are still undecided after phase 1 (returns
      // false if the queue is full; the caller then finishes it in place)
      auto enqueue = [&](int r, int col, uint32_t D, uint32_t cls) {
        const int slot = atomicAdd(qn, 1);
        if (slot >= QCAP) return false;
        q_pos[slot] = ((uint32_t)r << 8) | (uint32_t)col;
        q_d[slot] = D;
        q_cls[slot] = cls;
        return true;
      };
      // inner words of two adjacent rows (r, r+1) per thread: the two words
      // share the other colour's rows r and r+1 as neighbours
      auto phase1_pair = [&](int r, int col) {
        const uint32_t sa = So[r * SP + col];
        const uint32_t sb = So[(r + 1) * SP + col];
        const uint32_t u0 = Sn[(r - 1) * SP + col];
        const uint32_t m0 = Sn[r * SP + col];
        const uint32_t m1 = Sn[(r + 1) * SP + col];
        const uint32_t d1 = Sn[(r + 2) * SP + col];
        const int oa = (y0 + r + c) & 1;  // row r+1 has the other offset
        uint32_t side_a, side_b;
        if (oa == 0) {
          side_a = (m0 << 1) | (Sn[r * SP + col - 1] >> 31);
          side_b = (m1 >> 1) | (Sn[(r + 1) * SP + col + 1] << 31);
        } else {
          side_a = (m0 >> 1) | (Sn[r * SP + col + 1] << 31);
          side_b = (m1 << 1) | (Sn[(r + 1) * SP + col - 1] >> 31);
        }
        // both words have rows r and r+1 of the other colour as neighbours
        const uint32_t h01 = m0 ^ m1;
        const HalfClasses ka = classify_hs(sa, h01, m0, m1, u0, side_a);
        const HalfClasses kb = classify_hs(sb, h01, m0, m1, d1, side_b);
        const int gya = grow(r);
        const int gyb = gya + 1 == L ? 0 : gya + 1;
        const uint32_t gw = (uint32_t)(w0 + col - 4);  // inner column: no wrap
        const uint32_t ga = (uint32_t)gya * (uint32_t)Wc + gw;
        const uint32_t gb = (uint32_t)gyb * (uint32_t)Wc + gw;
        uint32_t Dv[2] = {~ka.ge2, ~kb.ge2}, accv[2] = {0u, 0u};
        const uint32_t gv[2] = {ga, gb}, clsv[2] = {ka.cls, kb.cls};
        planes8<2>(gv, t, rng.replica, c, rng, Dv, clsv, accv);
        const uint32_t Da = Dv[0], Db = Dv[1], acca = accv[0], accb = accv[1];
        So[r * SP + col] = sa ^ (ka.ge2 | acca);
        So[(r + 1) * SP + col] = sb ^ (kb.ge2 | accb);
        const bool ovfa = Da != 0u && !enqueue(r, col, Da, ka.cls);
        const bool ovfb = Db != 0u && !enqueue(r + 1, col, Db, kb.cls);
        if (__any_sync(0xffffffffu, ovfa || ovfb)) {  // queue full: finish in place
          uint32_t ea = ovfa ? Da : 0u, eb = ovfb ? Db : 0u, xa = 0, xb = 0;
          lazy_planes2<2, 8>(ga, gb, t, rng.replica, c, rng, ea, ka.cls, xa, eb, kb.cls, xb);
          if (ovfa) So[r * SP + col] ^= xa;
          if (ovfb) So[(r + 1) * SP + col] ^= xb;
        }
      };
      // three kinds of work item (row pairs, the odd last row, the halo
      // columns) dealt round-robin to the warps as one sequence, so the warps
      // that took one item more of a kind start the next kind later
      const int npairs = nrows >> 1;
      for (int item = warp; item < npairs * TWW; item += nwarps) {
        const int r = r_lo + 2 * (item / TWW);
        const int col = 4 + 32 * (item % TWW) + lane;
        phase1_pair(r, col);
      }
      int w1 = warp - (npairs * TWW) % nwarps;
      w1 += w1 < 0 ? nwarps : 0;
      if (nrows & 1) {  // odd row count: the last row alone
        for (int item = w1; item < TWW; item += nwarps)
          phase1(r_lo + nrows - 1, 4 + 32 * item + lane, true);
        w1 -= TWW % nwarps;
        w1 += w1 < 0 ? nwarps : 0;
      }
      for (int base = w1 * 32; base < 2 * nrows; base += blockDim.x) {
        const int idx = base + lane;
        const bool active = idx < 2 * nrows;
        const int r = r_lo + (active ? (idx >> 1) : 0);
        const int col = (idx & 1) ? 4 + TW : 3;
        phase1(r, col, active);
      }
      __syncthreads();

      // ---- phase 2: finish the queued words, all lanes busy ----
      const int n = min(*qn, QCAP);
      if (tid == 0) q_n[(h + 1) & 1] = 0;
      for (int base = warp * 32; base < n; base += blockDim.x) {
        const int e = base + lane;
        const bool act = e < n;
        const uint32_t pos = act ? q_pos[e] : (3u | ((uint32_t)r_lo << 8));
        uint32_t D = act ? q_d[e] : 0u, acc = 0;
        const uint32_t cls = act ? q_cls[e] : 0u;
        const int r = (int)(pos >> 8), col = (int)(pos & 255u);
        const uint32_t g = (uint32_t)grow(r) * (uint32_t)Wc + (uint32_t)gcol(col);
        lazy_planes<2, 8>(g, t, rng.replica, c, rng, D, cls, acc);
        if (act && acc) So[r * SP + col] ^= acc;
      }
      if (c == 1 && slots.slot[sw] >= 0) {
        __syncthreads();
        unsigned long long anti = 0, ones = 0;
        for (int item = warp; item < Ty * TWW; item += nwarps) {
          const int r = H + item / TWW;
          const int col = 4 + 32 * (item % TWW) + lane;
          const uint32_t ns = S1[r * SP + col];
          const uint32_t up = S0[(r - 1) * SP + col];
          const uint32_t dn = S0[(r + 1) * SP + col];
          const uint32_t mid = S0[r * SP + col];
          const int o = (y0 + r + 1) & 1;
          const uint32_t side = o == 0 ? ((mid << 1) | (S0[r * SP + col - 1] >> 31))
                                       : ((mid >> 1) | (S0[r * SP + col + 1] << 31));
          anti += __popc(ns ^ up) + __popc(ns ^ dn) + __popc(ns ^ mid) + __popc(ns ^ side);
          ones += __popc(ns) + __popc(mid);
        }
        anti = warp_sum_u64(anti);
        ones = warp_sum_u64(ones);
        if (lane == 0) {
          atomicAdd(&s_anti[sw], anti);
          atomicAdd(&s_ones[sw], ones);
        }
      }
      __syncthreads();
    }
    constexpr int QIN = TW / 4;
    for (int i = tid; i < 2 * Ty * QIN; i += blockDim.x) {
      const int c = i >= Ty * QIN;
      const int rem = i - c * Ty * QIN;
      const int r = rem / QIN, q = rem - (rem / QIN) * QIN;
      const uint4 v = reinterpret_cast<const uint4*>(S + c * SR * SP + (H + r) * SP + 4)[q];
      *reinterpret_cast<uint4*>(out + (size_t)c * L * Wc + (size_t)(y0 + r) * Wc + w0 + 4 * q) = v;
    }
    __syncthreads();
  }
  if (tid < K && slots.slot[tid] >= 0) {
    unsigned long long* dst = rec + 2 * (size_t)slots.slot[tid];
    if (s_anti[tid]) atomicAdd(dst, s_anti[tid]);
    if (s_ones[tid]) atomicAdd(dst + 1, s_ones[tid]);
  }
}

template <int K>
cudaError_t launch_tiled_k(const BitsLattice& in, uint32_t* out, const RngParams& rng,
                                  uint32_t sweep0, const RecordSlots& slots,
                                  unsigned long long* rec, int n_ty, int Tw, int grid, int block,
                                  cudaStream_t s) {
  const size_t smem = tiled_smem_bytes(in.L, K, n_ty, Tw);
  cudaError_t e = cudaFuncSetAttribute(k_tiled_bits<K>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_tiled_bits<K><<<grid, block, smem, s>>>(in.planes, out, in.L, in.Wc, n_ty, Tw, sweep0, rng,
                                             slots, rec);
  return cudaGetLastError();
}

template <int K, int TWW, int MINB>
cudaError_t launch_tiled32_v(const BitsLattice& in, uint32_t* out, const RngParams& rng,
                             uint32_t sweep0, const RecordSlots& slots, unsigned long long* rec,
                             int n_ty, int grid, size_t smem, int per_sm, cudaStream_t s) {
  static DeviceCache configured;  // per instantiation and device
  if ((long long)smem > configured.get()) {
    cudaError_t e = cudaFuncSetAttribute(k_tiled32_bits<K, TWW, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured.set((long long)smem);
  }
  const int n_tiles = n_ty * (in.Wc / (32 * TWW));
  if (grid <= 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = per_sm * sms;
  }
  if (grid > n_tiles) grid = n_tiles;
  if (grid < 1) grid = 1;
  k_tiled32_bits<K, TWW, MINB><<<grid, 256, smem, s>>>(in.planes, out, in.L, in.Wc, n_ty, sweep0,
                                                       rng, slots, rec);
  return cudaGetLastError();
}

// Resident CTAs per SM of the 3-CTA variant decide the variant: three or more
// run it, fewer (tiles too tall for three CTAs' shared memory) run the 2-CTA
// variant with its larger register budget.
template <int K, int TWW>
cudaError_t launch_tiled32_k(const BitsLattice& in, uint32_t* out, const RngParams& rng,
                                    uint32_t sweep0, const RecordSlots& slots,
                                    unsigned long long* rec, int n_ty, int grid, cudaStream_t s) {
  const size_t smem = tiled32_smem_bytes(in.L, K, n_ty, 32 * TWW);
  // CTAs per SM of the 3-CTA variant, cached per device as (smem << 20 | CTAs)
  static DeviceCache occ;
  int per_sm = 0;
  const long long memo = occ.get();
  if ((memo >> 20) == (long long)smem) {
    per_sm = (int)(memo & 0xfffff);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_tiled32_bits<K, TWW, 3>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tiled32_bits<K, TWW, 3>, 256, smem);
    if (e != cudaSuccess) return e;
    occ.set(((long long)smem << 20) | (long long)per_sm);
  }
  if (per_sm >= 3)
    return launch_tiled32_v<K, TWW, 3>(in, out, rng, sweep0, slots, rec, n_ty, grid, smem, per_sm, s);
  return launch_tiled32_v<K, TWW, 2>(in, out, rng, sweep0, slots, rec, n_ty, grid, smem,
                                     per_sm < 1 ? 1 : per_sm, s);
}

}  // namespace
}  // namespace ising

#define ISING_TILED_INSTANTIATE(K)                                                         \
  namespace ising {                                                                        \
  cudaError_t launch_tiled_k##K(const BitsLattice& in, uint32_t* out, const RngParams& rng,   \
                                uint32_t sweep0, const RecordSlots& slots,                 \
                                unsigned long long* rec, int n_ty, int Tw, int grid,       \
                                int block, cudaStream_t s) {                               \
    return launch_tiled_k<K>(in, out, rng, sweep0, slots, rec, n_ty, Tw, grid, block, s);    \
  }                                                                                        \
  cudaError_t launch_tiled32_k##K##_w1(const BitsLattice& in, uint32_t* out,                \
                                       const RngParams& rng, uint32_t sweep0,             \
                                       const RecordSlots& slots, unsigned long long* rec, \
                                       int n_ty, int grid, cudaStream_t s) {              \
    return launch_tiled32_k<K, 1>(in, out, rng, sweep0, slots, rec, n_ty, grid, s);        \
  }                                                                                        \
  cudaError_t launch_tiled32_k##K##_w2(const BitsLattice& in, uint32_t* out,                \
                                       const RngParams& rng, uint32_t sweep0,             \
                                       const RecordSlots& slots, unsigned long long* rec, \
                                       int n_ty, int grid, cudaStream_t s) {              \
    return launch_tiled32_k<K, 2>(in, out, rng, sweep0, slots, rec, n_ty, grid, s);        \
  }                                                                                        \
  }
