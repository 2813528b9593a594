// Swendsen-Wang cluster update on the packed lattice (Swendsen & Wang, PRL 58,
// 86 (1987)); the paper points to cluster updates as the step beyond its
// single-site Monte Carlo.  One step:
//   1. every bond between equal spins is active iff u < floor((1 - e^{-2 beta}) 2^32),
//      u = word (b & 3) of Philox(b >> 2, step, replica, SW_BOND << 16),
//      b = 2 (y L + x) + dir (dir 0: bond to x+1, 1: to y+1);
//   2. clusters = connected components of the active bonds, found by a lock-free
//      union-find whose links always point from the larger to the smaller site
//      index, so each cluster's root is its smallest site whatever the order in
//      which threads link.  When L >= 2048 is a multiple of the 128 x 64 tile, each CTA
//      first labels its tile's inner bonds in shared memory (k_sw_local) and
//      only the bonds crossing tile edges go through the global forest
//      (k_sw_edges); otherwise every bond does (k_sw_bonds);
//   3. each cluster flips iff bit 31 of word (m & 3) of
//      Philox(m >> 2, step, replica, SW_FLIP << 16), m = its root.
// The outcome depends only on (seed, step, replica, spins): bit-identical to
// any sequential implementation of the same rule.
#include <cuda_runtime.h>

#include "internal.h"
#include "ising_device.cuh"

namespace ising {
namespace {

constexpr uint32_t kTagSWBond = 10, kTagSWFlip = 11;

__device__ __forceinline__ int bit_at(const uint32_t* planes, int L, int Wc, int x, int y) {
  const int c = (x + y) & 1, j = x >> 1;
  return (__ldcg(&planes[(size_t)c * L * Wc + (size_t)y * Wc + (j >> 5)]) >> (j & 31)) & 1;
}

__device__ __forceinline__ uint32_t find_root(uint32_t* parent, uint32_t a) {
  // links only go to smaller indices: the walk strictly decreases and ends.
  // Path halving (parent[a] = grandparent) keeps the trees shallow; it only
  // ever stores an ancestor of a, which stays in a's set (sets never split).
  while (true) {
    const uint32_t p = __ldcg(&parent[a]);
    if (p == a) return a;
    const uint32_t gp = __ldcg(&parent[p]);
    if (gp != p) __stcg(&parent[a], gp);
    a = gp;
  }
}

// Read-only walk for the roots pass: a halving store there could overwrite, with
// a mere ancestor, the root that the site's own thread has just stored.
__device__ __forceinline__ uint32_t find_root_ro(const uint32_t* parent, uint32_t a) {
  while (true) {
    const uint32_t p = __ldcg(&parent[a]);
    if (p == a) return a;
    a = p;
  }
}

__device__ __forceinline__ void unite(uint32_t* parent, uint32_t a, uint32_t b) {
  while (true) {
    a = find_root(parent, a);
    b = find_root(parent, b);
    if (a == b) return;
    if (a < b) {
      const uint32_t t = a;
      a = b;
      b = t;
    }
    const uint32_t old = atomicCAS(&parent[a], a, b);  // link the larger root below the smaller
    if (old == a) return;
    a = old;  // a got linked meanwhile: retry from there
  }
}

// Labelling kernels may be gated on a device flag (Wolff steps label the
// lattice only when the bounded growth from the seed gave up); null = always run.
__device__ __forceinline__ bool gated_off(const uint32_t* gate) { return gate && *gate == 0; }

__global__ void k_sw_init(uint32_t* __restrict__ parent, long long N, const uint32_t* gate) {
  if (gated_off(gate)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    parent[i] = (uint32_t)i;
}

// One thread per pair of sites (a = 2p, 2p + 1): the four bonds of the pair use
// the four words of one Philox block.
__global__ void __launch_bounds__(256) k_sw_bonds(const uint32_t* __restrict__ planes, int L,
                                                  int Wc, uint32_t step, uint32_t thr,
                                                  RngParams rng, uint32_t* __restrict__ parent,
                                                  FastDiv fL, uint32_t bond_tag, const uint32_t* gate,
                                                  const uint32_t* step_ptr) {
  if (gated_off(gate)) return;
  if (step_ptr) step = *step_ptr;
  const long long N = (long long)L * L;
  for (long long pr = blockIdx.x * (long long)blockDim.x + threadIdx.x; 2 * pr < N;
       pr += (long long)gridDim.x * blockDim.x) {
    const uint4 r = philox10_rk(make_uint4((uint32_t)pr, step, rng.replica, bond_tag << 16),
                                rng.rk0, rng.rk1);
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long a = 2 * pr + h;
      if (a >= N) break;
      const int y = (int)fdiv((uint32_t)a, fL), x = (int)((uint32_t)a - (uint32_t)y * (uint32_t)L);
      const int sa = bit_at(planes, L, Wc, x, y);
#pragma unroll
      for (int dir = 0; dir < 2; ++dir) {
        const int xn = dir == 0 ? (x + 1 == L ? 0 : x + 1) : x;
        const int yn = dir == 0 ? y : (y + 1 == L ? 0 : y + 1);
        if (bit_at(planes, L, Wc, xn, yn) != sa) continue;
        if (w[2 * h + dir] >= thr) continue;  // bond 2a + dir -> word (2a + dir) & 3
        unite(parent, (uint32_t)a, (uint32_t)yn * (uint32_t)L + (uint32_t)xn);
      }
    }
  }
}

// Roots decide their flip; every site records its root (only the site's own
// thread writes parent[i] here, so afterwards parent[i] is i's root).
__global__ void k_sw_roots(uint32_t* __restrict__ parent, long long N, uint32_t step,
                           RngParams rng, uint8_t* __restrict__ flip) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const uint32_t m = find_root_ro(parent, (uint32_t)i);
    parent[i] = m;  // compress: every site now points at its root
    if (m == (uint32_t)i) {
      const uint4 r = philox10_rk(make_uint4(m >> 2, step, rng.replica, kTagSWFlip << 16),
                                  rng.rk0, rng.rk1);
      const uint32_t w = (m & 3) == 0 ? r.x : ((m & 3) == 1 ? r.y : ((m & 3) == 2 ? r.z : r.w));
      flip[i] = (uint8_t)(w >> 31);
    }
  }
}

// One thread per packed word: XOR in the flips of its sites' clusters.
__global__ void k_sw_apply(uint32_t* __restrict__ planes, int L, int Wc,
                           const uint32_t* __restrict__ parent, const uint8_t* __restrict__ flip,
                           FastDiv fplane, FastDiv fwc) {
  const int n = L / 2;
  const uint32_t words = 2u * (uint32_t)L * (uint32_t)Wc;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x) {
    const int c = (int)fdiv(i, fplane);
    const uint32_t rem = i - (uint32_t)c * fplane.d;
    const int y = (int)fdiv(rem, fwc), w = (int)(rem - (uint32_t)y * (uint32_t)Wc);
    uint32_t mask = 0;
    for (int b = 0; b < 32; ++b) {
      const int j = 32 * w + b;
      if (j >= n) break;
      const int x = 2 * j + ((y + c) & 1);
      const uint32_t m = parent[(size_t)y * L + x];  // the root (compressed above)
      mask |= (uint32_t)flip[m] << b;
    }
    planes[i] ^= mask;
  }
}

// ---- two-level labelling: union-find inside a TX x TY tile in shared memory,
// then only the bonds that cross tile edges in global memory ----
constexpr int kTileX = 128, kTileY = 64, kTileSites = kTileX * kTileY, kTileThreads = 512;

__device__ __forceinline__ uint32_t sfind(volatile uint32_t* lab, uint32_t a) {
  while (true) {
    const uint32_t p = lab[a];
    if (p == a) return a;
    const uint32_t gp = lab[p];
    if (gp != p) lab[a] = gp;  // an ancestor: stays in a's set
    a = gp;
  }
}

__device__ __forceinline__ void sunite(uint32_t* lab, uint32_t a, uint32_t b) {
  while (true) {
    a = sfind(lab, a);
    b = sfind(lab, b);
    if (a == b) return;
    if (a < b) {
      const uint32_t t = a;
      a = b;
      b = t;
    }
    const uint32_t old = atomicCAS(&lab[a], a, b);
    if (old == a) return;
    a = old;
  }
}

// One CTA per tile: spins in, local clusters of the tile's inner bonds, and
// parent[site] = global index of its local root (the smallest global index of
// the local cluster: inside a tile local and global order agree); mark[site] = 2
// for local roots, 0 otherwise.  Labelling: horizontal runs first (each site
// labelled with the start of its run by a warp max-scan, no atomics), then the
// vertical bonds unite runs (skipping a bond whose left neighbour already joined
// the same two runs), then every label is resolved to its root.
__global__ void __launch_bounds__(kTileThreads, 4) k_sw_local(const uint32_t* __restrict__ planes, int L, int Wc,
                                                           uint32_t step, uint32_t thr, RngParams rng,
                                                           uint32_t* __restrict__ parent,
                                                           uint8_t* __restrict__ mark, uint32_t bond_tag,
                                                           const uint32_t* gate, const uint32_t* step_ptr) {
  if (gated_off(gate)) return;
  if (step_ptr) step = *step_ptr;
  __shared__ uint32_t lab[kTileSites];
  // vertical bonds that need a union, compacted so that every lane of a warp
  // works on one (a full list makes the scan unite in place)
  constexpr int kUnionCap = 4096;
  __shared__ uint16_t ulist[kUnionCap];
  __shared__ int s_nu;
  if (threadIdx.x == 0) s_nu = 0;
  // per site: bit 0 spin, bit 1 bond li -> li + 1 active, bit 2 bond li -> li + TX
  // active (bonds inside the tile only)
  __shared__ __align__(16) uint8_t st[kTileSites];
  const int tiles_x = L / kTileX;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  const int x0 = tx * kTileX, y0 = ty * kTileY;
  // spins: one thread per (row, 64-site column block) reads the two colour
  // words of the block and writes 64 spin bytes as 16 four-byte stores
  constexpr int kWordsRow = kTileX / 64;
  for (int i = threadIdx.x; i < kTileY * kWordsRow; i += blockDim.x) {
    const int ly = i / kWordsRow, wi = i - ly * kWordsRow;
    const int y = y0 + ly;
    const int ce = y & 1;  // the colour whose sites sit at even x
    const uint32_t we = __ldg(&planes[(size_t)ce * L * Wc + (size_t)y * Wc + (x0 >> 6) + wi]);
    const uint32_t wo = __ldg(&planes[(size_t)(1 - ce) * L * Wc + (size_t)y * Wc + (x0 >> 6) + wi]);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&st[ly * kTileX + 64 * wi]);
#pragma unroll
    for (int b = 0; b < 32; b += 2) {
      // bytes x = 2b, 2b + 1, 2b + 2, 2b + 3: even, odd, even, odd sites
      const uint32_t e = (we >> b) & 3u, o = (wo >> b) & 3u;
      dst[b >> 1] = (e & 1u) | ((o & 1u) << 8) | ((e & 2u) << 15) | ((o & 2u) << 23);
    }
  }
  __syncthreads();
  // inner bonds: one thread per site pair (one Philox block for its four bonds)
  for (int pp = threadIdx.x; pp < kTileSites / 2; pp += blockDim.x) {
    const int ly = pp / (kTileX / 2), lx0 = 2 * (pp - ly * (kTileX / 2));
    const long long a0 = (long long)(y0 + ly) * L + x0 + lx0;
    const uint4 r = philox10_rk(make_uint4((uint32_t)(a0 >> 1), step, rng.replica, bond_tag << 16),
                                rng.rk0, rng.rk1);
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      // other threads rewrite only the bond bits of their own sites: spin bits read here are stable
      const int lx = lx0 + h, li = ly * kTileX + lx;
      const uint8_t me = st[li] & 1u;
      const bool hbond = lx + 1 < kTileX && w[2 * h] < thr && me == (st[li + 1] & 1u);
      const bool vbond = ly + 1 < kTileY && w[2 * h + 1] < thr && me == (st[li + kTileX] & 1u);
      st[li] = (uint8_t)(me | (hbond ? 2u : 0u) | (vbond ? 4u : 0u));
    }
  }
  __syncthreads();
  // horizontal runs: one warp per row, four consecutive sites per lane; the
  // same pass lists the vertical bonds that need a union (warp ballots, one
  // shared-memory atomic per warp per row)
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int ly = warp; ly < kTileY; ly += nwarps) {
      const int base = ly * kTileX + 4 * lane;
      // this lane's four flag bytes, the byte left of them, and the same in the row below
      const uint32_t cw = *reinterpret_cast<const uint32_t*>(&st[base]);
      const uint32_t pb = lane > 0 ? st[base - 1] : 0u;
      const bool below = ly + 1 < kTileY;
      const uint32_t dw = below ? *reinterpret_cast<const uint32_t*>(&st[base + kTileX]) : 0u;
      const uint32_t dpb = (below && lane > 0) ? st[base - 1 + kTileX] : 0u;
      int start[4], last = -1;
      bool need[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int lx = 4 * lane + k;
        const uint32_t own = (cw >> (8 * k)) & 0xffu;
        const uint32_t left = k == 0 ? pb : (cw >> (8 * (k - 1))) & 0xffu;
        const uint32_t below_left = k == 0 ? dpb : (dw >> (8 * (k - 1))) & 0xffu;
        if (lx == 0 || !(left & 2u)) last = lx;
        start[k] = last;
        // a vertical bond needs a union unless the left neighbour's vertical
        // bond already joined the same two runs
        need[k] = (own & 4u) && !(lx > 0 && (left & 6u) == 6u && (below_left & 2u));
      }
      // carry: the last run start of lanes below (inclusive max-scan)
      int carry = last;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, carry, off);
        if (lane >= off) carry = max(carry, v);
      }
      int prev = __shfl_up_sync(0xffffffffu, carry, 1);
      if (lane == 0) prev = -1;
#pragma unroll
      for (int k = 0; k < 4; ++k) lab[base + k] = (uint32_t)(ly * kTileX + (start[k] >= 0 ? start[k] : prev));
      uint32_t m[4];
      int total = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        m[k] = __ballot_sync(0xffffffffu, need[k]);
        total += __popc(m[k]);
      }
      int slot0 = 0;
      if (lane == 0 && total) slot0 = atomicAdd(&s_nu, total);
      slot0 = __shfl_sync(0xffffffffu, slot0, 0);
      const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (need[k]) {
          const int slot = slot0 + __popc(m[k] & lt);
          if (slot < kUnionCap) ulist[slot] = (uint16_t)(base + k);
        }
        slot0 += __popc(m[k]);
      }
    }
  }
  __syncthreads();
  // vertical bonds unite runs, every lane of a warp on a listed bond; if the
  // list overflowed (not at beta_c tile sizes), every needed bond is united
  // by a scan instead (uniting listed bonds twice is harmless)
  if (s_nu <= kUnionCap) {
    for (int i = threadIdx.x; i < s_nu; i += blockDim.x) {
      const uint32_t li = ulist[i];
      sunite(lab, li + kTileX, li);
    }
  } else {
    for (int li = threadIdx.x; li < kTileSites; li += blockDim.x) {
      const int lx = li % kTileX;
      if ((st[li] & 4u) && !(lx > 0 && (st[li - 1] & 6u) == 6u && (st[li - 1 + kTileX] & 2u)))
        sunite(lab, (uint32_t)(li + kTileX), (uint32_t)li);
    }
  }
  __syncthreads();
  // Roots.  Every label is a run start (the runs pass sets run starts, unions
  // link roots, path halving stores grandparents), so once each run start
  // knows its root, the root of site li is that of run start lab[li].  Run
  // starts walk read-only (labels < 2^13 in the low half of each word) and
  // store their root in the high half of their own word, which no walk reads.
  for (int li = threadIdx.x; li < kTileSites; li += blockDim.x) {
    const int lx = li % kTileX;
    if (lx == 0 || !(st[li - 1] & 2u)) {
      uint32_t a = (uint32_t)li;
      while (true) {
        const uint32_t p = lab[a] & 0xffffu;
        if (p == a) break;
        a = p;
      }
      lab[li] = (lab[li] & 0xffffu) | (a << 16);
    }
  }
  __syncthreads();
  for (int li = threadIdx.x; li < kTileSites; li += blockDim.x) {
    const uint32_t r = lab[lab[li] & 0xffffu] >> 16;
    const int ly = li / kTileX, lx = li - ly * kTileX;
    const int ry = (int)r / kTileX, rx = (int)r - ry * kTileX;
    const size_t g = (size_t)(y0 + ly) * L + x0 + lx;
    parent[g] = (uint32_t)((size_t)(y0 + ry) * L + x0 + rx);
    mark[g] = (uint8_t)(r == (uint32_t)li ? 2 : 0);
  }
}

// After the edge unions: every local root (mark 2) finds its final root; a
// non-final one stores it (its own entry only), a final root draws its
// cluster's coin into mark[] (0 / 1) and leaves its entry alone.
__global__ void __launch_bounds__(256) k_sw_resolve(uint32_t* __restrict__ parent, uint8_t* __restrict__ mark,
                                                    long long N, uint32_t step, RngParams rng) {
  // A warp takes 512 sites at a time (16 marks per lane from one 16-byte load;
  // N is a multiple of 16 on the tiled path), lists their local roots in shared
  // memory (prefix sum over the lanes), then resolves the list with every lane
  // busy instead of each lane walking its own roots while the others wait.
  __shared__ uint32_t roots[8][512];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long n16 = N >> 4;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long c0 = ((long long)blockIdx.x * (blockDim.x >> 5) + warp) * 32; c0 < n16; c0 += warps * 32) {
    const long long i16 = c0 + lane;
    uint32_t z[4] = {0u, 0u, 0u, 0u};
    int cnt = 0;
    if (i16 < n16) {
      const uint4 m4 = reinterpret_cast<const uint4*>(mark)[i16];
      const uint32_t w[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        // bytes equal to 2 are the zero bytes of x; the high bit of each zero
        // byte of x, exactly (seven-bit sums cannot carry into the next byte)
        const uint32_t x = w[q] ^ 0x02020202u;
        z[q] = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);
        cnt += __popc(z[q]);
      }
    }
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int pos = incl - cnt;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      while (z[q]) {
        const int byte = (__ffs(z[q]) - 1) >> 3;
        z[q] &= z[q] - 1;
        roots[warp][pos++] = (uint32_t)((i16 << 4) + 4 * q + byte);
      }
    __syncwarp();
    // two walks per lane, interleaved so that both loads are in flight
    for (int e = lane; e < total; e += 64) {
      const bool two = e + 32 < total;
      const uint32_t ia = roots[warp][e], ib = two ? roots[warp][e + 32] : ia;
      uint32_t a = ia, b = ib;
      bool da = false, db = !two;
      while (!(da && db)) {
        if (!da) {
          const uint32_t p = __ldcg(&parent[a]);
          if (p == a) da = true; else a = p;
        }
        if (!db) {
          const uint32_t p = __ldcg(&parent[b]);
          if (p == b) db = true; else b = p;
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !two) break;
        const uint32_t i = h ? ib : ia, m = h ? b : a;
        if (m == i) {
          const uint4 r = philox10_rk(make_uint4(m >> 2, step, rng.replica, kTagSWFlip << 16), rng.rk0, rng.rk1);
          const uint32_t wd = (m & 3) == 0 ? r.x : ((m & 3) == 1 ? r.y : ((m & 3) == 2 ? r.z : r.w));
          mark[i] = (uint8_t)(wd >> 31);
        } else {
          parent[i] = m;
        }
      }
    }
    __syncwarp();
  }
}

// Every non-final local root (still mark 2) takes the coin of its final root
// (its parent entry after k_sw_resolve, whose mark is 0 / 1).  Afterwards
// mark[parent[site]] is every site's coin: a site's entry points at a local
// root (the tile pass sets it; unions link only roots, and path halving moves
// it to another local root), and every local root now holds its cluster's coin.
__global__ void k_sw_coin_copy(const uint32_t* __restrict__ parent, uint8_t* __restrict__ mark,
                               long long N) {
  const long long n16 = N >> 4;  // 16 marks per thread and iteration, as k_sw_resolve
  for (long long i16 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i16 < n16;
       i16 += (long long)gridDim.x * blockDim.x) {
    const uint4 m4 = reinterpret_cast<const uint4*>(mark)[i16];
    const uint32_t w[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t x = w[q] ^ 0x02020202u;
      uint32_t z = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);
      while (z) {
        const int byte = (__ffs(z) - 1) >> 3;
        z &= z - 1;
        const long long i = (i16 << 4) + 4 * q + byte;
        mark[i] = mark[parent[i]];
      }
    }
  }
}

// One warp per 64 consecutive sites of a row (both colours): lane l reads the
// parent entries of sites 64 w + 2 l and 64 w + 2 l + 1 with one 8-byte load
// (each entry a local root), gathers their coins, and two ballots assemble the
// flip masks of packed word w of the two colour planes (site x of row y is bit
// (x >> 1) & 31 of word x >> 6 of colour (x + y) & 1).  The parent array is read
// once, contiguously.  Needs L % 64 == 0 (the tiled path's lattices).
__global__ void __launch_bounds__(256) k_sw_apply2(uint32_t* __restrict__ planes, int L, int Wc,
                                                   const uint32_t* __restrict__ parent,
                                                   const uint8_t* __restrict__ coin) {
  // four segments per warp and iteration, their loads in flight together; lanes
  // 0..3 apply the flip masks of segments 0..3
  constexpr int kU = 4;
  const int lane = threadIdx.x & 31;
  const uint32_t segs = (uint32_t)L * (uint32_t)Wc;  // 64-site row segments
  const uint32_t warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t i0 = warp0 * kU; i0 < segs; i0 += nwarps * kU) {
    uint2 pr[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const uint32_t i = i0 + u < segs ? i0 + u : i0;
      const uint32_t y = i / (uint32_t)Wc, w = i - y * (uint32_t)Wc;
      pr[u] = __ldg(reinterpret_cast<const uint2*>(parent + (size_t)y * L + 64 * w + 2 * lane));
    }
    bool f[kU][2];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      f[u][0] = __ldg(&coin[pr[u].x]) != 0;  // x even: colour y & 1
      f[u][1] = __ldg(&coin[pr[u].y]) != 0;  // x odd: the other colour
    }
    uint32_t mine0 = 0, mine1 = 0;
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const uint32_t m0 = __ballot_sync(0xffffffffu, f[u][0]);
      const uint32_t m1 = __ballot_sync(0xffffffffu, f[u][1]);
      if (lane == u) {
        mine0 = m0;
        mine1 = m1;
      }
    }
    const uint32_t i = i0 + (uint32_t)lane;
    if (lane < kU && i < segs) {
      const uint32_t y = i / (uint32_t)Wc, w = i - y * (uint32_t)Wc;
      const uint32_t c0 = y & 1u;
      if (mine0) planes[(size_t)c0 * L * Wc + (size_t)y * Wc + w] ^= mine0;
      if (mine1) planes[(size_t)(c0 ^ 1u) * L * Wc + (size_t)y * Wc + w] ^= mine1;
    }
  }
}

// Bonds across tile edges (right edge: dir 0 from the last column; bottom edge:
// dir 1 from the last row; periodic), united in the global forest.
__global__ void __launch_bounds__(256) k_sw_edges(const uint32_t* __restrict__ planes, int L, int Wc,
                                                  uint32_t step, uint32_t thr, RngParams rng,
                                                  uint32_t* __restrict__ parent, uint32_t bond_tag,
                                                  const uint32_t* gate, const uint32_t* step_ptr) {
  if (gated_off(gate)) return;
  if (step_ptr) step = *step_ptr;
  const int tiles_x = L / kTileX;
  const long long n_tiles = (long long)tiles_x * (L / kTileY);
  const long long total = n_tiles * (kTileX + kTileY);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long tile = i / (kTileX + kTileY);
    const int k = (int)(i - tile * (kTileX + kTileY));
    const int tx = (int)(tile % tiles_x), ty = (int)(tile / tiles_x);
    int x, y, dir;
    if (k < kTileY) {
      x = tx * kTileX + kTileX - 1;
      y = ty * kTileY + k;
      dir = 0;
    } else {
      x = tx * kTileX + (k - kTileY);
      y = ty * kTileY + kTileY - 1;
      dir = 1;
    }
    const int xn = dir == 0 ? (x + 1 == L ? 0 : x + 1) : x;
    const int yn = dir == 0 ? y : (y + 1 == L ? 0 : y + 1);
    if (bit_at(planes, L, Wc, x, y) != bit_at(planes, L, Wc, xn, yn)) continue;
    const long long a = (long long)y * L + x;
    const uint4 r = philox10_rk(make_uint4((uint32_t)(a >> 1), step, rng.replica, bond_tag << 16),
                                rng.rk0, rng.rk1);
    const int wsel = 2 * (int)(a & 1) + dir;
    const uint32_t u = wsel == 0 ? r.x : (wsel == 1 ? r.y : (wsel == 2 ? r.z : r.w));
    if (u >= thr) continue;
    unite(parent, (uint32_t)a, (uint32_t)yn * (uint32_t)L + (uint32_t)xn);
  }
}

int grid_of(long long items) {
  long long g = (items + 255) / 256;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (int)g;
}

}  // namespace

bool sw_tiled(int L) { return L % kTileX == 0 && L % kTileY == 0 && L >= 2048; }

cudaError_t launch_cluster_labels(const BitsLattice& lat, uint32_t step, uint32_t thr, uint32_t bond_tag,
                                  const RngParams& rng, uint32_t* parent, uint8_t* mark,
                                  const uint32_t* gate, cudaStream_t s, const uint32_t* step_ptr) {
  const long long N = (long long)lat.L * lat.L;
  cudaError_t e;
  // tiles only pay when there are enough of them to fill the GPU (>= 512 CTAs)
  if (sw_tiled(lat.L)) {
    const long long tiles = (long long)(lat.L / kTileX) * (lat.L / kTileY);
    k_sw_local<<<(unsigned)tiles, kTileThreads, 0, s>>>(lat.planes, lat.L, lat.Wc, step, thr, rng, parent,
                                                        mark, bond_tag, gate, step_ptr);
    e = cudaGetLastError();
    if (e) return e;
    k_sw_edges<<<grid_of(tiles * (kTileX + kTileY)), 256, 0, s>>>(lat.planes, lat.L, lat.Wc, step, thr, rng,
                                                                  parent, bond_tag, gate, step_ptr);
    return cudaGetLastError();
  }
  k_sw_init<<<grid_of(N), 256, 0, s>>>(parent, N, gate);
  e = cudaGetLastError();
  if (e) return e;
  k_sw_bonds<<<grid_of((N + 1) / 2), 256, 0, s>>>(lat.planes, lat.L, lat.Wc, step, thr, rng, parent,
                                                  make_fastdiv((uint32_t)lat.L), bond_tag, gate, step_ptr);
  return cudaGetLastError();
}

cudaError_t launch_sw_step(const BitsLattice& lat, uint32_t step, uint32_t thr,
                           const RngParams& rng, uint32_t* parent, uint8_t* flip,
                           cudaStream_t s) {
  const long long N = (long long)lat.L * lat.L;
  cudaError_t e = launch_cluster_labels(lat, step, thr, kTagSWBond, rng, parent, flip, nullptr, s);
  if (e) return e;
  if (sw_tiled(lat.L)) {
    k_sw_resolve<<<grid_of(N), 256, 0, s>>>(parent, flip, N, step, rng);
    e = cudaGetLastError();
    if (e) return e;
    k_sw_coin_copy<<<grid_of(N), 256, 0, s>>>(parent, flip, N);
    e = cudaGetLastError();
    if (e) return e;
    k_sw_apply2<<<grid_of((long long)lat.L * lat.Wc * 32), 256, 0, s>>>(lat.planes, lat.L, lat.Wc,
                                                                        parent, flip);
    return cudaGetLastError();
  }
  k_sw_roots<<<grid_of(N), 256, 0, s>>>(parent, N, step, rng, flip);
  e = cudaGetLastError();
  if (e) return e;
  k_sw_apply<<<grid_of(2LL * lat.L * lat.Wc), 256, 0, s>>>(lat.planes, lat.L, lat.Wc, parent, flip,
                                                            make_fastdiv((uint32_t)lat.L * (uint32_t)lat.Wc),
                                                            make_fastdiv((uint32_t)lat.Wc));
  return cudaGetLastError();
}

}  // namespace ising
