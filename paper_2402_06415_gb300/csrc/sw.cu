// Swendsen-Wang cluster update on the packed lattice (Swendsen & Wang, PRL 58,
// 86 (1987)); the paper points to cluster updates as the step beyond its
// single-site Monte Carlo.  One step:
//   1. every bond between equal spins is active iff u < floor((1 - e^{-2 beta}) 2^32),
//      u = word (b & 3) of Philox(b >> 2, step, replica, SW_BOND << 16),
//      b = 2 (y L + x) + dir (dir 0: bond to x+1, 1: to y+1);
//   2. clusters = connected components of the active bonds, found by a lock-free
//      union-find whose links always point from the larger to the smaller site
//      index, so each cluster's root is its smallest site whatever the order in
//      which threads link;
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

__global__ void k_sw_init(uint32_t* __restrict__ parent, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    parent[i] = (uint32_t)i;
}

// One thread per pair of sites (a = 2p, 2p + 1): the four bonds of the pair use
// the four words of one Philox block.
__global__ void __launch_bounds__(256) k_sw_bonds(const uint32_t* __restrict__ planes, int L,
                                                  int Wc, uint32_t step, uint32_t thr,
                                                  RngParams rng, uint32_t* __restrict__ parent) {
  const long long N = (long long)L * L;
  for (long long pr = blockIdx.x * (long long)blockDim.x + threadIdx.x; 2 * pr < N;
       pr += (long long)gridDim.x * blockDim.x) {
    const uint4 r = philox10_rk(make_uint4((uint32_t)pr, step, rng.replica, kTagSWBond << 16),
                                rng.rk0, rng.rk1);
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long a = 2 * pr + h;
      if (a >= N) break;
      const int y = (int)(a / L), x = (int)(a - (a / L) * L);
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
                           const uint32_t* __restrict__ parent, const uint8_t* __restrict__ flip) {
  const int n = L / 2;
  const long long words = 2LL * L * Wc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < words;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / ((long long)L * Wc));
    const long long rem = i - (long long)c * L * Wc;
    const int y = (int)(rem / Wc), w = (int)(rem - (rem / Wc) * Wc);
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

int grid_of(long long items) {
  long long g = (items + 255) / 256;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (int)g;
}

}  // namespace

cudaError_t launch_sw_step(const BitsLattice& lat, uint32_t step, uint32_t thr,
                           const RngParams& rng, uint32_t* parent, uint8_t* flip,
                           cudaStream_t s) {
  const long long N = (long long)lat.L * lat.L;
  k_sw_init<<<grid_of(N), 256, 0, s>>>(parent, N);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  k_sw_bonds<<<grid_of((N + 1) / 2), 256, 0, s>>>(lat.planes, lat.L, lat.Wc, step, thr, rng, parent);
  e = cudaGetLastError();
  if (e) return e;
  k_sw_roots<<<grid_of(N), 256, 0, s>>>(parent, N, step, rng, flip);
  e = cudaGetLastError();
  if (e) return e;
  k_sw_apply<<<grid_of(2LL * lat.L * lat.Wc), 256, 0, s>>>(lat.planes, lat.L, lat.Wc, parent, flip);
  return cudaGetLastError();
}

}  // namespace ising
