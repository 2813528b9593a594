// Cluster steps (Swendsen-Wang and Wolff) as one persistent cooperative
// kernel per call, for lattices below the tiled-labelling size.  Below L = 2048
// a step's kernels each have little work and the step is bound by launch
// latency; here every CTA stays resident and a step is three phases between
// bounded grid barriers:
//   1. parent[i] = i for every site (and the previous step's observables);
//   2. bond draws and lock-free unions (links from the larger root to the
//      smaller, so each cluster's root is its smallest site);
//   3. every site walks to its root and flips iff: (SW) bit 31 of word (m & 3)
//      of Philox(m >> 2, step, replica, SW_FLIP << 16), m its root; (Wolff) its
//      root is the root of the seed site m = floor(u N / 2^32),
//      u = word 0 of Philox(0, step, replica, WOLFF_SEED << 16).
// Bond draws use the tag of the method (SW_BOND 10, WOLFF_BOND 17), so the
// chain is the same as the kernel-per-phase path's, bit for bit.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "ising_device.cuh"

namespace ising {
namespace {

constexpr uint32_t kTagSWBond = 10, kTagSWFlip = 11, kTagWolffSeed = 16, kTagWolffBond = 17;
constexpr int kPersistThreads = 256;

__device__ __forceinline__ uint32_t bit_at(const uint32_t* planes, int L, int Wc, int x, int y) {
  const int c = (x + y) & 1, j = x >> 1;
  return (__ldcg(&planes[(size_t)c * L * Wc + (size_t)y * Wc + (j >> 5)]) >> (j & 31)) & 1u;
}

__device__ __forceinline__ uint32_t find_root_ro(const uint32_t* parent, uint32_t a) {
  while (true) {
    const uint32_t p = __ldcg(&parent[a]);
    if (p == a) return a;
    a = p;
  }
}

__device__ __forceinline__ uint32_t find_root(uint32_t* parent, uint32_t a) {
  // path halving stores only ancestors of a (sets never split)
  while (true) {
    const uint32_t p = __ldcg(&parent[a]);
    if (p == a) return a;
    const uint32_t gp = __ldcg(&parent[p]);
    if (gp != p) __stcg(&parent[a], gp);
    a = gp;
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
    const uint32_t old = atomicCAS(&parent[a], a, b);
    if (old == a) return;
    a = old;
  }
}

__device__ __forceinline__ uint32_t pick(const uint4& r, uint32_t k) {
  return k == 0 ? r.x : (k == 1 ? r.y : (k == 2 ? r.z : r.w));
}

// Anti-parallel bonds (from every colour-0 site to its four neighbours) and up
// spins, added into dst[0], dst[1]; every thread of the grid calls it.
__device__ void measure_into(const uint32_t* planes, int L, int Wc, unsigned long long* dst) {
  const int n = L / 2;
  const long long words = (long long)L * Wc;
  const uint32_t* p0 = planes;
  const uint32_t* p1 = planes + (size_t)L * Wc;
  unsigned long long anti = 0, ones = 0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < words;
       idx += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(idx / Wc), w = (int)(idx - (idx / Wc) * Wc);
    const uint32_t* rm = p1 + (size_t)y * Wc;
    const uint32_t valid = valid_mask(w, Wc, n);
    const uint32_t s = __ldcg(&p0[(size_t)y * Wc + w]);
    const uint32_t up = __ldcg(&p1[(size_t)(y == 0 ? L - 1 : y - 1) * Wc + w]);
    const uint32_t dn = __ldcg(&p1[(size_t)(y == L - 1 ? 0 : y + 1) * Wc + w]);
    const uint32_t mid = __ldcg(&rm[w]);
    const uint32_t side = side_word([rm](int ww) { return __ldcg(&rm[ww]); }, w, Wc, n, y & 1);
    anti += __popc((s ^ up) & valid) + __popc((s ^ dn) & valid) + __popc((s ^ mid) & valid) +
            __popc((s ^ side) & valid);
    ones += __popc(s & valid) + __popc(mid & valid);
  }
  anti = warp_sum_u64(anti);
  ones = warp_sum_u64(ones);
  if ((threadIdx.x & 31) == 0) {
    if (anti) atomicAdd(&dst[0], anti);
    if (ones) atomicAdd(&dst[1], ones);
  }
}

template <bool WOLFF>
__global__ void __launch_bounds__(kPersistThreads)
    k_cluster_persist(uint32_t* __restrict__ planes, int L, int Wc, uint32_t step0, int n_steps, int measure_every,
                      uint32_t thr, RngParams rng, uint32_t* __restrict__ parent, unsigned long long* __restrict__ rec,
                      long long rec0, long long rec_cap, GridCtl* gctl, long long limit, WolffCtl* __restrict__ wctl,
                      FastDiv fL, FastDiv fplane, FastDiv fwc) {
  __shared__ uint32_t s_root, s_count;
  const uint32_t N = (uint32_t)L * (uint32_t)L;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const uint32_t bond_tag = WOLFF ? kTagWolffBond : kTagSWBond;
  long long pending = -1;  // record slot of the previous step, filled in the next phase 1
  const long long m = measure_every;
  const long long rec_before = m > 0 ? (long long)step0 / m : 0;  // records of steps < step0
  for (int s = 0; s < n_steps; ++s) {
    const uint32_t t = step0 + (uint32_t)s;
    // ---- phase 1 ----
    for (long long i = tid; i < N; i += nth) parent[i] = (uint32_t)i;
    if (pending >= 0) measure_into(planes, L, Wc, rec + 2 * pending);
    if (WOLFF && tid == 0) wctl->last_size = 0;  // phase 3 adds this step's cluster
    if (!grid_sync_bounded(gctl, limit)) return;
    // ---- phase 2: one thread per site pair, one Philox block for its four bonds ----
    for (long long pr = tid; 2 * pr < N; pr += nth) {
      const uint4 r = philox10_rk(make_uint4((uint32_t)pr, t, rng.replica, bond_tag << 16), rng.rk0, rng.rk1);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t a = 2 * (uint32_t)pr + h;
        if (a >= N) break;
        const int y = (int)fdiv(a, fL), x = (int)(a - (uint32_t)y * (uint32_t)L);
        const uint32_t sa = bit_at(planes, L, Wc, x, y);
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
          const int xn = dir == 0 ? (x + 1 == L ? 0 : x + 1) : x;
          const int yn = dir == 0 ? y : (y + 1 == L ? 0 : y + 1);
          if (bit_at(planes, L, Wc, xn, yn) != sa) continue;
          if (pick(r, 2 * h + dir) >= thr) continue;  // bond 2a + dir -> word (2a + dir) & 3
          unite(parent, a, (uint32_t)yn * (uint32_t)L + (uint32_t)xn);
        }
      }
    }
    if (!grid_sync_bounded(gctl, limit)) return;
    // ---- phase 3: flip (one warp per packed word, one lane per site) ----
    if (threadIdx.x == 0) {
      if (WOLFF) {
        const uint4 r = philox10_rk(make_uint4(0u, t, rng.replica, kTagWolffSeed << 16), rng.rk0, rng.rk1);
        const uint32_t seed_site = __umulhi(r.x, N);
        s_root = find_root_ro(parent, seed_site);
        if (blockIdx.x == 0) wctl->seed_site = seed_site;
      }
      s_count = 0;
    }
    __syncthreads();
    const int n = L / 2;
    const uint32_t words = 2u * (uint32_t)L * (uint32_t)Wc;
    const int lane = threadIdx.x & 31;
    uint32_t count = 0;
    for (uint32_t i = (uint32_t)(tid >> 5); i < words; i += (uint32_t)(nth >> 5)) {
      const int c = (int)fdiv(i, fplane);
      const uint32_t rem = i - (uint32_t)c * fplane.d;
      const int y = (int)fdiv(rem, fwc), w = (int)(rem - (uint32_t)y * (uint32_t)Wc);
      const int j = 32 * w + lane;
      bool f = false;
      if (j < n) {
        const int x = 2 * j + ((y + c) & 1);
        const uint32_t root = find_root_ro(parent, (uint32_t)y * (uint32_t)L + (uint32_t)x);
        if (WOLFF) {
          f = root == s_root;
        } else {
          const uint4 r = philox10_rk(make_uint4(root >> 2, t, rng.replica, kTagSWFlip << 16), rng.rk0, rng.rk1);
          f = (pick(r, root & 3u) >> 31) != 0;
        }
      }
      const uint32_t mask = __ballot_sync(0xffffffffu, f);
      if (lane == 0 && mask) {
        planes[i] ^= mask;
        count += __popc(mask);
      }
    }
    if (WOLFF) {
      if (lane == 0 && count) atomicAdd(&s_count, count);
      __syncthreads();
      if (threadIdx.x == 0 && s_count) {
        atomicAdd(&wctl->last_size, s_count);
        atomicAdd(&wctl->flipped, (unsigned long long)s_count);
      }
      if (tid == 0) {
        wctl->labelled += 1;
        wctl->need_label = 0;
      }
    }
    pending = -1;
    if (m > 0 && ((long long)t + 1) % m == 0) {
      // k-th record of this launch: records of steps <= t minus those before step0
      const long long k = ((long long)t + 1) / m - rec_before - 1;
      pending = (rec0 + k) % rec_cap;
      if (tid == 0) rec[2 * pending] = rec[2 * pending + 1] = 0ull;
    }
    if (!grid_sync_bounded(gctl, limit)) return;
  }
  if (pending >= 0) measure_into(planes, L, Wc, rec + 2 * pending);
}

}  // namespace

cudaError_t launch_cluster_persist(const BitsLattice& lat, bool wolff, uint32_t step0, int n_steps,
                                   int measure_every, uint32_t thr, const RngParams& rng, uint32_t* parent,
                                   unsigned long long* rec, long long rec0, long long rec_cap, GridCtl* gctl,
                                   WolffCtl* wctl, int sms, cudaStream_t s) {
  static DeviceCache occ[2];
  const void* fn = wolff ? (const void*)k_cluster_persist<true> : (const void*)k_cluster_persist<false>;
  long long per_sm = occ[wolff].get();
  if (!per_sm) {
    int b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kPersistThreads, 0);
    if (e) return e;
    per_sm = b > 0 ? b : 1;
    occ[wolff].set(per_sm);
  }
  const long long N = (long long)lat.L * lat.L;
  const long long want = (N / 2 + kPersistThreads - 1) / kPersistThreads;
  const long long grid = std::max(1LL, std::min(want, per_sm * sms));
  cudaError_t e = cudaMemsetAsync(&gctl->count, 0, sizeof(unsigned int), s);
  if (e) return e;
  uint32_t* planes = lat.planes;
  int L = lat.L, Wc = lat.Wc, n = n_steps, m = measure_every;
  uint32_t t0 = step0, th = thr;
  RngParams r = rng;
  long long r0 = rec0, cap = rec_cap, limit = kClusterSpinLimit;
  FastDiv fL = make_fastdiv((uint32_t)L), fplane = make_fastdiv((uint32_t)L * (uint32_t)Wc),
          fwc = make_fastdiv((uint32_t)Wc);
  void* args[] = {&planes, &L, &Wc, &t0, &n, &m, &th, &r, &parent, &rec, &r0, &cap, &gctl, &limit, &wctl,
                  &fL, &fplane, &fwc};
  return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kPersistThreads), args, 0, s);
}

}  // namespace ising
