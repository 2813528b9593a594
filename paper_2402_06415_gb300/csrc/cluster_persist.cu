// Cluster steps (Swendsen-Wang and Wolff) as one persistent cooperative
// kernel per call, for small lattices (by default L < 768), where a step's
// kernels each have little work and the step is bound by launch latency; here
// every CTA stays resident and a step is three phases between bounded grid
// barriers:
//   1. one warp per row draws the row's bonds and labels its horizontal runs
//      (each site's parent = the first site of its run, by a warp max-scan, no
//      atomics), and the previous step's observables are summed;
//   2. the vertical bonds and each row's wrap bond unite runs, lock-free, links
//      always from the larger root to the smaller, so each cluster's root is its
//      smallest site;
//   3. every site walks to its root and flips iff: (SW) bit 31 of word (m & 3)
//      of Philox(m >> 2, step, replica, SW_FLIP << 16), m its root; (Wolff) its
//      root is the root of the seed site m = floor(u N / 2^32),
//      u = word 0 of Philox(0, step, replica, WOLFF_SEED << 16).
// Bond draws use the tag of the method (SW_BOND 10, WOLFF_BOND 17), so the
// chain is the same as the kernel-per-phase path's, bit for bit.  Lattices of
// at most 4096 sites run the same steps in one CTA with the whole lattice in
// shared memory (k_cluster_smem), where the label walks cost shared-memory
// rather than L2 latency and a step needs only CTA barriers.
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
                      uint32_t thr, RngParams rng, uint32_t* __restrict__ parent, uint8_t* __restrict__ mark,
                      unsigned long long* __restrict__ rec,
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
    // ---- phase 1: bond draws and horizontal runs, one warp per row ----
    // Every site's parent becomes the first site of its run of active
    // horizontal bonds (runs stop at x = L - 1; the wrap bond joins in phase 2),
    // and mark[] keeps bit 1 = bond to x+1 active, bit 2 = bond to y+1 active.
    {
      const int lane = threadIdx.x & 31;
      const int k = (((L + 31) >> 5) + 1) & ~1;  // sites per lane, even so pairs stay whole
      for (long long row = tid >> 5; row < L; row += nth >> 5) {
        const int y = (int)row, yn = y + 1 == L ? 0 : y + 1;
        const int x0 = lane * k;
        const uint32_t base = (uint32_t)y * (uint32_t)L;
        unsigned long long hbits = 0;  // bonds to x+1 of the lane's first 64 sites, in registers
        for (int q = 0; q < k && x0 + q < L; q += 2) {
          const int x = x0 + q;
          const uint4 r = philox10_rk(make_uint4((base + (uint32_t)x) >> 1, t, rng.replica, bond_tag << 16),
                                      rng.rk0, rng.rk1);
          const uint32_t s0 = bit_at(planes, L, Wc, x, y), s1 = bit_at(planes, L, Wc, x + 1, y);
          const uint32_t s2 = bit_at(planes, L, Wc, x + 2 == L ? 0 : x + 2, y);
          const uint32_t d0 = bit_at(planes, L, Wc, x, yn), d1 = bit_at(planes, L, Wc, x + 1, yn);
          const bool h0 = r.x < thr && s0 == s1, v0 = r.y < thr && s0 == d0;
          const bool h1 = r.z < thr && s1 == s2, v1 = r.w < thr && s1 == d1;
          mark[base + x] = (uint8_t)((h0 ? 2u : 0u) | (v0 ? 4u : 0u));
          mark[base + x + 1] = (uint8_t)((h1 ? 2u : 0u) | (v1 ? 4u : 0u));
          if (q < 64) hbits |= ((unsigned long long)h0 | ((unsigned long long)h1 << 1)) << q;
        }
        const int nq = max(0, min(k, L - x0));  // sites of this lane
        // bond x -> x + 1 of this lane's sites: registers, or (past 64 sites a
        // lane, L > 2048) this thread's own mark[] stores above
        const uint8_t* own = mark + base + x0;
        auto hb = [hbits, own](int q) { return q < 64 ? ((hbits >> q) & 1ull) != 0 : (own[q] & 2u) != 0; };
        // whether the previous lane's last bond to the right is active (then this
        // lane's first site continues that run)
        const bool open_right = nq > 0 && hb(nq - 1);
        const bool enters = __shfl_up_sync(0xffffffffu, open_right, 1) && lane > 0;
        int last = -1;  // the last run start in this lane's sites
        for (int q = 0; q < nq; ++q)
          if (q == 0 ? !enters : !hb(q - 1)) last = x0 + q;
        int carry = last;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, carry, off);
          if (lane >= off) carry = max(carry, v);
        }
        int cur = __shfl_up_sync(0xffffffffu, carry, 1);
        if (lane == 0) cur = 0;
        for (int q = 0; q < nq; ++q) {
          const int x = x0 + q;
          if (q == 0 ? !enters : !hb(q - 1)) cur = x;
          parent[base + x] = base + (uint32_t)cur;
        }
      }
    }
    if (pending >= 0) measure_into(planes, L, Wc, rec + 2 * pending);
    if (WOLFF && tid == 0) wctl->last_size = 0;  // phase 3 adds this step's cluster
    if (!grid_sync_bounded(gctl, limit)) return;
    // ---- phase 2: vertical bonds and the wrap bond of each row unite runs ----
    for (long long i = tid; i < N; i += nth) {
      const uint32_t b = __ldcg(&mark[i]);
      if (!(b & 6u)) continue;
      const uint32_t a = (uint32_t)i;
      const uint32_t y = fdiv(a, fL), x = a - y * (uint32_t)L;
      if (b & 4u) {
        const uint32_t an = (y + 1 == (uint32_t)L ? 0u : y + 1) * (uint32_t)L + x;
        // the left neighbour's vertical bond already joined the same two runs
        const bool skip = x > 0 && (__ldcg(&mark[a - 1]) & 6u) == 6u && (__ldcg(&mark[an - 1]) & 2u);
        if (!skip) unite(parent, a, an);
      }
      if ((b & 2u) && x + 1 == (uint32_t)L) unite(parent, a, a - x);
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


// ---- whole lattice in one CTA's shared memory (L * L <= 65536) ----
// The same three steps with every access in shared memory: labels are 16-bit
// site indices (lab), st[] holds per site bit 0 spin, bit 1 bond to x+1, bit 2
// bond to y+1, bit 3 the coin of a Swendsen-Wang root.  Spins are read from the
// packed planes once per call and written back at its end.
constexpr int kSmemThreads = 1024;
constexpr int kSmemMaxSites = 65536;  // 16-bit labels
// One SM does all the work here: measured on GB300 it beats the grid kernel's
// L2-latency-bound phases up to about 64 x 64 sites (16 x 16: 4.8 vs 28 us per
// step) and loses beyond (128 x 128: 91 vs 41 us).
constexpr int kSmemAutoMaxSites = 4096;  // 12 KB of shared memory
static_assert(kSmemAutoMaxSites <= kSmemMaxSites, "labels are 16-bit");

__device__ __forceinline__ uint32_t sfind16(uint16_t* lab, uint32_t a) {
  volatile uint16_t* v = lab;
  while (true) {
    const uint32_t p = v[a];
    if (p == a) return a;
    const uint32_t gp = v[p];
    if (gp != p) v[a] = (uint16_t)gp;  // an ancestor: stays in a's set
    a = gp;
  }
}

__device__ __forceinline__ uint32_t sfind16_ro(const uint16_t* lab, uint32_t a) {
  const volatile uint16_t* v = lab;
  while (true) {
    const uint32_t p = v[a];
    if (p == a) return a;
    a = p;
  }
}

__device__ __forceinline__ void sunite16(uint16_t* lab, uint32_t a, uint32_t b) {
  while (true) {
    a = sfind16(lab, a);
    b = sfind16(lab, b);
    if (a == b) return;
    if (a < b) {
      const uint32_t t = a;
      a = b;
      b = t;
    }
    const uint32_t old = atomicCAS(reinterpret_cast<unsigned short*>(&lab[a]), (unsigned short)a, (unsigned short)b);
    if (old == a) return;
    a = old;
  }
}

template <bool WOLFF>
__global__ void __launch_bounds__(kSmemThreads, 1)
    k_cluster_smem(uint32_t* __restrict__ planes, int L, int Wc, uint32_t step0, int n_steps, int measure_every,
                   uint32_t thr, RngParams rng, unsigned long long* __restrict__ rec, long long rec0,
                   long long rec_cap, WolffCtl* __restrict__ wctl, FastDiv fL, FastDiv fplane, FastDiv fwc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const uint32_t N = (uint32_t)L * (uint32_t)L;
  uint16_t* lab = reinterpret_cast<uint16_t*>(smraw);
  uint8_t* st = smraw + 2 * (size_t)N;
  __shared__ unsigned long long s_anti, s_ones;
  __shared__ uint32_t s_root, s_count;
  const uint32_t tid = threadIdx.x, nth = blockDim.x;
  const int lane = (int)(tid & 31), warp = (int)(tid >> 5), nwarps = (int)(nth >> 5);
  const uint32_t bond_tag = WOLFF ? kTagWolffBond : kTagSWBond;
  for (uint32_t li = tid; li < N; li += nth) {
    const uint32_t y = fdiv(li, fL), x = li - y * (uint32_t)L;
    st[li] = (uint8_t)bit_at(planes, L, Wc, (int)x, (int)y);
  }
  __syncthreads();
  const long long m = measure_every;
  const long long rec_before = m > 0 ? (long long)step0 / m : 0;
  const int k = (((L + 31) >> 5) + 1) & ~1;  // sites per lane, even so pairs stay whole
  for (int s = 0; s < n_steps; ++s) {
    const uint32_t t = step0 + (uint32_t)s;
    // bonds and horizontal runs, one warp per row
    for (int y = warp; y < L; y += nwarps) {
      const int yn = y + 1 == L ? 0 : y + 1;
      const uint32_t base = (uint32_t)y * (uint32_t)L, below = (uint32_t)yn * (uint32_t)L;
      const int x0 = lane * k;
      for (int q = 0; q < k && x0 + q < L; q += 2) {
        const uint32_t x = (uint32_t)(x0 + q);
        const uint4 r = philox10_rk(make_uint4((base + x) >> 1, t, rng.replica, bond_tag << 16), rng.rk0, rng.rk1);
        // bit 0 of every byte is stable while other threads rewrite bits 1-3
        const uint32_t s0 = st[base + x] & 1u, s1 = st[base + x + 1] & 1u;
        const uint32_t s2 = st[base + (x + 2 == (uint32_t)L ? 0u : x + 2)] & 1u;
        const uint32_t d0 = st[below + x] & 1u, d1 = st[below + x + 1] & 1u;
        const bool h0 = r.x < thr && s0 == s1, v0 = r.y < thr && s0 == d0;
        const bool h1 = r.z < thr && s1 == s2, v1 = r.w < thr && s1 == d1;
        st[base + x] = (uint8_t)(s0 | (h0 ? 2u : 0u) | (v0 ? 4u : 0u));
        st[base + x + 1] = (uint8_t)(s1 | (h1 ? 2u : 0u) | (v1 ? 4u : 0u));
      }
      const int nq = max(0, min(k, L - x0));
      auto hb = [&](int q) { return (st[base + x0 + q] & 2u) != 0; };
      const bool open_right = nq > 0 && hb(nq - 1);
      const bool enters = __shfl_up_sync(0xffffffffu, open_right, 1) && lane > 0;
      int last = -1;
      for (int q = 0; q < nq; ++q)
        if (q == 0 ? !enters : !hb(q - 1)) last = x0 + q;
      int carry = last;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, carry, off);
        if (lane >= off) carry = max(carry, v);
      }
      int cur = __shfl_up_sync(0xffffffffu, carry, 1);
      if (lane == 0) cur = 0;
      for (int q = 0; q < nq; ++q) {
        if (q == 0 ? !enters : !hb(q - 1)) cur = x0 + q;
        lab[base + x0 + q] = (uint16_t)(base + (uint32_t)cur);
      }
    }
    __syncthreads();
    // vertical bonds and each row's wrap bond unite runs
    for (uint32_t li = tid; li < N; li += nth) {
      const uint32_t b = st[li];
      if (!(b & 6u)) continue;
      const uint32_t y = fdiv(li, fL), x = li - y * (uint32_t)L;
      if (b & 4u) {
        const uint32_t an = (y + 1 == (uint32_t)L ? 0u : y + 1) * (uint32_t)L + x;
        const bool skip = x > 0 && (st[li - 1] & 6u) == 6u && (st[an - 1] & 2u);
        if (!skip) sunite16(lab, li, an);
      }
      if ((b & 2u) && x + 1 == (uint32_t)L) sunite16(lab, li, li - x);
    }
    __syncthreads();
    for (uint32_t li = tid; li < N; li += nth) lab[li] = (uint16_t)sfind16_ro(lab, li);
    if (tid == 0) {
      s_anti = 0;
      s_ones = 0;
      s_count = 0;
      if (WOLFF) {
        const uint4 r = philox10_rk(make_uint4(0u, t, rng.replica, kTagWolffSeed << 16), rng.rk0, rng.rk1);
        wctl->seed_site = __umulhi(r.x, N);
      }
    }
    __syncthreads();
    if (WOLFF) {
      if (tid == 0) s_root = lab[__umulhi(philox10_rk(make_uint4(0u, t, rng.replica, kTagWolffSeed << 16), rng.rk0,
                                                      rng.rk1).x, N)];
    } else {
      for (uint32_t li = tid; li < N; li += nth)
        if (lab[li] == li) {
          const uint4 r = philox10_rk(make_uint4(li >> 2, t, rng.replica, kTagSWFlip << 16), rng.rk0, rng.rk1);
          st[li] |= (uint8_t)((pick(r, li & 3u) >> 31) << 3);
        }
    }
    __syncthreads();
    uint32_t count = 0;
    for (uint32_t li = tid; li < N; li += nth) {
      const uint32_t root = lab[li];
      const bool f = WOLFF ? root == s_root : ((st[root] >> 3) & 1u) != 0;
      if (f) {
        st[li] ^= 1u;  // the owner's read-modify-write keeps bit 3, which others read
        ++count;
      }
    }
    if (WOLFF) {
      count = __reduce_add_sync(0xffffffffu, count);
      if (lane == 0 && count) atomicAdd(&s_count, count);
    }
    __syncthreads();
    if (m > 0 && ((long long)t + 1) % m == 0) {
      unsigned long long anti = 0, ones = 0;
      for (uint32_t li = tid; li < N; li += nth) {
        const uint32_t y = fdiv(li, fL), x = li - y * (uint32_t)L;
        const uint32_t sv = st[li] & 1u;
        const uint32_t right = st[y * (uint32_t)L + (x + 1 == (uint32_t)L ? 0u : x + 1)] & 1u;
        const uint32_t down = st[(y + 1 == (uint32_t)L ? 0u : y + 1) * (uint32_t)L + x] & 1u;
        anti += (sv ^ right) + (sv ^ down);
        ones += sv;
      }
      anti = warp_sum_u64(anti);
      ones = warp_sum_u64(ones);
      if (lane == 0) {
        atomicAdd(&s_anti, anti);
        atomicAdd(&s_ones, ones);
      }
      __syncthreads();
      if (tid == 0) {
        const long long slot = (rec0 + ((long long)t + 1) / m - rec_before - 1) % rec_cap;
        rec[2 * slot] = s_anti;
        rec[2 * slot + 1] = s_ones;
      }
    }
    if (WOLFF && tid == 0) {
      wctl->last_size = s_count;
      wctl->flipped += s_count;
      wctl->labelled += 1;
      wctl->need_label = 0;
    }
    __syncthreads();
  }
  const int n = L / 2;
  const uint32_t words = 2u * (uint32_t)L * (uint32_t)Wc;
  for (uint32_t i = tid; i < words; i += nth) {
    const uint32_t c = fdiv(i, fplane), rem = i - c * fplane.d;
    const uint32_t y = fdiv(rem, fwc), w = rem - y * (uint32_t)Wc;
    uint32_t word = 0;
    for (int b = 0; b < 32; ++b) {
      const int j = 32 * (int)w + b;
      if (j >= n) break;
      const uint32_t x = 2u * (uint32_t)j + ((y + c) & 1u);
      word |= (uint32_t)(st[y * (uint32_t)L + x] & 1u) << b;
    }
    planes[i] = word;
  }
}
}  // namespace

cudaError_t launch_cluster_persist(const BitsLattice& lat, bool wolff, uint32_t step0, int n_steps,
                                   int measure_every, uint32_t thr, const RngParams& rng, uint32_t* parent,
                                   uint8_t* mark, unsigned long long* rec, long long rec0, long long rec_cap, GridCtl* gctl,
                                   WolffCtl* wctl, int sms, cudaStream_t s) {
  const long long N = (long long)lat.L * lat.L;
  const FastDiv fL = make_fastdiv((uint32_t)lat.L), fplane = make_fastdiv((uint32_t)lat.L * (uint32_t)lat.Wc),
                fwc = make_fastdiv((uint32_t)lat.Wc);
  if (N <= kSmemAutoMaxSites) {
    const size_t smem = 3 * (size_t)N;
    if (wolff)
      k_cluster_smem<true><<<1, kSmemThreads, smem, s>>>(lat.planes, lat.L, lat.Wc, step0, n_steps, measure_every, thr,
                                                         rng, rec, rec0, rec_cap, wctl, fL, fplane, fwc);
    else
      k_cluster_smem<false><<<1, kSmemThreads, smem, s>>>(lat.planes, lat.L, lat.Wc, step0, n_steps, measure_every,
                                                          thr, rng, rec, rec0, rec_cap, wctl, fL, fplane, fwc);
    return cudaGetLastError();
  }
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
  // one thread per site in the union and flip phases (one warp per 32-site word)
  const long long want = (N + kPersistThreads - 1) / kPersistThreads;
  const long long grid = std::max(1LL, std::min(want, per_sm * sms));
  cudaError_t e = cudaMemsetAsync(&gctl->count, 0, sizeof(unsigned int), s);
  if (e) return e;
  uint32_t* planes = lat.planes;
  int L = lat.L, Wc = lat.Wc, n = n_steps, m = measure_every;
  uint32_t t0 = step0, th = thr;
  RngParams r = rng;
  long long r0 = rec0, cap = rec_cap, limit = kClusterSpinLimit;
  FastDiv fl = fL, fp = fplane, fw = fwc;
  void* args[] = {&planes, &L, &Wc, &t0, &n, &m, &th, &r, &parent, &mark, &rec, &r0, &cap, &gctl, &limit, &wctl,
                  &fl, &fp, &fw};
  return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kPersistThreads), args, 0, s);
}

}  // namespace ising
