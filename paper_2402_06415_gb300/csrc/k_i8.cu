// int8 (+-1 per byte) checkerboard Metropolis kernels.
//
// One warp handles one 32-site group (32 colour-c sites of a row, lane i =
// site j = 32w + i).  The group's 32 plane words come from 8 Philox blocks (one
// per lane 0..7); a 32 x 32 bit transpose by warp ballots gives every lane its
// full 32-bit uniform, which is compared with the integer threshold directly.
// This is a second, independent route to the same decisions as the bit-sliced
// path in k_bits.cu.
#include "internal.h"
#include "ising_device.cuh"

namespace ising {
namespace {

constexpr unsigned kAll = 0xffffffffu;

__device__ __forceinline__ uint32_t group_uniform(uint32_t g, uint32_t t, uint32_t rep,
                                                  uint32_t c, uint32_t k0, uint32_t k1) {
  const int lane = threadIdx.x & 31;
  uint4 r = make_uint4(0u, 0u, 0u, 0u);
  if (lane < 8) r = philox10(make_uint4(g, t, rep, ctr_w(kTagMet, c, (uint32_t)lane)), k0, k1);
  const int src = lane >> 2;
  const uint32_t a = __shfl_sync(kAll, r.x, src);
  const uint32_t b = __shfl_sync(kAll, r.y, src);
  const uint32_t d = __shfl_sync(kAll, r.z, src);
  const uint32_t e = __shfl_sync(kAll, r.w, src);
  const int q = lane & 3;
  const uint32_t P = q == 0 ? a : (q == 1 ? b : (q == 2 ? d : e));  // plane `lane`
  uint32_t u = 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const uint32_t m = __ballot_sync(kAll, (P >> i) & 1u);  // bit k = bit i of plane k
    if (lane == i) u = __brev(m);                            // plane 0 -> bit 31
  }
  return u;
}

__device__ __forceinline__ int8_t at(const int8_t* s, int L, int x, int y) {
  x = x < 0 ? x + L : (x >= L ? x - L : x);
  y = y < 0 ? y + L : (y >= L ? y - L : y);
  return s[y * L + x];
}

// Half sweep of one group (whole warp).  Returns nothing; updates s in place.
__device__ __forceinline__ void group_update(int8_t* s, int L, int Wc, int y, int w, int c,
                                             uint32_t t, const RngParams& rng) {
  const int lane = threadIdx.x & 31;
  const uint32_t g = (uint32_t)y * Wc + w;
  const uint32_t u = group_uniform(g, t, rng.replica, (uint32_t)c, rng.key0, rng.key1);
  const int j = 32 * w + lane;
  if (j < L / 2) {
    const int x = 2 * j + ((y + c) & 1);
    const int8_t v = s[y * L + x];
    const int n = (at(s, L, x + 1, y) != v) + (at(s, L, x - 1, y) != v) +
                  (at(s, L, x, y + 1) != v) + (at(s, L, x, y - 1) != v);
    const bool flip = n >= 2 || (n == 1 && u < rng.t4) || (n == 0 && u < rng.t8);
    if (flip) s[y * L + x] = (int8_t)-v;
  }
}

// Counts antiparallel bonds (right and down neighbour of every site) and up
// spins of s over the threads of the calling block; returns the block totals
// in thread 0.
__device__ void block_count(const int8_t* s, int L, unsigned long long& anti_out,
                            unsigned long long& ones_out) {
  __shared__ unsigned long long sh[2][32];
  unsigned long long anti = 0, ones = 0;
  for (int i = threadIdx.x; i < L * L; i += blockDim.x) {
    const int y = i / L, x = i - (i / L) * L;
    const int8_t v = s[i];
    anti += (at(s, L, x + 1, y) != v) + (at(s, L, x, y + 1) != v);
    ones += v > 0;
  }
  anti = warp_sum_u64(anti);
  ones = warp_sum_u64(ones);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) {
    sh[0][warp] = anti;
    sh[1][warp] = ones;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    anti = lane < nw ? sh[0][lane] : 0ull;
    ones = lane < nw ? sh[1][lane] : 0ull;
    anti = warp_sum_u64(anti);
    ones = warp_sum_u64(ones);
  }
  anti_out = anti;
  ones_out = ones;
}

__global__ void k_init_i8(int8_t* __restrict__ s, int L, RngParams rng) {
  const int Wc = (L / 2 + 31) / 32;
  const long long N = (long long)L * L;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / L), x = (int)(i - (i / L) * L);
    const int c = (x + y) & 1, j = x >> 1;
    const uint32_t g = (uint32_t)y * Wc + (uint32_t)(j >> 5);
    const uint4 r = philox10(make_uint4(g, 0u, rng.replica, ctr_w(kTagInit, c, 0)), rng.key0,
                             rng.key1);
    s[i] = ((r.x >> (j & 31)) & 1u) ? 1 : -1;
  }
}

// Whole lattice in shared memory of one CTA; n_sweeps sweeps; after sweep t
// with (t+1) % measure_every == 0 the (anti, ones) counts go to record slot
// (slot0 + (t - first_t) / measure_every) % cap.
__global__ void __launch_bounds__(1024) k_resident_i8(int8_t* __restrict__ g_s, int L,
                                                      RngParams rng, uint32_t t0, int n_sweeps,
                                                      int measure_every, uint32_t first_t,
                                                      long long slot0, long long cap,
                                                      unsigned long long* __restrict__ rec) {
  extern __shared__ int8_t s[];
  const int N = L * L;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s[i] = g_s[i];
  __syncthreads();
  const int Wc = (L / 2 + 31) / 32;
  const int groups = L * Wc;
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int k = 0; k < n_sweeps; ++k) {
    const uint32_t t = t0 + (uint32_t)k;
    for (int c = 0; c < 2; ++c) {
      for (int gi = warp; gi < groups; gi += nwarps) group_update(s, L, Wc, gi / Wc, gi % Wc, c, t, rng);
      __syncthreads();
    }
    if (measure_every > 0 && ((unsigned long long)t + 1) % (unsigned)measure_every == 0) {
      unsigned long long anti, ones;
      block_count(s, L, anti, ones);
      if (threadIdx.x == 0) {
        const long long slot = (slot0 + (long long)(t - first_t) / measure_every) % cap;
        rec[2 * slot] = anti;
        rec[2 * slot + 1] = ones;
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) g_s[i] = s[i];
}

__global__ void __launch_bounds__(256) k_half_sweep_i8(int8_t* __restrict__ s, int L,
                                                       RngParams rng, int c, uint32_t t) {
  const int Wc = (L / 2 + 31) / 32;
  const long long groups = (long long)L * Wc;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long gi = warp; gi < groups; gi += nw)
    group_update(s, L, Wc, (int)(gi / Wc), (int)(gi % Wc), c, t, rng);
}

__global__ void __launch_bounds__(256) k_measure_i8(const int8_t* __restrict__ s, int L,
                                                    unsigned long long* __restrict__ out2) {
  __shared__ unsigned long long sh[2][32];
  unsigned long long anti = 0, ones = 0;
  const long long N = (long long)L * L;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / L), x = (int)(i - (i / L) * L);
    const int8_t v = s[i];
    anti += (at(s, L, x + 1, y) != v) + (at(s, L, x, y + 1) != v);
    ones += v > 0;
  }
  anti = warp_sum_u64(anti);
  ones = warp_sum_u64(ones);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh[0][warp] = anti;
    sh[1][warp] = ones;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    anti = warp_sum_u64(lane < nw ? sh[0][lane] : 0ull);
    ones = warp_sum_u64(lane < nw ? sh[1][lane] : 0ull);
    if (lane == 0) {
      atomicAdd(out2, anti);
      atomicAdd(out2 + 1, ones);
    }
  }
}

int grid_for(long long items, int block) {
  long long g = (items + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 152 * 64) g = 152 * 64;
  return (int)g;
}

}  // namespace

cudaError_t launch_init_i8(int8_t* s, int L, const RngParams& rng, cudaStream_t st) {
  k_init_i8<<<grid_for((long long)L * L, 256), 256, 0, st>>>(s, L, rng);
  return cudaGetLastError();
}

size_t resident_i8_smem_bytes(int L) { return (size_t)L * (size_t)L; }

cudaError_t launch_resident_sweep_i8(int8_t* s, int L, const RngParams& rng, uint32_t sweep0,
                                     int n_sweeps, int measure_every, uint32_t rec_first_t,
                                     long long rec_slot0, long long rec_cap,
                                     unsigned long long* rec, cudaStream_t st) {
  const size_t smem = resident_i8_smem_bytes(L);
  cudaError_t e = cudaFuncSetAttribute(k_resident_i8, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_resident_i8<<<1, 1024, smem, st>>>(s, L, rng, sweep0, n_sweeps, measure_every, rec_first_t,
                                       rec_slot0, rec_cap, rec);
  return cudaGetLastError();
}

cudaError_t launch_half_sweep_i8(int8_t* s, int L, const RngParams& rng, int colour,
                                 uint32_t sweep, unsigned long long* rec, cudaStream_t st) {
  const long long groups = (long long)L * ((L / 2 + 31) / 32);
  k_half_sweep_i8<<<grid_for(groups * 32, 256), 256, 0, st>>>(s, L, rng, colour, sweep);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || rec == nullptr) return e;
  return launch_measure_i8(s, L, rec, st);
}

cudaError_t launch_measure_i8(const int8_t* s, int L, unsigned long long* out2, cudaStream_t st) {
  k_measure_i8<<<grid_for((long long)L * L, 256), 256, 0, st>>>(s, L, out2);
  return cudaGetLastError();
}

}  // namespace ising
