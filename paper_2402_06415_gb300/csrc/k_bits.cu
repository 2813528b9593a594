// Multi-spin-coded (1 bit per spin) checkerboard Metropolis kernels.
//
// Layout: two colour planes, plane c = [L rows][pitch words]; word w of row y
// holds the colour-c sites j = 32w .. 32w+31 of that row (x = 2j + ((y+c)&1)).
// A half sweep updates every colour-c site from its four colour-(1-c)
// neighbours (arXiv 2402.06415, Results A / Fig. 2: bipartite update); one
// thread handles one 32-site word.
#include "internal.h"
#include "ising_device.cuh"

namespace ising {
namespace {

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

__global__ void k_init_bits(uint32_t* __restrict__ planes, int L, int Wc, int pitch,
                            RngParams rng) {
  const int n = L / 2;
  const long long per_plane = (long long)L * Wc;
  const long long total = 2 * per_plane;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / per_plane);
    const long long rem = i - c * per_plane;
    const int y = (int)(rem / Wc), w = (int)(rem - (long long)y * Wc);
    const uint32_t g = (uint32_t)y * (uint32_t)Wc + (uint32_t)w;
    const uint4 r = philox10(make_uint4(g, 0u, rng.replica, ctr_w(kTagInit, c, 0)), rng.key0,
                             rng.key1);
    planes[(size_t)c * L * pitch + (size_t)y * pitch + w] = r.x & valid_mask(w, Wc, n);
  }
}

// One half sweep of colour c, in place.  With MEASURE (colour 1 only) it also
// counts, after the update, the antiparallel bonds of every colour-1 site (each
// bond of the lattice exactly once) and the up spins of both colours.
template <bool MEASURE>
__global__ void __launch_bounds__(256) k_half_sweep_bits(uint32_t* __restrict__ planes, int L,
                                                         int Wc, int pitch, int c, uint32_t t,
                                                         RngParams rng,
                                                         unsigned long long* __restrict__ rec) {
  const int n = L / 2;
  const long long words = (long long)L * Wc;
  uint32_t* own = planes + (size_t)c * L * pitch;
  const uint32_t* oth = planes + (size_t)(1 - c) * L * pitch;
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  unsigned long long anti = 0, ones = 0;
  for (long long base = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); base < words;
       base += stride) {
    const long long idx = base + lane;
    const bool active = idx < words;
    int y = 0, w = 0;
    if (active) {
      y = (int)(idx / Wc);
      w = (int)(idx - (long long)y * Wc);
    }
    const uint32_t* rm = oth + (size_t)y * pitch;
    const uint32_t* ru = oth + (size_t)(y == 0 ? L - 1 : y - 1) * pitch;
    const uint32_t* rd = oth + (size_t)(y == L - 1 ? 0 : y + 1) * pitch;
    uint32_t valid = 0, s = 0, up = 0, dn = 0, mid = 0, side = 0;
    if (active) {
      valid = valid_mask(w, Wc, n);
      s = own[(size_t)y * pitch + w];
      up = ru[w];
      dn = rd[w];
      mid = rm[w];
      side = side_word([rm](int ww) { return rm[ww]; }, w, Wc, n, (y + c) & 1);
    }
    const Classes k = classify(s, up, dn, mid, side);
    const uint32_t f = flip_mask(k, valid, (uint32_t)y * Wc + w, t, rng.replica, c, rng.key0,
                                 rng.key1, rng.t4, rng.t8);
    if (active) {
      const uint32_t ns = s ^ f;
      own[(size_t)y * pitch + w] = ns;
      if (MEASURE) {
        anti += __popc((ns ^ up) & valid) + __popc((ns ^ dn) & valid) +
                __popc((ns ^ mid) & valid) + __popc((ns ^ side) & valid);
        ones += __popc(ns & valid) + __popc(mid & valid);
      }
    }
  }
  if (MEASURE) block_add2(anti, ones, rec);
}

// Observables of the current configuration: antiparallel bonds counted from
// every colour-0 site to its four colour-1 neighbours, and up spins.
__global__ void __launch_bounds__(256) k_measure_bits(const uint32_t* __restrict__ planes, int L,
                                                      int Wc, int pitch,
                                                      unsigned long long* __restrict__ out2) {
  const int n = L / 2;
  const long long words = (long long)L * Wc;
  const uint32_t* p0 = planes;
  const uint32_t* p1 = planes + (size_t)L * pitch;
  unsigned long long anti = 0, ones = 0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < words;
       idx += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(idx / Wc), w = (int)(idx - (idx / Wc) * Wc);
    const uint32_t* rm = p1 + (size_t)y * pitch;
    const uint32_t valid = valid_mask(w, Wc, n);
    const uint32_t s = p0[(size_t)y * pitch + w];
    const uint32_t up = p1[(size_t)(y == 0 ? L - 1 : y - 1) * pitch + w];
    const uint32_t dn = p1[(size_t)(y == L - 1 ? 0 : y + 1) * pitch + w];
    const uint32_t mid = rm[w];
    const uint32_t side = side_word([rm](int ww) { return rm[ww]; }, w, Wc, n, y & 1);
    anti += __popc((s ^ up) & valid) + __popc((s ^ dn) & valid) + __popc((s ^ mid) & valid) +
            __popc((s ^ side) & valid);
    ones += __popc(s & valid) + __popc(mid & valid);
  }
  block_add2(anti, ones, out2);
}

__global__ void k_unpack_bits(const uint32_t* __restrict__ planes, int L, int Wc, int pitch,
                              int8_t* __restrict__ spins) {
  const long long N = (long long)L * L;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(i / L), x = (int)(i - (i / L) * L);
    const int c = (x + y) & 1, j = x >> 1;
    const uint32_t wv = planes[(size_t)c * L * pitch + (size_t)y * pitch + (j >> 5)];
    spins[i] = ((wv >> (j & 31)) & 1u) ? 1 : -1;
  }
}

__global__ void k_pack_bits(uint32_t* __restrict__ planes, int L, int Wc, int pitch,
                            const int8_t* __restrict__ spins) {
  const int n = L / 2;
  const long long total = 2LL * L * Wc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / ((long long)L * Wc));
    const long long rem = i - (long long)c * L * Wc;
    const int y = (int)(rem / Wc), w = (int)(rem - (rem / Wc) * Wc);
    uint32_t v = 0;
    for (int b = 0; b < 32; ++b) {
      const int j = 32 * w + b;
      if (j >= n) break;
      const int x = 2 * j + ((y + c) & 1);
      if (spins[(size_t)y * L + x] > 0) v |= 1u << b;
    }
    planes[(size_t)c * L * pitch + (size_t)y * pitch + w] = v;
  }
}

int grid_for(long long items, int block) {
  long long g = (items + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 152 * 64) g = 152 * 64;
  return (int)g;
}

}  // namespace

// Per-K tiled launchers (k_tiled_k<K>.cu).
#define ISING_TILED_DECLARE(K)                                                                   \
  cudaError_t launch_tiled_k##K(const BitsLattice&, uint32_t*, const RngParams&, uint32_t,       \
                                const RecordSlots&, unsigned long long*, int, int, int, int,     \
                                cudaStream_t);                                                   \
  cudaError_t launch_tiled32_k##K##_w1(const BitsLattice&, uint32_t*, const RngParams&, uint32_t, \
                                       const RecordSlots&, unsigned long long*, int, int,        \
                                       cudaStream_t);                                            \
  cudaError_t launch_tiled32_k##K##_w2(const BitsLattice&, uint32_t*, const RngParams&, uint32_t, \
                                       const RecordSlots&, unsigned long long*, int, int,        \
                                       cudaStream_t);
ISING_TILED_DECLARE(1)
ISING_TILED_DECLARE(2)
ISING_TILED_DECLARE(3)
ISING_TILED_DECLARE(4)
ISING_TILED_DECLARE(5)
ISING_TILED_DECLARE(6)
ISING_TILED_DECLARE(7)
ISING_TILED_DECLARE(8)
#undef ISING_TILED_DECLARE

cudaError_t launch_init_bits(const BitsLattice& lat, const RngParams& rng, cudaStream_t s) {
  const long long items = 2LL * lat.L * lat.Wc;
  k_init_bits<<<grid_for(items, 256), 256, 0, s>>>(lat.planes, lat.L, lat.Wc, lat.pitch, rng);
  return cudaGetLastError();
}

cudaError_t launch_half_sweep_bits(const BitsLattice& lat, const RngParams& rng, int colour,
                                   uint32_t sweep, unsigned long long* rec, int grid, int block,
                                   cudaStream_t s) {
  const long long words = (long long)lat.L * lat.Wc;
  if (block <= 0) block = 256;
  if (grid <= 0) grid = grid_for(words, block);
  if (rec)
    k_half_sweep_bits<true><<<grid, block, 0, s>>>(lat.planes, lat.L, lat.Wc, lat.pitch, colour,
                                                   sweep, rng, rec);
  else
    k_half_sweep_bits<false><<<grid, block, 0, s>>>(lat.planes, lat.L, lat.Wc, lat.pitch,
                                                    colour, sweep, rng, nullptr);
  return cudaGetLastError();
}

size_t tiled_smem_bytes(int L, int k, int n_tile_rows, int tile_words) {
  const int Ty_max = (L + n_tile_rows - 1) / n_tile_rows;
  return 2ull * (size_t)(Ty_max + 4 * k) * (size_t)(tile_words + 8) * sizeof(uint32_t);
}


cudaError_t launch_tiled_sweep_bits(const BitsLattice& in, uint32_t* out, const RngParams& rng,
                                    uint32_t sweep0, int k, const RecordSlots& slots,
                                    unsigned long long* rec, int n_ty, int Tw, int grid,
                                    int block, cudaStream_t s) {
  const int n_tiles = n_ty * (in.Wc / Tw);
  if (block <= 0) block = 256;
  if (grid <= 0 || grid > n_tiles) grid = n_tiles;
  switch (k) {
    case 1: return launch_tiled_k1(in, out, rng, sweep0, slots, rec, n_ty, Tw, grid, block, s);
    case 2: return launch_tiled_k2(in, out, rng, sweep0, slots, rec, n_ty, Tw, grid, block, s);
    case 3: return launch_tiled_k3(in, out, rng, sweep0, slots, rec, n_ty, Tw, grid, block, s);
    case 4: return launch_tiled_k4(in, out, rng, sweep0, slots, rec, n_ty, Tw, grid, block, s);
    case 5: return launch_tiled_k5(in, out, rng, sweep0, slots, rec, n_ty, Tw, grid, block, s);
    case 6: return launch_tiled_k6(in, out, rng, sweep0, slots, rec, n_ty, Tw, grid, block, s);
    case 7: return launch_tiled_k7(in, out, rng, sweep0, slots, rec, n_ty, Tw, grid, block, s);
    case 8: return launch_tiled_k8(in, out, rng, sweep0, slots, rec, n_ty, Tw, grid, block, s);
    default: return cudaErrorInvalidValue;
  }
}

size_t tiled32_smem_bytes(int L, int k, int n_tile_rows, int tile_words) {
  const int Ty_max = (L + n_tile_rows - 1) / n_tile_rows;
  return 2ull * (size_t)(Ty_max + 4 * k) * (size_t)(tile_words + 8) * sizeof(uint32_t);
}


template <int TWW>
static cudaError_t launch_tiled32_w(const BitsLattice& in, uint32_t* out, const RngParams& rng,
                                    uint32_t sweep0, int k, const RecordSlots& slots,
                                    unsigned long long* rec, int n_ty, int grid, cudaStream_t s) {
  switch (k) {
    case 1: return TWW == 1 ? launch_tiled32_k1_w1(in, out, rng, sweep0, slots, rec, n_ty, grid, s)
                            : launch_tiled32_k1_w2(in, out, rng, sweep0, slots, rec, n_ty, grid, s);
    case 2: return TWW == 1 ? launch_tiled32_k2_w1(in, out, rng, sweep0, slots, rec, n_ty, grid, s)
                            : launch_tiled32_k2_w2(in, out, rng, sweep0, slots, rec, n_ty, grid, s);
    case 3: return TWW == 1 ? launch_tiled32_k3_w1(in, out, rng, sweep0, slots, rec, n_ty, grid, s)
                            : launch_tiled32_k3_w2(in, out, rng, sweep0, slots, rec, n_ty, grid, s);
    case 4: return TWW == 1 ? launch_tiled32_k4_w1(in, out, rng, sweep0, slots, rec, n_ty, grid, s)
                            : launch_tiled32_k4_w2(in, out, rng, sweep0, slots, rec, n_ty, grid, s);
    case 5: return TWW == 1 ? launch_tiled32_k5_w1(in, out, rng, sweep0, slots, rec, n_ty, grid, s)
                            : launch_tiled32_k5_w2(in, out, rng, sweep0, slots, rec, n_ty, grid, s);
    case 6: return TWW == 1 ? launch_tiled32_k6_w1(in, out, rng, sweep0, slots, rec, n_ty, grid, s)
                            : launch_tiled32_k6_w2(in, out, rng, sweep0, slots, rec, n_ty, grid, s);
    case 7: return TWW == 1 ? launch_tiled32_k7_w1(in, out, rng, sweep0, slots, rec, n_ty, grid, s)
                            : launch_tiled32_k7_w2(in, out, rng, sweep0, slots, rec, n_ty, grid, s);
    case 8: return TWW == 1 ? launch_tiled32_k8_w1(in, out, rng, sweep0, slots, rec, n_ty, grid, s)
                            : launch_tiled32_k8_w2(in, out, rng, sweep0, slots, rec, n_ty, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tiled32_sweep_bits(const BitsLattice& in, uint32_t* out, const RngParams& rng,
                                      uint32_t sweep0, int k, const RecordSlots& slots,
                                      unsigned long long* rec, int n_ty, int tile_words, int grid,
                                      cudaStream_t s) {
  if (tile_words == 32) return launch_tiled32_w<1>(in, out, rng, sweep0, k, slots, rec, n_ty, grid, s);
  if (tile_words == 64) return launch_tiled32_w<2>(in, out, rng, sweep0, k, slots, rec, n_ty, grid, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_measure_bits(const BitsLattice& lat, unsigned long long* out2,
                                cudaStream_t s) {
  const long long words = (long long)lat.L * lat.Wc;
  k_measure_bits<<<grid_for(words, 256), 256, 0, s>>>(lat.planes, lat.L, lat.Wc, lat.pitch, out2);
  return cudaGetLastError();
}

cudaError_t launch_unpack_bits(const BitsLattice& lat, int8_t* spins, cudaStream_t s) {
  const long long N = (long long)lat.L * lat.L;
  k_unpack_bits<<<grid_for(N, 256), 256, 0, s>>>(lat.planes, lat.L, lat.Wc, lat.pitch, spins);
  return cudaGetLastError();
}

cudaError_t launch_pack_bits(const BitsLattice& lat, const int8_t* spins, cudaStream_t s) {
  const long long items = 2LL * lat.L * lat.Wc;
  k_pack_bits<<<grid_for(items, 256), 256, 0, s>>>(lat.planes, lat.L, lat.Wc, lat.pitch, spins);
  return cudaGetLastError();
}

}  // namespace ising
