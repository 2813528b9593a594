// Learned block proposal: CNN inference on tensor cores fused with the exact
// Metropolis-Hastings block update, and FP32 training kernels.
//
// Not in the paper (its MC is single-site Metropolis, Results A /
// Supplementary MC steps 1-3); the block update is an extra move of the same
// Markov chain and leaves its Boltzmann distribution invariant.
//
// Network (C = 32 channels): three 3 x 3 convolutions with zero padding on the
// (B+2) x (B+2) frame around a B x B block, 2 -> C -> C -> 1 channels, ReLU after
// the first two.  Frame channel 0 = boundary spins on the four edges of the
// ring (corners and interior 0), channel 1 = 1 on those edge sites.  Logits of
// the interior drive the proposal p_i = sigmoid(logit_i), quantised to the
// integer P_i in [1, 2^32 - 1]; a new spin is +1 iff u_i < P_i.  The move is
// accepted iff u' < exp(-beta dE + log q(old) - log q(new)) in FP32, log q from
// the same integers P_i, so the chain is exact up to FP32 rounding of the
// acceptance probability.
//
// Inference keeps BF16 weights and FP32 accumulation; the first-layer
// activations (the tensor-core A operand) are a BF16 hi + lo pair (two MMAs per
// step into the same accumulator), the second-layer ones FP32:
// layer 2 (K = 9 C = 288) runs on the tensor cores as an implicit GEMM over
// frame positions (mma.sync m16n8k16, A gathered by ldmatrix straight from the
// zero-padded activation grid); layers 1 and 3 (K = 18 and 288 with one
// output channel) run on the CUDA cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "ising.h"
#include "ising_device.cuh"
#include "nn_common.cuh"

namespace ising {
namespace {

using namespace nnc;

struct InferSmem {
  // layer-1 activations as a BF16 pair hi + lo (hi = bf16(h), lo = bf16(h - hi)):
  // the tensor-core A operand with ~16 mantissa bits
  __nv_bfloat16 h1[(kMaxB + 4) * (kMaxB + 4) * kCP];
  __nv_bfloat16 h1lo[(kMaxB + 4) * (kMaxB + 4) * kCP];
  float h2[(kMaxB + 4) * (kMaxB + 4) * kC];            // FP32: layer-3 input
  __nv_bfloat16 w2t[kC * kK2P];
  float w1[kOffB1 + kC];   // W1 then b1
  float w3[kC * 9 + 1];    // W3 then b3
  float b2[kC];
  float logit[kMaxB * kMaxB];
  int8_t win[(kMaxB + 2) * (kMaxB + 2)];
  int8_t nw[kMaxB * kMaxB];
  float red_lq[kInferThreads / 32];
  int red_de[kInferThreads / 32];
  int accept;
  // Positions whose values depend on the window.  The input is nonzero only on
  // the ring (frame distance 0), so layer-1 outputs at frame distance >= 2,
  // layer-2 outputs at distance >= 3 and logits at distance >= 4 are the same
  // for every window: computed once per CTA (first window), then only these
  // lists are recomputed.  d = min(fy, fx, F-1-fy, F-1-fx).
  int16_t var1[(kMaxB + 2) * (kMaxB + 2)];  // frame positions, d <= 1
  int16_t var2[(kMaxB + 2) * (kMaxB + 2)];  // frame positions, d <= 2
  int16_t var3[kMaxB * kMaxB];              // interior indices iy B + ix, d <= 3
  int n_var1, n_var2, n_var3;
};

// Builds the variable-position lists (warp 0, ballot compaction; the order of
// a list does not matter).  Call before the first window, then __syncthreads().
__device__ void build_var_lists(InferSmem& S, int B) {
  if (threadIdx.x >= 32) return;
  const int F = B + 2, lane = threadIdx.x;
  int n1 = 0, n2 = 0, n3 = 0;
  for (int p0 = 0; p0 < F * F; p0 += 32) {
    const int p = p0 + lane;
    const int fy = p / F, fx = p - (p / F) * F;
    const int d = min(min(fy, fx), min(F - 1 - fy, F - 1 - fx));
    const bool in = p < F * F;
    const unsigned below = (1u << lane) - 1u;
    const unsigned b1 = __ballot_sync(0xffffffffu, in && d <= 1);
    const unsigned b2 = __ballot_sync(0xffffffffu, in && d <= 2);
    const unsigned b3 = __ballot_sync(0xffffffffu, in && d >= 1 && d <= 3);
    if (in && d <= 1) S.var1[n1 + __popc(b1 & below)] = (int16_t)p;
    if (in && d <= 2) S.var2[n2 + __popc(b2 & below)] = (int16_t)p;
    if (in && d >= 1 && d <= 3) S.var3[n3 + __popc(b3 & below)] = (int16_t)((fy - 1) * B + fx - 1);
    n1 += __popc(b1);
    n2 += __popc(b2);
    n3 += __popc(b3);
  }
  if (lane == 0) {
    S.n_var1 = n1;
    S.n_var2 = n2;
    S.n_var3 = n3;
  }
}

// Per-network cache of the window-independent activations, one slot per block
// size B in {2, 4, 8, 16}: the bytes of h1, h1lo, h2 (with their zero padding)
// followed by the logits, as a CTA holds them after processing any window.  It
// lives behind the re-laid-out W2 in the same allocation and is rebuilt by
// k_nn_const whenever weights are loaded.
constexpr size_t kActBytes = sizeof(__nv_bfloat16) * 2 * (kMaxB + 4) * (kMaxB + 4) * kCP +
                             sizeof(float) * (kMaxB + 4) * (kMaxB + 4) * kC;
constexpr size_t kCacheSlot = ((kActBytes + sizeof(float) * kMaxB * kMaxB) + 255) / 256 * 256;
constexpr size_t kW2tBytes = ((size_t)kC * kK2P * sizeof(__nv_bfloat16) + 255) / 256 * 256;

static_assert(offsetof(InferSmem, h1) == 0 && offsetof(InferSmem, w2t) == kActBytes && kActBytes % 16 == 0,
              "the activation cache copies the leading h1 / h1lo / h2 grids as one block");
static_assert(offsetof(InferSmem, w2t) % 16 == 0 && (kC * kK2P * 2) % 16 == 0, "W2 is copied as uint4");

__host__ __device__ inline int cache_slot_of(int B) {
  return B == 2 ? 0 : (B == 4 ? 1 : (B == 8 ? 2 : (B == 16 ? 3 : -1)));
}

// Loads weights into shared memory and zeroes the padding of the grids; with a
// cache slot, the grids and logits come from it instead (returns true: only the
// window-dependent positions need computing).
__device__ bool load_weights(InferSmem& S, const __nv_bfloat16* __restrict__ w,
                             const __nv_bfloat16* __restrict__ w2t, int B, bool use_cache) {
  const int FP = frame_of(B) + 2;
  for (int i = threadIdx.x; i < kOffB1 + kC; i += blockDim.x) S.w1[i] = bf(w[kOffW1 + i]);
  for (int i = threadIdx.x; i < kC * 9 + 1; i += blockDim.x) S.w3[i] = bf(w[kOffW3 + i]);
  for (int i = threadIdx.x; i < kC; i += blockDim.x) S.b2[i] = bf(w[kOffB2 + i]);
  {
    const uint4* src = reinterpret_cast<const uint4*>(w2t);
    uint4* dst = reinterpret_cast<uint4*>(S.w2t);
    for (int i = threadIdx.x; i < kC * kK2P * 2 / 16; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  const int slot = use_cache ? cache_slot_of(B) : -1;
  if (slot >= 0) {
    const uint4* src = reinterpret_cast<const uint4*>(reinterpret_cast<const char*>(w2t) + kW2tBytes +
                                                      (size_t)slot * kCacheSlot);
    uint4* dst = reinterpret_cast<uint4*>(&S);  // h1, h1lo, h2 lead the struct
    for (int i = threadIdx.x; i < (int)(kActBytes / 16); i += blockDim.x) dst[i] = __ldg(src + i);
    const float* lsrc = reinterpret_cast<const float*>(reinterpret_cast<const char*>(src) + kActBytes);
    for (int i = threadIdx.x; i < kMaxB * kMaxB; i += blockDim.x) S.logit[i] = __ldg(lsrc + i);
    return true;
  }
  const __nv_bfloat16 z = __float2bfloat16(0.f);
  for (int i = threadIdx.x; i < FP * FP * kCP; i += blockDim.x) {
    S.h1[i] = z;
    S.h1lo[i] = z;
  }
  for (int i = threadIdx.x; i < FP * FP * kC; i += blockDim.x) S.h2[i] = 0.f;
  return false;
}

// Layer 1 on the CUDA cores: h1 = relu(conv(frame)) on the F x F frame (all
// positions when full, else the window-dependent ones).  The input is nonzero
// only on ring sites, so each (position, 4-channel group) task visits only its
// ring taps (a 9-bit mask, ascending tap order as in the plain convolution).
__device__ void layer1(InferSmem& S, int B, bool full) {
  const int F = frame_of(B), FP = F + 2;
  const int np = full ? F * F : S.n_var1;
  for (int task = threadIdx.x; task < np * (kC / 4); task += blockDim.x) {
    const int cg = task & (kC / 4 - 1), k = task / (kC / 4);
    const int p = full ? k : S.var1[k];
    const int fy = p / F, fx = p - (p / F) * F;
    unsigned mask = 0;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int yy = fy + t / 3 - 1, xx = fx + t % 3 - 1;
      if (yy >= 0 && yy < F && xx >= 0 && xx < F && ring_edge(yy, xx, F)) mask |= 1u << t;
    }
    float z[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) z[j] = S.w1[kOffB1 + 4 * cg + j];
    while (mask) {
      const int t = __ffs(mask) - 1;
      mask &= mask - 1;
      const float sv = (float)S.win[(fy + t / 3 - 1) * F + fx + t % 3 - 1];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = 4 * cg + j;
        z[j] += S.w1[(c * 2 + 0) * 9 + t] * sv + S.w1[(c * 2 + 1) * 9 + t];
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = 4 * cg + j;
      const float h = fmaxf(z[j], 0.f);
      const __nv_bfloat16 hi = __float2bfloat16(h);
      S.h1[((fy + 1) * FP + fx + 1) * kCP + c] = hi;
      S.h1lo[((fy + 1) * FP + fx + 1) * kCP + c] = __float2bfloat16(h - __bfloat162float(hi));
    }
  }
}

// Layer 2 on the tensor cores: implicit GEMM, M = F^2 positions, N = 32
// channels, K = 288 (tap-major, 16 channels per step).
__device__ void layer2(InferSmem& S, int B, bool full) {
  const int F = frame_of(B), FP = F + 2, M = full ? F * F : S.n_var2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int n_mt = (M + 15) / 16;
  for (int mt = warp; mt < n_mt; mt += nwarps) {
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    // this lane's A row (output position) for ldmatrix.x4
    const int row = mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
    // padding rows: any valid address, results dropped
    const int p = row >= M ? 0 : (full ? row : S.var2[row]);
    const int py = p / F, px = p - (p / F) * F;
    const int acol = (lane >> 4) * 8;
#pragma unroll 1
    for (int kc = 0; kc < 18; ++kc) {
      const int tap = kc >> 1, ci0 = (kc & 1) * 16;
      const int dy = tap / 3, dx = tap - (tap / 3) * 3;
      const int aoff = ((py + dy) * FP + px + dx) * kCP + ci0 + acol;
      uint32_t a0, a1, a2, a3, l0, l1, l2, l3;
      asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                   : "=r"(a0), "=r"(a1), "=r"(a2), "=r"(a3)
                   : "r"(smem_addr(&S.h1[aoff])));
      asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                   : "=r"(l0), "=r"(l1), "=r"(l2), "=r"(l3)
                   : "r"(smem_addr(&S.h1lo[aoff])));
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const __nv_bfloat16* brow =
            &S.w2t[(nt * 8 + (lane & 7)) * kK2P + kc * 16 + ((lane >> 3) & 1) * 8];
        uint32_t b0, b1;
        asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
                     : "=r"(b0), "=r"(b1)
                     : "r"(smem_addr(brow)));
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
            "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
            : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
            "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
            : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
            : "r"(l0), "r"(l1), "r"(l2), "r"(l3), "r"(b0), "r"(b1));
      }
    }
    const int g = lane >> 2, t2 = (lane & 3) * 2;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int rr = mt * 16 + g + half * 8;
      if (rr >= M) continue;
      const int pp = full ? rr : S.var2[rr];
      const int fy = pp / F, fx = pp - (pp / F) * F;
      float* dst = &S.h2[((fy + 1) * FP + fx + 1) * kC];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int c = nt * 8 + t2;
        dst[c] = fmaxf(acc[nt][half * 2 + 0] + S.b2[c], 0.f);
        dst[c + 1] = fmaxf(acc[nt][half * 2 + 1] + S.b2[c + 1], 0.f);
      }
    }
  }
}

// Layer 3 on the CUDA cores: logits of the B x B interior (all, or the
// window-dependent ones).  Eight lanes per logit, four channels each over the
// nine taps, then a three-step shuffle sum.
__device__ void layer3(InferSmem& S, int B, bool full) {
  const int F = frame_of(B), FP = F + 2;
  const int n = full ? B * B : S.n_var3;
  const int sub = threadIdx.x & 7, c0 = 4 * sub;
  const int rounds = (n + (int)(blockDim.x >> 3) - 1) / (int)(blockDim.x >> 3);
  for (int r = 0; r < rounds; ++r) {
    const int k = r * (int)(blockDim.x >> 3) + (int)(threadIdx.x >> 3);
    float z = 0.f;
    int i = 0;
    if (k < n) {
      i = full ? k : S.var3[k];
      const int iy = i / B, ix = i - (i / B) * B;
      const int fy = iy + 1, fx = ix + 1;
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const float4 h = *reinterpret_cast<const float4*>(&S.h2[((fy + dy) * FP + fx + dx) * kC + c0]);
          const int t = dy * 3 + dx;
          z += S.w3[(c0 + 0) * 9 + t] * h.x + S.w3[(c0 + 1) * 9 + t] * h.y +
               S.w3[(c0 + 2) * 9 + t] * h.z + S.w3[(c0 + 3) * 9 + t] * h.w;
        }
    }
    z += __shfl_xor_sync(0xffffffffu, z, 4);
    z += __shfl_xor_sync(0xffffffffu, z, 2);
    z += __shfl_xor_sync(0xffffffffu, z, 1);
    if (k < n && sub == 0) S.logit[i] = z + S.w3[kC * 9];
  }
}

struct PassParams {
  uint32_t* planes;  // packed lattice [2][L][Wc]
  int L, Wc, B, colour;
  uint32_t pass;     // block-pass counter (Philox)
  RngParams rng;
  float beta;
  unsigned long long* stats;  // [0] proposed, [1] accepted
};

// One exact block MH update of square (bx, by) of a lattice (whole CTA).
__device__ void process_block(InferSmem& S, uint32_t* planes, int L, int Wc, int B, int colour,
                              int ox, int oy, int bx, int by, uint32_t pass, uint32_t replica,
                              const RngParams& rng, float beta, unsigned long long* stats, bool full) {
  const int F = frame_of(B);
  const int nbx = L / B;
  const int x0 = ox + bx * B, y0 = oy + by * B;  // interior origin (mod L)
  const uint32_t gid = (uint32_t)(by * nbx + bx);
  for (int i = threadIdx.x; i < F * F; i += blockDim.x) {
    const int fy = i / F, fx = i - (i / F) * F;
    int y = y0 - 1 + fy, x = x0 - 1 + fx;
    y = (y % L + L) % L;
    x = (x % L + L) % L;
    S.win[i] = (int8_t)get_spin(planes, L, Wc, y, x);
  }
  __syncthreads();
  layer1(S, B, full);
  __syncthreads();
  layer2(S, B, full);
  __syncthreads();
  layer3(S, B, full);
  __syncthreads();
  // proposal draw, log q terms and local energy terms
  float lq = 0.f;
  int de = 0;
  const int i = threadIdx.x;
  int old_s = 0, new_s = 0;
  if (i < B * B) {
    const int iy = i / B, ix = i - (i / B) * B;
    const uint32_t Pq = quantise_p(S.logit[i]);
    const uint4 r = philox10_rk(
        make_uint4(gid, pass, replica, ctr_w(kTagBlkSample, colour, i >> 2)), rng.rk0, rng.rk1);
    const uint32_t u = (i & 3) == 0 ? r.x : ((i & 3) == 1 ? r.y : ((i & 3) == 2 ? r.z : r.w));
    new_s = u < Pq ? 1 : -1;
    old_s = S.win[(iy + 1) * F + ix + 1];
    S.nw[i] = (int8_t)new_s;
    lq = log2_q_term(Pq, old_s) - log2_q_term(Pq, new_s);
  }
  __syncthreads();
  if (i < B * B) {
    const int iy = i / B, ix = i - (i / B) * B;
    const int fy = iy + 1, fx = ix + 1;
    // bonds to the right and down (interior or boundary), plus left / up
    // bonds to the boundary: every bond touching the interior once
    const int o_r = S.win[fy * F + fx + 1], o_d = S.win[(fy + 1) * F + fx];
    const int n_r = ix + 1 < B ? S.nw[i + 1] : o_r;
    const int n_d = iy + 1 < B ? S.nw[i + B] : o_d;
    int e_old = -old_s * (o_r + o_d), e_new = -new_s * (n_r + n_d);
    if (ix == 0) {
      const int l = S.win[fy * F + fx - 1];
      e_old -= old_s * l;
      e_new -= new_s * l;
    }
    if (iy == 0) {
      const int u = S.win[(fy - 1) * F + fx];
      e_old -= old_s * u;
      e_new -= new_s * u;
    }
    de = e_new - e_old;
  }
  float lqs = lq;
  int des = de;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lqs += __shfl_xor_sync(0xffffffffu, lqs, o);
    des += __shfl_xor_sync(0xffffffffu, des, o);
  }
  if ((threadIdx.x & 31) == 0) {
    S.red_lq[threadIdx.x >> 5] = lqs;
    S.red_de[threadIdx.x >> 5] = des;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float sl = 0.f;
    int sd = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      sl += S.red_lq[k];
      sd += S.red_de[k];
    }
    const float log_alpha = -beta * (float)sd + 0.69314718f * sl;
    const uint4 r = philox10_rk(make_uint4(gid, pass, replica, ctr_w(kTagBlkAccept, colour, 0)),
                                rng.rk0, rng.rk1);
    const float ua = (float)(r.x >> 8) * (1.0f / 16777216.0f);
    S.accept = (log_alpha >= 0.f || ua < expf(log_alpha)) ? 1 : 0;
    atomicAdd(&stats[0], 1ull);
    if (S.accept) atomicAdd(&stats[1], 1ull);
  }
  __syncthreads();
  if (S.accept && i < B * B && new_s != old_s) {
    const int iy = i / B, ix = i - (i / B) * B;
    const int y = (y0 + iy) % L, x = (x0 + ix) % L;
    const int c = (x + y) & 1, j = x >> 1;
    atomicXor(&planes[(size_t)c * L * Wc + (size_t)y * Wc + (j >> 5)], 1u << (j & 31));
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kInferThreads) k_nn_block_pass(PassParams P,
                                                           const __nv_bfloat16* __restrict__ w,
                                                           const __nv_bfloat16* __restrict__ w2t) {
  extern __shared__ uint4 smem_raw[];
  InferSmem& S = *reinterpret_cast<InferSmem*>(smem_raw);
  const int B = P.B, L = P.L;
  const int nbx = L / B, half = nbx / 2;
  const int n_blocks = nbx * half;  // squares of this colour
  int ox, oy;
  block_offset(P.pass, P.rng.replica, P.rng, B, ox, oy);
  bool full = !load_weights(S, w, w2t, B, true);
  build_var_lists(S, B);
  __syncthreads();
  for (int blk = blockIdx.x; blk < n_blocks; blk += gridDim.x) {
    const int by = blk / half, bx = 2 * (blk - by * half) + ((by + P.colour) & 1);
    process_block(S, P.planes, L, P.Wc, B, P.colour, ox, oy, bx, by, P.pass, P.rng.replica, P.rng,
                  P.beta, P.stats, full);
    full = false;
  }
}

// The same pass over every replica of a batch: replica r has its packed
// lattice at spins + off[r], size L of its ladder, the beta of its current
// temperature slot, Philox replica id r.  Work unit u (squares of this colour,
// all replicas) maps to (r, square) through the prefix sums unit0[r].
struct BatchPassParams {
  uint32_t* spins;
  const long long* off;
  const int* lad_L;
  const int* slot_of;
  const float* beta_of_slot;
  const long long* unit0;  // [n_rep + 1]
  int n_rep, n_beta, B, colour;
  uint32_t pass;
  RngParams rng;           // key and round keys; replica set per unit
  unsigned long long* stats;
};

__global__ void __launch_bounds__(kInferThreads) k_nn_batch_block_pass(BatchPassParams P,
                                                                 const __nv_bfloat16* __restrict__ w,
                                                                 const __nv_bfloat16* __restrict__ w2t) {
  extern __shared__ uint4 smem_raw[];
  InferSmem& S = *reinterpret_cast<InferSmem*>(smem_raw);
  const int B = P.B;
  bool full = !load_weights(S, w, w2t, B, true);
  build_var_lists(S, B);
  __syncthreads();
  const long long total = P.unit0[P.n_rep];
  for (long long u = blockIdx.x; u < total; u += gridDim.x) {
    int lo = 0, hi = P.n_rep;  // unit0[lo] <= u < unit0[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (P.unit0[mid] <= u) lo = mid; else hi = mid;
    }
    const int r = lo;
    const int L = P.lad_L[r / P.n_beta];
    const int Wc = (L / 2 + 31) / 32;
    const int nbx = L / B, half = nbx / 2;
    const int blk = (int)(u - P.unit0[r]);
    const int by = blk / half, bx = 2 * (blk - by * half) + ((by + P.colour) & 1);
    int ox, oy;
    block_offset(P.pass, (uint32_t)r, P.rng, B, ox, oy);
    const float beta = P.beta_of_slot[P.slot_of[r]];
    process_block(S, P.spins + P.off[r], L, Wc, B, P.colour, ox, oy, bx, by, P.pass, (uint32_t)r,
                  P.rng, beta, P.stats, full);
    full = false;
  }
}

// Logits of windows [n][F][F] (int8 spins incl. interior, which is ignored).
__global__ void __launch_bounds__(kInferThreads) k_nn_logits(const int8_t* __restrict__ windows, int n,
                                                       int B, const __nv_bfloat16* __restrict__ w,
                                                       const __nv_bfloat16* __restrict__ w2t,
                                                       float* __restrict__ out) {
  extern __shared__ uint4 smem_raw[];
  InferSmem& S = *reinterpret_cast<InferSmem*>(smem_raw);
  const int F = frame_of(B);
  load_weights(S, w, w2t, B, false);
  build_var_lists(S, B);
  __syncthreads();
  bool full = true;
  for (int k = blockIdx.x; k < n; k += gridDim.x) {
    for (int i = threadIdx.x; i < F * F; i += blockDim.x) S.win[i] = windows[(size_t)k * F * F + i];
    __syncthreads();
    layer1(S, B, full);
    __syncthreads();
    layer2(S, B, full);
    __syncthreads();
    layer3(S, B, full);
    __syncthreads();
    full = false;
    for (int i = threadIdx.x; i < B * B; i += blockDim.x) out[(size_t)k * B * B + i] = S.logit[i];
    __syncthreads();
  }
}

// Builds the cache slot of block size B = 2 << blockIdx.x: a full pass over a
// window of +1 ring spins (any window gives the same window-independent part).
__global__ void __launch_bounds__(kInferThreads) k_nn_const(const __nv_bfloat16* __restrict__ w,
                                                           __nv_bfloat16* __restrict__ w2t) {
  extern __shared__ uint4 smem_raw[];
  InferSmem& S = *reinterpret_cast<InferSmem*>(smem_raw);
  const int B = 2 << blockIdx.x, F = frame_of(B);
  load_weights(S, w, w2t, B, false);
  build_var_lists(S, B);
  for (int i = threadIdx.x; i < F * F; i += blockDim.x) S.win[i] = 1;
  __syncthreads();
  layer1(S, B, true);
  __syncthreads();
  layer2(S, B, true);
  __syncthreads();
  layer3(S, B, true);
  __syncthreads();
  uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<char*>(w2t) + kW2tBytes +
                                        (size_t)cache_slot_of(B) * kCacheSlot);
  const uint4* src = reinterpret_cast<const uint4*>(&S);
  for (int i = threadIdx.x; i < (int)(kActBytes / 16); i += blockDim.x) dst[i] = src[i];
  float* ldst = reinterpret_cast<float*>(reinterpret_cast<char*>(dst) + kActBytes);
  for (int i = threadIdx.x; i < kMaxB * kMaxB; i += blockDim.x) ldst[i] = S.logit[i];
}

// ---------------------------------------------------------------------------
// Training (FP32 on the CUDA cores): one sample per (window, network stage of
// the plan): input = the spins known before that stage and their mask, loss
// terms BCE(logit_i, (s_i + 1) / 2) at the stage's sites; loss = their sum over
// all samples / number of windows (for the one-shot plan: the mean over windows
// of the sum over the interior).  Gradients accumulated with atomics.
// ---------------------------------------------------------------------------
struct TrainSmem {
  float prm[kNParams];
  float gacc[kNParams];  // this CTA's gradient sums over its samples (flushed once)
  float x0[(kMaxB + 2) * (kMaxB + 2)];   // ring spins
  float x1[(kMaxB + 2) * (kMaxB + 2)];   // ring mask
  float h1[(kMaxB + 2) * (kMaxB + 2) * kC];
  float h2[(kMaxB + 2) * (kMaxB + 2) * kC];  // later: g_h1 -> g_z1
  float gz2[(kMaxB + 2) * (kMaxB + 2) * kC];
  float g3[(kMaxB + 2) * (kMaxB + 2)];
  float tgt[kMaxB * kMaxB];
  uint8_t tmask[kMaxB * kMaxB];  // sites of the sample's stage (the loss terms)
  float red[kThreads / 32];
};

__device__ __forceinline__ float at(const float* m, int F, int y, int x, int C, int c) {
  return (y < 0 || y >= F || x < 0 || x >= F) ? 0.f : m[(y * F + x) * C + c];
}

__global__ void __launch_bounds__(kThreads) k_nn_train(const int8_t* __restrict__ windows, int n,
                                                      int B, const StagedPlan* __restrict__ plan,
                                                      const float* __restrict__ params,
                                                      float* __restrict__ grads,
                                                      float* __restrict__ loss) {
  extern __shared__ uint4 smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  const int F = frame_of(B), FF = F * F;
  const float invn = 1.f / (float)n;
  for (int i = threadIdx.x; i < kNParams; i += blockDim.x) {
    S.prm[i] = params[i];
    S.gacc[i] = 0.f;
  }
  __syncthreads();
  const float* W1 = S.prm + kOffW1;
  const float* b1 = S.prm + kOffB1;
  const float* W2 = S.prm + kOffW2;
  const float* b2 = S.prm + kOffB2;
  const float* W3 = S.prm + kOffW3;
  const float b3 = S.prm[kOffB3];
  float my_loss = 0.f;
  const int n_net = plan->n_net;
  const int total = n * n_net;
  for (int smp = blockIdx.x; smp < total; smp += gridDim.x) {
    const int k = smp / n_net;
    const int stage = plan->net_ids[smp - k * n_net];
    const int8_t* win = windows + (size_t)k * FF;
    for (int i = threadIdx.x; i < FF; i += blockDim.x) {
      const int fy = i / F, fx = i - (i / F) * F;
      const bool e = known_at(*plan, fy, fx, stage);
      S.x0[i] = e ? (float)win[i] : 0.f;
      S.x1[i] = e ? 1.f : 0.f;
      if (fy >= 1 && fy <= B && fx >= 1 && fx <= B) {
        const int ii = (fy - 1) * B + fx - 1;
        S.tgt[ii] = win[i] > 0 ? 1.f : 0.f;
        S.tmask[ii] = plan->stage_of[ii] == stage ? 1 : 0;
      }
    }
    __syncthreads();
    // forward
    for (int i = threadIdx.x; i < FF * kC; i += blockDim.x) {
      const int c = i % kC, p = i / kC, fy = p / F, fx = p - (p / F) * F;
      float z = b1[c];
      for (int t = 0; t < 9; ++t) {
        const int yy = fy + t / 3 - 1, xx = fx + t % 3 - 1;
        if (yy < 0 || yy >= F || xx < 0 || xx >= F) continue;
        z += W1[(c * 2) * 9 + t] * S.x0[yy * F + xx] + W1[(c * 2 + 1) * 9 + t] * S.x1[yy * F + xx];
      }
      S.h1[p * kC + c] = fmaxf(z, 0.f);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < FF * kC; i += blockDim.x) {
      const int o = i % kC, p = i / kC, fy = p / F, fx = p - (p / F) * F;
      float z = b2[o];
      for (int t = 0; t < 9; ++t) {
        const int yy = fy + t / 3 - 1, xx = fx + t % 3 - 1;
        if (yy < 0 || yy >= F || xx < 0 || xx >= F) continue;
        const float* h = &S.h1[(yy * F + xx) * kC];
        for (int c = 0; c < kC; ++c) z += W2[(o * kC + c) * 9 + t] * h[c];
      }
      S.h2[p * kC + o] = fmaxf(z, 0.f);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < FF; p += blockDim.x) {
      const int fy = p / F, fx = p - (p / F) * F;
      float g = 0.f;
      if (fy >= 1 && fy <= B && fx >= 1 && fx <= B && S.tmask[(fy - 1) * B + fx - 1]) {
        float z = b3;
        for (int t = 0; t < 9; ++t) {
          const int yy = fy + t / 3 - 1, xx = fx + t % 3 - 1;
          const float* h = &S.h2[(yy * F + xx) * kC];
          for (int c = 0; c < kC; ++c) z += W3[c * 9 + t] * h[c];
        }
        const float y = S.tgt[(fy - 1) * B + fx - 1];
        my_loss += (fmaxf(z, 0.f) - z * y + log1pf(expf(-fabsf(z)))) * invn;
        g = (1.f / (1.f + expf(-z)) - y) * invn;
      }
      S.g3[p] = g;
    }
    __syncthreads();
    // layer 3 weight gradients; g_z2 = (W3^T * g3) . (h2 > 0)
    for (int i = threadIdx.x; i < kC * 9 + 1; i += blockDim.x) {
      float s = 0.f;
      if (i == kC * 9) {
        for (int p = 0; p < FF; ++p) s += S.g3[p];
        S.gacc[kOffB3] += s;
      } else {
        const int c = i / 9, t = i % 9, dy = t / 3 - 1, dx = t % 3 - 1;
        for (int p = 0; p < FF; ++p) {
          if (S.g3[p] == 0.f) continue;
          const int fy = p / F, fx = p - (p / F) * F;
          s += S.g3[p] * at(S.h2, F, fy + dy, fx + dx, kC, c);
        }
        S.gacc[kOffW3 + i] += s;
      }
    }
    for (int i = threadIdx.x; i < FF * kC; i += blockDim.x) {
      const int c = i % kC, q = i / kC, qy = q / F, qx = q - (q / F) * F;
      float s = 0.f;
      for (int t = 0; t < 9; ++t) {
        const int py = qy - (t / 3 - 1), px = qx - (t % 3 - 1);
        if (py < 0 || py >= F || px < 0 || px >= F) continue;
        s += W3[c * 9 + t] * S.g3[py * F + px];
      }
      S.gz2[i] = S.h2[i] > 0.f ? s : 0.f;
    }
    __syncthreads();
    // layer 2 weight and bias gradients
    for (int i = threadIdx.x; i < kC * kC * 9 + kC; i += blockDim.x) {
      float s = 0.f;
      if (i >= kC * kC * 9) {
        const int o = i - kC * kC * 9;
        for (int p = 0; p < FF; ++p) s += S.gz2[p * kC + o];
        S.gacc[kOffB2 + o] += s;
      } else {
        const int o = i / (kC * 9), c = (i / 9) % kC, t = i % 9, dy = t / 3 - 1, dx = t % 3 - 1;
        for (int p = 0; p < FF; ++p) {
          const float g = S.gz2[p * kC + o];
          if (g == 0.f) continue;
          const int fy = p / F, fx = p - (p / F) * F;
          s += g * at(S.h1, F, fy + dy, fx + dx, kC, c);
        }
        S.gacc[kOffW2 + i] += s;
      }
    }
    __syncthreads();
    // g_z1 = (W2^T * g_z2) . (h1 > 0), written over h2
    for (int i = threadIdx.x; i < FF * kC; i += blockDim.x) {
      const int c = i % kC, q = i / kC, qy = q / F, qx = q - (q / F) * F;
      float s = 0.f;
      for (int t = 0; t < 9; ++t) {
        const int py = qy - (t / 3 - 1), px = qx - (t % 3 - 1);
        if (py < 0 || py >= F || px < 0 || px >= F) continue;
        const float* g = &S.gz2[(py * F + px) * kC];
        for (int o = 0; o < kC; ++o) s += W2[(o * kC + c) * 9 + t] * g[o];
      }
      S.h2[i] = S.h1[i] > 0.f ? s : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kC * 2 * 9 + kC; i += blockDim.x) {
      float s = 0.f;
      if (i >= kC * 18) {
        const int o = i - kC * 18;
        for (int p = 0; p < FF; ++p) s += S.h2[p * kC + o];
        S.gacc[kOffB1 + o] += s;
      } else {
        const int o = i / 18, ci = (i / 9) % 2, t = i % 9, dy = t / 3 - 1, dx = t % 3 - 1;
        const float* xin = ci == 0 ? S.x0 : S.x1;
        for (int p = 0; p < FF; ++p) {
          const float g = S.h2[p * kC + o];
          if (g == 0.f) continue;
          const int fy = p / F + dy, fx = p - (p / F) * F + dx;
          if (fy < 0 || fy >= F || fx < 0 || fx >= F) continue;
          s += g * xin[fy * F + fx];
        }
        S.gacc[kOffW1 + i] += s;
      }
    }
    __syncthreads();
  }
  // gradients: one global add per parameter and CTA (each parameter's sum is
  // written by one thread per sample, so the shared sums need no atomics)
  for (int i = threadIdx.x; i < kNParams; i += blockDim.x)
    if (S.gacc[i] != 0.f) atomicAdd(&grads[i], S.gacc[i]);
  // loss
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_loss += __shfl_xor_sync(0xffffffffu, my_loss, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, my_loss);
}

// Adam on the FP32 master weights, then the BF16 copies for inference.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1,
                       float c2, __nv_bfloat16* __restrict__ wbf, __nv_bfloat16* __restrict__ w2t) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParams; i += gridDim.x * blockDim.x) {
    if (lr != 0.f) {
      const float gi = g[i];
      const float mi = b1 * m[i] + (1.f - b1) * gi;
      const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
      m[i] = mi;
      v[i] = vi;
      p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
    const __nv_bfloat16 b = __float2bfloat16(p[i]);
    wbf[i] = b;
    if (i >= kOffW2 && i < kOffB2) {
      const int r = i - kOffW2, co = r / (kC * 9), ci = (r / 9) % kC, tap = r % 9;
      w2t[co * kK2P + tap * kC + ci] = b;
    }
  }
}

// BF16 blob (kNParams values) -> re-laid-out W2.
__global__ void k_relayout(const __nv_bfloat16* __restrict__ wbf, __nv_bfloat16* __restrict__ w2t) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kC * kK2P; i += gridDim.x * blockDim.x) {
    const int co = i / kK2P, k = i % kK2P;
    __nv_bfloat16 v = __float2bfloat16(0.f);
    if (k < kK2) {
      const int tap = k / kC, ci = k % kC;
      v = wbf[kOffW2 + (co * kC + ci) * 9 + tap];
    }
    w2t[i] = v;
  }
}

size_t infer_smem() { return sizeof(InferSmem); }
size_t train_smem() { return sizeof(TrainSmem); }

int nfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

#define NTRY(expr)                                                                      \
  do {                                                                                  \
    cudaError_t e__ = (expr);                                                           \
    if (e__ != cudaSuccess) return nfail(ISING_ECUDA, "%s: %s", #expr, cudaGetErrorString(e__)); \
  } while (0)

int sms_of_current() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

// ---- interface used by api.cu for block passes on a context ----
cudaError_t nn_alloc_weights(__nv_bfloat16** wbf, __nv_bfloat16** w2t) {
  cudaError_t e = cudaMalloc((void**)wbf, kNParams * sizeof(__nv_bfloat16));
  if (e) return e;
  // re-laid-out W2, then the four activation-cache slots
  return cudaMalloc((void**)w2t, kW2tBytes + 4 * kCacheSlot);
}

cudaError_t nn_load_blob(__nv_bfloat16* wbf, __nv_bfloat16* w2t, const void* host_blob,
                         cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(wbf, host_blob, kNParams * sizeof(__nv_bfloat16),
                                  cudaMemcpyHostToDevice, s);
  if (e) return e;
  k_relayout<<<(kC * kK2P + 255) / 256, 256, 0, s>>>(wbf, w2t);
  e = cudaGetLastError();
  if (e) return e;
  static DeviceCache attr;
  if (!attr.get()) {
    e = cudaFuncSetAttribute(k_nn_const, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)infer_smem());
    if (e) return e;
    attr.set(1);
  }
  k_nn_const<<<4, kInferThreads, infer_smem(), s>>>(wbf, w2t);
  e = cudaGetLastError();
  if (e) return e;
  return cudaStreamSynchronize(s);
}

size_t nn_blob_bytes() { return kNParams * sizeof(__nv_bfloat16); }

cudaError_t nn_block_pass(uint32_t* planes, int L, int Wc, int B, uint32_t pass, int colour,
                          const RngParams& rng, double beta, const __nv_bfloat16* wbf,
                          const __nv_bfloat16* w2t, unsigned long long* stats, cudaStream_t s) {
  static DeviceCache attr;
  if (!attr.get()) {
    cudaError_t e = cudaFuncSetAttribute(k_nn_block_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)infer_smem());
    if (e) return e;
    attr.set(1);
  }
  PassParams P;
  P.planes = planes;
  P.L = L;
  P.Wc = Wc;
  P.B = B;
  P.colour = colour;
  P.pass = pass;
  P.rng = rng;
  P.beta = (float)beta;
  P.stats = stats;
  const int n_blocks = (L / B) * (L / B) / 2;
  const int grid = std::max(1, std::min(n_blocks, 2 * sms_of_current()));
  k_nn_block_pass<<<grid, kInferThreads, infer_smem(), s>>>(P, wbf, w2t);
  return cudaGetLastError();
}

cudaError_t nn_batch_block_pass(uint32_t* spins, const long long* off, const int* lad_L,
                                const int* slot_of, const float* beta_of_slot,
                                const long long* unit0, long long total_units, int n_rep,
                                int n_beta, int B, int colour, uint32_t pass, const RngParams& rng,
                                const __nv_bfloat16* wbf, const __nv_bfloat16* w2t,
                                unsigned long long* stats, cudaStream_t s) {
  static DeviceCache attr;
  if (!attr.get()) {
    cudaError_t e = cudaFuncSetAttribute(k_nn_batch_block_pass,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)infer_smem());
    if (e) return e;
    attr.set(1);
  }
  BatchPassParams P;
  P.spins = spins;
  P.off = off;
  P.lad_L = lad_L;
  P.slot_of = slot_of;
  P.beta_of_slot = beta_of_slot;
  P.unit0 = unit0;
  P.n_rep = n_rep;
  P.n_beta = n_beta;
  P.B = B;
  P.colour = colour;
  P.pass = pass;
  P.rng = rng;
  P.stats = stats;
  const long long g = std::min<long long>(total_units, 2LL * sms_of_current());
  k_nn_batch_block_pass<<<(int)std::max<long long>(g, 1), kInferThreads, infer_smem(), s>>>(P, wbf, w2t);
  return cudaGetLastError();
}

}  // namespace ising

using namespace ising;

struct ising_nn {
  int B = 16;
  int kind = kProposalOneShot;
  int engine = kEngineMmaSync;  // layer-2 engine of the staged inference entry points
  int train_prec = kTrainFp32;   // FP32 CUDA-core or BF16 tensor-core training kernel
  StagedPlan* plan = nullptr;  // device copy of the proposal plan
  int n_net = 1;
  cudaStream_t stream = nullptr;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
  __nv_bfloat16 *wbf = nullptr, *w2t = nullptr;
  int64_t step = 0;
};

namespace {

// loss and gradients of count windows with the trainer's kernel
cudaError_t launch_train(ising_nn* n, const int8_t* dev_windows, int count) {
  if (n->train_prec == kTrainBf16Tc)
    return nn_train_tc(dev_windows, count, n->plan, n->n_net, n->p, n->g, n->loss, sms_of_current(),
                       n->stream);
  const int grid = std::max(1, std::min(count * n->n_net, sms_of_current()));
  k_nn_train<<<grid, kThreads, train_smem(), n->stream>>>(dev_windows, count, n->B, n->plan, n->p, n->g,
                                                          n->loss);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

int ising_nn_param_count(void) { return kNParams; }

int ising_nn_create(ising_nn** out, int block, int channels, void* stream) {
  if (!out) return nfail(ISING_EINVAL, "null output pointer");
  *out = nullptr;
  if (channels != kC) return nfail(ISING_EINVAL, "channels must be 32");
  if (block != 2 && block != 4 && block != 8 && block != 16)
    return nfail(ISING_EINVAL, "block must be 2, 4, 8 or 16");
  ising_nn* n = new (std::nothrow) ising_nn();
  if (!n) return nfail(ISING_ENOMEM, "host allocation failed");
  n->B = block;
  n->stream = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  float** fp[] = {&n->p, &n->g, &n->m, &n->v};
  for (float** q : fp)
    if (!e) e = cudaMalloc((void**)q, kNParams * sizeof(float));
  if (!e) e = cudaMalloc((void**)&n->loss, sizeof(float));
  if (!e) e = nn_alloc_weights(&n->wbf, &n->w2t);
  if (!e) e = nn_upload_plan(block, kProposalOneShot, &n->plan, &n->n_net, n->stream);
  if (!e) e = cudaMemset(n->p, 0, kNParams * 4);
  if (!e) e = cudaMemset(n->m, 0, kNParams * 4);
  if (!e) e = cudaMemset(n->v, 0, kNParams * 4);
  if (!e) e = cudaMemset(n->w2t, 0, kC * kK2P * 2);
  if (e) {
    cudaGetLastError();
    ising_nn_destroy(n);
    return nfail(ISING_ENOMEM, "nn allocation: %s", cudaGetErrorString(e));
  }
  if (cudaFuncSetAttribute(k_nn_logits, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)infer_smem()) ||
      cudaFuncSetAttribute(k_nn_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)train_smem())) {
    ising_nn_destroy(n);
    return nfail(ISING_ECUDA, "shared-memory attribute");
  }
  *out = n;
  set_last_error("");
  return ISING_OK;
}

int ising_nn_set_params(ising_nn* n, const float* host, int count) {
  if (!n || !host || count != kNParams) return nfail(ISING_EINVAL, "need %d parameters", kNParams);
  NTRY(cudaMemcpyAsync(n->p, host, kNParams * 4, cudaMemcpyHostToDevice, n->stream));
  NTRY(cudaMemsetAsync(n->m, 0, kNParams * 4, n->stream));
  NTRY(cudaMemsetAsync(n->v, 0, kNParams * 4, n->stream));
  n->step = 0;
  k_adam<<<(kNParams + 255) / 256, 256, 0, n->stream>>>(n->p, n->g, n->m, n->v, 0.f, 0.f, 0.f, 0.f,
                                                        1.f, 1.f, n->wbf, n->w2t);
  NTRY(cudaGetLastError());
  NTRY(cudaStreamSynchronize(n->stream));
  set_last_error("");
  return ISING_OK;
}

int ising_nn_get_params(ising_nn* n, float* host, int count) {
  if (!n || !host || count != kNParams) return nfail(ISING_EINVAL, "need %d parameters", kNParams);
  NTRY(cudaMemcpyAsync(host, n->p, kNParams * 4, cudaMemcpyDeviceToHost, n->stream));
  NTRY(cudaStreamSynchronize(n->stream));
  set_last_error("");
  return ISING_OK;
}

int ising_nn_export(ising_nn* n, void* host_bf16, size_t bytes) {
  if (!n || !host_bf16 || bytes != nn_blob_bytes())
    return nfail(ISING_EINVAL, "blob must be %zu bytes", nn_blob_bytes());
  NTRY(cudaMemcpyAsync(host_bf16, n->wbf, bytes, cudaMemcpyDeviceToHost, n->stream));
  NTRY(cudaStreamSynchronize(n->stream));
  set_last_error("");
  return ISING_OK;
}

int ising_nn_logits(ising_nn* n, const int8_t* dev_windows, int count, float* dev_logits) {
  if (!n || (count > 0 && (!dev_windows || !dev_logits))) return nfail(ISING_EINVAL, "bad arguments");
  if (count <= 0) return ISING_OK;
  const int grid = std::max(1, std::min(count, 2 * sms_of_current()));
  k_nn_logits<<<grid, kInferThreads, infer_smem(), n->stream>>>(dev_windows, count, n->B, n->wbf,
                                                           n->w2t, dev_logits);
  NTRY(cudaGetLastError());
  set_last_error("");
  return ISING_OK;
}

int ising_nn_loss_grad(ising_nn* n, const int8_t* dev_windows, int count, float* loss,
                       float* host_grads) {
  if (!n || !dev_windows || count <= 0) return nfail(ISING_EINVAL, "bad arguments");
  NTRY(cudaMemsetAsync(n->g, 0, kNParams * 4, n->stream));
  NTRY(cudaMemsetAsync(n->loss, 0, 4, n->stream));
  NTRY(launch_train(n, dev_windows, count));
  if (loss) NTRY(cudaMemcpyAsync(loss, n->loss, 4, cudaMemcpyDeviceToHost, n->stream));
  if (host_grads) NTRY(cudaMemcpyAsync(host_grads, n->g, kNParams * 4, cudaMemcpyDeviceToHost, n->stream));
  NTRY(cudaStreamSynchronize(n->stream));
  set_last_error("");
  return ISING_OK;
}

int ising_nn_train_step(ising_nn* n, const int8_t* dev_windows, int count, float lr, float* loss) {
  if (!n || !dev_windows || count <= 0 || !(lr >= 0.f)) return nfail(ISING_EINVAL, "bad arguments");
  NTRY(cudaMemsetAsync(n->g, 0, kNParams * 4, n->stream));
  NTRY(cudaMemsetAsync(n->loss, 0, 4, n->stream));
  NTRY(launch_train(n, dev_windows, count));
  n->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
  k_adam<<<(kNParams + 255) / 256, 256, 0, n->stream>>>(n->p, n->g, n->m, n->v, lr, b1, b2, 1e-8f,
                                                        c1, c2, n->wbf, n->w2t);
  NTRY(cudaGetLastError());
  if (loss) {
    NTRY(cudaMemcpyAsync(loss, n->loss, 4, cudaMemcpyDeviceToHost, n->stream));
    NTRY(cudaStreamSynchronize(n->stream));
  }
  set_last_error("");
  return ISING_OK;
}

int ising_nn_apply_grads(ising_nn* n, const float* host_grads, int count, float lr) {
  if (!n || !host_grads || count != kNParams || !(lr >= 0.f))
    return nfail(ISING_EINVAL, "need %d gradients and lr >= 0", kNParams);
  NTRY(cudaMemcpyAsync(n->g, host_grads, kNParams * 4, cudaMemcpyHostToDevice, n->stream));
  n->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
  k_adam<<<(kNParams + 255) / 256, 256, 0, n->stream>>>(n->p, n->g, n->m, n->v, lr, b1, b2, 1e-8f,
                                                        c1, c2, n->wbf, n->w2t);
  NTRY(cudaGetLastError());
  NTRY(cudaStreamSynchronize(n->stream));
  set_last_error("");
  return ISING_OK;
}

int ising_nn_set_proposal(ising_nn* n, int kind) {
  if (!n) return nfail(ISING_EINVAL, "null trainer");
  if (kind != kProposalOneShot && kind != kProposalStaged)
    return nfail(ISING_EINVAL, "proposal kind must be ISING_PROPOSAL_ONESHOT or ISING_PROPOSAL_STAGED");
  NTRY(nn_upload_plan(n->B, kind, &n->plan, &n->n_net, n->stream));
  n->kind = kind;
  set_last_error("");
  return ISING_OK;
}

int ising_nn_set_train_precision(ising_nn* n, int precision) {
  if (!n) return nfail(ISING_EINVAL, "null trainer");
  if (precision != kTrainFp32 && precision != kTrainBf16Tc)
    return nfail(ISING_EINVAL, "precision must be ISING_NN_TRAIN_FP32 or ISING_NN_TRAIN_BF16_TC");
  n->train_prec = precision;
  set_last_error("");
  return ISING_OK;
}

int ising_nn_set_engine(ising_nn* n, int engine) {
  if (!n) return nfail(ISING_EINVAL, "null trainer");
  if (engine != kEngineMmaSync && engine != kEngineTcgen05)
    return nfail(ISING_EINVAL, "engine must be ISING_NN_ENGINE_MMA_SYNC or ISING_NN_ENGINE_TCGEN05");
  n->engine = engine;
  set_last_error("");
  return ISING_OK;
}

int ising_nn_stage_logits(ising_nn* n, const int8_t* dev_windows, int count, int stage, double beta,
                          float* dev_logits) {
  if (!n || (count > 0 && (!dev_windows || !dev_logits)) || count < 0)
    return nfail(ISING_EINVAL, "bad arguments");
  int n_stages = 0;
  NTRY(nn_plan_stages(n->B, n->kind, &n_stages));
  if (stage < 0 || stage >= n_stages) return nfail(ISING_EINVAL, "stage %d out of range [0, %d)", stage, n_stages);
  if (!(beta >= 0.0) || !std::isfinite(beta)) return nfail(ISING_EINVAL, "beta must be finite and >= 0");
  if (count == 0) return ISING_OK;
  NTRY(nn_stage_logits(dev_windows, count, n->plan, stage, (float)beta, n->engine, n->wbf, n->w2t,
                       dev_logits, n->stream));
  set_last_error("");
  return ISING_OK;
}

int ising_nn_log_q(ising_nn* n, const int8_t* dev_windows, int count, double beta, float* dev_log_q) {
  if (!n || (count > 0 && (!dev_windows || !dev_log_q)) || count < 0)
    return nfail(ISING_EINVAL, "bad arguments");
  if (!(beta >= 0.0) || !std::isfinite(beta)) return nfail(ISING_EINVAL, "beta must be finite and >= 0");
  if (count == 0) return ISING_OK;
  NTRY(nn_log_q(dev_windows, count, n->plan, (float)beta, n->engine, n->wbf, n->w2t, dev_log_q,
                n->stream));
  set_last_error("");
  return ISING_OK;
}

int ising_nn_destroy(ising_nn* n) {
  if (!n) return ISING_OK;
  cudaStreamSynchronize(n->stream);
  cudaFree(n->p);
  cudaFree(n->g);
  cudaFree(n->m);
  cudaFree(n->v);
  cudaFree(n->loss);
  cudaFree(n->wbf);
  cudaFree(n->w2t);
  cudaFree(n->plan);
  delete n;
  return ISING_OK;
}

}  // extern "C"
