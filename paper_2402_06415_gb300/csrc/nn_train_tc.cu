// CNN training on the tensor cores: loss and gradients of the block proposal's
// maximum-likelihood objective (the same samples, inputs, loss terms and
// normalisation as the FP32 kernel k_nn_train in nn.cu) with the three
// contractions of the 32 -> 32 convolution on warp-level mma.sync
// (m16n8k16, BF16 operands, FP32 accumulation):
//   forward        z2[p][o]  = sum_{t,c} h1[p + d_t][c] W2[o][c][t]
//   input gradient g1[q][c]  = sum_{t,o} gz2[q - d_t][o] W2[o][c][t]
//   weight gradient dW2[o][c][t] += sum_p gz2[p][o] h1[p + d_t][c]
// (p, q frame positions, d_t the offset of tap t, zero outside the frame).
// Layers 1 and 3 (2 -> 32 and 32 -> 1 channels, a few per cent of the work) run
// in FP32 on the CUDA cores.  Activations and dL/dz2 are rounded to BF16 for the
// MMA operands (the master weights stay FP32, the operands see them in BF16),
// so gradients agree with the FP32 kernel to BF16 rounding, not bit for bit.
// Each CTA keeps its weight-gradient sums (dW2 in the accumulator registers of
// its warps, the rest in shared memory) over all its samples and adds them to
// the global gradient once.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "nn_common.cuh"

namespace ising {
namespace nnc {
namespace {

constexpr int kG = kMaxB + 4;     // padded grid side: frame plus a zero border
constexpr int kGrid = kG * kG;    // 400 grid positions
constexpr int kZeroPos = 0;       // a grid corner: always zero (padding rows)

struct TrainTcSmem {
  __nv_bfloat16 w2f[kC * kK2P];  // forward B operand: [o][t * 32 + c]
  __nv_bfloat16 w2r[kC * kK2P];  // input-gradient B operand: [c][t * 32 + o]
  __nv_bfloat16 h1[kGrid * kCP];   // layer-1 output, zero outside the frame
  __nv_bfloat16 h2[kGrid * kCP];   // layer-2 output, zero outside the frame
  __nv_bfloat16 gz2[kGrid * kCP];  // dL/dz2, zero outside the frame
  float gz1[kMaxFrame * kC];       // dL/dz1 (FP32, frame positions)
  float w1t[18 * kC];              // W1 as [ci * 9 + t][c] (lanes = channels)
  float b1[kC], b2[kC], w3[kC * 9 + 1];
  float xg[2][kGrid];              // input channels on the padded grid (zero border)
  float g3g[kGrid];                // dL/dz3 on the padded grid (zero outside the sites)
  float red[8][kC * 18 + kC];      // per-warp layer-1 gradient sums, reduced at the end
  float tgt[kMaxB * kMaxB];
  uint8_t tmask[kMaxB * kMaxB];
  int16_t sites[kMaxB * kMaxB];    // frame positions of this sample's loss terms
  int n_sites;
  // this CTA's gradient sums (dW2 lives in registers)
  float gw1[kC * 18], gb1[kC], gb2[kC], gw3[kC * 9], gb3;
};

__device__ __forceinline__ int grid_of_frame(int p, int F) { return (p / F + 1) * kG + p % F + 1; }
__device__ __forceinline__ int tap_off(int t) { return (t / 3 - 1) * kG + (t % 3 - 1); }

__device__ __forceinline__ void ldm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(addr));
}
__device__ __forceinline__ void ldm_x2_t(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
      "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Implicit GEMM over the frame positions (rows) with N = 32 channels and
// K = 9 taps x 32 channels: acc[p][n] = sum_{t,k} act[g(p) + sign * d_t][k] B[n][t * 32 + k].
// sign = +1: forward (B = w2f); sign = -1: input gradient (B = w2r).  The
// epilogue gets (frame position, channel, value) for every valid output.
template <typename Epi>
__device__ __forceinline__ void conv_gemm(const __nv_bfloat16* act, const __nv_bfloat16* Bm, int F, int sign,
                                          Epi epi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int FF = F * F;
  const int n_mt = (FF + 15) / 16;
  for (int mt = warp; mt < n_mt; mt += nwarps) {
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    const int row = mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
    const int gpos = row < FF ? grid_of_frame(row, F) : -1;
    const int acol = (lane >> 4) * 8;
#pragma unroll 2
    for (int kc = 0; kc < 18; ++kc) {
      const int tap = kc >> 1, k0 = (kc & 1) * 16;
      // padding rows read the zero corner (results dropped)
      const int ga = gpos >= 0 ? gpos + sign * tap_off(tap) : kZeroPos;
      uint32_t a0, a1, a2, a3;
      ldm_x4(smem_addr(act + ga * kCP + k0 + acol), a0, a1, a2, a3);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        uint32_t b0, b1;
        ldm_x2(smem_addr(Bm + (nt * 8 + (lane & 7)) * kK2P + kc * 16 + ((lane >> 3) & 1) * 8), b0, b1);
        mma_bf16(acc[nt], a0, a1, a2, a3, b0, b1);
      }
    }
    const int g = lane >> 2, t2 = (lane & 3) * 2;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int p = mt * 16 + g + half * 8;
      if (p >= FF) continue;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        epi(p, nt * 8 + t2, acc[nt][half * 2 + 0]);
        epi(p, nt * 8 + t2 + 1, acc[nt][half * 2 + 1]);
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_nn_train_tc(const int8_t* __restrict__ windows, int n,
                                                             const StagedPlan* __restrict__ plan,
                                                             const float* __restrict__ params,
                                                             float* __restrict__ grads,
                                                             float* __restrict__ loss) {
  extern __shared__ uint4 smem_raw[];
  TrainTcSmem& S = *reinterpret_cast<TrainTcSmem*>(smem_raw);
  const int B = plan->B, F = frame_of(B), FF = F * F;
  const float invn = 1.f / (float)n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // weights: FP32 for layers 1 and 3, BF16 operand layouts of W2
  for (int i = threadIdx.x; i < kC * kC * 9; i += blockDim.x) {
    const int o = i / (kC * 9), c = (i / 9) % kC, t = i % 9;  // W2[o][c][t]
    const __nv_bfloat16 v = __float2bfloat16_rn(params[kOffW2 + i]);
    S.w2f[o * kK2P + t * kC + c] = v;
    S.w2r[c * kK2P + t * kC + o] = v;
  }
  for (int i = threadIdx.x; i < kC * 18; i += blockDim.x) {
    const int c = i / 18, j = i % 18;  // W1[c][ci][t], j = ci * 9 + t
    S.w1t[j * kC + c] = params[kOffW1 + i];
    S.gw1[i] = 0.f;
  }
  for (int i = threadIdx.x; i < kC * 9 + 1; i += blockDim.x) S.w3[i] = params[kOffW3 + i];
  for (int i = threadIdx.x; i < kC * 9; i += blockDim.x) S.gw3[i] = 0.f;
  for (int i = threadIdx.x; i < kC; i += blockDim.x) {
    S.b1[i] = params[kOffB1 + i];
    S.b2[i] = params[kOffB2 + i];
    S.gb1[i] = 0.f;
    S.gb2[i] = 0.f;
  }
  if (threadIdx.x == 0) S.gb3 = 0.f;
  // grids start (and outside the frame stay) zero
  const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
  for (int i = threadIdx.x; i < kGrid * kCP; i += blockDim.x) S.h1[i] = S.h2[i] = S.gz2[i] = z;
  for (int i = threadIdx.x; i < kGrid; i += blockDim.x) S.xg[0][i] = S.xg[1][i] = S.g3g[i] = 0.f;
  __syncthreads();

  // dW2 accumulators: warp w owns tap w (both 16-row o tiles x four 8-column c
  // tiles) and one tile of tap 8 (o tile w >> 2, c tile w & 3)
  float dw[9][4];
#pragma unroll
  for (int a = 0; a < 9; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) dw[a][b] = 0.f;
  // layer-1 gradient sums of this thread: channel o = lane, positions of
  // warp `warp`'s slice, all samples (j = ci * 9 + t; gw1s[18] = bias)
  float gw1s[19];
#pragma unroll
  for (int j = 0; j < 19; ++j) gw1s[j] = 0.f;
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
      const int gi = grid_of_frame(i, F);
      S.xg[0][gi] = e ? (float)win[i] : 0.f;
      S.xg[1][gi] = e ? 1.f : 0.f;
      S.g3g[gi] = 0.f;
      if (fy >= 1 && fy <= B && fx >= 1 && fx <= B) {
        const int ii = (fy - 1) * B + fx - 1;
        S.tgt[ii] = win[i] > 0 ? 1.f : 0.f;
        S.tmask[ii] = plan->stage_of[ii] == stage ? 1 : 0;
      }
    }
    if (threadIdx.x == 0) {
      int m = 0;
      for (int ii = 0; ii < B * B; ++ii)
        if (plan->stage_of[ii] == stage) S.sites[m++] = (int16_t)((ii / B + 1) * F + ii % B + 1);
      S.n_sites = m;
    }
    __syncthreads();
    // layer 1 (FP32): h1 = relu(W1 * x + b1), stored in BF16; lanes = channels
    for (int i = threadIdx.x; i < FF * kC; i += blockDim.x) {
      const int c = i % kC, p = i / kC, gp = grid_of_frame(p, F);
      float zz = S.b1[c];
#pragma unroll
      for (int t = 0; t < 9; ++t)
        zz += S.w1t[t * kC + c] * S.xg[0][gp + tap_off(t)] + S.w1t[(9 + t) * kC + c] * S.xg[1][gp + tap_off(t)];
      S.h1[gp * kCP + c] = __float2bfloat16_rn(fmaxf(zz, 0.f));
    }
    __syncthreads();
    // layer 2 forward on the tensor cores
    conv_gemm(S.h1, S.w2f, F, +1, [&](int p, int o, float v) {
      S.h2[grid_of_frame(p, F) * kCP + o] = __float2bfloat16_rn(fmaxf(v + S.b2[o], 0.f));
    });
    __syncthreads();
    // layer 3 and the loss at this sample's sites: eight lanes per site
    for (int base = warp * 4; base < S.n_sites; base += (int)(blockDim.x >> 3)) {
      const int si = base + (lane >> 3);
      const int sub = lane & 7, c0 = 4 * sub;
      float zz = 0.f;
      int p = 0;
      if (si < S.n_sites) {
        p = S.sites[si];
        const int gp = grid_of_frame(p, F);
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          const __nv_bfloat16* h = &S.h2[(gp + tap_off(t)) * kCP + c0];
          zz += S.w3[(c0 + 0) * 9 + t] * bf(h[0]) + S.w3[(c0 + 1) * 9 + t] * bf(h[1]) +
                S.w3[(c0 + 2) * 9 + t] * bf(h[2]) + S.w3[(c0 + 3) * 9 + t] * bf(h[3]);
        }
      }
      zz += __shfl_xor_sync(0xffffffffu, zz, 4);
      zz += __shfl_xor_sync(0xffffffffu, zz, 2);
      zz += __shfl_xor_sync(0xffffffffu, zz, 1);
      if (si < S.n_sites && sub == 0) {
        zz += S.w3[kC * 9];
        const int fy = p / F, fx = p - (p / F) * F;
        const float y = S.tgt[(fy - 1) * B + fx - 1];
        my_loss += (fmaxf(zz, 0.f) - zz * y + log1pf(expf(-fabsf(zz)))) * invn;
        S.g3g[grid_of_frame(p, F)] = (1.f / (1.f + expf(-zz)) - y) * invn;
      }
    }
    __syncthreads();
    // layer 3 gradients (FP32) and dL/dz2 = (W3^T g3) . (h2 > 0), stored in BF16
    for (int i = threadIdx.x; i < kC * 9 + 1; i += blockDim.x) {
      float s = 0.f;
      for (int j = 0; j < S.n_sites; ++j) {
        const int gp = grid_of_frame(S.sites[j], F);
        if (i == kC * 9) {
          s += S.g3g[gp];
        } else {
          const int c = i / 9, t = i % 9;
          s += S.g3g[gp] * bf(S.h2[(gp + tap_off(t)) * kCP + c]);
        }
      }
      if (i == kC * 9)
        S.gb3 += s;
      else
        S.gw3[i] += s;
    }
    for (int i = threadIdx.x; i < FF * kC; i += blockDim.x) {
      const int c = i % kC, q = i / kC, gqp = grid_of_frame(q, F);
      float s = 0.f;
#pragma unroll
      for (int t = 0; t < 9; ++t) s += S.w3[c * 9 + t] * S.g3g[gqp - tap_off(t)];
      const int gq = gqp * kCP + c;
      const float v = bf(S.h2[gq]) > 0.f ? s : 0.f;
      S.gz2[gq] = __float2bfloat16_rn(v);
      S.gz1[q * kC + c] = v;  // FP32 dL/dz2 for the bias sum below (overwritten by g1)
    }
    __syncthreads();
    // bias of layer 2 from the FP32 dL/dz2 (one thread per channel)
    if (threadIdx.x < kC) {
      float s = 0.f;
      for (int q = 0; q < FF; ++q) s += S.gz1[q * kC + threadIdx.x];
      S.gb2[threadIdx.x] += s;
    }
    // weight gradient of layer 2 on the tensor cores: K = frame positions
    {
      const int n_kt = (FF + 15) / 16;
      for (int kt = 0; kt < n_kt; ++kt) {
        // this lane's frame position in the A (gz2^T) and B (h1) tiles
        const int pa = kt * 16 + (lane & 7) + ((lane >> 4) << 3);          // A: mat = lane >> 3, rows p
        const int pb = kt * 16 + (lane & 7) + (((lane >> 3) & 1) << 3);    // B: rows p
        const int ga = pa < FF ? grid_of_frame(pa, F) : -1;
        const int gb = pb < FF ? grid_of_frame(pb, F) : -1;
        const int oa = ((lane >> 3) & 1) * 8;   // A column (o) offset within the 16-row tile
        const int cb = (lane >> 4) * 8;         // B column (c) offset: second n tile
        // A tiles: gz2^T for o tiles 0 and 1
        uint32_t a[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
          ldm_x4_t(smem_addr(S.gz2 + (ga >= 0 ? ga : kZeroPos) * kCP + mt * 16 + oa), a[mt][0], a[mt][1],
                   a[mt][2], a[mt][3]);
        // tap `warp`: both o tiles, four c tiles
        {
          const int t = warp;
          const int gbt = gb >= 0 ? gb + tap_off(t) : kZeroPos;
#pragma unroll
          for (int np = 0; np < 2; ++np) {
            uint32_t b0, b1, b2, b3;
            ldm_x4_t(smem_addr(S.h1 + gbt * kCP + np * 16 + cb), b0, b1, b2, b3);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
              mma_bf16(dw[mt * 4 + np * 2 + 0], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
              mma_bf16(dw[mt * 4 + np * 2 + 1], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b2, b3);
            }
          }
        }
        // tap 8: o tile warp >> 2, c tile warp & 3
        {
          const int mt = warp >> 2, nt = warp & 3;
          const int gbt = gb >= 0 ? gb + tap_off(8) : kZeroPos;
          uint32_t b0, b1;
          ldm_x2_t(smem_addr(S.h1 + gbt * kCP + nt * 8), b0, b1);
          mma_bf16(dw[8], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
        }
      }
    }
    __syncthreads();
    // input gradient of layer 2 on the tensor cores: dL/dz1 = (W2^T * gz2) . (h1 > 0)
    conv_gemm(S.gz2, S.w2r, F, -1, [&](int q, int c, float v) {
      S.gz1[q * kC + c] = bf(S.h1[grid_of_frame(q, F) * kCP + c]) > 0.f ? v : 0.f;
    });
    __syncthreads();
    // layer 1 gradients (FP32): lane = output channel, warp = a slice of the
    // positions, sums kept in registers over all samples
    for (int p = warp; p < FF; p += (int)(blockDim.x >> 5)) {
      const float g = S.gz1[p * kC + lane];
      const int gp = grid_of_frame(p, F);
      gw1s[18] += g;
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        gw1s[t] += g * S.xg[0][gp + tap_off(t)];
        gw1s[9 + t] += g * S.xg[1][gp + tap_off(t)];
      }
    }
    __syncthreads();
  }
  // flush this CTA's sums
  {
    const int g = lane >> 2, t2 = (lane & 3) * 2;
    auto put = [&](const float (&d)[4], int t, int mt, int nt) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int o = mt * 16 + g + (e >> 1) * 8, c = nt * 8 + t2 + (e & 1);
        if (d[e] != 0.f) atomicAdd(&grads[kOffW2 + (o * kC + c) * 9 + t], d[e]);
      }
    };
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) put(dw[mt * 4 + nt], warp, mt, nt);
    put(dw[8], 8, warp >> 2, warp & 3);
  }
  // layer-1 sums: reduce the warps' partial sums in shared memory
#pragma unroll
  for (int j = 0; j < 18; ++j) S.red[warp][lane * 18 + j] = gw1s[j];
  S.red[warp][kC * 18 + lane] = gw1s[18];
  __syncthreads();
  for (int i = threadIdx.x; i < kC * 18 + kC; i += blockDim.x) {
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += S.red[w][i];
    if (i < kC * 18)
      S.gw1[i] += s;  // [o][ci * 9 + t] = W1[o][ci][t]
    else
      S.gb1[i - kC * 18] += s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kC * 18; i += blockDim.x)
    if (S.gw1[i] != 0.f) atomicAdd(&grads[kOffW1 + i], S.gw1[i]);
  for (int i = threadIdx.x; i < kC * 9; i += blockDim.x)
    if (S.gw3[i] != 0.f) atomicAdd(&grads[kOffW3 + i], S.gw3[i]);
  for (int i = threadIdx.x; i < kC; i += blockDim.x) {
    if (S.gb1[i] != 0.f) atomicAdd(&grads[kOffB1 + i], S.gb1[i]);
    if (S.gb2[i] != 0.f) atomicAdd(&grads[kOffB2 + i], S.gb2[i]);
  }
  if (threadIdx.x == 0 && S.gb3 != 0.f) atomicAdd(&grads[kOffB3], S.gb3);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_loss += __shfl_xor_sync(0xffffffffu, my_loss, o);
  if (lane == 0) atomicAdd(loss, my_loss);
}

}  // namespace

size_t nn_train_tc_smem() { return sizeof(TrainTcSmem); }

cudaError_t nn_train_tc(const int8_t* windows, int count, const StagedPlan* d_plan, int n_net,
                        const float* params, float* grads, float* loss, int grid, cudaStream_t s) {
  static DeviceCache attr;
  if (!attr.get()) {
    cudaError_t e = cudaFuncSetAttribute(k_nn_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(TrainTcSmem));
    if (e) return e;
    attr.set(1);
  }
  const int g = std::max(1, std::min(count * n_net, grid));
  k_nn_train_tc<<<g, kThreads, sizeof(TrainTcSmem), s>>>(windows, count, d_plan, params, grads, loss);
  return cudaGetLastError();
}

}  // namespace nnc
}  // namespace ising
