// Shared pieces of the learned block proposal (nn.cu: one-shot pass and
// training; nn_staged.cu: staged pass): network layout, Philox tags, the
// proposal plan (stage schedule and per-stage position lists) and small device
// helpers.  The block move has no counterpart in the paper; it is an extra
// exact move of the same Markov chain (Results A / Supplementary MC steps are
// single-site Metropolis).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "ising_device.cuh"

namespace ising {
namespace nnc {

constexpr int kC = 32;
constexpr int kCP = 40;     // channel stride of activation grids (conflict-free ldmatrix rows)
constexpr int kK2 = 9 * kC; // 288
constexpr int kK2P = 296;   // row stride of the re-laid-out W2
constexpr int kOffW1 = 0, kOffB1 = 576, kOffW2 = 608, kOffB2 = 9824, kOffW3 = 9856,
              kOffB3 = 10144, kNParams = 10145;
constexpr uint32_t kTagBlkSample = 4, kTagBlkAccept = 5, kTagBlkOffset = 6;
constexpr int kMaxB = 16;
constexpr int kThreads = 256;       // training kernels
constexpr int kInferThreads = 512;  // inference / block-pass kernels

// ---- proposal plan -------------------------------------------------------
// ONESHOT: one network stage with every interior site, ring-edge input.
// STAGED: network stages (class-0 / class-1 sites of one depth band) and exact
// stages (sites whose conditional, unknown neighbours summed out, is exact);
// the schedule is built on the host by build_plan (nn_staged.cu).
constexpr int kProposalOneShot = 0;
constexpr int kProposalStaged = 1;
// layer-2 engine of the staged proposal: warp-level mma.sync on the listed
// positions (default) or tcgen05 tiles with TMEM accumulators
constexpr int kEngineMmaSync = 0;
constexpr int kEngineTcgen05 = 1;
constexpr int kMaxStages = 32;
constexpr int kMaxFrame = (kMaxB + 2) * (kMaxB + 2);
constexpr int kMaxNetStages = 12;
constexpr int kMaxList = kMaxNetStages * kMaxFrame;  // l1 / l2 entries over all network stages

struct alignas(16) StagedPlan {
  int B, kind, n_stages, n_net;
  uint8_t exact[kMaxStages];           // 1 = exact stage, 0 = network stage
  uint8_t stage_of[kMaxB * kMaxB];     // interior index iy * B + ix -> its stage
  int16_t net_ids[kMaxStages];         // the network stages, in order
  // per stage k: frame positions fy * F + fx of layer-1 outputs [off1[k], off1[k+1]),
  // of layer-2 outputs [off2[k], off2[k+1]) (network stages only; the positions
  // the stage's logits read), and interior indices of the stage's sites
  // [off3[k], off3[k+1])
  int16_t off1[kMaxStages + 1], off2[kMaxStages + 1], off3[kMaxStages + 1];
  int16_t l1[kMaxList], l2[kMaxList], l3[kMaxB * kMaxB];
  // for each l1 entry: bit t (t = 3 (dy + 1) + dx + 1) set iff the input tap at
  // offset (dy, dx) is a known site before the entry's stage
  uint16_t m1[kMaxList];
};
static_assert(sizeof(StagedPlan) % 16 == 0, "the plan is copied to shared memory as uint4");

// Builds the plan of block size B (2..16, even) and kind; returns false for
// unsupported arguments.
bool build_plan(int B, int kind, StagedPlan* out);

__host__ __device__ constexpr int frame_of(int B) { return B + 2; }

__device__ __forceinline__ float bf(const __nv_bfloat16& v) { return __bfloat162float(v); }

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// is frame position (fy, fx) on one of the four ring edges (not a corner)?
__host__ __device__ __forceinline__ bool ring_edge(int fy, int fx, int F) {
  const bool ey = (fy == 0 || fy == F - 1) && fx >= 1 && fx <= F - 2;
  const bool ex = (fx == 0 || fx == F - 1) && fy >= 1 && fy <= F - 2;
  return ey || ex;
}

// P_i = clamp(rint(sigmoid(l) 2^32), 1, 2^32 - 1).  p 2^32 is exact in FP32
// (a power-of-two scaling); rounding it to an integer (ties to even) and the
// saturating conversion give the same integer as the same steps in FP64.
__device__ __forceinline__ uint32_t quantise_p(float logit) {
  const float p = 1.f / (1.f + expf(-logit));
  const uint32_t v = __float2uint_rn(p * 4294967296.f);  // saturates at 2^32 - 1
  return v < 1u ? 1u : v;
}

// log2 of (P or 2^32 - P) / 2^32, the count rounded to FP32 first (P in
// [1, 2^32 - 1], so 2^32 - P = -P in 32-bit unsigned arithmetic)
__device__ __forceinline__ float log2_q_term(uint32_t P, int s) {
  const uint32_t num = s > 0 ? P : 0u - P;
  return log2f(__uint2float_rn(num)) - 32.f;
}

__device__ __forceinline__ int get_spin(const uint32_t* planes, int L, int Wc, int y, int x) {
  const int c = (x + y) & 1, j = x >> 1;
  const uint32_t w = __ldcg(&planes[(size_t)c * L * Wc + (size_t)y * Wc + (j >> 5)]);
  return ((w >> (j & 31)) & 1u) ? 1 : -1;
}

__device__ __forceinline__ void block_offset(uint32_t pass, uint32_t replica, const RngParams& rng,
                                             int B, int& ox, int& oy) {
  const uint4 r = philox10_rk(make_uint4(0u, pass, replica, ctr_w(kTagBlkOffset, 0, 0)), rng.rk0,
                              rng.rk1);
  ox = (int)(r.x % (uint32_t)B);
  oy = (int)(r.y % (uint32_t)B);
}

// is frame position (fy, fx) known before stage k of plan P?  (ring edges, and
// interior sites drawn by an earlier stage)
__device__ __forceinline__ bool known_at(const StagedPlan& P, int fy, int fx, int k) {
  const int F = P.B + 2;
  if (fy < 0 || fy >= F || fx < 0 || fx >= F) return false;
  if (fy >= 1 && fy <= P.B && fx >= 1 && fx <= P.B) return P.stage_of[(fy - 1) * P.B + fx - 1] < k;
  return ring_edge(fy, fx, F);
}

}  // namespace nnc
}  // namespace ising

namespace ising {
namespace nnc {

// ---- host launchers of the staged proposal (nn_staged.cu) ----
// Builds the plan of (B, kind) on the host and copies it to *d_plan
// (allocated on first use); *n_net = its number of network stages.
// Synchronises the stream.
cudaError_t nn_upload_plan(int B, int kind, StagedPlan** d_plan, int* n_net, cudaStream_t s);
// Number of stages of the plan of (B, kind) (host only).
cudaError_t nn_plan_stages(int B, int kind, int* n_stages);
// Logits of stage `stage` for windows [count][(B+2)^2] int8: network stages
// -> CNN logits at the stage's sites, exact stages -> exact log-odds there;
// other sites 0.  out [count][B*B].
cudaError_t nn_stage_logits(const int8_t* windows, int count, const StagedPlan* d_plan, int stage,
                            float beta, int engine, const __nv_bfloat16* wbf, const __nv_bfloat16* w2t,
                            float* out, cudaStream_t s);
// Teacher-forced natural log of the quantised proposal density of each
// window's interior given its ring.  out [count].
cudaError_t nn_log_q(const int8_t* windows, int count, const StagedPlan* d_plan, float beta, int engine,
                     const __nv_bfloat16* wbf, const __nv_bfloat16* w2t, float* out,
                     cudaStream_t s);
// Loss and gradient sums (added to grads, loss) of count windows on the tensor
// cores (nn_train_tc.cu): the objective of the FP32 training kernel with BF16
// operands and FP32 accumulation in the 32 -> 32 convolution; at most `grid`
// CTAs (one per SM fits).
cudaError_t nn_train_tc(const int8_t* windows, int count, const StagedPlan* d_plan, int n_net,
                        const float* params, float* grads, float* loss, int grid, cudaStream_t s);
// training precisions
constexpr int kTrainFp32 = 0;
constexpr int kTrainBf16Tc = 1;

}  // namespace nnc
}  // namespace ising
