// Staged learned block proposal: the B x B square is redrawn site by site in
// stages, each conditioned on the ring edges and on the sites drawn by the
// earlier stages.  Network stages run the CNN (BF16 weights, FP32
// accumulation; layer 2 on the tensor cores) on the spins known so far;
// exact stages draw sites whose conditional is known in closed form (their
// unknown neighbours summed out).  q(x) is the product of the quantised stage
// probabilities; the same stages evaluated on the current interior (teacher
// forcing) give q(old), so the Metropolis-Hastings test
// u' < exp(-beta dE + ln q(old) - ln q(new)) keeps the chain exact.
//
// Not in the paper (its Monte Carlo is single-site Metropolis, Results A /
// Supplementary MC steps); an extra exact move of the same Markov chain.
//
// Schedule (host, build_plan): site classes local to the square -- 0: i, j
// even; 1: i, j odd with ((i-1)/2 + (j-1)/2) even; 2: other i, j odd; 3: i + j
// odd -- and depth d = min(i, j, B-1-i, B-1-j).  For band k = d / 2 = 0, 1, ...:
// a network stage with the band's undrawn class-0 sites, one with its class-1
// sites, then the closure: repeatedly an exact stage with every undrawn site
// whose four neighbours are known, else with every undrawn class-2 site whose
// unknown neighbours have all their other neighbours known, until neither
// applies.  A last closure draws the rest.
//
// Exact log-odds of s_i = +1: sum over known neighbours n of 2 beta s_n, plus
// over unknown neighbours n of lcosh(beta (h_n + 1)) - lcosh(beta (h_n - 1)),
// h_n the sum of n's other three neighbours (all known by construction).
//
// One CTA per square, persistent over the squares of one colour; every stage
// computes layer 1 only where layer 2 reads it, layer 2 only where the stage's
// logits read it, and logits only at the stage's sites (position lists from
// the plan).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "ising.h"
#include "ising_device.cuh"
#include "nn_common.cuh"

namespace ising {
namespace nnc {

// ---------------------------------------------------------------------------
// host: the plan
// ---------------------------------------------------------------------------
namespace {

int site_class(int i, int j) {
  if ((i + j) & 1) return 3;
  if ((i & 1) == 0) return 0;
  return ((((i - 1) >> 1) + ((j - 1) >> 1)) & 1) == 0 ? 1 : 2;
}

struct Builder {
  int B, F;
  std::vector<uint8_t> known;     // F x F
  std::vector<uint8_t> drawn;     // B x B
  std::vector<std::vector<int>> stages;
  std::vector<uint8_t> exact;

  explicit Builder(int b) : B(b), F(b + 2), known((size_t)(b + 2) * (b + 2), 0), drawn((size_t)b * b, 0) {
    for (int fy = 0; fy < F; ++fy)
      for (int fx = 0; fx < F; ++fx) known[(size_t)fy * F + fx] = ring_edge(fy, fx, F) ? 1 : 0;
  }
  bool kn(int fy, int fx) const { return known[(size_t)fy * F + fx] != 0; }
  int stage_index_of(int iy, int ix) const {
    for (size_t k = 0; k < stages.size(); ++k)
      for (int i : stages[k])
        if (i == iy * B + ix) return (int)k;
    return 1 << 30;
  }
  void add(bool is_exact, const std::vector<int>& sites) {
    stages.push_back(sites);
    exact.push_back(is_exact ? 1 : 0);
    for (int i : sites) {
      drawn[i] = 1;
      known[(size_t)(i / B + 1) * F + (i % B) + 1] = 1;
    }
  }
  bool all_nbrs_known(int i) const {
    const int fy = i / B + 1, fx = i % B + 1;
    return kn(fy - 1, fx) && kn(fy + 1, fx) && kn(fy, fx - 1) && kn(fy, fx + 1);
  }
  // every unknown neighbour of i has its three other neighbours known
  bool drawable(int i) const {
    const int fy = i / B + 1, fx = i % B + 1;
    const int dy[4] = {-1, 1, 0, 0}, dx[4] = {0, 0, -1, 1};
    for (int d = 0; d < 4; ++d) {
      const int ny = fy + dy[d], nx = fx + dx[d];
      if (kn(ny, nx)) continue;
      for (int e = 0; e < 4; ++e) {
        const int my = ny + dy[e], mx = nx + dx[e];
        if (my == fy && mx == fx) continue;
        if (!kn(my, mx)) return false;
      }
    }
    return true;
  }
  void closure() {
    for (;;) {
      std::vector<int> x;
      for (int i = 0; i < B * B; ++i)
        if (!drawn[i] && all_nbrs_known(i)) x.push_back(i);
      if (!x.empty()) {
        add(true, x);
        continue;
      }
      for (int i = 0; i < B * B; ++i)
        if (!drawn[i] && site_class(i / B, i % B) == 2 && drawable(i)) x.push_back(i);
      if (!x.empty()) {
        add(true, x);
        continue;
      }
      return;
    }
  }
};

}  // namespace

bool build_plan(int B, int kind, StagedPlan* out) {
  if (B < 2 || B > kMaxB || (B & 1) || !out) return false;
  if (kind != kProposalOneShot && kind != kProposalStaged) return false;
  std::memset(out, 0, sizeof(StagedPlan));
  const int F = B + 2;
  Builder b(B);
  if (kind == kProposalOneShot) {
    std::vector<int> all;
    for (int i = 0; i < B * B; ++i) all.push_back(i);
    b.add(false, all);
  } else {
    const int n_bands = (B / 2 + 1) / 2;
    for (int k = 0; k < n_bands; ++k) {
      for (int cls = 0; cls < 2; ++cls) {
        std::vector<int> s;
        for (int i = 0; i < B * B; ++i) {
          const int iy = i / B, ix = i % B;
          const int d = std::min(std::min(iy, ix), std::min(B - 1 - iy, B - 1 - ix));
          if (!b.drawn[i] && site_class(iy, ix) == cls && d / 2 == k) s.push_back(i);
        }
        if (!s.empty()) b.add(false, s);
      }
      b.closure();
    }
    b.closure();
    for (int i = 0; i < B * B; ++i)
      if (!b.drawn[i]) return false;
  }
  const int S = (int)b.stages.size();
  if (S > kMaxStages) return false;
  out->B = B;
  out->kind = kind;
  out->n_stages = S;
  int n1 = 0, n2 = 0, n3 = 0, nn = 0;
  for (int k = 0; k < S; ++k) {
    out->exact[k] = b.exact[k];
    out->off1[k] = (int16_t)n1;
    out->off2[k] = (int16_t)n2;
    out->off3[k] = (int16_t)n3;
    std::vector<uint8_t> need2((size_t)F * F, 0), need1((size_t)F * F, 0);
    for (int i : b.stages[k]) {
      out->stage_of[i] = (uint8_t)k;
      out->l3[n3++] = (int16_t)i;
      if (!b.exact[k]) {
        const int fy = i / B + 1, fx = i % B + 1;
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) need2[(size_t)(fy + dy) * F + fx + dx] = 1;
      }
    }
    if (!b.exact[k]) {
      if (nn >= kMaxNetStages) return false;
      out->net_ids[nn++] = (int16_t)k;
      for (int p = 0; p < F * F; ++p) {
        if (!need2[p]) continue;
        const int py = p / F, px = p % F;
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int qy = py + dy, qx = px + dx;
            if (qy >= 0 && qy < F && qx >= 0 && qx < F) need1[(size_t)qy * F + qx] = 1;
          }
      }
      for (int p = 0; p < F * F; ++p) {
        if (need2[p]) {
          if (n2 >= kMaxList) return false;
          out->l2[n2++] = (int16_t)p;
        }
        if (need1[p]) {
          if (n1 >= kMaxList) return false;
          const int py = p / F, px = p % F;
          uint16_t m = 0;
          for (int t = 0; t < 9; ++t) {
            const int qy = py + t / 3 - 1, qx = px + t % 3 - 1;
            if (qy < 0 || qy >= F || qx < 0 || qx >= F) continue;
            const bool inner = qy >= 1 && qy <= B && qx >= 1 && qx <= B;
            const bool kn = inner ? (b.stage_index_of(qy - 1, qx - 1) < k) : ring_edge(qy, qx, F);
            if (kn) m |= (uint16_t)(1u << t);
          }
          out->m1[n1] = m;
          out->l1[n1++] = (int16_t)p;
        }
      }
    }
  }
  out->off1[S] = (int16_t)n1;
  out->off2[S] = (int16_t)n2;
  out->off3[S] = (int16_t)n3;
  out->n_net = nn;
  return true;
}

// ---------------------------------------------------------------------------
// device
// ---------------------------------------------------------------------------
namespace {

constexpr int kFP = kMaxB + 4;  // padded grid side (frame + zero border)

// tcgen05 operand layouts (K-major, no swizzle: core matrices of 8 rows x 16
// bytes, rows 16 bytes apart, 8-row groups 128 bytes apart).  h1 holds, per
// window and per 8-channel chunk, every grid position (kFP-stride grid of the
// frame and its zero border) as one 16-byte row, so the A operand of tap
// (dy, dx) for 128 consecutive positions is the same layout shifted by
// (dy kFP + dx) rows: no im2col copy.
constexpr int kTcPos = 528;  // positions per chunk: tiles start at the first frame position (>= 21),
                             // end <= 378 + 127, plus the largest tap shift 21
constexpr int kTcChunkBytes = kTcPos * 16;
constexpr int kTcWinBytes = (kC / 8) * kTcChunkBytes;  // 4 chunks
constexpr int kTcTiles = 3;                            // 128-position tiles per window (B <= 16)
constexpr int kTmemCols = 256;                         // 2 windows x 3 tiles x 32 columns, rounded up
constexpr int kW2Bytes = (kK2 / 8) * kC * 16;          // W2 as the B operand: [k chunk][n][8]
constexpr long long kTcWaitLimit = 2000000000LL;       // clock64 cycles an MMA wait may take (~1 s)
// instruction descriptor of tcgen05.mma kind::f16: D F32 (bits 4-5 = 1), A and
// B F16 (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0), N / 8 at bit 17,
// M / 16 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kC >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

// shared-memory matrix descriptor: start address, leading (K-direction) and
// stride (M/N-direction) byte offsets, all >> 4; descriptor version 1 (bit 46);
// no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      :
      : "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

// waits for phase `parity` of the mbarrier, at most kTcWaitLimit cycles
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > kTcWaitLimit) return false;
  }
}

// 32 consecutive 32-bit columns of the warp's 32 TMEM lanes (lane = row)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Two windows are evaluated side by side in every layer phase: window 0 =
// the square's ring plus the sites drawn so far (the proposal being drawn),
// window 1 = ring plus the current interior (teacher forcing for q(old)).
// Layer 2 runs in FP16 on the tensor cores (both operands): the activations
// are rounded to FP16 (11-bit significand; BF16's 8 bits left ~1 % logit
// errors), and the weights are the BF16 weight values held in FP16, which
// represents every BF16 value of magnitude 2^-14 .. 65504 exactly.
struct StagedSmem {
  alignas(128) unsigned char h1[2 * kTcWinBytes];  // layer-1 activations, FP16 [window][chunk][position][8]
  alignas(128) unsigned char w2[kW2Bytes];         // W2, FP16 [k chunk][output channel][8]
  float h2[2][kFP * kFP * kC];  // layer-2 activations (FP32) [window][position][channel chunk ^ (position & 7)][4]
  float w1[kOffB1 + kC];  // W1 then b1
  float w3[kC * 9 + 1];   // W3 then b3
  float b2[kC];
  float logit[2][kMaxB * kMaxB];
  float csum[4];              // exact-stage term of a summed neighbour, h = -3, -1, 1, 3
  uint32_t u[kMaxB * kMaxB];  // per-site draw uniforms
  int8_t win[2][kMaxFrame];
  float red_lq[kInferThreads / 32];
  int red_de[kInferThreads / 32];
  int accept;
  int tc_fail;          // an MMA wait ran out of time (results of this CTA are void)
  uint32_t tmem_base;   // TMEM address of the accumulators (written by tcgen05.alloc)
  alignas(8) unsigned long long mbar;  // completion barrier of the MMAs
  StagedPlan plan;
};
static_assert(offsetof(StagedSmem, plan) % 16 == 0, "uint4 copies into shared memory");
static_assert(sizeof(StagedSmem) <= 227 * 1024, "one CTA per SM must fit");

__device__ __forceinline__ __half* h1_at(StagedSmem& S, int w, int g, int c) {
  return reinterpret_cast<__half*>(S.h1 + w * kTcWinBytes + (c >> 3) * kTcChunkBytes + g * 16 + (c & 7) * 2);
}

__device__ void load_all(StagedSmem& S, const __nv_bfloat16* __restrict__ w,
                         const __nv_bfloat16* __restrict__ w2t, const StagedPlan* __restrict__ plan) {
  for (int i = threadIdx.x; i < kOffB1 + kC; i += blockDim.x) S.w1[i] = bf(w[kOffW1 + i]);
  for (int i = threadIdx.x; i < kC * 9 + 1; i += blockDim.x) S.w3[i] = bf(w[kOffW3 + i]);
  for (int i = threadIdx.x; i < kC; i += blockDim.x) S.b2[i] = bf(w[kOffB2 + i]);
  // W2 as the K-major B operand: element (k chunk, output channel n, e) holds
  // W2[n][ci][tap] with k = 8 chunk + e = 32 tap + ci (the A operand's order)
  __half* w2h = reinterpret_cast<__half*>(S.w2);
  for (int i = threadIdx.x; i < kK2 * kC; i += blockDim.x) {
    const int kch = i >> 8, n = (i >> 3) & 31, k = 8 * kch + (i & 7);
    w2h[i] = __float2half_rn(bf(w2t[n * kK2P + (k >> 5) * kC + (k & 31)]));
  }
  {
    const uint4* src = reinterpret_cast<const uint4*>(plan);
    uint4* dst = reinterpret_cast<uint4*>(&S.plan);
    for (int i = threadIdx.x; i < (int)(sizeof(StagedPlan) / 16); i += blockDim.x) dst[i] = __ldg(src + i);
  }
  // Only the one-position border of the padded grid is read without being
  // written first (every frame position a tap of a needed output reads was
  // computed in the same stage), so only the border is zeroed.
  const int FB = __ldg(&plan->B) + 4;  // frame + border extent in the kFP-stride grid
  for (int t = threadIdx.x; t < 2 * 4 * FB; t += blockDim.x) {
    const int wi = t / (4 * FB), e = t - wi * 4 * FB, side = e / FB, o = e - side * FB;
    const int gy = side == 0 ? 0 : (side == 1 ? FB - 1 : o);
    const int gx = side < 2 ? o : (side == 2 ? 0 : FB - 1);
    const int g = gy * kFP + gx;
    for (int ch = 0; ch < kC / 8; ++ch)
      *reinterpret_cast<uint4*>(S.h1 + wi * kTcWinBytes + ch * kTcChunkBytes + g * 16) = make_uint4(0, 0, 0, 0);
  }
  if (threadIdx.x == 0) {
    S.tc_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
}

// Tensor memory for the layer-2 accumulators: allocated by warp 0 after
// load_all, before any MMA; every thread reads the address after the barrier.
__device__ void tmem_setup(StagedSmem& S) {
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&S.tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Frees the tensor memory (every MMA has completed and every tcgen05.ld has
// been waited for by then).
__device__ void tmem_teardown(StagedSmem& S) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_base), "r"(kTmemCols)
                 : "memory");
}

// Layer-1 weights as per-lane mma.sync B fragments (FP16 pairs), built once
// per CTA.  Layer 1 is a GEMM with K = 9 taps x 2 input channels, ordered
// k = 2 t + ch and padded to 32: k-step 0 holds taps 0..7, k-step 1 tap 8.
// For lane (g = lane / 4, q = lane % 4) and n-tile nt (channel n = 8 nt + g):
// kb0 = (W1[n][0][q], W1[n][1][q]), kb1 = taps q + 4, kb2 = tap 8 (q = 0 only).
struct L1Frag {
  uint32_t kb0[4], kb1[4], kb2[4];
};

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ L1Frag layer1_frags(const StagedSmem& S) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  L1Frag f;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int n = nt * 8 + g;
    f.kb0[nt] = pack_h2(S.w1[(n * 2 + 0) * 9 + q], S.w1[(n * 2 + 1) * 9 + q]);
    f.kb1[nt] = pack_h2(S.w1[(n * 2 + 0) * 9 + q + 4], S.w1[(n * 2 + 1) * 9 + q + 4]);
    f.kb2[nt] = q == 0 ? pack_h2(S.w1[(n * 2 + 0) * 9 + 8], S.w1[(n * 2 + 1) * 9 + 8]) : 0u;
  }
  return f;
}

// A-fragment half pair (spin x known, known) of the input tap at window index
// p + off (tap t of the 3 x 3 stencil); taps outside the frame or not yet
// known (bit t of mask clear) give (0, 0).
__device__ __forceinline__ uint32_t l1_tap(const int8_t* w, int p, int off, unsigned mask, int t) {
  if (!((mask >> t) & 1u)) return 0u;
  return pack_h2((float)w[p + off], 1.f);
}

// Layer 1 on the tensor cores for windows 0 .. nw-1 at the listed frame
// positions (known-tap masks from the plan): mma.sync m16n8k16 FP16 -> FP32
// (K = 18 is too small for a tcgen05 tile to pay), A fragments built in
// registers from the spin grid; epilogue bias + ReLU, FP16 into the layer-2
// operand layout.
__device__ void layer1t(StagedSmem& S, const L1Frag& f, int nw, const int16_t* list,
                        const uint16_t* masks, int n) {
  const int F = S.plan.B + 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int rows = nw * n;
  const int n_mt = (rows + 15) / 16;
  // window-index offsets of this lane's taps q, q + 4 and 8
  const int off0 = (q / 3 - 1) * F + q % 3 - 1;
  const int off1 = ((q + 4) / 3 - 1) * F + (q + 4) % 3 - 1;
  const int off2 = F + 1;
  for (int mt = warp; mt < n_mt; mt += nwarps) {
    uint32_t a[2][3];  // [row g / g + 8][tap q, tap q + 4, tap 8]
    int pos[2], wsel[2];  // grid position and window of rows g and g + 8
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = mt * 16 + g + 8 * h;
      a[h][0] = a[h][1] = a[h][2] = 0u;
      pos[h] = -1;
      wsel[h] = 0;
      if (r < rows) {
        const int wi = r >= n ? 1 : 0;
        const int idx = r - wi * n;
        const int p = list[idx];
        const unsigned m = masks[idx];
        const int fy = p / F, fx = p - (p / F) * F;
        const int8_t* w = S.win[wi];
        a[h][0] = l1_tap(w, p, off0, m, q);
        a[h][1] = l1_tap(w, p, off1, m, q + 4);
        a[h][2] = q == 0 ? l1_tap(w, p, off2, m, 8) : 0u;
        pos[h] = (fy + 1) * kFP + fx + 1;
        wsel[h] = wi;
      }
    }
    float acc[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[nt][j] = 0.f;
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, "
          "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
          : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
          : "r"(a[0][0]), "r"(a[1][0]), "r"(a[0][1]), "r"(a[1][1]), "r"(f.kb0[nt]), "r"(f.kb1[nt]));
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, "
          "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
          : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
          : "r"(a[0][2]), "r"(a[1][2]), "r"(0u), "r"(0u), "r"(f.kb2[nt]), "r"(0u));
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (pos[h] < 0) continue;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int c = nt * 8 + 2 * q;
        const __half2 v = __floats2half2_rn(fmaxf(acc[nt][2 * h] + S.w1[kOffB1 + c], 0.f),
                                            fmaxf(acc[nt][2 * h + 1] + S.w1[kOffB1 + c + 1], 0.f));
        *reinterpret_cast<__half2*>(h1_at(S, wsel[h], pos[h], c)) = v;
      }
    }
  }
}

// frame-row offset of 3 x 3 tap t (t = 3 dy + dx, dy, dx in 0..2)
__device__ __forceinline__ constexpr int tap_row(int t) { return (t / 3 - 1) * kFP + (t % 3 - 1); }

// Layer 2 with warp-level MMA for windows 0 .. nw-1 at the listed frame
// positions only: implicit GEMM, M = nw x positions, N = 32 channels,
// K = 288 (tap-major, 16 channels per step), mma.sync m16n8k16 FP16 -> FP32.
// ldmatrix gathers the A rows (one row address per lane) and the W2 rows from
// the same shared-memory layouts the tcgen05 path reads (every (position,
// 8-channel chunk) and (k chunk, output channel) is one 16-byte row).
__device__ void layer2_mma(StagedSmem& S, int nw, const int16_t* list, int M) {
  const int F = S.plan.B + 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int rows = nw * M;
  const int n_mt = (rows + 15) / 16;
  // B rows for ldmatrix.x4: matrix m = lane / 8 is (n-tile 2 np + m / 2, k chunk + m % 2)
  const uint32_t bbase = smem_addr(S.w2) + (uint32_t)((((lane >> 3) & 1) * kC + (lane >> 4) * 8 + (lane & 7)) * 16);
  for (int mt = warp; mt < n_mt; mt += nwarps) {
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    int row = mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
    if (row >= rows) row = 0;  // padding rows: any valid row, results dropped
    const int wi = row >= M ? 1 : 0;
    const int p = list[row - wi * M];
    const int g = (p / F + 1) * kFP + p % F + 1;
    // A rows: window wi, grid position g, channel chunk lane / 16 of the k step
    const uint32_t abase = smem_addr(S.h1) + (uint32_t)(wi * kTcWinBytes + (lane >> 4) * kTcChunkBytes + g * 16);
#pragma unroll
    for (int kc = 0; kc < 18; ++kc) {
      const int tap = kc >> 1, half = kc & 1;
      uint32_t a0, a1, a2, a3;
      asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                   : "=r"(a0), "=r"(a1), "=r"(a2), "=r"(a3)
                   : "r"(abase + (uint32_t)(2 * half * kTcChunkBytes + tap_row(tap) * 16)));
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        uint32_t b0, b1, b2, b3;
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                     : "=r"(b0), "=r"(b1), "=r"(b2), "=r"(b3)
                     : "r"(bbase + (uint32_t)(((4 * tap + 2 * half) * kC + 16 * np) * 16)));
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, "
            "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
            : "+f"(acc[2 * np][0]), "+f"(acc[2 * np][1]), "+f"(acc[2 * np][2]), "+f"(acc[2 * np][3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, "
            "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
            : "+f"(acc[2 * np + 1][0]), "+f"(acc[2 * np + 1][1]), "+f"(acc[2 * np + 1][2]),
              "+f"(acc[2 * np + 1][3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b2), "r"(b3));
      }
    }
    const int gq = lane >> 2, t2 = (lane & 3) * 2;
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      const int rr = mt * 16 + gq + hf * 8;
      if (rr >= rows) continue;
      const int ow = rr >= M ? 1 : 0;
      const int pp = list[rr - ow * M];
      const int pg = (pp / F + 1) * kFP + pp % F + 1;
      float* dst = &S.h2[ow][pg * kC];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int c = nt * 8 + t2;  // channels c, c + 1: one 4-channel chunk (swizzled)
        *reinterpret_cast<float2*>(dst + 4 * ((c >> 2) ^ (pg & 7)) + (c & 3)) =
            make_float2(fmaxf(acc[nt][hf * 2 + 0] + S.b2[c], 0.f), fmaxf(acc[nt][hf * 2 + 1] + S.b2[c + 1], 0.f));
      }
    }
  }
}

// Layer 2 on the 5th-generation tensor cores for windows 0 .. nw-1: implicit
// GEMM over the grid positions from the first to the last listed one (the
// listed positions are the ones the stage's logits read), in tiles of
// M = 128 positions, N = 32 channels, K = 288 in 18 steps of 16 (tap-major,
// two 8-channel chunks per step).  One thread issues tcgen05.mma with both
// operands in shared memory (A = the activation grid shifted by the tap, B =
// W2) and accumulators in tensor memory, then commits to an mbarrier; after
// the (bounded) wait every warp reads its 32 TMEM lanes of a tile with
// tcgen05.ld and writes bias + ReLU in FP32 to h2.  Rows of the range that no
// listed position needs are computed from stale inputs and never read.
__device__ void layer2_tc(StagedSmem& S, int nw, const int16_t* list, int M, uint32_t& parity) {
  const int F = S.plan.B + 2;
  const int pf0 = list[0], pf1 = list[M - 1];
  const int g0 = (pf0 / F + 1) * kFP + pf0 % F + 1;
  const int g1 = (pf1 / F + 1) * kFP + pf1 % F + 1;
  const int ntiles = (g1 - g0) / 128 + 1;
  // the layer-1 stores of every thread become visible to the async proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // the start-address field is the descriptor's low 14 bits (address / 16,
    // all shared-memory addresses < 2^18), so a descriptor for address + off
    // is the descriptor plus off / 16: one base descriptor per operand, and
    // compile-time offsets per tap and channel half
    const uint64_t bdesc0 = umma_desc(smem_addr(S.w2), kC * 16, 128);
    for (int w = 0; w < nw; ++w)
      for (int j = 0; j < ntiles; ++j) {
        const uint32_t d = S.tmem_base + (uint32_t)((w * kTcTiles + j) * kC);
        const uint64_t adesc0 = umma_desc(smem_addr(S.h1) + (uint32_t)(w * kTcWinBytes) +
                                              (uint32_t)(g0 + 128 * j) * 16u,
                                          kTcChunkBytes, 128);
#pragma unroll
        for (int t = 0; t < 9; ++t) {
#pragma unroll
          for (int kc = 0; kc < 2; ++kc) {
            const int64_t aoff = (2 * kc * kTcChunkBytes + tap_row(t) * 16) / 16;
            const int64_t boff = ((4 * t + 2 * kc) * kC * 16) / 16;
            umma_f16(d, adesc0 + (uint64_t)aoff, bdesc0 + (uint64_t)boff, (t | kc) != 0);
          }
        }
      }
    umma_commit(smem_addr(&S.mbar));
  }
  const bool ok = mbar_wait(smem_addr(&S.mbar), parity);
  parity ^= 1u;
  if (!ok) S.tc_fail = 1;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3;
  // warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows of its quadrant)
  for (int job = warp >> 2; job < nw * ntiles; job += (int)(blockDim.x >> 7)) {
    const int w = job / ntiles, j = job - (job / ntiles) * ntiles;
    uint32_t r[32];
    tmem_ld32(S.tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)((w * kTcTiles + j) * kC), r);
    const int g = g0 + 128 * j + 32 * q + lane;
    const int gy = g / kFP, gx = g - (g / kFP) * kFP;
    if (g <= g1 && gx >= 1 && gx <= F && gy >= 1 && gy <= F) {
      float* dst = &S.h2[w][g * kC];
      // 16-byte chunk c4 of the row goes to chunk c4 ^ (g & 7): the eight
      // lanes of a store phase (consecutive rows) hit eight different chunks
#pragma unroll
      for (int c = 0; c < kC; c += 4)
        *reinterpret_cast<float4*>(dst + 4 * ((c >> 2) ^ (g & 7))) =
            make_float4(fmaxf(__uint_as_float(r[c]) + S.b2[c], 0.f), fmaxf(__uint_as_float(r[c + 1]) + S.b2[c + 1], 0.f),
                        fmaxf(__uint_as_float(r[c + 2]) + S.b2[c + 2], 0.f),
                        fmaxf(__uint_as_float(r[c + 3]) + S.b2[c + 3], 0.f));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// Layer 3 (CUDA cores) for windows 0 .. nw-1: logits at the listed interior
// indices; eight lanes per logit, four channels each over the nine taps,
// shuffle sum.
__device__ void layer3s(StagedSmem& S, int nw, const int16_t* list, int n) {
  const int B = S.plan.B;
  const int sub = threadIdx.x & 7, c0 = 4 * sub;
  const int per = (int)(blockDim.x >> 3);
  const int total = nw * n;
  const int rounds = (total + per - 1) / per;
  for (int r = 0; r < rounds; ++r) {
    const int k = r * per + (int)(threadIdx.x >> 3);
    float z = 0.f;
    int i = 0, wi = 0;
    if (k < total) {
      wi = k >= n ? 1 : 0;
      i = list[k - wi * n];
      const int iy = i / B, ix = i - (i / B) * B;
      const int fy = iy + 1, fx = ix + 1;
      const float* h2 = S.h2[wi];
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const int gp = (fy + dy) * kFP + fx + dx;
          const float4 h = *reinterpret_cast<const float4*>(&h2[gp * kC + 4 * (sub ^ (gp & 7))]);
          const int t = dy * 3 + dx;
          z += S.w3[(c0 + 0) * 9 + t] * h.x + S.w3[(c0 + 1) * 9 + t] * h.y +
               S.w3[(c0 + 2) * 9 + t] * h.z + S.w3[(c0 + 3) * 9 + t] * h.w;
        }
    }
    z += __shfl_xor_sync(0xffffffffu, z, 4);
    z += __shfl_xor_sync(0xffffffffu, z, 2);
    z += __shfl_xor_sync(0xffffffffu, z, 1);
    if (k < total && sub == 0) S.logit[wi][i] = z + S.w3[kC * 9];
  }
}

// log cosh(x) + log 2 (the constant cancels in the exact log-odds)
__device__ __forceinline__ float lcosh2(float x) {
  const float a = fabsf(x);
  return a + log1pf(expf(-2.f * a));
}

// The exact-stage contribution lcosh(beta (h + 1)) - lcosh(beta (h - 1)) of a
// summed neighbour whose other three neighbours sum to h (odd, |h| <= 3), for
// the four values of h (threads 0..3; the caller synchronises).
__device__ __forceinline__ void exact_table(StagedSmem& S, float beta) {
  if (threadIdx.x < 4) {
    const float h = (float)(2 * (int)threadIdx.x - 3);
    S.csum[threadIdx.x] = lcosh2(beta * (h + 1.f)) - lcosh2(beta * (h - 1.f));
  }
}

// Exact log-odds of s_i = +1 at stage k for window w (interior index i).
__device__ float exact_logodds(const StagedSmem& S, const int8_t* w, int k, int i, float beta) {
  const int B = S.plan.B, F = B + 2;
  const int fy = i / B + 1, fx = i - (i / B) * B + 1;
  float l = 0.f;
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const int ny = fy + (d == 0 ? -1 : (d == 1 ? 1 : 0));
    const int nx = fx + (d == 2 ? -1 : (d == 3 ? 1 : 0));
    if (known_at(S.plan, ny, nx, k)) {
      l += 2.f * beta * (float)w[ny * F + nx];
    } else {
      // h = the summed neighbour's other three neighbours: its four minus this
      // site's entry (0 in window 0, where the site is not drawn yet; its
      // current spin in window 1)
      int h = -w[fy * F + fx];
      h += w[(ny - 1) * F + nx] + w[(ny + 1) * F + nx] + w[ny * F + nx - 1] + w[ny * F + nx + 1];
      l += S.csum[(h + 3) >> 1];
    }
  }
  return l;
}

// Network logits of stage k for windows 0 .. nw-1 at the stage's sites
// (S.logit[w]); the caller synchronises before, this returns after the last
// phase without a final barrier.
__device__ void net_eval(StagedSmem& S, const L1Frag& f, int nw, int k, uint32_t& parity, bool tc) {
  const StagedPlan& P = S.plan;
  layer1t(S, f, nw, P.l1 + P.off1[k], P.m1 + P.off1[k], P.off1[k + 1] - P.off1[k]);
  if (tc) {
    layer2_tc(S, nw, P.l2 + P.off2[k], P.off2[k + 1] - P.off2[k], parity);  // synchronises first
  } else {
    __syncthreads();
    layer2_mma(S, nw, P.l2 + P.off2[k], P.off2[k + 1] - P.off2[k]);
  }
  __syncthreads();
  layer3s(S, nw, P.l3 + P.off3[k], P.off3[k + 1] - P.off3[k]);
}

// One staged MH update of square (bx, by) of a lattice (whole CTA).
__device__ void process_square(StagedSmem& S, const L1Frag& f1, uint32_t& parity, bool tc, uint32_t* planes,
                               int L, int Wc, int colour, int ox, int oy, int bx, int by,
                               uint32_t pass, uint32_t replica, const RngParams& rng, float beta,
                               unsigned long long* stats) {
  const StagedPlan& P = S.plan;
  const int B = P.B, F = B + 2, BB = B * B;
  const int nbx = L / B;
  const int x0 = ox + bx * B, y0 = oy + by * B;  // interior origin (mod L)
  const uint32_t gid = (uint32_t)(by * nbx + bx);
  for (int i = threadIdx.x; i < F * F; i += blockDim.x) {
    const int fy = i / F, fx = i - (i / F) * F;
    int8_t v = 0;
    const bool inner = fy >= 1 && fy <= B && fx >= 1 && fx <= B;
    if (inner || ring_edge(fy, fx, F)) {
      int y = y0 - 1 + fy, x = x0 - 1 + fx;
      y = (y % L + L) % L;
      x = (x % L + L) % L;
      v = (int8_t)get_spin(planes, L, Wc, y, x);
    }
    S.win[1][i] = v;
    S.win[0][i] = inner ? 0 : v;
  }
  for (int q = threadIdx.x; q < BB / 4; q += blockDim.x) {
    const uint4 r = philox10_rk(make_uint4(gid, pass, replica, ctr_w(kTagBlkSample, colour, q)),
                                rng.rk0, rng.rk1);
    S.u[4 * q + 0] = r.x;
    S.u[4 * q + 1] = r.y;
    S.u[4 * q + 2] = r.z;
    S.u[4 * q + 3] = r.w;
  }
  exact_table(S, beta);
  __syncthreads();
  float lq = 0.f;  // log2 q(old) - log2 q(new) over this thread's draws
  for (int k = 0; k < P.n_stages; ++k) {
    // thread t draws the t-th site of the stage (consecutive threads, so only
    // the first few warps do this phase's work)
    const int t = threadIdx.x;
    const bool mine = t < P.off3[k + 1] - P.off3[k];
    const int si = mine ? P.l3[P.off3[k] + t] : 0;
    const int sf = (si / B + 1) * F + si % B + 1;
    if (P.exact[k]) {
      // a site's exact conditional reads only sites known before stage k, so
      // it is drawn at once (no other site of the stage reads it)
      if (mine) {
        const uint32_t Pn = quantise_p(exact_logodds(S, S.win[0], k, si, beta));
        const int s = S.u[si] < Pn ? 1 : -1;
        lq += log2_q_term(quantise_p(exact_logodds(S, S.win[1], k, si, beta)), S.win[1][sf]) -
              log2_q_term(Pn, s);
        S.win[0][sf] = (int8_t)s;
      }
    } else {
      net_eval(S, f1, 2, k, parity, tc);
      __syncthreads();
      if (mine) {
        const uint32_t Pn = quantise_p(S.logit[0][si]);
        const int s = S.u[si] < Pn ? 1 : -1;
        lq += log2_q_term(quantise_p(S.logit[1][si]), S.win[1][sf]) - log2_q_term(Pn, s);
        S.win[0][sf] = (int8_t)s;
      }
    }
    __syncthreads();
  }
  // bond energy change over the bonds touching the interior
  const int i = threadIdx.x;
  const int fi = i < BB ? (i / B + 1) * F + i % B + 1 : 0;
  int de = 0;
  if (i < BB) {
    const int fy = i / B + 1, fx = i % B + 1;
    const int8_t* wn = S.win[0];
    const int8_t* wo = S.win[1];
    const int os = wo[fi], ns = wn[fi];
    // bonds to the right and down (interior or ring), plus left / up bonds to
    // the ring: every bond touching the interior once
    int e_old = -os * (wo[fy * F + fx + 1] + wo[(fy + 1) * F + fx]);
    int e_new = -ns * (wn[fy * F + fx + 1] + wn[(fy + 1) * F + fx]);
    if (fx == 1) {
      e_old -= os * wo[fy * F];
      e_new -= ns * wn[fy * F];
    }
    if (fy == 1) {
      e_old -= os * wo[fx];
      e_new -= ns * wn[fx];
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
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      sl += S.red_lq[w];
      sd += S.red_de[w];
    }
    const float log_alpha = -beta * (float)sd + 0.69314718f * sl;
    const uint4 r = philox10_rk(make_uint4(gid, pass, replica, ctr_w(kTagBlkAccept, colour, 0)),
                                rng.rk0, rng.rk1);
    const float ua = (float)(r.x >> 8) * (1.0f / 16777216.0f);
    S.accept = (log_alpha >= 0.f || ua < expf(log_alpha)) ? 1 : 0;
    if (S.tc_fail) {  // a tensor-core wait ran out: no move, the host is told
      S.accept = 0;
      atomicAdd(&stats[2], 1ull);
    }
    atomicAdd(&stats[0], 1ull);
    if (S.accept) atomicAdd(&stats[1], 1ull);
  }
  __syncthreads();
  if (S.accept && i < BB && S.win[0][fi] != S.win[1][fi]) {
    const int y = (y0 + i / B) % L, x = (x0 + i % B) % L;
    const int c = (x + y) & 1, j = x >> 1;
    atomicXor(&planes[(size_t)c * L * Wc + (size_t)y * Wc + (j >> 5)], 1u << (j & 31));
  }
  __syncthreads();
}

struct StagedPassParams {
  uint32_t* planes;  // packed lattice [2][L][Wc]
  int L, Wc, colour;
  int tc;            // layer 2 on tcgen05 (1) or mma.sync (0)
  uint32_t pass;
  RngParams rng;
  float beta;
  unsigned long long* stats;  // [0] proposed, [1] accepted
};

__global__ void __launch_bounds__(kInferThreads, 1) k_nn_staged_pass(StagedPassParams Q,
                                                             const StagedPlan* __restrict__ plan,
                                                             const __nv_bfloat16* __restrict__ w,
                                                             const __nv_bfloat16* __restrict__ w2t) {
  extern __shared__ uint4 smem_raw[];
  StagedSmem& S = *reinterpret_cast<StagedSmem*>(smem_raw);
  load_all(S, w, w2t, plan);
  __syncthreads();
  if (Q.tc) tmem_setup(S);
  const L1Frag f1 = layer1_frags(S);
  uint32_t parity = 0;  // phase of the MMA completion barrier
  const int B = S.plan.B, L = Q.L;
  const int nbx = L / B, half = nbx / 2;
  const int n_sq = nbx * half;
  int ox, oy;
  block_offset(Q.pass, Q.rng.replica, Q.rng, B, ox, oy);
  for (int blk = blockIdx.x; blk < n_sq; blk += gridDim.x) {
    const int by = blk / half, bx = 2 * (blk - by * half) + ((by + Q.colour) & 1);
    process_square(S, f1, parity, Q.tc != 0, Q.planes, L, Q.Wc, Q.colour, ox, oy, bx, by, Q.pass,
                   Q.rng.replica, Q.rng, Q.beta, Q.stats);
  }
  if (Q.tc) tmem_teardown(S);
}

struct StagedBatchParams {
  uint32_t* spins;
  const long long* off;
  const int* lad_L;
  const int* slot_of;
  const float* beta_of_slot;
  const long long* unit0;  // [n_rep + 1]
  int n_rep, n_beta, colour;
  int tc;  // layer 2 on tcgen05 (1) or mma.sync (0)
  uint32_t pass;
  RngParams rng;
  unsigned long long* stats;
};

__global__ void __launch_bounds__(kInferThreads, 1) k_nn_staged_batch_pass(StagedBatchParams Q,
                                                                   const StagedPlan* __restrict__ plan,
                                                                   const __nv_bfloat16* __restrict__ w,
                                                                   const __nv_bfloat16* __restrict__ w2t) {
  extern __shared__ uint4 smem_raw[];
  StagedSmem& S = *reinterpret_cast<StagedSmem*>(smem_raw);
  load_all(S, w, w2t, plan);
  __syncthreads();
  if (Q.tc) tmem_setup(S);
  const L1Frag f1 = layer1_frags(S);
  uint32_t parity = 0;  // phase of the MMA completion barrier
  const int B = S.plan.B;
  const long long total = Q.unit0[Q.n_rep];
  for (long long u = blockIdx.x; u < total; u += gridDim.x) {
    int lo = 0, hi = Q.n_rep;  // unit0[lo] <= u < unit0[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (Q.unit0[mid] <= u) lo = mid; else hi = mid;
    }
    const int r = lo;
    const int L = Q.lad_L[r / Q.n_beta];
    const int Wc = (L / 2 + 31) / 32;
    const int nbx = L / B, half = nbx / 2;
    const int blk = (int)(u - Q.unit0[r]);
    const int by = blk / half, bx = 2 * (blk - by * half) + ((by + Q.colour) & 1);
    int ox, oy;
    block_offset(Q.pass, (uint32_t)r, Q.rng, B, ox, oy);
    const float beta = Q.beta_of_slot[Q.slot_of[r]];
    process_square(S, f1, parity, Q.tc != 0, Q.spins + Q.off[r], L, Wc, Q.colour, ox, oy, bx, by, Q.pass,
                   (uint32_t)r, Q.rng, beta, Q.stats);
  }
  if (Q.tc) tmem_teardown(S);
}

// Stage logits of windows (tests and diagnostics): window k in S.win[0].
__global__ void __launch_bounds__(kInferThreads, 1) k_nn_stage_logits(const int8_t* __restrict__ windows,
                                                              int n, int stage, float beta, int tc,
                                                              const StagedPlan* __restrict__ plan,
                                                              const __nv_bfloat16* __restrict__ w,
                                                              const __nv_bfloat16* __restrict__ w2t,
                                                              float* __restrict__ out) {
  extern __shared__ uint4 smem_raw[];
  StagedSmem& S = *reinterpret_cast<StagedSmem*>(smem_raw);
  load_all(S, w, w2t, plan);
  __syncthreads();
  if (tc) tmem_setup(S);
  const L1Frag f1 = layer1_frags(S);
  uint32_t parity = 0;  // phase of the MMA completion barrier
  const int B = S.plan.B, F = B + 2, BB = B * B;
  for (int k = blockIdx.x; k < n; k += gridDim.x) {
    for (int i = threadIdx.x; i < F * F; i += blockDim.x) S.win[0][i] = windows[(size_t)k * F * F + i];
    for (int i = threadIdx.x; i < BB; i += blockDim.x) S.logit[0][i] = 0.f;
    exact_table(S, beta);
    __syncthreads();
    if (S.plan.exact[stage]) {
      for (int i = threadIdx.x; i < BB; i += blockDim.x)
        if (S.plan.stage_of[i] == stage) S.logit[0][i] = exact_logodds(S, S.win[0], stage, i, beta);
    } else {
      net_eval(S, f1, 1, stage, parity, tc != 0);
    }
    __syncthreads();
    const float nan = __int_as_float(0x7fc00000);
    for (int i = threadIdx.x; i < BB; i += blockDim.x)
      out[(size_t)k * BB + i] = S.tc_fail ? nan : (S.plan.stage_of[i] == stage ? S.logit[0][i] : 0.f);
    __syncthreads();
  }
  if (tc) tmem_teardown(S);
}

// Teacher-forced ln q of windows (tests and diagnostics): window k in S.win[1],
// the same per-stage evaluation as q(old) in process_square.
__global__ void __launch_bounds__(kInferThreads, 1) k_nn_log_q(const int8_t* __restrict__ windows, int n,
                                                       float beta, int tc, const StagedPlan* __restrict__ plan,
                                                       const __nv_bfloat16* __restrict__ w,
                                                       const __nv_bfloat16* __restrict__ w2t,
                                                       float* __restrict__ out) {
  extern __shared__ uint4 smem_raw[];
  StagedSmem& S = *reinterpret_cast<StagedSmem*>(smem_raw);
  load_all(S, w, w2t, plan);
  __syncthreads();
  if (tc) tmem_setup(S);
  const L1Frag f1 = layer1_frags(S);
  uint32_t parity = 0;  // phase of the MMA completion barrier
  const StagedPlan& P = S.plan;
  const int B = P.B, F = B + 2;
  for (int k = blockIdx.x; k < n; k += gridDim.x) {
    for (int t = threadIdx.x; t < F * F; t += blockDim.x) {
      const int8_t v = windows[(size_t)k * F * F + t];
      S.win[1][t] = v;
      S.win[0][t] = v;  // layer phases run on windows 0 and 1; both hold the window here
    }
    exact_table(S, beta);
    __syncthreads();
    float lq = 0.f;
    for (int st = 0; st < P.n_stages; ++st) {
      const int t = threadIdx.x;
      const bool mine = t < P.off3[st + 1] - P.off3[st];
      const int si = mine ? P.l3[P.off3[st] + t] : 0;
      const int sf = (si / B + 1) * F + si % B + 1;
      if (P.exact[st]) {
        if (mine) lq += log2_q_term(quantise_p(exact_logodds(S, S.win[1], st, si, beta)), S.win[1][sf]);
      } else {
        net_eval(S, f1, 2, st, parity, tc != 0);
        __syncthreads();
        if (mine) lq += log2_q_term(quantise_p(S.logit[1][si]), S.win[1][sf]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lq += __shfl_xor_sync(0xffffffffu, lq, o);
    if ((threadIdx.x & 31) == 0) S.red_lq[threadIdx.x >> 5] = lq;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w8 = 0; w8 < (int)(blockDim.x >> 5); ++w8) t += S.red_lq[w8];
      out[k] = S.tc_fail ? __int_as_float(0x7fc00000) : 0.69314718f * t;
    }
    __syncthreads();
  }
  if (tc) tmem_teardown(S);
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

template <typename K>
cudaError_t allow_smem(K kernel, DeviceCache& attr) {
  if (attr.get()) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(StagedSmem));
  if (e == cudaSuccess) attr.set(1);
  return e;
}

}  // namespace

cudaError_t nn_upload_plan(int B, int kind, StagedPlan** d_plan, int* n_net, cudaStream_t s) {
  std::vector<StagedPlan> h(1);
  if (!build_plan(B, kind, h.data())) return cudaErrorInvalidValue;
  if (!*d_plan) {
    cudaError_t e = cudaMalloc((void**)d_plan, sizeof(StagedPlan));
    if (e) return e;
  }
  cudaError_t e = cudaMemcpyAsync(*d_plan, h.data(), sizeof(StagedPlan), cudaMemcpyHostToDevice, s);
  if (e) return e;
  if (n_net) *n_net = h[0].n_net;
  return cudaStreamSynchronize(s);  // h lives on this stack frame
}

cudaError_t nn_plan_stages(int B, int kind, int* n_stages) {
  std::vector<StagedPlan> h(1);
  if (!build_plan(B, kind, h.data())) return cudaErrorInvalidValue;
  *n_stages = h[0].n_stages;
  return cudaSuccess;
}

cudaError_t nn_stage_logits(const int8_t* windows, int count, const StagedPlan* d_plan, int stage,
                            float beta, int engine, const __nv_bfloat16* wbf, const __nv_bfloat16* w2t,
                            float* out, cudaStream_t s) {
  static DeviceCache attr;
  cudaError_t e = allow_smem(k_nn_stage_logits, attr);
  if (e) return e;
  const int grid = std::max(1, std::min(count, 2 * sm_count()));
  k_nn_stage_logits<<<grid, kInferThreads, sizeof(StagedSmem), s>>>(windows, count, stage, beta, engine,
                                                                   d_plan, wbf, w2t, out);
  return cudaGetLastError();
}

cudaError_t nn_log_q(const int8_t* windows, int count, const StagedPlan* d_plan, float beta, int engine,
                     const __nv_bfloat16* wbf, const __nv_bfloat16* w2t, float* out,
                     cudaStream_t s) {
  static DeviceCache attr;
  cudaError_t e = allow_smem(k_nn_log_q, attr);
  if (e) return e;
  const int grid = std::max(1, std::min(count, 2 * sm_count()));
  k_nn_log_q<<<grid, kInferThreads, sizeof(StagedSmem), s>>>(windows, count, beta, engine, d_plan, wbf, w2t,
                                                             out);
  return cudaGetLastError();
}

}  // namespace nnc

cudaError_t nn_staged_block_pass(uint32_t* planes, int L, int Wc, const nnc::StagedPlan* d_plan, int B,
                                 uint32_t pass, int colour, const RngParams& rng, double beta, int engine,
                                 const __nv_bfloat16* wbf, const __nv_bfloat16* w2t,
                                 unsigned long long* stats, cudaStream_t s) {
  using namespace nnc;
  static DeviceCache attr;
  cudaError_t e = allow_smem(k_nn_staged_pass, attr);
  if (e) return e;
  StagedPassParams Q;
  Q.planes = planes;
  Q.L = L;
  Q.Wc = Wc;
  Q.colour = colour;
  Q.tc = engine;
  Q.pass = pass;
  Q.rng = rng;
  Q.beta = (float)beta;
  Q.stats = stats;
  const int n_sq = (L / B) * (L / B) / 2;
  const int grid = std::max(1, std::min(n_sq, sm_count()));
  k_nn_staged_pass<<<grid, kInferThreads, sizeof(StagedSmem), s>>>(Q, d_plan, wbf, w2t);
  return cudaGetLastError();
}

cudaError_t nn_batch_staged_block_pass(uint32_t* spins, const long long* off, const int* lad_L,
                                       const int* slot_of, const float* beta_of_slot,
                                       const long long* unit0, long long total_units, int n_rep,
                                       int n_beta, const nnc::StagedPlan* d_plan, int colour,
                                       uint32_t pass, const RngParams& rng, int engine,
                                       const __nv_bfloat16* wbf, const __nv_bfloat16* w2t,
                                       unsigned long long* stats, cudaStream_t s) {
  using namespace nnc;
  static DeviceCache attr;
  cudaError_t e = allow_smem(k_nn_staged_batch_pass, attr);
  if (e) return e;
  StagedBatchParams Q;
  Q.spins = spins;
  Q.off = off;
  Q.lad_L = lad_L;
  Q.slot_of = slot_of;
  Q.beta_of_slot = beta_of_slot;
  Q.unit0 = unit0;
  Q.n_rep = n_rep;
  Q.n_beta = n_beta;
  Q.colour = colour;
  Q.tc = engine;
  Q.pass = pass;
  Q.rng = rng;
  Q.stats = stats;
  const long long g = std::min<long long>(total_units, (long long)sm_count());
  k_nn_staged_batch_pass<<<(int)std::max<long long>(g, 1), kInferThreads, sizeof(StagedSmem), s>>>(
      Q, d_plan, wbf, w2t);
  return cudaGetLastError();
}

}  // namespace ising

extern "C" int ising_proposal_schedule(int block, int kind, uint8_t* stage_of_site, uint8_t* stage_exact,
                                       int capacity, int* n_stages) {
  using namespace ising::nnc;
  std::vector<StagedPlan> h(1);
  if (!stage_of_site || !stage_exact || !n_stages || !build_plan(block, kind, h.data())) {
    ising::set_last_error("block must be even in [2, 16], kind ONESHOT or STAGED, pointers non-null");
    return ISING_EINVAL;
  }
  *n_stages = h[0].n_stages;
  if (capacity < h[0].n_stages) {
    ising::set_last_error("capacity below the number of stages");
    return ISING_EINVAL;
  }
  std::memcpy(stage_of_site, h[0].stage_of, (size_t)block * block);
  std::memcpy(stage_exact, h[0].exact, (size_t)h[0].n_stages);
  ising::set_last_error("");
  return ISING_OK;
}
