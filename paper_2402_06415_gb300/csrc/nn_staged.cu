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

struct StagedSmem {
  // layer-1 activations as a BF16 pair hi + lo (the tensor-core A operand with
  // ~16 mantissa bits), layer-2 activations in FP32; zero border of one
  __nv_bfloat16 h1[kFP * kFP * kCP];
  __nv_bfloat16 h1lo[kFP * kFP * kCP];
  float h2[kFP * kFP * kC];
  __nv_bfloat16 w2t[kC * kK2P];
  float w1[kOffB1 + kC];  // W1 then b1
  float w3[kC * 9 + 1];   // W3 then b3
  float b2[kC];
  float logit[kMaxB * kMaxB];
  uint32_t u[kMaxB * kMaxB];  // per-site draw uniforms
  int8_t win[kMaxFrame];      // ring + the sites drawn so far (new interior)
  int8_t wold[kMaxFrame];     // ring + current interior
  float red_lq[kInferThreads / 32];
  int red_de[kInferThreads / 32];
  int accept;
  StagedPlan plan;
};
static_assert(offsetof(StagedSmem, w2t) % 16 == 0 && offsetof(StagedSmem, plan) % 16 == 0,
              "uint4 copies into shared memory");

__device__ void load_all(StagedSmem& S, const __nv_bfloat16* __restrict__ w,
                         const __nv_bfloat16* __restrict__ w2t, const StagedPlan* __restrict__ plan) {
  for (int i = threadIdx.x; i < kOffB1 + kC; i += blockDim.x) S.w1[i] = bf(w[kOffW1 + i]);
  for (int i = threadIdx.x; i < kC * 9 + 1; i += blockDim.x) S.w3[i] = bf(w[kOffW3 + i]);
  for (int i = threadIdx.x; i < kC; i += blockDim.x) S.b2[i] = bf(w[kOffB2 + i]);
  {
    const uint4* src = reinterpret_cast<const uint4*>(w2t);
    uint4* dst = reinterpret_cast<uint4*>(S.w2t);
    for (int i = threadIdx.x; i < kC * kK2P * 2 / 16; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  {
    const uint4* src = reinterpret_cast<const uint4*>(plan);
    uint4* dst = reinterpret_cast<uint4*>(&S.plan);
    for (int i = threadIdx.x; i < (int)(sizeof(StagedPlan) / 16); i += blockDim.x) dst[i] = __ldg(src + i);
  }
  const __nv_bfloat16 z = __float2bfloat16(0.f);
  for (int i = threadIdx.x; i < kFP * kFP * kCP; i += blockDim.x) {
    S.h1[i] = z;
    S.h1lo[i] = z;
  }
  for (int i = threadIdx.x; i < kFP * kFP * kC; i += blockDim.x) S.h2[i] = 0.f;
}

// Layer 1 (CUDA cores) at the listed frame positions: input channel 0 = spin
// of w where known before stage k, channel 1 = known mask; only known taps
// contribute (ascending tap order).
__device__ void layer1s(StagedSmem& S, const int8_t* w, int k, const int16_t* list, int n) {
  const int B = S.plan.B, F = B + 2, FP = F + 2;
  for (int task = threadIdx.x; task < n * (kC / 4); task += blockDim.x) {
    const int cg = task & (kC / 4 - 1), idx = task / (kC / 4);
    const int p = list[idx];
    const int fy = p / F, fx = p - (p / F) * F;
    unsigned mask = 0;
#pragma unroll
    for (int t = 0; t < 9; ++t)
      if (known_at(S.plan, fy + t / 3 - 1, fx + t % 3 - 1, k)) mask |= 1u << t;
    float z[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) z[j] = S.w1[kOffB1 + 4 * cg + j];
    while (mask) {
      const int t = __ffs(mask) - 1;
      mask &= mask - 1;
      const float sv = (float)w[(fy + t / 3 - 1) * F + fx + t % 3 - 1];
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

// Layer 2 on the tensor cores at the listed frame positions: implicit GEMM,
// M = positions, N = 32 channels, K = 288 (tap-major, 16 channels per step),
// mma.sync m16n8k16 BF16 -> FP32, A rows gathered by ldmatrix straight from
// the zero-padded activation grid (hi and lo parts into one accumulator).
__device__ void layer2s(StagedSmem& S, const int16_t* list, int M) {
  const int F = S.plan.B + 2, FP = F + 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int n_mt = (M + 15) / 16;
  for (int mt = warp; mt < n_mt; mt += nwarps) {
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    const int row = mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
    const int p = row >= M ? list[0] : list[row];  // padding rows: any valid row, results dropped
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
      const int pp = list[rr];
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

// Layer 3 (CUDA cores): logits at the listed interior indices; eight lanes
// per logit, four channels each over the nine taps, shuffle sum.
__device__ void layer3s(StagedSmem& S, const int16_t* list, int n) {
  const int B = S.plan.B, F = B + 2, FP = F + 2;
  const int sub = threadIdx.x & 7, c0 = 4 * sub;
  const int per = (int)(blockDim.x >> 3);
  const int rounds = (n + per - 1) / per;
  for (int r = 0; r < rounds; ++r) {
    const int k = r * per + (int)(threadIdx.x >> 3);
    float z = 0.f;
    int i = 0;
    if (k < n) {
      i = list[k];
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

// log cosh(x) + log 2 (the constant cancels in the exact log-odds)
__device__ __forceinline__ float lcosh2(float x) {
  const float a = fabsf(x);
  return a + log1pf(expf(-2.f * a));
}

// Exact log-odds of s_i = +1 at stage k for window w (interior index i).
__device__ float exact_logodds(const StagedSmem& S, const int8_t* w, int k, int i, float beta) {
  const int B = S.plan.B, F = B + 2;
  const int fy = i / B + 1, fx = i - (i / B) * B + 1;
  const int dy[4] = {-1, 1, 0, 0}, dx[4] = {0, 0, -1, 1};
  float l = 0.f;
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const int ny = fy + dy[d], nx = fx + dx[d];
    if (known_at(S.plan, ny, nx, k)) {
      l += 2.f * beta * (float)w[ny * F + nx];
    } else {
      int h = 0;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int my = ny + dy[e], mx = nx + dx[e];
        if (my == fy && mx == fx) continue;
        h += w[my * F + mx];
      }
      l += lcosh2(beta * (float)(h + 1)) - lcosh2(beta * (float)(h - 1));
    }
  }
  return l;
}

// Logits of stage k for window w at the stage's sites (S.logit); the caller
// synchronises before and after.
__device__ void stage_eval(StagedSmem& S, const int8_t* w, int k, float beta) {
  const StagedPlan& P = S.plan;
  const int a = P.off3[k], b = P.off3[k + 1];
  if (P.exact[k]) {
    for (int t = a + (int)threadIdx.x; t < b; t += blockDim.x) {
      const int i = P.l3[t];
      S.logit[i] = exact_logodds(S, w, k, i, beta);
    }
    return;
  }
  layer1s(S, w, k, P.l1 + P.off1[k], P.off1[k + 1] - P.off1[k]);
  __syncthreads();
  layer2s(S, P.l2 + P.off2[k], P.off2[k + 1] - P.off2[k]);
  __syncthreads();
  layer3s(S, P.l3 + a, b - a);
}

// Teacher-forced log2 q of the interior of S.wold (every thread returns its
// own sites' share; sum over the CTA for the total).
__device__ float log2_q_old(StagedSmem& S, float beta) {
  const StagedPlan& P = S.plan;
  const int B = P.B, F = B + 2;
  const int i = threadIdx.x;
  const int my_stage = i < B * B ? P.stage_of[i] : -1;
  float lq = 0.f;
  for (int k = 0; k < P.n_stages; ++k) {
    stage_eval(S, S.wold, k, beta);
    __syncthreads();
    if (my_stage == k) lq += log2_q_term(quantise_p(S.logit[i]), S.wold[(i / B + 1) * F + i % B + 1]);
    __syncthreads();
  }
  return lq;
}

// One staged MH update of square (bx, by) of a lattice (whole CTA).
__device__ void process_square(StagedSmem& S, uint32_t* planes, int L, int Wc, int colour, int ox,
                               int oy, int bx, int by, uint32_t pass, uint32_t replica,
                               const RngParams& rng, float beta, unsigned long long* stats) {
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
    S.wold[i] = v;
    S.win[i] = inner ? 0 : v;
  }
  for (int q = threadIdx.x; q < BB / 4; q += blockDim.x) {
    const uint4 r = philox10_rk(make_uint4(gid, pass, replica, ctr_w(kTagBlkSample, colour, q)),
                                rng.rk0, rng.rk1);
    S.u[4 * q + 0] = r.x;
    S.u[4 * q + 1] = r.y;
    S.u[4 * q + 2] = r.z;
    S.u[4 * q + 3] = r.w;
  }
  __syncthreads();
  const int i = threadIdx.x;
  const int my_stage = i < BB ? P.stage_of[i] : -1;
  const int fi = i < BB ? (i / B + 1) * F + i % B + 1 : 0;
  float lq = 0.f;  // log2 q(old) - log2 q(new), this thread's sites
  for (int k = 0; k < P.n_stages; ++k) {
    stage_eval(S, S.win, k, beta);
    __syncthreads();
    if (my_stage == k) {
      const uint32_t Pq = quantise_p(S.logit[i]);
      const int s = S.u[i] < Pq ? 1 : -1;
      lq -= log2_q_term(Pq, s);
      S.win[fi] = (int8_t)s;  // read by later stages only
    }
    __syncthreads();
    stage_eval(S, S.wold, k, beta);
    __syncthreads();
    if (my_stage == k) lq += log2_q_term(quantise_p(S.logit[i]), S.wold[fi]);
    __syncthreads();
  }
  // bond energy change over the bonds touching the interior
  int de = 0;
  if (i < BB) {
    const int fy = i / B + 1, fx = i % B + 1;
    const int os = S.wold[fi], ns = S.win[fi];
    // bonds to the right and down (interior or ring), plus left / up bonds to
    // the ring: every bond touching the interior once
    int e_old = -os * (S.wold[fy * F + fx + 1] + S.wold[(fy + 1) * F + fx]);
    int e_new = -ns * (S.win[fy * F + fx + 1] + S.win[(fy + 1) * F + fx]);
    if (fx == 1) {
      e_old -= os * S.wold[fy * F];
      e_new -= ns * S.win[fy * F];
    }
    if (fy == 1) {
      e_old -= os * S.wold[fx];
      e_new -= ns * S.win[fx];
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
    atomicAdd(&stats[0], 1ull);
    if (S.accept) atomicAdd(&stats[1], 1ull);
  }
  __syncthreads();
  if (S.accept && i < BB && S.win[fi] != S.wold[fi]) {
    const int y = (y0 + i / B) % L, x = (x0 + i % B) % L;
    const int c = (x + y) & 1, j = x >> 1;
    atomicXor(&planes[(size_t)c * L * Wc + (size_t)y * Wc + (j >> 5)], 1u << (j & 31));
  }
  __syncthreads();
}

struct StagedPassParams {
  uint32_t* planes;  // packed lattice [2][L][Wc]
  int L, Wc, colour;
  uint32_t pass;
  RngParams rng;
  float beta;
  unsigned long long* stats;  // [0] proposed, [1] accepted
};

__global__ void __launch_bounds__(kInferThreads) k_nn_staged_pass(StagedPassParams Q,
                                                             const StagedPlan* __restrict__ plan,
                                                             const __nv_bfloat16* __restrict__ w,
                                                             const __nv_bfloat16* __restrict__ w2t) {
  extern __shared__ uint4 smem_raw[];
  StagedSmem& S = *reinterpret_cast<StagedSmem*>(smem_raw);
  load_all(S, w, w2t, plan);
  __syncthreads();
  const int B = S.plan.B, L = Q.L;
  const int nbx = L / B, half = nbx / 2;
  const int n_sq = nbx * half;
  int ox, oy;
  block_offset(Q.pass, Q.rng.replica, Q.rng, B, ox, oy);
  for (int blk = blockIdx.x; blk < n_sq; blk += gridDim.x) {
    const int by = blk / half, bx = 2 * (blk - by * half) + ((by + Q.colour) & 1);
    process_square(S, Q.planes, L, Q.Wc, Q.colour, ox, oy, bx, by, Q.pass, Q.rng.replica, Q.rng,
                   Q.beta, Q.stats);
  }
}

struct StagedBatchParams {
  uint32_t* spins;
  const long long* off;
  const int* lad_L;
  const int* slot_of;
  const float* beta_of_slot;
  const long long* unit0;  // [n_rep + 1]
  int n_rep, n_beta, colour;
  uint32_t pass;
  RngParams rng;
  unsigned long long* stats;
};

__global__ void __launch_bounds__(kInferThreads) k_nn_staged_batch_pass(StagedBatchParams Q,
                                                                   const StagedPlan* __restrict__ plan,
                                                                   const __nv_bfloat16* __restrict__ w,
                                                                   const __nv_bfloat16* __restrict__ w2t) {
  extern __shared__ uint4 smem_raw[];
  StagedSmem& S = *reinterpret_cast<StagedSmem*>(smem_raw);
  load_all(S, w, w2t, plan);
  __syncthreads();
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
    process_square(S, Q.spins + Q.off[r], L, Wc, Q.colour, ox, oy, bx, by, Q.pass, (uint32_t)r, Q.rng,
                   beta, Q.stats);
  }
}

// Stage logits of windows (tests and diagnostics).
__global__ void __launch_bounds__(kInferThreads) k_nn_stage_logits(const int8_t* __restrict__ windows,
                                                              int n, int stage, float beta,
                                                              const StagedPlan* __restrict__ plan,
                                                              const __nv_bfloat16* __restrict__ w,
                                                              const __nv_bfloat16* __restrict__ w2t,
                                                              float* __restrict__ out) {
  extern __shared__ uint4 smem_raw[];
  StagedSmem& S = *reinterpret_cast<StagedSmem*>(smem_raw);
  load_all(S, w, w2t, plan);
  __syncthreads();
  const int B = S.plan.B, F = B + 2, BB = B * B;
  for (int k = blockIdx.x; k < n; k += gridDim.x) {
    for (int i = threadIdx.x; i < F * F; i += blockDim.x) S.win[i] = windows[(size_t)k * F * F + i];
    for (int i = threadIdx.x; i < BB; i += blockDim.x) S.logit[i] = 0.f;
    __syncthreads();
    stage_eval(S, S.win, stage, beta);
    __syncthreads();
    for (int i = threadIdx.x; i < BB; i += blockDim.x)
      out[(size_t)k * BB + i] = S.plan.stage_of[i] == stage ? S.logit[i] : 0.f;
    __syncthreads();
  }
}

// Teacher-forced ln q of windows (tests and diagnostics).
__global__ void __launch_bounds__(kInferThreads) k_nn_log_q(const int8_t* __restrict__ windows, int n,
                                                       float beta, const StagedPlan* __restrict__ plan,
                                                       const __nv_bfloat16* __restrict__ w,
                                                       const __nv_bfloat16* __restrict__ w2t,
                                                       float* __restrict__ out) {
  extern __shared__ uint4 smem_raw[];
  StagedSmem& S = *reinterpret_cast<StagedSmem*>(smem_raw);
  load_all(S, w, w2t, plan);
  __syncthreads();
  const int F = S.plan.B + 2;
  for (int k = blockIdx.x; k < n; k += gridDim.x) {
    for (int i = threadIdx.x; i < F * F; i += blockDim.x) S.wold[i] = windows[(size_t)k * F * F + i];
    __syncthreads();
    float lq = log2_q_old(S, beta);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lq += __shfl_xor_sync(0xffffffffu, lq, o);
    if ((threadIdx.x & 31) == 0) S.red_lq[threadIdx.x >> 5] = lq;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w8 = 0; w8 < (int)(blockDim.x >> 5); ++w8) t += S.red_lq[w8];
      out[k] = 0.69314718f * t;
    }
    __syncthreads();
  }
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
                            float beta, const __nv_bfloat16* wbf, const __nv_bfloat16* w2t,
                            float* out, cudaStream_t s) {
  static DeviceCache attr;
  cudaError_t e = allow_smem(k_nn_stage_logits, attr);
  if (e) return e;
  const int grid = std::max(1, std::min(count, 2 * sm_count()));
  k_nn_stage_logits<<<grid, kInferThreads, sizeof(StagedSmem), s>>>(windows, count, stage, beta, d_plan,
                                                                   wbf, w2t, out);
  return cudaGetLastError();
}

cudaError_t nn_log_q(const int8_t* windows, int count, const StagedPlan* d_plan, float beta,
                     const __nv_bfloat16* wbf, const __nv_bfloat16* w2t, float* out,
                     cudaStream_t s) {
  static DeviceCache attr;
  cudaError_t e = allow_smem(k_nn_log_q, attr);
  if (e) return e;
  const int grid = std::max(1, std::min(count, 2 * sm_count()));
  k_nn_log_q<<<grid, kInferThreads, sizeof(StagedSmem), s>>>(windows, count, beta, d_plan, wbf, w2t, out);
  return cudaGetLastError();
}

}  // namespace nnc

cudaError_t nn_staged_block_pass(uint32_t* planes, int L, int Wc, const nnc::StagedPlan* d_plan, int B,
                                 uint32_t pass, int colour, const RngParams& rng, double beta,
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
                                       uint32_t pass, const RngParams& rng, const __nv_bfloat16* wbf,
                                       const __nv_bfloat16* w2t, unsigned long long* stats,
                                       cudaStream_t s) {
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
