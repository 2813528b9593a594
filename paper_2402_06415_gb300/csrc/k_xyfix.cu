// Fixed-point XY model sweep for the operand-precision study (arXiv 2402.06415,
// Supplementary "Operand bit width optimization trial", Tab. S3): spin angles
// are fixed-point numbers with F fractional bits (the paper's (m, n) types with
// m - n = F), the random words keep their full 32 bits.  All arithmetic is
// integer, so the chain is exactly reproducible:
//   angle grid k 2^-F, k in [0, K), K = round(2 pi 2^F); tables C[k], S[k] =
//   cos, sin of the grid angle rounded to F fractional bits; local field
//   (hx, hy) = sum of the four neighbours' table entries; proposal
//   k' = floor(u1 K / 2^32); dE = -round(((C[k'] - C[k]) hx + (S[k'] - S[k]) hy)
//   / 2^F) (nearest, ties up; Eq. S1 with its sign corrected, local-field
//   form); accept iff dE <= 0 or u2 < A[dE] = floor(exp(-beta dE 2^-F) 2^32)
//   (with ISING_XYFIX_QUANTISE_P the probability is first truncated to F
//   fractional bits: A[dE] = floor(exp(-beta dE 2^-F) 2^F) 2^(32-F)).
// Layout: angle indices (int32) in two colour planes [2][L][L/2] (site (x, y) of
// colour (x + y) & 1 at y (L/2) + (x >> 1)); tables in device memory (read
// through the read-only cache).  Counter map: start k = floor(w K / 2^32), w =
// word (n & 3) of Philox(n >> 2, 0, r, XYFIX_INIT << 16); sweep t, colour c:
// Philox(j >> 1, t, r, XYFIX_MET << 16 | c << 8), words 2(j & 1), 2(j & 1) + 1.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <vector>

#include "internal.h"
#include "ising.h"
#include "ising_device.cuh"

namespace ising {
namespace {

constexpr uint32_t kTagXYFixMet = 14, kTagXYFixInit = 15;

struct FixTables {
  const int2* trig;        // [K] (C, S)
  const uint32_t* accept;  // [n_accept], index dE (scale 2^-F)
  int n_accept;
  uint32_t K;
  int F;
  FastDiv fh;              // division by L / 2
};

__global__ void k_xyfix_init(int32_t* __restrict__ kp, int L, uint32_t K, RngParams rng) {
  const long long N = (long long)L * L;
  const int half = L / 2;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(n / L), x = (int)(n - (n / L) * L);
    const uint4 r = philox10_rk(make_uint4((uint32_t)(n >> 2), 0u, rng.replica, kTagXYFixInit << 16),
                                rng.rk0, rng.rk1);
    const uint32_t w = (n & 3) == 0 ? r.x : ((n & 3) == 1 ? r.y : ((n & 3) == 2 ? r.z : r.w));
    kp[(size_t)((x + y) & 1) * L * half + (size_t)y * half + (x >> 1)] =
        (int32_t)(((unsigned long long)w * K) >> 32);
  }
}

// State loads / stores: plain in the per-half-sweep kernels, L2-only in the
// persistent kernel (its CTAs read what other SMs wrote after a grid barrier).
template <bool CG>
__device__ __forceinline__ int32_t ld_k(const int32_t* p) {
  if (CG) return __ldcg(p);
  return *p;
}
template <bool CG>
__device__ __forceinline__ void st_k(int32_t* p, int32_t v) {
  if (CG) __stcg(p, v);
  else *p = v;
}

// Trials of the colour-compact sites j = 2b, 2b + 1 of colour c; returns the
// number accepted.
template <bool CG>
__device__ __forceinline__ unsigned int xyfix_pair(int32_t* __restrict__ own, const int32_t* __restrict__ oth,
                                                   int L, uint32_t nk, uint32_t b, int c, uint32_t t,
                                                   const RngParams& rng, const FixTables& tb) {
  const int half = L / 2;
  const long long round_half = 1LL << (tb.F - 1);
  unsigned int acc = 0;
  const uint4 r = philox10_rk(make_uint4(b, t, rng.replica, (kTagXYFixMet << 16) | ((uint32_t)c << 8)),
                              rng.rk0, rng.rk1);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const uint32_t j = 2 * b + h;
    if (j >= nk) break;
    const int y = (int)fdiv(j, tb.fh), jj = (int)(j - (uint32_t)y * (uint32_t)half);
    const int o = (y + c) & 1;
    const int jr = o == 0 ? jj : (jj + 1 == half ? 0 : jj + 1);
    const int jl = o == 0 ? (jj == 0 ? half - 1 : jj - 1) : jj;
    const int yd = y + 1 == L ? 0 : y + 1, yu = y == 0 ? L - 1 : y - 1;
    const int2 a = __ldg(&tb.trig[ld_k<CG>(oth + (size_t)y * half + jr)]);
    const int2 bl = __ldg(&tb.trig[ld_k<CG>(oth + (size_t)y * half + jl)]);
    const int2 d = __ldg(&tb.trig[ld_k<CG>(oth + (size_t)yd * half + jj)]);
    const int2 e = __ldg(&tb.trig[ld_k<CG>(oth + (size_t)yu * half + jj)]);
    const long long hx = (long long)a.x + bl.x + d.x + e.x;
    const long long hy = (long long)a.y + bl.y + d.y + e.y;
    const uint32_t w1 = h == 0 ? r.x : r.z, w2 = h == 0 ? r.y : r.w;
    const int32_t k2 = (int32_t)(((unsigned long long)w1 * tb.K) >> 32);
    const int32_t k1 = ld_k<CG>(own + j);
    const int2 t1 = __ldg(&tb.trig[k1]), t2 = __ldg(&tb.trig[k2]);
    const long long p = (long long)(t2.x - t1.x) * hx + (long long)(t2.y - t1.y) * hy;
    const long long dE = -((p + round_half) >> tb.F);
    bool ok = dE <= 0;
    if (!ok) ok = w2 < __ldg(&tb.accept[dE < tb.n_accept ? dE : tb.n_accept - 1]);
    if (ok) {
      st_k<CG>(own + j, k2);
      ++acc;
    }
  }
  return acc;
}

__device__ __forceinline__ void fix_add_accepted(unsigned long long* accepted, unsigned int acc) {
  if (!accepted) return;
  unsigned int s = acc;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(accepted, (unsigned long long)s);
}

// One half sweep of colour c; thread = one Philox block = colour-compact sites
// j = 2b and 2b + 1.
__global__ void __launch_bounds__(256) k_xyfix_half(int32_t* __restrict__ kp, int L, int c, uint32_t t,
                                                    RngParams rng, FixTables tb,
                                                    unsigned long long* __restrict__ accepted) {
  const int half = L / 2;
  const uint32_t nk = (uint32_t)L * (uint32_t)half;
  int32_t* own = kp + (size_t)c * L * half;
  const int32_t* oth = kp + (size_t)(1 - c) * L * half;
  unsigned int acc = 0;
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; 2 * b < nk; b += gridDim.x * blockDim.x)
    acc += xyfix_pair<false>(own, oth, L, nk, b, c, t, rng, tb);
  fix_add_accepted(accepted, acc);
}

// out3[0] += sum over bonds of C C' + S S' (each bond once: colour-0 site times
// its four colour-1 neighbours); out3[1..2] += sum C, sum S.
template <bool CG>
__device__ __forceinline__ void xyfix_measure_part(const int32_t* __restrict__ kp, int L,
                                                   const int2* __restrict__ trig,
                                                   unsigned long long* __restrict__ out3, const FastDiv& fh) {
  const int half = L / 2;
  const uint32_t nk = (uint32_t)L * (uint32_t)half;
  const int32_t* p0 = kp;
  const int32_t* p1 = kp + (size_t)L * half;
  long long e = 0, mx = 0, my = 0;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nk; j += gridDim.x * blockDim.x) {
    const int y = (int)fdiv(j, fh), jj = (int)(j - (uint32_t)y * (uint32_t)half);
    const int o = y & 1;
    const int jr = o == 0 ? jj : (jj + 1 == half ? 0 : jj + 1);
    const int jl = o == 0 ? (jj == 0 ? half - 1 : jj - 1) : jj;
    const int yd = y + 1 == L ? 0 : y + 1, yu = y == 0 ? L - 1 : y - 1;
    const int2 s = __ldg(&trig[ld_k<CG>(p0 + j)]);
    const int2 a = __ldg(&trig[ld_k<CG>(p1 + (size_t)y * half + jr)]);
    const int2 b = __ldg(&trig[ld_k<CG>(p1 + (size_t)y * half + jl)]);
    const int2 d = __ldg(&trig[ld_k<CG>(p1 + (size_t)yd * half + jj)]);
    const int2 f = __ldg(&trig[ld_k<CG>(p1 + (size_t)yu * half + jj)]);
    e += (long long)s.x * ((long long)a.x + b.x + d.x + f.x) + (long long)s.y * ((long long)a.y + b.y + d.y + f.y);
    const int2 s1 = __ldg(&trig[ld_k<CG>(p1 + j)]);
    mx += (long long)s.x + s1.x;
    my += (long long)s.y + s1.y;
  }
  const unsigned long long se = warp_sum_u64((unsigned long long)e);
  const unsigned long long sx = warp_sum_u64((unsigned long long)mx);
  const unsigned long long sy = warp_sum_u64((unsigned long long)my);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out3[0], se);
    atomicAdd(&out3[1], sx);
    atomicAdd(&out3[2], sy);
  }
}

__global__ void __launch_bounds__(256) k_xyfix_measure(const int32_t* __restrict__ kp, int L,
                                                       const int2* __restrict__ trig,
                                                       unsigned long long* __restrict__ out3, FastDiv fh) {
  xyfix_measure_part<false>(kp, L, trig, out3, fh);
}

// Persistent form for small lattices (as for the floating-point XY kernel): n
// sweeps from t0 in one launch; PM 0: one CTA with __syncthreads(); 1: one
// thread-block cluster with the hardware cluster barrier; 2: cooperative grid
// with the bounded grid barrier (state through L2 in 1 and 2); record slot
// zeroed by CTA 0 in the half sweep before.
template <int PM>
__device__ __forceinline__ bool fix_sync(GridCtl* ctl, long long limit) {
  if (PM == 2) return grid_sync_bounded(ctl, limit);
  if (PM == 1) cooperative_groups::this_cluster().sync();
  else __syncthreads();
  return true;
}

template <int PM>
__global__ void __launch_bounds__(PM == 2 ? 256 : 1024) k_xyfix_persist(int32_t* __restrict__ kp, int L, RngParams rng,
                                                       FixTables tb, uint32_t t0, int n, int m,
                                                       unsigned long long* __restrict__ rec, long long rec0,
                                                       long long rec_cap,
                                                       unsigned long long* __restrict__ accepted,
                                                       GridCtl* ctl, long long limit) {
  const int half = L / 2;
  const uint32_t nk = (uint32_t)L * (uint32_t)half;
  unsigned int acc = 0;
  long long ri = rec0;
  for (int s = 0; s < n; ++s) {
    const uint32_t t = t0 + (uint32_t)s;
    const bool meas = m > 0 && ((long long)t + 1) % m == 0;
    unsigned long long* slot = rec + 3 * (ri % rec_cap);
    bool ok = true;
    for (int c = 0; c < 2 && ok; ++c) {
      int32_t* own = kp + (size_t)c * L * half;
      const int32_t* oth = kp + (size_t)(1 - c) * L * half;
      for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; 2 * b < nk; b += gridDim.x * blockDim.x)
        acc += xyfix_pair<PM != 0>(own, oth, L, nk, b, c, t, rng, tb);
      if (meas && c == 1 && blockIdx.x == 0 && threadIdx.x == 0) slot[0] = slot[1] = slot[2] = 0ull;
      ok = fix_sync<PM>(ctl, limit);
    }
    if (ok && meas) {
      xyfix_measure_part<PM != 0>(kp, L, tb.trig, slot, tb.fh);
      ++ri;
      ok = fix_sync<PM>(ctl, limit);
    }
    if (!ok) break;
  }
  fix_add_accepted(accepted, acc);
}

// to_dev = 0: planes -> row-major [L][L]; 1: the reverse (host is the source).
__global__ void k_xyfix_layout(int32_t* __restrict__ kp, int L, int32_t* __restrict__ rm, int to_dev) {
  const long long N = (long long)L * L;
  const int half = L / 2;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(n / L), x = (int)(n - (n / L) * L);
    const size_t idx = (size_t)((x + y) & 1) * L * half + (size_t)y * half + (x >> 1);
    if (to_dev) kp[idx] = rm[n];
    else rm[n] = kp[idx];
  }
}

int ffail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

#define FTRY(expr)                                                                        \
  do {                                                                                    \
    cudaError_t e__ = (expr);                                                             \
    if (e__ != cudaSuccess) return ffail(ISING_ECUDA, "%s: %s", #expr, cudaGetErrorString(e__)); \
  } while (0)

int fgrid(long long items) {
  long long g = (items + 255) / 256;
  return (int)std::max(1LL, std::min(g, 152LL * 32));
}

}  // namespace
}  // namespace ising

using namespace ising;

struct ising_xyfix {
  int L = 0, F = 0;
  uint32_t K = 0;
  double beta = 0;
  uint64_t seed = 0;
  int64_t sweep = 0;
  cudaStream_t stream = nullptr;
  int32_t* kp = nullptr;
  int2* trig = nullptr;
  uint32_t* accept = nullptr;
  int n_accept = 0;
  unsigned long long* rec = nullptr;  // ring [65536][3]
  int64_t rec_count = 0;
  unsigned long long* accepted = nullptr;
  int64_t launches = 0;
  int mode = 0;  // 0 auto, 1 one launch per half sweep, 2 persistent
  GridCtl* ctl = nullptr;
};

namespace {
constexpr int64_t kFixRec = 65536;
constexpr int kFixPersistMaxL = 256;               // automatic mode: persistent kernel up to here
constexpr long long kFixSpinLimit = 4000000000LL;  // ~2 s of SM clock per barrier

// Tables on the host.  Products and sums are kept in volatile temporaries so
// that no compiler fuses them: the entries must round exactly as written.
void build_fix_tables(int F, double beta, bool qp, uint32_t* K, std::vector<int2>& trig,
                      std::vector<uint32_t>& acc) {
  volatile double two_pi_scaled = 2.0 * 3.14159265358979323846 * std::ldexp(1.0, F);
  *K = (uint32_t)std::floor(two_pi_scaled + 0.5);
  const double sc = std::ldexp(1.0, F);
  trig.resize(*K);
  for (uint32_t k = 0; k < *K; ++k) {
    const double a = std::ldexp((double)k, -F);
    volatile double cs = std::cos(a) * sc;
    volatile double sn = std::sin(a) * sc;
    trig[k].x = (int32_t)std::floor(cs + 0.5);
    trig[k].y = (int32_t)std::floor(sn + 0.5);
  }
  // |dE| <= 8 (2^F + 1)^2 / 2^F + 1 < 9 2^F for F >= 5
  acc.assign((size_t)9 << F, 0xffffffffu);
  for (size_t e = 1; e < acc.size(); ++e) {
    const double dE = std::ldexp((double)e, -F);
    volatile double x = -beta * dE;
    // qp: the probability truncated to F fractional bits (ldexp scales exactly)
    const double t = qp ? std::ldexp(std::floor(std::ldexp(std::exp(x), F)), 32 - F)
                        : std::floor(std::exp(x) * 4294967296.0);
    acc[e] = t >= 4294967295.0 ? 0xffffffffu : (uint32_t)t;
  }
}
}  // namespace

extern "C" {

int ising_xyfix_create(ising_xyfix** out, int L, double beta, int frac_bits, int flags, void* stream) {
  if (!out) return ffail(ISING_EINVAL, "null output pointer");
  *out = nullptr;
  if (L < 2 || L > 32768 || (L & 1)) return ffail(ISING_EINVAL, "L must be even and in [2, 32768]");
  if (!std::isfinite(beta) || beta <= 0) return ffail(ISING_EINVAL, "beta must be finite and > 0");
  if (frac_bits < 6 || frac_bits > 16) return ffail(ISING_EINVAL, "frac_bits must be in [6, 16]");
  if (flags & ~ISING_XYFIX_QUANTISE_P) return ffail(ISING_EINVAL, "unknown flags 0x%x", flags);
  ising_xyfix* x = new (std::nothrow) ising_xyfix();
  if (!x) return ffail(ISING_ENOMEM, "host allocation failed");
  x->L = L;
  x->F = frac_bits;
  x->beta = beta;
  x->stream = (cudaStream_t)stream;
  std::vector<int2> trig;
  std::vector<uint32_t> acc;
  build_fix_tables(frac_bits, beta, (flags & ISING_XYFIX_QUANTISE_P) != 0, &x->K, trig, acc);
  x->n_accept = (int)acc.size();
  cudaError_t e = cudaMalloc((void**)&x->kp, (size_t)L * L * sizeof(int32_t));
  if (!e) e = cudaMalloc((void**)&x->trig, trig.size() * sizeof(int2));
  if (!e) e = cudaMalloc((void**)&x->accept, acc.size() * sizeof(uint32_t));
  if (!e) e = cudaMalloc((void**)&x->rec, kFixRec * 3 * sizeof(unsigned long long));
  if (!e) e = cudaMalloc((void**)&x->accepted, sizeof(unsigned long long));
  if (!e) e = cudaMalloc((void**)&x->ctl, sizeof(GridCtl));
  if (!e) e = cudaMemset(x->ctl, 0, sizeof(GridCtl));
  if (!e) e = cudaMemcpy(x->trig, trig.data(), trig.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(x->accept, acc.data(), acc.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e) {
    cudaGetLastError();
    cudaFree(x->kp);
    cudaFree(x->trig);
    cudaFree(x->accept);
    cudaFree(x->rec);
    cudaFree(x->accepted);
    cudaFree(x->ctl);
    delete x;
    return ffail(ISING_ENOMEM, "fixed-point XY allocation: %s", cudaGetErrorString(e));
  }
  *out = x;
  return ising_xyfix_seed(x, 0);
}

int ising_xyfix_seed(ising_xyfix* x, uint64_t seed) {
  if (!x) return ffail(ISING_EINVAL, "null context");
  x->seed = seed;
  x->sweep = 0;
  x->rec_count = 0;
  const RngParams rng = make_rng(seed, 0, 0, 0);
  k_xyfix_init<<<fgrid((long long)x->L * x->L), 256, 0, x->stream>>>(x->kp, x->L, x->K, rng);
  FTRY(cudaGetLastError());
  FTRY(cudaMemsetAsync(x->accepted, 0, sizeof(unsigned long long), x->stream));
  FTRY(cudaMemsetAsync(x->ctl, 0, sizeof(GridCtl), x->stream));
  set_last_error("");
  return ISING_OK;
}

int ising_xyfix_sweep(ising_xyfix* x, int n_sweeps, int measure_every) {
  if (!x) return ffail(ISING_EINVAL, "null context");
  if (n_sweeps < 0 || measure_every < 0) return ffail(ISING_EINVAL, "negative count");
  if (x->sweep + n_sweeps >= ((int64_t)1 << 32)) return ffail(ISING_EINVAL, "sweep counter overflow");
  NvtxRange nvtx("ising_xyfix_sweep");
  const RngParams rng = make_rng(x->seed, 0, 0, 0);
  const FixTables tb{x->trig, x->accept, x->n_accept, x->K, x->F, make_fastdiv((uint32_t)(x->L / 2))};
  if (x->mode == 2 || (x->mode == 0 && x->L <= kFixPersistMaxL)) {
    if (n_sweeps == 0) return ISING_OK;
    int dev = 0, sms = 0;
    FTRY(cudaGetDevice(&dev));
    FTRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long pairs = ((long long)x->L * (x->L / 2) + 1) / 2;
    // one CTA up to 256 site pairs, one cluster of 8 CTAs up to 8192, beyond a
    // cooperative grid
    const int pm = pairs <= 256 ? 0 : (pairs <= 8192 ? 1 : 2);
    const int threads = pm == 0 ? (int)(((pairs + 31) / 32) * 32)
                                : (pm == 1 ? (int)std::min<long long>(1024, ((pairs + 255) / 256) * 32) : 64);
    const long long grid =
        pm == 0 ? 1 : (pm == 1 ? 8 : std::max(1LL, std::min((pairs + threads - 1) / threads, (long long)sms)));
    if (pm == 2) FTRY(cudaMemsetAsync(&x->ctl->count, 0, sizeof(unsigned int), x->stream));
    int32_t* kp = x->kp;
    int L = x->L, n = n_sweeps, m = measure_every;
    RngParams r = rng;
    FixTables t = tb;
    uint32_t t0 = (uint32_t)x->sweep;
    unsigned long long* rec = x->rec;
    long long rec0 = x->rec_count, cap = kFixRec, limit = kFixSpinLimit;
    unsigned long long* acc = x->accepted;
    GridCtl* ctl = x->ctl;
    void* args[] = {&kp, &L, &r, &t, &t0, &n, &m, &rec, &rec0, &cap, &acc, &ctl, &limit};
    if (pm == 0) {
      FTRY(cudaLaunchKernel((const void*)k_xyfix_persist<0>, dim3(1), dim3(threads), args, 0, x->stream));
    } else if (pm == 1) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)grid);
      cfg.blockDim = dim3(threads);
      cfg.stream = x->stream;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)grid;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      FTRY(cudaLaunchKernelExC(&cfg, (const void*)k_xyfix_persist<1>, args));
    } else {
      FTRY(cudaLaunchCooperativeKernel((const void*)k_xyfix_persist<2>, dim3((unsigned)grid), dim3(threads),
                                       args, 0, x->stream));
    }
    ++x->launches;
    if (m > 0)
      for (int s = 0; s < n; ++s)
        if (((int64_t)x->sweep + s + 1) % m == 0) ++x->rec_count;
    x->sweep += n_sweeps;
    set_last_error("");
    return ISING_OK;
  }
  const long long blocks = ((long long)x->L * (x->L / 2) + 1) / 2;
  for (int s = 0; s < n_sweeps; ++s) {
    const uint32_t t = (uint32_t)(x->sweep + s);
    for (int c = 0; c < 2; ++c) {
      k_xyfix_half<<<fgrid(blocks), 256, 0, x->stream>>>(x->kp, x->L, c, t, rng, tb, x->accepted);
      FTRY(cudaGetLastError());
      ++x->launches;
    }
    if (measure_every > 0 && ((int64_t)t + 1) % measure_every == 0) {
      unsigned long long* slot = x->rec + 3 * (x->rec_count % kFixRec);
      FTRY(cudaMemsetAsync(slot, 0, 3 * sizeof(unsigned long long), x->stream));
      k_xyfix_measure<<<fgrid((long long)x->L * (x->L / 2)), 256, 0, x->stream>>>(x->kp, x->L, x->trig,
                                                                                   slot, tb.fh);
      FTRY(cudaGetLastError());
      ++x->launches;
      ++x->rec_count;
    }
  }
  x->sweep += n_sweeps;
  set_last_error("");
  return ISING_OK;
}

static int xyfix_status(ising_xyfix* x) {
  int st = 0;
  FTRY(cudaMemcpy(&st, &x->ctl->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) return ffail(ISING_ETIMEOUT, "grid barrier timed out in the persistent fixed-point XY kernel");
  return ISING_OK;
}

int ising_xyfix_set_mode(ising_xyfix* x, int mode) {
  if (!x) return ffail(ISING_EINVAL, "null context");
  if (mode < 0 || mode > 2) return ffail(ISING_EINVAL, "mode must be 0 (auto), 1 (per half sweep) or 2 (persistent)");
  x->mode = mode;
  set_last_error("");
  return ISING_OK;
}

int ising_xyfix_series(ising_xyfix* x, int64_t* E2, int64_t* Mx, int64_t* My, int n) {
  if (!x) return ffail(ISING_EINVAL, "null context");
  if (n < 0 || n > std::min<int64_t>(x->rec_count, kFixRec)) return ffail(ISING_EINVAL, "n exceeds records");
  std::vector<unsigned long long> h((size_t)3 * kFixRec);
  FTRY(cudaMemcpyAsync(h.data(), x->rec, h.size() * 8, cudaMemcpyDeviceToHost, x->stream));
  FTRY(cudaStreamSynchronize(x->stream));
  if (int st = xyfix_status(x)) return st;
  for (int i = 0; i < n; ++i) {
    const int64_t slot = (x->rec_count - n + i) % kFixRec;
    if (E2) E2[i] = (int64_t)h[3 * slot];
    if (Mx) Mx[i] = (int64_t)h[3 * slot + 1];
    if (My) My[i] = (int64_t)h[3 * slot + 2];
  }
  set_last_error("");
  return ISING_OK;
}

static int xyfix_layout(ising_xyfix* x, int32_t* host, int to_dev) {
  const long long N = (long long)x->L * x->L;
  int32_t* d = nullptr;
  FTRY(cudaMalloc((void**)&d, N * sizeof(int32_t)));
  cudaError_t e = cudaSuccess;
  if (to_dev) {
    for (long long i = 0; i < N; ++i)
      if (host[i] < 0 || (uint32_t)host[i] >= x->K) {
        cudaFree(d);
        return ffail(ISING_EINVAL, "angle index out of [0, K)");
      }
    e = cudaMemcpyAsync(d, host, N * sizeof(int32_t), cudaMemcpyHostToDevice, x->stream);
  }
  if (!e) {
    k_xyfix_layout<<<fgrid(N), 256, 0, x->stream>>>(x->kp, x->L, d, to_dev);
    e = cudaGetLastError();
  }
  if (!e && !to_dev) e = cudaMemcpyAsync(host, d, N * sizeof(int32_t), cudaMemcpyDeviceToHost, x->stream);
  if (!e) e = cudaStreamSynchronize(x->stream);
  cudaFree(d);
  if (e) return ffail(ISING_ECUDA, "angle copy: %s", cudaGetErrorString(e));
  if (int st = xyfix_status(x)) return st;
  set_last_error("");
  return ISING_OK;
}

int ising_xyfix_get_angles(ising_xyfix* x, int32_t* host_k) {
  if (!x || !host_k) return ffail(ISING_EINVAL, "null argument");
  return xyfix_layout(x, host_k, 0);
}

int ising_xyfix_set_angles(ising_xyfix* x, const int32_t* host_k) {
  if (!x || !host_k) return ffail(ISING_EINVAL, "null argument");
  return xyfix_layout(x, const_cast<int32_t*>(host_k), 1);
}

int ising_xyfix_info(ising_xyfix* x, int64_t* K, int64_t* accepted, int64_t* launches) {
  if (!x) return ffail(ISING_EINVAL, "null context");
  unsigned long long h = 0;
  FTRY(cudaMemcpyAsync(&h, x->accepted, 8, cudaMemcpyDeviceToHost, x->stream));
  FTRY(cudaStreamSynchronize(x->stream));
  if (int st = xyfix_status(x)) return st;
  if (K) *K = x->K;
  if (accepted) *accepted = (int64_t)h;
  if (launches) *launches = x->launches;
  set_last_error("");
  return ISING_OK;
}

int ising_xyfix_destroy(ising_xyfix* x) {
  if (!x) return ISING_OK;
  cudaStreamSynchronize(x->stream);
  cudaFree(x->kp);
  cudaFree(x->trig);
  cudaFree(x->accept);
  cudaFree(x->rec);
  cudaFree(x->accepted);
  cudaFree(x->ctl);
  delete x;
  return ISING_OK;
}

}  // extern "C"
