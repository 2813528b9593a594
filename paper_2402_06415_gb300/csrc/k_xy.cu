// Checkerboard Metropolis sweep of the 2D XY model: the paper's own Monte Carlo
// workload (arXiv 2402.06415, Eq. 1; Supplementary "Detail of the MC
// calculation for the XY model").  Each site holds the unit vector
// u = (cos theta, sin theta).  Per site: theta' = 2 pi U1, p = U2 (two 24-bit
// uniforms from one half of a Philox block), dE = -(u' - u) . h with h the sum
// of the four neighbour vectors (Eq. S1, sign corrected, in local-field form),
// accept iff dE <= 0 or p < exp(-beta dE).  Sublattice (x + y) even, then odd.
//
// cos, sin and exp are evaluated by this file's own routines: Cody-Waite
// reduction by pi/2 (two-part constant) or ln 2, then Taylor polynomials in
// Horner form with explicit fused multiply-adds.  All other arithmetic is
// single IEEE operations in a fixed order, so every decision is reproducible
// bit for bit by any implementation of the same recipe.
//
// Layout: two colour planes of [L][L/2] vectors (T2 = float2 or double2);
// site (x, y) of colour c = (x + y) & 1 is element y (L/2) + (x >> 1) of plane c.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

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

constexpr uint32_t kTagXYInit = 8, kTagXYMet = 9;

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float2; };
template <> struct Vec<double> { using type = double2; };

// ---- own elementary functions (double) ----
__device__ __forceinline__ void sincos_small(double r, double& s, double& c) {
  const double z = __dmul_rn(r, r);
  double pc = 1.0 / 20922789888000.0;
  pc = fma(pc, z, -1.0 / 87178291200.0);
  pc = fma(pc, z, 1.0 / 479001600.0);
  pc = fma(pc, z, -1.0 / 3628800.0);
  pc = fma(pc, z, 1.0 / 40320.0);
  pc = fma(pc, z, -1.0 / 720.0);
  pc = fma(pc, z, 1.0 / 24.0);
  pc = fma(pc, z, -0.5);
  pc = fma(pc, z, 1.0);
  double ps = 1.0 / 355687428096000.0;
  ps = fma(ps, z, -1.0 / 1307674368000.0);
  ps = fma(ps, z, 1.0 / 6227020800.0);
  ps = fma(ps, z, -1.0 / 39916800.0);
  ps = fma(ps, z, 1.0 / 362880.0);
  ps = fma(ps, z, -1.0 / 5040.0);
  ps = fma(ps, z, 1.0 / 120.0);
  ps = fma(ps, z, -1.0 / 6.0);
  ps = fma(ps, z, 1.0);
  c = pc;
  s = __dmul_rn(ps, r);
}

__device__ __forceinline__ void own_sincos(double x, double& s, double& c) {
  const double k = rint(__dmul_rn(x, 0.6366197723675814));
  double r = fma(-k, 1.5707963267948966, x);
  r = fma(-k, 6.123233995736766e-17, r);
  double ss, cc;
  sincos_small(r, ss, cc);
  const int q = ((int)k) & 3;
  s = q == 0 ? ss : (q == 1 ? cc : (q == 2 ? -ss : -cc));
  c = q == 0 ? cc : (q == 1 ? -ss : (q == 2 ? -cc : ss));
}

__device__ __forceinline__ double own_exp(double x) {
  if (x < -700.0) return 0.0;
  const double k = rint(__dmul_rn(x, 1.4426950408889634));
  double r = fma(-k, 0.6931471805599453, x);
  r = fma(-k, 2.3190468138462996e-17, r);
  double p = 1.0 / 6227020800.0;
  p = fma(p, r, 1.0 / 479001600.0);
  p = fma(p, r, 1.0 / 39916800.0);
  p = fma(p, r, 1.0 / 3628800.0);
  p = fma(p, r, 1.0 / 362880.0);
  p = fma(p, r, 1.0 / 40320.0);
  p = fma(p, r, 1.0 / 5040.0);
  p = fma(p, r, 1.0 / 720.0);
  p = fma(p, r, 1.0 / 120.0);
  p = fma(p, r, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  p = fma(p, r, 1.0);
  // p 2^k with 2^k built from its exponent field (k in [-1010, 0], a normal
  // number): a multiplication by a power of two is exact, or correctly rounded
  // when the product is subnormal, i.e. the same result as ldexp
  return p * __longlong_as_double((long long)((int)k + 1023) << 52);
}

// ---- own elementary functions (float) ----
__device__ __forceinline__ void sincos_small(float r, float& s, float& c) {
  const float z = __fmul_rn(r, r);
  float pc = 1.0f / 40320.0f;
  pc = fmaf(pc, z, -1.0f / 720.0f);
  pc = fmaf(pc, z, 1.0f / 24.0f);
  pc = fmaf(pc, z, -0.5f);
  pc = fmaf(pc, z, 1.0f);
  float ps = 1.0f / 362880.0f;
  ps = fmaf(ps, z, -1.0f / 5040.0f);
  ps = fmaf(ps, z, 1.0f / 120.0f);
  ps = fmaf(ps, z, -1.0f / 6.0f);
  ps = fmaf(ps, z, 1.0f);
  c = pc;
  s = __fmul_rn(ps, r);
}

__device__ __forceinline__ void own_sincos(float x, float& s, float& c) {
  const float k = rintf(__fmul_rn(x, 0.636619747f));
  float r = fmaf(-k, 1.57079637f, x);
  r = fmaf(-k, -4.37113883e-08f, r);
  float ss, cc;
  sincos_small(r, ss, cc);
  const int q = ((int)k) & 3;
  s = q == 0 ? ss : (q == 1 ? cc : (q == 2 ? -ss : -cc));
  c = q == 0 ? cc : (q == 1 ? -ss : (q == 2 ? -cc : ss));
}

__device__ __forceinline__ float own_exp(float x) {
  if (x < -87.0f) return 0.0f;
  const float k = rintf(__fmul_rn(x, 1.44269502f));
  float r = fmaf(-k, 0.693147182f, x);
  r = fmaf(-k, -1.90465421e-09f, r);
  float p = 1.0f / 40320.0f;
  p = fmaf(p, r, 1.0f / 5040.0f);
  p = fmaf(p, r, 1.0f / 720.0f);
  p = fmaf(p, r, 1.0f / 120.0f);
  p = fmaf(p, r, 1.0f / 24.0f);
  p = fmaf(p, r, 1.0f / 6.0f);
  p = fmaf(p, r, 0.5f);
  p = fmaf(p, r, 1.0f);
  p = fmaf(p, r, 1.0f);
  // p 2^k, 2^k from its exponent field (k in [-126, 0]): same result as ldexpf
  return p * __int_as_float(((int)k + 127) << 23);
}

template <typename T> __device__ __forceinline__ T two_pi();
template <> __device__ __forceinline__ double two_pi<double>() { return 6.283185307179586; }
template <> __device__ __forceinline__ float two_pi<float>() { return 6.28318548f; }
template <typename T> __device__ __forceinline__ T inv24();
template <> __device__ __forceinline__ double inv24<double>() { return 1.0 / 16777216.0; }
template <> __device__ __forceinline__ float inv24<float>() { return 1.0f / 16777216.0f; }

template <typename T> __device__ __forceinline__ T mul_rn(T a, T b);
template <> __device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }
template <> __device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <typename T> __device__ __forceinline__ T add_rn(T a, T b);
template <> __device__ __forceinline__ double add_rn<double>(double a, double b) { return __dadd_rn(a, b); }
template <> __device__ __forceinline__ float add_rn<float>(float a, float b) { return __fadd_rn(a, b); }
template <typename T> __device__ __forceinline__ T sub_rn(T a, T b);
template <> __device__ __forceinline__ double sub_rn<double>(double a, double b) { return __dsub_rn(a, b); }
template <> __device__ __forceinline__ float sub_rn<float>(float a, float b) { return __fsub_rn(a, b); }

template <typename T>
__device__ __forceinline__ T angle_of(uint32_t w) {
  return mul_rn<T>(two_pi<T>(), mul_rn<T>((T)(w >> 8), inv24<T>()));
}

template <typename T>
__global__ void k_xy_init(typename Vec<T>::type* __restrict__ u, int L, RngParams rng) {
  const long long N = (long long)L * L;
  const int half = L / 2;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(n / L), x = (int)(n - (n / L) * L);
    const uint4 r = philox10_rk(make_uint4((uint32_t)(n >> 2), 0u, rng.replica, kTagXYInit << 16),
                                rng.rk0, rng.rk1);
    const uint32_t w = (n & 3) == 0 ? r.x : ((n & 3) == 1 ? r.y : ((n & 3) == 2 ? r.z : r.w));
    T s, c;
    own_sincos(angle_of<T>(w), s, c);
    const int col = (x + y) & 1;
    typename Vec<T>::type v;
    v.x = c;
    v.y = s;
    u[(size_t)col * L * half + (size_t)y * half + (x >> 1)] = v;
  }
}

// The acceptance decision p < own_exp(x) (x = -beta dE < 0), decided first from
// the hardware exponential __expf: its documented error on this range is at most
// 2 + 1.173 |x| ulp (about 1e-5 relative for x >= -80), the rounding of x to
// float adds at most |x| 2^-24 relative, so when p lies outside
// e (1 -+ 1e-4) the exact own_exp gives the same answer and is skipped; inside
// that band (rare), or for x < -80 with p = 0, own_exp decides.  For x < -80,
// exp(x) < 2^-115 < p whenever p > 0 (p is a multiple of 2^-24).
template <typename T>
__device__ __forceinline__ bool accept_exp(T p, T x) {
  if (x >= (T)-80) {
    const float e = __expf((float)x);
    const float pf = (float)p;  // exact: p = k 2^-24, k < 2^24
    if (pf < e * 0.9999f) return true;
    if (pf > e * 1.0001f) return false;
  } else if (p > (T)0) {
    return false;
  }
  return p < own_exp(x);
}

// Loads and stores of the state: plain in the one-launch-per-half-sweep
// kernels; through L2 only (no L1) in the persistent kernel, whose CTAs read
// what other SMs wrote after a grid barrier.
template <bool CG, typename V>
__device__ __forceinline__ V ld_state(const V* p) {
  if (CG) return __ldcg(p);
  return *p;
}
template <bool CG, typename V>
__device__ __forceinline__ void st_state(V* p, V v) {
  if (CG) __stcg(p, v);
  else *p = v;
}

// Metropolis trials of the two colour-compact sites k = 2b, 2b + 1 of colour
// c (one Philox block); returns how many were accepted.
template <typename T, bool CG>
__device__ __forceinline__ unsigned int xy_pair(typename Vec<T>::type* __restrict__ own,
                                                const typename Vec<T>::type* __restrict__ oth, int L,
                                                uint32_t nk, uint32_t b, int c, uint32_t t, T beta,
                                                const RngParams& rng, const FastDiv& fh) {
  using V = typename Vec<T>::type;
  const int half = L / 2;
  unsigned int acc = 0;
  const uint4 r = philox10_rk(make_uint4(b, t, rng.replica, (kTagXYMet << 16) | ((uint32_t)c << 8)),
                              rng.rk0, rng.rk1);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const uint32_t k = 2 * b + h;
    if (k >= nk) break;
    const int y = (int)fdiv(k, fh), j = (int)(k - (uint32_t)y * (uint32_t)half);
    const int o = (y + c) & 1;  // x = 2 j + o
    const int jr = o == 0 ? j : (j + 1 == half ? 0 : j + 1);   // x + 1
    const int jl = o == 0 ? (j == 0 ? half - 1 : j - 1) : j;   // x - 1
    const int yd = y + 1 == L ? 0 : y + 1, yu = y == 0 ? L - 1 : y - 1;
    const V a = ld_state<CG>(oth + (size_t)y * half + jr);
    const V bl = ld_state<CG>(oth + (size_t)y * half + jl);
    const V d = ld_state<CG>(oth + (size_t)yd * half + j);
    const V e = ld_state<CG>(oth + (size_t)yu * half + j);
    T hx = add_rn<T>(a.x, bl.x);
    hx = add_rn<T>(hx, d.x);
    hx = add_rn<T>(hx, e.x);
    T hy = add_rn<T>(a.y, bl.y);
    hy = add_rn<T>(hy, d.y);
    hy = add_rn<T>(hy, e.y);
    const uint32_t w1 = h == 0 ? r.x : r.z, w2 = h == 0 ? r.y : r.w;
    T sn, cs;
    own_sincos(angle_of<T>(w1), sn, cs);
    const T p = mul_rn<T>((T)(w2 >> 8), inv24<T>());
    V me = ld_state<CG>(own + k);
    const T dE = -fma(sub_rn<T>(cs, me.x), hx, mul_rn<T>(sub_rn<T>(sn, me.y), hy));
    if (dE <= (T)0 || accept_exp<T>(p, mul_rn<T>(-beta, dE))) {
      me.x = cs;
      me.y = sn;
      st_state<CG>(own + k, me);
      ++acc;
    }
  }
  return acc;
}

__device__ __forceinline__ void add_accepted(unsigned long long* accepted, unsigned int acc) {
  if (!accepted) return;
  unsigned int s = acc;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(accepted, (unsigned long long)s);
}

// One half sweep of colour c: thread = one Philox block = colour-compact sites
// k = 2b and 2b + 1.
template <typename T>
__global__ void __launch_bounds__(256) k_xy_half(typename Vec<T>::type* __restrict__ u, int L,
                                                 int c, uint32_t t, T beta, RngParams rng, FastDiv fh,
                                                 unsigned long long* __restrict__ accepted) {
  const int half = L / 2;
  const uint32_t nk = (uint32_t)L * (uint32_t)half;  // < 2^29 for L <= 32768
  typename Vec<T>::type* own = u + (size_t)c * L * half;
  const typename Vec<T>::type* oth = u + (size_t)(1 - c) * L * half;
  unsigned int acc = 0;
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; 2 * b < nk; b += gridDim.x * blockDim.x)
    acc += xy_pair<T, false>(own, oth, L, nk, b, c, t, beta, rng, fh);
  add_accepted(accepted, acc);
}

// E = -sum over colour-0 sites of u . (sum of its four neighbours) (every bond
// once), M = sum u; per-thread partials over a grid-stride range, accumulated
// in double and added to out3 by one atomic per warp.
template <typename T, bool CG>
__device__ __forceinline__ void xy_measure_part(const typename Vec<T>::type* __restrict__ u, int L,
                                                double* __restrict__ out3, const FastDiv& fh) {
  using V = typename Vec<T>::type;
  const int half = L / 2;
  const uint32_t nk = (uint32_t)L * (uint32_t)half;
  const V* p0 = u;
  const V* p1 = u + (size_t)L * half;
  double e = 0, mx = 0, my = 0;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nk; k += gridDim.x * blockDim.x) {
    const int y = (int)fdiv(k, fh), j = (int)(k - (uint32_t)y * (uint32_t)half);
    const int o = y & 1;
    const int jr = o == 0 ? j : (j + 1 == half ? 0 : j + 1);
    const int jl = o == 0 ? (j == 0 ? half - 1 : j - 1) : j;
    const int yd = y + 1 == L ? 0 : y + 1, yu = y == 0 ? L - 1 : y - 1;
    const V s = ld_state<CG>(p0 + k);
    const V a = ld_state<CG>(p1 + (size_t)y * half + jr), b = ld_state<CG>(p1 + (size_t)y * half + jl);
    const V d = ld_state<CG>(p1 + (size_t)yd * half + j), f = ld_state<CG>(p1 + (size_t)yu * half + j);
    const double hx = (double)a.x + b.x + d.x + f.x, hy = (double)a.y + b.y + d.y + f.y;
    e -= (double)s.x * hx + (double)s.y * hy;
    const V s1 = ld_state<CG>(p1 + k);
    mx += (double)s.x + (double)s1.x;
    my += (double)s.y + (double)s1.y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, off);
    mx += __shfl_xor_sync(0xffffffffu, mx, off);
    my += __shfl_xor_sync(0xffffffffu, my, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out3[0], e);
    atomicAdd(&out3[1], mx);
    atomicAdd(&out3[2], my);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_xy_measure(const typename Vec<T>::type* __restrict__ u,
                                                    int L, double* __restrict__ out3, FastDiv fh) {
  xy_measure_part<T, false>(u, L, out3, fh);
}

// Persistent form for small lattices: n sweeps (from sweep t0) in one launch,
// a barrier after each half sweep and each measurement.  PM = kOneCTA: one
// CTA, __syncthreads(), state through L1; kCluster: one thread-block cluster,
// the hardware cluster barrier (release / acquire), state through L2;
// kGrid: a cooperative grid (every CTA co-resident), the bounded grid barrier,
// state through L2.  Records go to ring slots rec0, rec0 + 1, ...; each slot is
// zeroed by CTA 0 in the half sweep before it is filled.
enum PersistMode { kOneCTA = 0, kCluster = 1, kGrid = 2 };

template <int PM>
__device__ __forceinline__ bool persist_sync(GridCtl* ctl, long long limit) {
  if (PM == kGrid) return grid_sync_bounded(ctl, limit);
  if (PM == kCluster) cooperative_groups::this_cluster().sync();
  else __syncthreads();
  return true;
}

template <typename T, int PM>
__global__ void __launch_bounds__(PM == kGrid ? 256 : 1024) k_xy_persist(typename Vec<T>::type* __restrict__ u, int L,
                                                    T beta, RngParams rng, uint32_t t0, int n, int m,
                                                    double* __restrict__ rec, long long rec0,
                                                    long long rec_cap,
                                                    unsigned long long* __restrict__ accepted,
                                                    GridCtl* ctl, long long limit, FastDiv fh) {
  using V = typename Vec<T>::type;
  const int half = L / 2;
  const uint32_t nk = (uint32_t)L * (uint32_t)half;
  unsigned int acc = 0;
  long long ri = rec0;
  for (int s = 0; s < n; ++s) {
    const uint32_t t = t0 + (uint32_t)s;
    const bool meas = m > 0 && ((long long)t + 1) % m == 0;
    double* slot = rec + 3 * (ri % rec_cap);
    bool ok = true;
    for (int c = 0; c < 2 && ok; ++c) {
      V* own = u + (size_t)c * L * half;
      const V* oth = u + (size_t)(1 - c) * L * half;
      for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; 2 * b < nk; b += gridDim.x * blockDim.x)
        acc += xy_pair<T, PM != kOneCTA>(own, oth, L, nk, b, c, t, beta, rng, fh);
      if (meas && c == 1 && blockIdx.x == 0 && threadIdx.x == 0) slot[0] = slot[1] = slot[2] = 0.0;
      ok = persist_sync<PM>(ctl, limit);
    }
    if (ok && meas) {
      xy_measure_part<T, PM != kOneCTA>(u, L, slot, fh);
      ++ri;
      ok = persist_sync<PM>(ctl, limit);
    }
    if (!ok) break;
  }
  add_accepted(accepted, acc);
}

// Self-test of the persistent kernels' barrier: CTA 0 never arrives, so every
// other CTA must give up after `limit` cycles and record the time-out.
__global__ void k_grid_barrier_selftest(GridCtl* ctl, long long limit) {
  if (blockIdx.x == 0) return;
  grid_sync_bounded(ctl, limit);
}

template <typename T>
__global__ void k_xy_to_host_layout(const typename Vec<T>::type* __restrict__ u, int L,
                                    double* __restrict__ out, int to_dev) {
  // to_dev = 0: planes -> [L][L][2] double; 1: the reverse (out is the source)
  using V = typename Vec<T>::type;
  const long long N = (long long)L * L;
  const int half = L / 2;
  V* uu = const_cast<V*>(u);
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(n / L), x = (int)(n - (n / L) * L);
    const size_t idx = (size_t)((x + y) & 1) * L * half + (size_t)y * half + (x >> 1);
    if (to_dev) {
      V v;
      v.x = (T)out[2 * n];
      v.y = (T)out[2 * n + 1];
      uu[idx] = v;
    } else {
      out[2 * n] = (double)u[idx].x;
      out[2 * n + 1] = (double)u[idx].y;
    }
  }
}

int xfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

#define XTRY(expr)                                                                        \
  do {                                                                                    \
    cudaError_t e__ = (expr);                                                             \
    if (e__ != cudaSuccess) return xfail(ISING_ECUDA, "%s: %s", #expr, cudaGetErrorString(e__)); \
  } while (0)

int grid_of(long long items) {
  long long g = (items + 255) / 256;
  return (int)std::max(1LL, std::min(g, 152LL * 32));
}

}  // namespace
}  // namespace ising

using namespace ising;

struct ising_xy {
  int L = 0, precision = 64;
  int mode = 0;                      // 0 auto, 1 one launch per half sweep, 2 persistent
  GridCtl* ctl = nullptr;            // persistent-kernel barrier and status
  int64_t launches = 0;
  double beta = 0;
  uint64_t seed = 0;
  int64_t sweep = 0;
  cudaStream_t stream = nullptr;
  void* u = nullptr;  // two colour planes of vectors
  double* rec = nullptr;  // ring [65536][3]
  int64_t rec_count = 0;
  unsigned long long* accepted = nullptr;
  double* host_scratch = nullptr;
};

namespace {
constexpr int64_t kXYRec = 65536;

// Largest L for which the automatic mode runs the persistent kernel.
constexpr int kXYPersistMaxL = 256;
constexpr long long kXYSpinLimit = 4000000000LL;  // ~2 s of SM clock per barrier

template <typename T>
cudaError_t xy_persist_t(ising_xy* x, int n, int m) {
  using V = typename Vec<T>::type;
  const RngParams rng = make_rng(x->seed, 0, 0, 0);
  const long long pairs = ((long long)x->L * (x->L / 2) + 1) / 2;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e) return e;
  // FP32: one CTA up to 256 site pairs, one cluster of 8 CTAs up to 8192;
  // FP64, which runs at a small fraction of the FP32 rate on this part: one CTA
  // only up to 32 pairs.  Beyond, a cooperative grid spreading the pairs over
  // the SMs (32 threads per CTA in FP64, 64 in FP32).
  const bool fp64 = sizeof(T) == 8;
  const int pm = pairs <= (fp64 ? 32 : 256) ? kOneCTA : (!fp64 && pairs <= 8192 ? kCluster : kGrid);
  int threads;
  long long grid;
  const void* fn;
  if (pm == kOneCTA) {
    threads = (int)(((pairs + 31) / 32) * 32);
    grid = 1;
    fn = (const void*)k_xy_persist<T, kOneCTA>;
  } else if (pm == kCluster) {
    threads = (int)std::min<long long>(1024, ((pairs + 8 * 32 - 1) / (8 * 32)) * 32);
    grid = 8;
    fn = (const void*)k_xy_persist<T, kCluster>;
  } else {
    threads = fp64 ? 32 : 64;
    grid = std::max(1LL, std::min((pairs + threads - 1) / threads, (long long)sms));
    fn = (const void*)k_xy_persist<T, kGrid>;
    e = cudaMemsetAsync(&x->ctl->count, 0, sizeof(unsigned int), x->stream);
    if (e) return e;
  }
  V* u = (V*)x->u;
  int L = x->L;
  T beta = (T)x->beta;
  uint32_t t0 = (uint32_t)x->sweep;
  long long rec0 = x->rec_count, cap = kXYRec, limit = kXYSpinLimit;
  double* rec = x->rec;
  unsigned long long* acc = x->accepted;
  GridCtl* ctl = x->ctl;
  RngParams r = rng;
  FastDiv fh = make_fastdiv((uint32_t)(x->L / 2));
  void* args[] = {&u, &L, &beta, &r, &t0, &n, &m, &rec, &rec0, &cap, &acc, &ctl, &limit, &fh};
  if (pm == kOneCTA) {
    e = cudaLaunchKernel(fn, dim3(1), dim3(threads), args, 0, x->stream);
  } else if (pm == kCluster) {
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
    e = cudaLaunchKernelExC(&cfg, fn, args);
  } else {
    e = cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(threads), args, 0, x->stream);
  }
  if (e) return e;
  ++x->launches;
  if (m > 0) {
    for (int s = 0; s < n; ++s)
      if (((int64_t)x->sweep + s + 1) % m == 0) ++x->rec_count;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t xy_sweep_t(ising_xy* x, int n, int m) {
  const bool persist = x->mode == 2 || (x->mode == 0 && x->L <= kXYPersistMaxL);
  if (persist) return n > 0 ? xy_persist_t<T>(x, n, m) : cudaSuccess;
  const RngParams rng = make_rng(x->seed, 0, 0, 0);
  const long long blocks = ((long long)x->L * (x->L / 2) + 1) / 2;
  using V = typename Vec<T>::type;
  for (int s = 0; s < n; ++s) {
    const uint32_t t = (uint32_t)(x->sweep + s);
    for (int c = 0; c < 2; ++c) {
      k_xy_half<T><<<grid_of(blocks), 256, 0, x->stream>>>((V*)x->u, x->L, c, t, (T)x->beta, rng,
                                                            make_fastdiv((uint32_t)(x->L / 2)), x->accepted);
      cudaError_t e = cudaGetLastError();
      if (e) return e;
      ++x->launches;
    }
    if (m > 0 && ((int64_t)t + 1) % m == 0) {
      double* slot = x->rec + 3 * (x->rec_count % kXYRec);
      cudaError_t e = cudaMemsetAsync(slot, 0, 3 * sizeof(double), x->stream);
      if (e) return e;
      k_xy_measure<T><<<grid_of((long long)x->L * (x->L / 2)), 256, 0, x->stream>>>(
          (const V*)x->u, x->L, slot, make_fastdiv((uint32_t)(x->L / 2)));
      e = cudaGetLastError();
      if (e) return e;
      ++x->launches;
      ++x->rec_count;
    }
  }
  return cudaSuccess;
}
}  // namespace

extern "C" {

int ising_xy_create(ising_xy** out, int L, double beta, int precision, void* stream) {
  if (!out) return xfail(ISING_EINVAL, "null output pointer");
  *out = nullptr;
  if (L < 2 || L > 32768 || (L & 1)) return xfail(ISING_EINVAL, "L must be even and in [2, 32768]");
  if (!std::isfinite(beta) || beta <= 0) return xfail(ISING_EINVAL, "beta must be finite and > 0");
  if (precision != 32 && precision != 64) return xfail(ISING_EINVAL, "precision must be 32 or 64");
  ising_xy* x = new (std::nothrow) ising_xy();
  if (!x) return xfail(ISING_ENOMEM, "host allocation failed");
  x->L = L;
  x->beta = beta;
  x->precision = precision;
  x->stream = (cudaStream_t)stream;
  const size_t bytes = (size_t)L * L * (precision == 64 ? 16 : 8);
  cudaError_t e = cudaMalloc(&x->u, bytes);
  if (!e) e = cudaMalloc((void**)&x->rec, kXYRec * 3 * sizeof(double));
  if (!e) e = cudaMalloc((void**)&x->accepted, sizeof(unsigned long long));
  if (!e) e = cudaMemset(x->accepted, 0, sizeof(unsigned long long));
  if (!e) e = cudaMalloc((void**)&x->ctl, sizeof(GridCtl));
  if (!e) e = cudaMemset(x->ctl, 0, sizeof(GridCtl));
  if (e) {
    cudaGetLastError();
    cudaFree(x->u);
    cudaFree(x->rec);
    cudaFree(x->accepted);
    cudaFree(x->ctl);
    delete x;
    return xfail(ISING_ENOMEM, "XY allocation: %s", cudaGetErrorString(e));
  }
  *out = x;
  return ising_xy_seed(x, 0);
}

int ising_xy_seed(ising_xy* x, uint64_t seed) {
  if (!x) return xfail(ISING_EINVAL, "null context");
  x->seed = seed;
  x->sweep = 0;
  x->rec_count = 0;
  const RngParams rng = make_rng(seed, 0, 0, 0);
  const long long N = (long long)x->L * x->L;
  if (x->precision == 64)
    k_xy_init<double><<<grid_of(N), 256, 0, x->stream>>>((double2*)x->u, x->L, rng);
  else
    k_xy_init<float><<<grid_of(N), 256, 0, x->stream>>>((float2*)x->u, x->L, rng);
  XTRY(cudaGetLastError());
  XTRY(cudaMemsetAsync(x->accepted, 0, sizeof(unsigned long long), x->stream));
  XTRY(cudaMemsetAsync(x->ctl, 0, sizeof(GridCtl), x->stream));
  set_last_error("");
  return ISING_OK;
}

int ising_xy_sweep(ising_xy* x, int n_sweeps, int measure_every) {
  if (!x) return xfail(ISING_EINVAL, "null context");
  if (n_sweeps < 0 || measure_every < 0) return xfail(ISING_EINVAL, "negative count");
  if (x->sweep + n_sweeps >= ((int64_t)1 << 32)) return xfail(ISING_EINVAL, "sweep counter overflow");
  NvtxRange nvtx("ising_xy_sweep");
  XTRY(x->precision == 64 ? xy_sweep_t<double>(x, n_sweeps, measure_every)
                          : xy_sweep_t<float>(x, n_sweeps, measure_every));
  x->sweep += n_sweeps;
  set_last_error("");
  return ISING_OK;
}

// After a synchronising call: ETIMEOUT if a persistent kernel's grid barrier
// gave up (the flag stays set until the next seed).
static int xy_status(ising_xy* x) {
  int st = 0;
  XTRY(cudaMemcpy(&st, &x->ctl->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) return xfail(ISING_ETIMEOUT, "grid barrier timed out in the persistent XY kernel");
  return ISING_OK;
}

int ising_selftest_grid_barrier(double timeout_s, int* timed_out) {
  if (!timed_out || !(timeout_s > 0) || timeout_s > 10) return xfail(ISING_EINVAL, "bad arguments");
  GridCtl* ctl = nullptr;
  XTRY(cudaMalloc((void**)&ctl, sizeof(GridCtl)));
  cudaError_t e = cudaMemset(ctl, 0, sizeof(GridCtl));
  if (!e) {
    GridCtl* c = ctl;
    long long limit = (long long)(timeout_s * 2.1e9);  // SM clock cycles (<= 2.1 GHz)
    void* args[] = {&c, &limit};
    e = cudaLaunchCooperativeKernel((const void*)k_grid_barrier_selftest, dim3(4), dim3(32), args, 0, 0);
  }
  if (!e) e = cudaDeviceSynchronize();
  GridCtl h{};
  if (!e) e = cudaMemcpy(&h, ctl, sizeof(GridCtl), cudaMemcpyDeviceToHost);
  cudaFree(ctl);
  if (e) return xfail(ISING_ECUDA, "barrier self-test: %s", cudaGetErrorString(e));
  *timed_out = h.status;
  set_last_error("");
  return ISING_OK;
}

int ising_xy_set_mode(ising_xy* x, int mode) {
  if (!x) return xfail(ISING_EINVAL, "null context");
  if (mode < 0 || mode > 2) return xfail(ISING_EINVAL, "mode must be 0 (auto), 1 (per half sweep) or 2 (persistent)");
  x->mode = mode;
  set_last_error("");
  return ISING_OK;
}

int ising_xy_launch_count(ising_xy* x, int64_t* count) {
  if (!x || !count) return xfail(ISING_EINVAL, "null argument");
  *count = x->launches;
  return ISING_OK;
}

int ising_xy_series(ising_xy* x, double* E, double* Mx, double* My, int n) {
  if (!x) return xfail(ISING_EINVAL, "null context");
  if (n < 0 || n > std::min<int64_t>(x->rec_count, kXYRec)) return xfail(ISING_EINVAL, "n exceeds records");
  std::vector<double> h((size_t)3 * kXYRec);
  XTRY(cudaMemcpyAsync(h.data(), x->rec, h.size() * 8, cudaMemcpyDeviceToHost, x->stream));
  XTRY(cudaStreamSynchronize(x->stream));
  if (int st = xy_status(x)) return st;
  for (int i = 0; i < n; ++i) {
    const int64_t slot = (x->rec_count - n + i) % kXYRec;
    if (E) E[i] = h[3 * slot];
    if (Mx) Mx[i] = h[3 * slot + 1];
    if (My) My[i] = h[3 * slot + 2];
  }
  set_last_error("");
  return ISING_OK;
}

int ising_xy_get_spins(ising_xy* x, double* host_uv) {
  if (!x || !host_uv) return xfail(ISING_EINVAL, "null argument");
  const long long N = (long long)x->L * x->L;
  double* d = nullptr;
  XTRY(cudaMalloc((void**)&d, N * 2 * sizeof(double)));
  if (x->precision == 64)
    k_xy_to_host_layout<double><<<grid_of(N), 256, 0, x->stream>>>((const double2*)x->u, x->L, d, 0);
  else
    k_xy_to_host_layout<float><<<grid_of(N), 256, 0, x->stream>>>((const float2*)x->u, x->L, d, 0);
  cudaError_t e = cudaGetLastError();
  if (!e) e = cudaMemcpyAsync(host_uv, d, N * 2 * sizeof(double), cudaMemcpyDeviceToHost, x->stream);
  if (!e) e = cudaStreamSynchronize(x->stream);
  cudaFree(d);
  if (e) return xfail(ISING_ECUDA, "get spins: %s", cudaGetErrorString(e));
  if (int st = xy_status(x)) return st;
  set_last_error("");
  return ISING_OK;
}

int ising_xy_set_spins(ising_xy* x, const double* host_uv) {
  if (!x || !host_uv) return xfail(ISING_EINVAL, "null argument");
  const long long N = (long long)x->L * x->L;
  double* d = nullptr;
  XTRY(cudaMalloc((void**)&d, N * 2 * sizeof(double)));
  cudaError_t e = cudaMemcpyAsync(d, host_uv, N * 2 * sizeof(double), cudaMemcpyHostToDevice, x->stream);
  if (!e) {
    if (x->precision == 64)
      k_xy_to_host_layout<double><<<grid_of(N), 256, 0, x->stream>>>((const double2*)x->u, x->L, d, 1);
    else
      k_xy_to_host_layout<float><<<grid_of(N), 256, 0, x->stream>>>((const float2*)x->u, x->L, d, 1);
    e = cudaGetLastError();
  }
  if (!e) e = cudaStreamSynchronize(x->stream);
  cudaFree(d);
  if (e) return xfail(ISING_ECUDA, "set spins: %s", cudaGetErrorString(e));
  set_last_error("");
  return ISING_OK;
}

int ising_xy_accepted(ising_xy* x, int64_t* accepted) {
  if (!x || !accepted) return xfail(ISING_EINVAL, "null argument");
  unsigned long long h = 0;
  XTRY(cudaMemcpyAsync(&h, x->accepted, 8, cudaMemcpyDeviceToHost, x->stream));
  XTRY(cudaStreamSynchronize(x->stream));
  if (int st = xy_status(x)) return st;
  *accepted = (int64_t)h;
  set_last_error("");
  return ISING_OK;
}

int ising_xy_destroy(ising_xy* x) {
  if (!x) return ISING_OK;
  cudaStreamSynchronize(x->stream);
  cudaFree(x->u);
  cudaFree(x->rec);
  cudaFree(x->accepted);
  cudaFree(x->ctl);
  delete x;
  return ISING_OK;
}

}  // extern "C"
