// Quadripartite Metropolis sweep of the Ising model on lattices with a
// four-site unit cell (arXiv 2402.06415, Results "optimising the partition",
// Fig. 5b/5d; Supplementary Fig. S4a-c): the four sites of a cell belong to four
// sublattices, none of which has an internal bond, so a sweep is four parallel
// steps (sublattice 0, 1, 2, 3).
//
// Lattices on Lc x Lc periodic cells:
//   SQUARE: square lattice of side 2 Lc, site (2X + i, 2Y + j) in sublattice
//     q = i + 2j; J1 on nearest neighbours, J2 on the diagonal (next-nearest)
//     neighbours.
//   SQOCT: square-octagon (4.8.8) lattice; cell sites A, B, C, D (q = 0..3)
//     form a J1 square A-B-C-D-A; J2 octagon bonds B(X,Y)-D(X+1,Y), A(X,Y)-C(X,Y+1).
// Flip of a site with a1 / a2 antiparallel J1 / J2 neighbours (z1, z2 of them):
// dE = 2 J1 (z1 - 2 a1) + 2 J2 (z2 - 2 a2); flip iff dE <= 0 or u < T(a1, a2) =
// floor(exp(-beta dE) 2^32), computed once on the host.
//
// Layout: one bit plane per sublattice, [4][Lc][Wq] u32 words, Wq = ceil(Lc/32),
// bit b of word w of row Y = cell X = 32 w + b (1 = spin up); padding bits 0.
// One thread per word: neighbour words of the other three planes (a one-bit
// funnel shift for the x-offset cells), bit-sliced counts of antiparallel J1 and
// J2 neighbours, class masks, then a lazy bit-serial compare u < T against the
// per-lane threshold, MSB first, generating Philox planes only while lanes are
// undecided.  Uniform of lane b: u = sum_k bit_b(P_k) 2^(31-k), P_{4m+k} = word
// k of Philox(g, t, replica, QUAD_MET << 16 | q << 8 | m), g = Y Wq + w.
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

constexpr uint32_t kTagQuadInit = 12, kTagQuadMet = 13;
constexpr int kMaxClasses = 25;

struct QuadGeom {
  int Lc, Wq, nlast;  // nlast: valid bits of a row's last word (1..32)
  FastDiv fw;         // division by Wq
};

// Decision table of one (lattice, beta, J1, J2): class c = a1 (z2 + 1) + a2.
struct QuadTable {
  uint32_t always;            // classes with dE <= 0
  int n_vals;                 // distinct thresholds of the other classes
  uint32_t val[kMaxClasses];  // the thresholds
  uint32_t cls[kMaxClasses];  // bitset of the classes holding val[d]
  uint32_t lm[kMaxClasses][32];  // all ones iff bit 31 - k of val[d] is set
};

struct Count3 {  // bit-sliced 3-bit counter per lane (counts 0..4)
  uint32_t c0 = 0, c1 = 0, c2 = 0;
  __device__ __forceinline__ void add(uint32_t x) {
    const uint32_t k0 = c0 & x;
    c0 ^= x;
    const uint32_t k1 = c1 & k0;
    c1 ^= k0;
    c2 |= k1;
  }
  __device__ __forceinline__ uint32_t eq(int v) const {
    return ((v & 1) ? c0 : ~c0) & ((v & 2) ? c1 : ~c1) & ((v & 4) ? c2 : ~c2);
  }
};

// Neighbour-plane loads: through the read-only path from global memory (G), or
// plain loads from shared memory in the persistent single-CTA kernel.
template <bool G>
__device__ __forceinline__ uint32_t ldw(const uint32_t* p) {
  if (G) return __ldg(p);
  return *p;
}

// Word whose bit b holds the spin of cell X = 32 w + b + DX (periodic in X) of a row.
template <int DX, bool G = true>
__device__ __forceinline__ uint32_t xword(const uint32_t* __restrict__ row, const QuadGeom& g, int w) {
  const uint32_t cur = ldw<G>(row + w);
  if (DX == 0) return cur;
  if (DX > 0) {
    const bool last = w == g.Wq - 1;
    const uint32_t nxt = ldw<G>(row + (last ? 0 : w + 1));
    const int valid = last ? g.nlast : 32;
    return (cur >> 1) | ((nxt & 1u) << (valid - 1));
  }
  const bool first = w == 0;
  const uint32_t prv = ldw<G>(row + (first ? g.Wq - 1 : w - 1));
  const int pvalid = first ? g.nlast : 32;
  return (cur << 1) | ((prv >> (pvalid - 1)) & 1u);
}

template <bool G>
__device__ __forceinline__ uint32_t xword_dir(const uint32_t* row, const QuadGeom& g, int w, int dx) {
  return dx > 0 ? xword<1, G>(row, g, w) : xword<-1, G>(row, g, w);
}

// Antiparallel J1 / J2 neighbour counts of the 32 sites of word (q, Y, w).
template <int LAT, bool G = true>
__device__ __forceinline__ void count_anti(const uint32_t* __restrict__ planes, const QuadGeom& g,
                                           int q, int Y, int w, uint32_t me, Count3& n1, Count3& n2) {
  const size_t plane = (size_t)g.Lc * g.Wq;
  const int Yp = Y + 1 == g.Lc ? 0 : Y + 1, Ym = Y == 0 ? g.Lc - 1 : Y - 1;
  if (LAT == ISING_QUAD_SQUARE) {
    const int sx = (q & 1) ? 1 : -1;
    const int Yn = (q & 2) ? Yp : Ym;
    const uint32_t* rx = planes + (size_t)(q ^ 1) * plane + (size_t)Y * g.Wq;
    const uint32_t* ry0 = planes + (size_t)(q ^ 2) * plane + (size_t)Y * g.Wq;
    const uint32_t* ry1 = planes + (size_t)(q ^ 2) * plane + (size_t)Yn * g.Wq;
    const uint32_t* rd0 = planes + (size_t)(q ^ 3) * plane + (size_t)Y * g.Wq;
    const uint32_t* rd1 = planes + (size_t)(q ^ 3) * plane + (size_t)Yn * g.Wq;
    n1.add(me ^ xword<0, G>(rx, g, w));
    n1.add(me ^ xword_dir<G>(rx, g, w, sx));
    n1.add(me ^ xword<0, G>(ry0, g, w));
    n1.add(me ^ xword<0, G>(ry1, g, w));
    n2.add(me ^ xword<0, G>(rd0, g, w));
    n2.add(me ^ xword_dir<G>(rd0, g, w, sx));
    n2.add(me ^ xword<0, G>(rd1, g, w));
    n2.add(me ^ xword_dir<G>(rd1, g, w, sx));
  } else {
    const int nxt = (q + 1) & 3, prv = (q + 3) & 3;
    n1.add(me ^ xword<0, G>(planes + (size_t)nxt * plane + (size_t)Y * g.Wq, g, w));
    n1.add(me ^ xword<0, G>(planes + (size_t)prv * plane + (size_t)Y * g.Wq, g, w));
    uint32_t o;
    if (q == 0) o = xword<0, G>(planes + 2 * plane + (size_t)Yp * g.Wq, g, w);
    else if (q == 1) o = xword<1, G>(planes + 3 * plane + (size_t)Y * g.Wq, g, w);
    else if (q == 2) o = xword<0, G>(planes + 0 * plane + (size_t)Ym * g.Wq, g, w);
    else o = xword<-1, G>(planes + 1 * plane + (size_t)Y * g.Wq, g, w);
    n2.add(me ^ o);
  }
}

__device__ __forceinline__ uint32_t valid_bits(const QuadGeom& g, int w) {
  return (w == g.Wq - 1 && g.nlast < 32) ? ((1u << g.nlast) - 1u) : 0xffffffffu;
}

// Metropolis trials of the 32 sites of word i = Y Wq + w of sublattice q.
// All 32 lanes of the warp call it together (warp vote); lanes past the end pass
// active = false (any in-range i) and change nothing.
template <int LAT, int NV, bool G>
__device__ __forceinline__ void quad_word(uint32_t* __restrict__ planes, const QuadGeom& g, int q,
                                          long long i, bool active, uint32_t t, const RngParams& rng,
                                          const QuadTable& tab) {
  constexpr int Z2 = LAT == ISING_QUAD_SQUARE ? 4 : 1;
  constexpr int Z1 = LAT == ISING_QUAD_SQUARE ? 4 : 2;
  if (!active) i = 0;
  const int Y = (int)fdiv((uint32_t)i, g.fw), w = (int)((uint32_t)i - (uint32_t)Y * (uint32_t)g.Wq);
  uint32_t* own = planes + (size_t)q * g.Lc * g.Wq + i;
  const uint32_t me = *own;
  const uint32_t valid = active ? valid_bits(g, w) : 0u;
  Count3 n1, n2;
  count_anti<LAT, G>(planes, g, q, Y, w, me, n1, n2);
  uint32_t e2[Z2 + 1];
#pragma unroll
  for (int a2 = 0; a2 <= Z2; ++a2) e2[a2] = n2.eq(a2);
  uint32_t always = 0, vm[NV];
#pragma unroll
  for (int d = 0; d < NV; ++d) vm[d] = 0;
#pragma unroll
  for (int a1 = 0; a1 <= Z1; ++a1) {
    const uint32_t e1 = n1.eq(a1);
#pragma unroll
    for (int a2 = 0; a2 <= Z2; ++a2) {
      const int c = a1 * (Z2 + 1) + a2;
      const uint32_t cm = e1 & e2[a2];
      always |= cm & (0u - ((tab.always >> c) & 1u));
#pragma unroll
      for (int d = 0; d < NV; ++d) vm[d] |= cm & (0u - ((tab.cls[d] >> c) & 1u));
    }
  }
  uint32_t und = ~always & valid, lt = 0;
  const uint32_t g_idx = (uint32_t)i;
  // planes block by block while any lane of the warp is undecided; the level is
  // a compile-time index, so each threshold-bit mask is a constant operand
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    if (!__any_sync(0xffffffffu, und != 0u)) break;
    const uint4 r = philox10_rk(make_uint4(g_idx, t, rng.replica, (kTagQuadMet << 16) | ((uint32_t)q << 8) | (uint32_t)m),
                                rng.rk0, rng.rk1);
    const uint32_t pw[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int lvl = 4 * m + k;
      uint32_t tm = 0;
#pragma unroll
      for (int d = 0; d < NV; ++d) tm |= vm[d] & tab.lm[d][lvl];
      lt |= und & ~pw[k] & tm;
      und &= ~(pw[k] ^ tm);
    }
  }
  const uint32_t flip = (always | lt) & valid;
  if (active && flip) *own = me ^ flip;
}

template <int LAT, int NV>
__global__ void __launch_bounds__(256) k_quad_quarter(uint32_t* __restrict__ planes, QuadGeom g, int q,
                                                      uint32_t t, RngParams rng, QuadTable tab) {
  const long long words = (long long)g.Lc * g.Wq;
  const int lane = threadIdx.x & 31;
  for (long long base = (blockIdx.x * (long long)blockDim.x + threadIdx.x) - lane; base < words;
       base += (long long)gridDim.x * blockDim.x)
    quad_word<LAT, NV, true>(planes, g, q, base + lane, base + lane < words, t, rng, tab);
}

__global__ void k_quad_init(uint32_t* __restrict__ planes, QuadGeom g, RngParams rng) {
  const long long words = (long long)g.Lc * g.Wq;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 4 * words;
       i += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(i / words);
    const long long gi = i - (long long)q * words;
    const int w = (int)(gi % g.Wq);
    const uint4 r = philox10_rk(make_uint4((uint32_t)gi, 0u, rng.replica, (kTagQuadInit << 16) | ((uint32_t)q << 8)),
                                rng.rk0, rng.rk1);
    planes[i] = r.x & valid_bits(g, w);
  }
}

// Bond sums of word i of the 4 Lc Wq words: (2 B1, 2 B2, M) contributions (each
// bond is seen from both ends).
template <int LAT, bool G>
__device__ __forceinline__ void quad_measure_word(const uint32_t* __restrict__ planes, const QuadGeom& g,
                                                  long long i, long long& b1, long long& b2, long long& m) {
  constexpr int Z1 = LAT == ISING_QUAD_SQUARE ? 4 : 2;
  constexpr int Z2 = LAT == ISING_QUAD_SQUARE ? 4 : 1;
  const long long words = (long long)g.Lc * g.Wq;
  const int q = (int)(i / words);
  const long long gi = i - (long long)q * words;
  const int Y = (int)fdiv((uint32_t)gi, g.fw), w = (int)((uint32_t)gi - (uint32_t)Y * (uint32_t)g.Wq);
  const uint32_t v = valid_bits(g, w);
  const uint32_t me = planes[i];
  Count3 n1, n2;
  count_anti<LAT, G>(planes, g, q, Y, w, me, n1, n2);
  const int nv = __popc(v);
  const int anti1 = __popc(n1.c0 & v) + 2 * __popc(n1.c1 & v) + 4 * __popc(n1.c2 & v);
  const int anti2 = __popc(n2.c0 & v) + 2 * __popc(n2.c1 & v) + 4 * __popc(n2.c2 & v);
  b1 += (long long)Z1 * nv - 2LL * anti1;
  b2 += (long long)Z2 * nv - 2LL * anti2;
  m += 2LL * __popc(me & v) - nv;
}

// rec[0] += 2 B1, rec[1] += 2 B2, rec[2] += M.
template <int LAT>
__global__ void __launch_bounds__(256) k_quad_measure(const uint32_t* __restrict__ planes, QuadGeom g,
                                                      unsigned long long* __restrict__ rec) {
  const long long words = (long long)g.Lc * g.Wq;
  long long b1 = 0, b2 = 0, m = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 4 * words;
       i += (long long)gridDim.x * blockDim.x)
    quad_measure_word<LAT, true>(planes, g, i, b1, b2, m);
  const unsigned long long s1 = warp_sum_u64((unsigned long long)b1);
  const unsigned long long s2 = warp_sum_u64((unsigned long long)b2);
  const unsigned long long s3 = warp_sum_u64((unsigned long long)m);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&rec[0], s1);
    atomicAdd(&rec[1], s2);
    atomicAdd(&rec[2], s3);
  }
}

// Small lattices (the paper's N = 16 ... 4096 and up to 256^2 cells): the whole
// lattice in shared memory, one CTA, n sweeps in one launch with __syncthreads()
// between quarter sweeps; records (2 B1, 2 B2, M) written to ring slots rec0, ...
template <int LAT, int NV>
__global__ void __launch_bounds__(1024) k_quad_persist(uint32_t* __restrict__ planes, QuadGeom g, uint32_t t0,
                                                       int n, int meas_every, RngParams rng, QuadTable tab,
                                                       unsigned long long* __restrict__ rec, long long rec0,
                                                       long long rec_cap) {
  extern __shared__ uint32_t sp[];
  __shared__ long long red[3][32];
  const long long words = (long long)g.Lc * g.Wq;
  for (long long i = threadIdx.x; i < 4 * words; i += blockDim.x) sp[i] = planes[i];
  __syncthreads();
  long long ri = rec0;
  for (int s = 0; s < n; ++s) {
    const uint32_t t = t0 + (uint32_t)s;
    for (int q = 0; q < 4; ++q) {
      for (long long base = threadIdx.x & ~31; base < words; base += blockDim.x)
        quad_word<LAT, NV, false>(sp, g, q, base + (threadIdx.x & 31), base + (threadIdx.x & 31) < words, t,
                                  rng, tab);
      __syncthreads();
    }
    if (meas_every > 0 && ((long long)t + 1) % meas_every == 0) {
      long long b1 = 0, b2 = 0, m = 0;
      for (long long i = threadIdx.x; i < 4 * words; i += blockDim.x) quad_measure_word<LAT, false>(sp, g, i, b1, b2, m);
      b1 = (long long)warp_sum_u64((unsigned long long)b1);
      b2 = (long long)warp_sum_u64((unsigned long long)b2);
      m = (long long)warp_sum_u64((unsigned long long)m);
      const int wid = threadIdx.x >> 5;
      if ((threadIdx.x & 31) == 0) {
        red[0][wid] = b1;
        red[1][wid] = b2;
        red[2][wid] = m;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        long long a = 0, b = 0, c = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
          a += red[0][k];
          b += red[1][k];
          c += red[2][k];
        }
        unsigned long long* slot = rec + 3 * (ri % rec_cap);
        slot[0] = (unsigned long long)a;
        slot[1] = (unsigned long long)b;
        slot[2] = (unsigned long long)c;
      }
      ++ri;
      __syncthreads();
    }
  }
  for (long long i = threadIdx.x; i < 4 * words; i += blockDim.x) planes[i] = sp[i];
}

int qfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

#define QTRY(expr)                                                                        \
  do {                                                                                    \
    cudaError_t e__ = (expr);                                                             \
    if (e__ != cudaSuccess) return qfail(ISING_ECUDA, "%s: %s", #expr, cudaGetErrorString(e__)); \
  } while (0)

int qgrid(long long items) {
  long long g = (items + 255) / 256;
  return (int)std::max(1LL, std::min(g, 152LL * 32));
}

// Classes and thresholds for one (lattice, beta, J1, J2).  The products are
// kept in volatile temporaries so that no compiler contracts them into a fused
// multiply-add: the table must round exactly as written.
bool build_table(int lattice, double beta, double J1, double J2, QuadTable* tab) {
  const int z1 = lattice == ISING_QUAD_SQUARE ? 4 : 2, z2 = lattice == ISING_QUAD_SQUARE ? 4 : 1;
  QuadTable t{};
  for (int a1 = 0; a1 <= z1; ++a1)
    for (int a2 = 0; a2 <= z2; ++a2) {
      const int c = a1 * (z2 + 1) + a2;
      volatile double p1 = 2.0 * J1 * (double)(z1 - 2 * a1);
      volatile double p2 = 2.0 * J2 * (double)(z2 - 2 * a2);
      const double dE = p1 + p2;
      if (dE <= 0.0) {
        t.always |= 1u << c;
        continue;
      }
      volatile double x = -beta * dE;
      const double f = std::floor(std::exp(x) * 4294967296.0);
      const uint32_t thr = f >= 4294967295.0 ? 0xffffffffu : (uint32_t)f;
      int d = 0;
      while (d < t.n_vals && t.val[d] != thr) ++d;
      if (d == t.n_vals) {
        if (t.n_vals == kMaxClasses) return false;
        t.val[t.n_vals++] = thr;
      }
      t.cls[d] |= 1u << c;
    }
  for (int d = 0; d < t.n_vals; ++d)
    for (int k = 0; k < 32; ++k) t.lm[d][k] = ((t.val[d] >> (31 - k)) & 1u) ? 0xffffffffu : 0u;
  *tab = t;
  return true;
}

}  // namespace
}  // namespace ising

using namespace ising;

struct ising_quad {
  int lattice = 0, Lc = 0;
  QuadGeom geom{};
  double beta = 0, J1 = 1, J2 = 0;
  QuadTable tab{};
  uint64_t seed = 0;
  uint32_t replica = 0;
  int64_t sweep = 0;
  cudaStream_t stream = nullptr;
  uint32_t* planes = nullptr;
  unsigned long long* rec = nullptr;  // ring [65536][3]
  int64_t rec_count = 0;
  int64_t launches = 0;
};

namespace {
constexpr int64_t kQuadRec = 65536;

template <int LAT, int NV>
cudaError_t launch_quarter(ising_quad* x, int q, uint32_t t, const RngParams& rng) {
  k_quad_quarter<LAT, NV><<<qgrid((long long)x->Lc * x->geom.Wq), 256, 0, x->stream>>>(
      x->planes, x->geom, q, t, rng, x->tab);
  return cudaGetLastError();
}

template <int LAT>
cudaError_t quarter_dispatch(ising_quad* x, int q, uint32_t t, const RngParams& rng) {
  const int nv = x->tab.n_vals;
  if (nv <= 2) return launch_quarter<LAT, 2>(x, q, t, rng);
  if (nv <= 8) return launch_quarter<LAT, 8>(x, q, t, rng);
  if (LAT == ISING_QUAD_SQUARE) return launch_quarter<LAT, kMaxClasses>(x, q, t, rng);
  return cudaErrorInvalidValue;  // the square-octagon lattice has at most 6 classes
}

constexpr int kQuadPersistMaxLc = 256;  // shared memory: 4 Lc ceil(Lc/32) words <= 32 KB

template <int LAT, int NV>
cudaError_t launch_persist(ising_quad* x, int n, int m, const RngParams& rng) {
  const long long words = (long long)x->Lc * x->geom.Wq;
  const int threads = (int)std::min<long long>(1024, ((words + 31) / 32) * 32);
  const size_t smem = (size_t)4 * words * sizeof(uint32_t);
  k_quad_persist<LAT, NV><<<1, threads, smem, x->stream>>>(x->planes, x->geom, (uint32_t)x->sweep, n, m, rng,
                                                           x->tab, x->rec, x->rec_count, kQuadRec);
  return cudaGetLastError();
}

template <int LAT>
cudaError_t persist_dispatch(ising_quad* x, int n, int m, const RngParams& rng) {
  const int nv = x->tab.n_vals;
  if (nv <= 2) return launch_persist<LAT, 2>(x, n, m, rng);
  if (nv <= 8) return launch_persist<LAT, 8>(x, n, m, rng);
  if (LAT == ISING_QUAD_SQUARE) return launch_persist<LAT, kMaxClasses>(x, n, m, rng);
  return cudaErrorInvalidValue;
}

cudaError_t quad_sweeps(ising_quad* x, int n, int m) {
  const RngParams rng = make_rng(x->seed, x->replica, 0, 0);
  if (x->Lc <= kQuadPersistMaxLc && n > 0) {
    cudaError_t e = x->lattice == ISING_QUAD_SQUARE ? persist_dispatch<ISING_QUAD_SQUARE>(x, n, m, rng)
                                                    : persist_dispatch<ISING_QUAD_SQOCT>(x, n, m, rng);
    if (e) return e;
    ++x->launches;
    if (m > 0)
      for (int s = 0; s < n; ++s)
        if ((x->sweep + s + 1) % m == 0) ++x->rec_count;
    return cudaSuccess;
  }
  for (int s = 0; s < n; ++s) {
    const uint32_t t = (uint32_t)(x->sweep + s);
    for (int q = 0; q < 4; ++q) {
      cudaError_t e = x->lattice == ISING_QUAD_SQUARE ? quarter_dispatch<ISING_QUAD_SQUARE>(x, q, t, rng)
                                                      : quarter_dispatch<ISING_QUAD_SQOCT>(x, q, t, rng);
      if (e) return e;
      ++x->launches;
    }
    if (m > 0 && ((int64_t)t + 1) % m == 0) {
      unsigned long long* slot = x->rec + 3 * (x->rec_count % kQuadRec);
      cudaError_t e = cudaMemsetAsync(slot, 0, 3 * sizeof(unsigned long long), x->stream);
      if (e) return e;
      const int grid = qgrid(4LL * x->Lc * x->geom.Wq);
      if (x->lattice == ISING_QUAD_SQUARE)
        k_quad_measure<ISING_QUAD_SQUARE><<<grid, 256, 0, x->stream>>>(x->planes, x->geom, slot);
      else
        k_quad_measure<ISING_QUAD_SQOCT><<<grid, 256, 0, x->stream>>>(x->planes, x->geom, slot);
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

int ising_quad_create(ising_quad** out, int lattice, int Lc, double beta, double J1, double J2,
                      void* stream) {
  if (!out) return qfail(ISING_EINVAL, "null output pointer");
  *out = nullptr;
  if (lattice != ISING_QUAD_SQUARE && lattice != ISING_QUAD_SQOCT)
    return qfail(ISING_EINVAL, "unknown lattice %d", lattice);
  if (Lc < 2 || Lc > 16384) return qfail(ISING_EINVAL, "Lc must be in [2, 16384] (got %d)", Lc);
  if (!std::isfinite(beta) || beta <= 0) return qfail(ISING_EINVAL, "beta must be finite and > 0");
  if (!std::isfinite(J1) || !std::isfinite(J2)) return qfail(ISING_EINVAL, "couplings must be finite");
  ising_quad* x = new (std::nothrow) ising_quad();
  if (!x) return qfail(ISING_ENOMEM, "host allocation failed");
  x->lattice = lattice;
  x->Lc = Lc;
  x->geom.Lc = Lc;
  x->geom.Wq = (Lc + 31) / 32;
  x->geom.nlast = Lc - 32 * (x->geom.Wq - 1);
  x->geom.fw = make_fastdiv((uint32_t)x->geom.Wq);
  x->beta = beta;
  x->J1 = J1;
  x->J2 = J2;
  x->stream = (cudaStream_t)stream;
  if (!build_table(lattice, beta, J1, J2, &x->tab)) {
    delete x;
    return qfail(ISING_EINTERNAL, "threshold table overflow");
  }
  const size_t bytes = (size_t)4 * Lc * x->geom.Wq * sizeof(uint32_t);
  cudaError_t e = cudaMalloc((void**)&x->planes, bytes);
  if (!e) e = cudaMalloc((void**)&x->rec, kQuadRec * 3 * sizeof(unsigned long long));
  if (e) {
    cudaGetLastError();
    cudaFree(x->planes);
    cudaFree(x->rec);
    delete x;
    return qfail(ISING_ENOMEM, "quad allocation: %s", cudaGetErrorString(e));
  }
  *out = x;
  return ising_quad_seed(x, 0);
}

int ising_quad_seed(ising_quad* x, uint64_t seed) {
  if (!x) return qfail(ISING_EINVAL, "null context");
  x->seed = seed;
  x->sweep = 0;
  x->rec_count = 0;
  const RngParams rng = make_rng(seed, x->replica, 0, 0);
  k_quad_init<<<qgrid(4LL * x->Lc * x->geom.Wq), 256, 0, x->stream>>>(x->planes, x->geom, rng);
  QTRY(cudaGetLastError());
  set_last_error("");
  return ISING_OK;
}

int ising_quad_set_replica(ising_quad* x, uint32_t replica) {
  if (!x) return qfail(ISING_EINVAL, "null context");
  x->replica = replica;
  return ising_quad_seed(x, x->seed);
}

int ising_quad_sweep(ising_quad* x, int n_sweeps, int measure_every) {
  if (!x) return qfail(ISING_EINVAL, "null context");
  if (n_sweeps < 0 || measure_every < 0) return qfail(ISING_EINVAL, "negative count");
  if (x->sweep + n_sweeps >= ((int64_t)1 << 32)) return qfail(ISING_EINVAL, "sweep counter overflow");
  NvtxRange nvtx("ising_quad_sweep");
  QTRY(quad_sweeps(x, n_sweeps, measure_every));
  x->sweep += n_sweeps;
  set_last_error("");
  return ISING_OK;
}

int ising_quad_series(ising_quad* x, int64_t* B1, int64_t* B2, int64_t* M, int n) {
  if (!x) return qfail(ISING_EINVAL, "null context");
  if (n < 0 || n > std::min<int64_t>(x->rec_count, kQuadRec)) return qfail(ISING_EINVAL, "n exceeds records");
  std::vector<unsigned long long> h((size_t)3 * kQuadRec);
  QTRY(cudaMemcpyAsync(h.data(), x->rec, h.size() * 8, cudaMemcpyDeviceToHost, x->stream));
  QTRY(cudaStreamSynchronize(x->stream));
  for (int i = 0; i < n; ++i) {
    const int64_t slot = (x->rec_count - n + i) % kQuadRec;
    if (B1) B1[i] = (int64_t)h[3 * slot] / 2;
    if (B2) B2[i] = (int64_t)h[3 * slot + 1] / 2;
    if (M) M[i] = (int64_t)h[3 * slot + 2];
  }
  set_last_error("");
  return ISING_OK;
}

int ising_quad_get_spins(ising_quad* x, int8_t* host_out) {
  if (!x || !host_out) return qfail(ISING_EINVAL, "null argument");
  const int Lc = x->Lc, Wq = x->geom.Wq;
  std::vector<uint32_t> h((size_t)4 * Lc * Wq);
  QTRY(cudaMemcpyAsync(h.data(), x->planes, h.size() * 4, cudaMemcpyDeviceToHost, x->stream));
  QTRY(cudaStreamSynchronize(x->stream));
  for (int q = 0; q < 4; ++q)
    for (int Y = 0; Y < Lc; ++Y)
      for (int X = 0; X < Lc; ++X) {
        const uint32_t wv = h[((size_t)q * Lc + Y) * Wq + (X >> 5)];
        host_out[((size_t)q * Lc + Y) * Lc + X] = ((wv >> (X & 31)) & 1u) ? 1 : -1;
      }
  set_last_error("");
  return ISING_OK;
}

int ising_quad_set_spins(ising_quad* x, const int8_t* host_in) {
  if (!x || !host_in) return qfail(ISING_EINVAL, "null argument");
  const int Lc = x->Lc, Wq = x->geom.Wq;
  std::vector<uint32_t> h((size_t)4 * Lc * Wq, 0u);
  for (int q = 0; q < 4; ++q)
    for (int Y = 0; Y < Lc; ++Y)
      for (int X = 0; X < Lc; ++X) {
        const int8_t v = host_in[((size_t)q * Lc + Y) * Lc + X];
        if (v != 1 && v != -1) return qfail(ISING_EINVAL, "spins must be +1 or -1");
        if (v == 1) h[((size_t)q * Lc + Y) * Wq + (X >> 5)] |= 1u << (X & 31);
      }
  QTRY(cudaMemcpyAsync(x->planes, h.data(), h.size() * 4, cudaMemcpyHostToDevice, x->stream));
  QTRY(cudaStreamSynchronize(x->stream));
  set_last_error("");
  return ISING_OK;
}

int ising_quad_launch_count(ising_quad* x, int64_t* count) {
  if (!x || !count) return qfail(ISING_EINVAL, "null argument");
  *count = x->launches;
  return ISING_OK;
}

int ising_quad_destroy(ising_quad* x) {
  if (!x) return ISING_OK;
  cudaStreamSynchronize(x->stream);
  cudaFree(x->planes);
  cudaFree(x->rec);
  delete x;
  return ISING_OK;
}

}  // extern "C"
