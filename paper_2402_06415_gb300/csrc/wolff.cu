// Wolff single-cluster update on the packed lattice (Wolff, PRL 62, 361
// (1989)), the second cluster method next to Swendsen-Wang (the paper's
// Discussion names cluster algorithms as the next step).  Step n:
//   seed site m = floor(u N / 2^32), u = word 0 of Philox(0, n, replica, WOLFF_SEED << 16);
//   a bond b = 2 (y L + x) + dir (dir 0: to x+1, 1: to y+1) between equal spins is
//   active iff u < floor((1 - e^{-2 beta}) 2^32), u = word (b & 3) of
//   Philox(b >> 2, n, replica, WOLFF_BOND << 16);
//   the connected cluster of active bonds that holds m flips.
// The cluster is a connected component, so it does not depend on how it is
// found.  Two ways, bit-identical:
//   * growth (k_wolff_grow): one CTA grows the cluster level by level from the
//     seed, its member list and a visited hash set in shared memory; the work
//     is proportional to the cluster's surface, which is what makes Wolff
//     cheap away from criticality.  Growth is bounded (sites and levels); past
//     either bound it gives up and records that the lattice must be labelled;
//   * labelling: the Swendsen-Wang connected-component kernels (sw.cu) run on
//     the Wolff bond draws, gated on that flag, and k_wolff_apply flips the
//     sites whose root is the seed's root.
// After a step that gave up, the next 15 steps go straight to labelling
// (a critical cluster grows over hundreds of levels, where one CTA's level
// barriers cost more than labelling the whole lattice); every 16th retries.
#include <cuda_runtime.h>

#include "internal.h"
#include "ising_device.cuh"

namespace ising {
namespace {

constexpr uint32_t kTagWolffSeed = 16, kTagWolffBond = 17;
constexpr int kGrowThreads = 1024;
constexpr uint32_t kEmpty = 0xffffffffu;

__device__ __forceinline__ uint32_t site_word(uint32_t a, int L, int Wc, const FastDiv& fL, uint32_t* bit) {
  const uint32_t y = fdiv(a, fL), x = a - y * (uint32_t)L;
  const uint32_t c = (x + y) & 1u, j = x >> 1;
  *bit = 1u << (j & 31u);
  return c * (uint32_t)L * (uint32_t)Wc + y * (uint32_t)Wc + (j >> 5);
}

__device__ __forceinline__ uint32_t spin_at(const uint32_t* planes, uint32_t a, int L, int Wc, const FastDiv& fL) {
  uint32_t bit;
  const uint32_t w = site_word(a, L, Wc, fL, &bit);
  return (__ldcg(&planes[w]) & bit) ? 1u : 0u;
}

// Knuth's multiplicative hash; the top hash_bits bits index the table.
__device__ __forceinline__ uint32_t m_hash(uint32_t a) { return a * 2654435761u; }

__device__ __forceinline__ uint32_t pick(const uint4& r, uint32_t k) {
  return k == 0 ? r.x : (k == 1 ? r.y : (k == 2 ? r.z : r.w));
}

// Shared-memory layout of the growth kernel: hash[cap] (open addressing on the
// site index, at most half full) then list[max_sites].
size_t grow_hash_cap(int max_sites) {
  size_t cap = 1;
  while (cap < 2 * (size_t)max_sites) cap <<= 1;
  return cap;
}

__global__ void __launch_bounds__(kGrowThreads) k_wolff_grow(uint32_t* __restrict__ planes, int L, int Wc,
                                                             uint32_t step, uint32_t thr, RngParams rng,
                                                             int max_sites, int max_levels, uint32_t hash_bits,
                                                             WolffCtl* __restrict__ ctl, FastDiv fL,
                                                             const uint32_t* step_ptr,
                                                             cudaGraphConditionalHandle cond, int set_cond) {
  extern __shared__ uint32_t sm[];
  // graph path: the step index lives on the device (read before the first
  // barrier; thread 0 advances it after the last one)
  if (step_ptr) step = *step_ptr;
  const uint32_t cap = 1u << hash_bits;
  uint32_t* hash = sm;
  uint32_t* list = sm + cap;
  const volatile uint32_t* vhash = hash;  // other threads insert while this one reads
  __shared__ uint32_t s_tail, s_lo, s_hi, s_s0, s_m;
  __shared__ int s_state;  // 0 growing, 1 cluster complete, 2 gave up
  const uint32_t N = (uint32_t)L * (uint32_t)L;
  for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) hash[i] = kEmpty;
  if (threadIdx.x == 0) {
    const uint4 r = philox10_rk(make_uint4(0u, step, rng.replica, kTagWolffSeed << 16), rng.rk0, rng.rk1);
    const uint32_t m = __umulhi(r.x, N);
    ctl->seed_site = m;
    s_m = m;
    // after a give-up, skip growth for 15 steps (the run counter tells which)
    const uint32_t run = ctl->gave_up_run;
    const bool skip = run > 0 && (run & 15u) != 0;
    s_state = (skip || max_sites < 5) ? 2 : 0;
    s_s0 = spin_at(planes, m, L, Wc, fL);
    list[0] = m;
    s_tail = 1;
    s_lo = 0;
    s_hi = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) hash[m_hash(s_m) >> (32 - hash_bits)] = s_m;
  __syncthreads();
  const uint32_t s0 = s_s0;
  int level = 0;
  while (true) {
    const uint32_t lo = s_lo, hi = s_hi;
    if (s_state != 0) break;
    // one thread per (frontier site, direction)
    for (uint32_t i = threadIdx.x; i < 4u * (hi - lo); i += blockDim.x) {
      const uint32_t a = list[lo + (i >> 2)], dir = i & 3u;
      const uint32_t y = fdiv(a, fL), x = a - y * (uint32_t)L;
      const uint32_t xr = x + 1 == (uint32_t)L ? 0u : x + 1, xl = x == 0 ? (uint32_t)L - 1 : x - 1;
      const uint32_t yd = y + 1 == (uint32_t)L ? 0u : y + 1, yu = y == 0 ? (uint32_t)L - 1 : y - 1;
      uint32_t b, bond;
      if (dir == 0) {
        b = y * L + xr;
        bond = 2 * a;
      } else if (dir == 1) {
        b = yd * L + x;
        bond = 2 * a + 1;
      } else if (dir == 2) {
        b = y * L + xl;
        bond = 2 * b;
      } else {
        b = yu * L + x;
        bond = 2 * b + 1;
      }
      if (spin_at(planes, b, L, Wc, fL) != s0) continue;
      // already a member: skip the draw (the component does not change)
      uint32_t h = m_hash(b) >> (32 - hash_bits);
      bool seen = false;
      for (uint32_t probe = 0; probe < cap; ++probe) {
        const uint32_t v = vhash[h];
        if (v == b) {
          seen = true;
          break;
        }
        if (v == kEmpty) break;
        h = (h + 1) & (cap - 1);
      }
      if (seen) continue;
      const uint4 r = philox10_rk(make_uint4(bond >> 2, step, rng.replica, kTagWolffBond << 16), rng.rk0,
                                  rng.rk1);
      if (pick(r, bond & 3u) >= thr) continue;
      // claim b in the hash set; the thread that inserts it appends it
      h = m_hash(b) >> (32 - hash_bits);
      bool mine = false;
      for (uint32_t probe = 0; probe < cap; ++probe) {
        const uint32_t old = atomicCAS(&hash[h], kEmpty, b);
        if (old == kEmpty) {
          mine = true;
          break;
        }
        if (old == b) break;
        h = (h + 1) & (cap - 1);
      }
      if (mine) list[atomicAdd(&s_tail, 1u)] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t nlo = hi, nhi = s_tail;
      ++level;
      if (nhi == nlo)
        s_state = 1;
      // the next level appends at most 4 sites per frontier site
      else if (level >= max_levels || (uint64_t)nhi + 4ull * (nhi - nlo) > (uint64_t)max_sites)
        s_state = 2;
      s_lo = nlo;
      s_hi = nhi;
    }
    __syncthreads();
  }
  const uint32_t total = s_hi;
  if (s_state == 1) {
    for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) {
      uint32_t bit;
      const uint32_t w = site_word(list[i], L, Wc, fL, &bit);
      atomicXor(&planes[w], bit);
    }
  }
  if (threadIdx.x == 0) {
    if (s_state == 1) {
      ctl->need_label = 0;
      ctl->last_size = total;
      ctl->flipped += total;
      ctl->grown += 1;
      ctl->gave_up_run = 0;
    } else {
      ctl->need_label = 1;
      ctl->last_size = 0;  // k_wolff_apply adds the cluster's size
      ctl->labelled += 1;
      ctl->gave_up_run += 1;
    }
    // graph path: the labelling nodes run only when growth gave up, with this
    // step's index; the next growth node takes the next one
    if (set_cond) {
      ctl->step_body = step;
      ctl->step = step + 1u;
      cudaGraphSetConditional(cond, s_state == 1 ? 0u : 1u);
    }
  }
}

__global__ void k_wolff_set_step(WolffCtl* ctl, uint32_t step) { ctl->step = step; }

__device__ __forceinline__ uint32_t find_root_ro(const uint32_t* parent, uint32_t a) {
  while (true) {
    const uint32_t p = __ldcg(&parent[a]);
    if (p == a) return a;
    a = p;
  }
}

// Gated on need_label: every site that may head a subtree (mark 2 after the
// tiled labelling; every site otherwise) stores its final root in its own
// entry, so parent[parent[i]] is every site's root afterwards.
__global__ void __launch_bounds__(256) k_wolff_resolve(uint32_t* __restrict__ parent,
                                                       const uint8_t* __restrict__ mark, long long N, bool tiled,
                                                       const WolffCtl* __restrict__ ctl) {
  if (ctl->need_label == 0) return;
  if (!tiled) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
      parent[i] = find_root_ro(parent, (uint32_t)i);
    return;
  }
  // tiled path: a warp lists the local roots (mark 2) of 512 sites in shared
  // memory (16 marks per lane from one 16-byte load, prefix sum over the
  // lanes) and walks them with every lane busy
  __shared__ uint32_t roots[8][512];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long n16 = N >> 4;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long c0 = ((long long)blockIdx.x * (blockDim.x >> 5) + warp) * 32; c0 < n16; c0 += warps * 32) {
    const long long i16 = c0 + lane;
    uint32_t z[4] = {0u, 0u, 0u, 0u};
    int cnt = 0;
    if (i16 < n16) {
      const uint4 m4 = reinterpret_cast<const uint4*>(mark)[i16];
      const uint32_t w[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        // the high bit of each byte equal to 2, exactly
        const uint32_t x = w[q] ^ 0x02020202u;
        z[q] = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);
        cnt += __popc(z[q]);
      }
    }
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int pos = incl - cnt;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      while (z[q]) {
        const int byte = (__ffs(z[q]) - 1) >> 3;
        z[q] &= z[q] - 1;
        roots[warp][pos++] = (uint32_t)((i16 << 4) + 4 * q + byte);
      }
    __syncwarp();
    // two walks per lane, interleaved so that both loads are in flight
    for (int e = lane; e < total; e += 64) {
      const bool two = e + 32 < total;
      const uint32_t ia = roots[warp][e], ib = two ? roots[warp][e + 32] : ia;
      uint32_t a = ia, b = ib;
      bool da = false, db = !two;
      while (!(da && db)) {
        if (!da) {
          const uint32_t p = __ldcg(&parent[a]);
          if (p == a) da = true; else a = p;
        }
        if (!db) {
          const uint32_t p = __ldcg(&parent[b]);
          if (p == b) db = true; else b = p;
        }
      }
      parent[ia] = a;
      if (two) parent[ib] = b;
    }
    __syncwarp();
  }
}

// Gated on need_label: one warp per packed word, one lane per site; the lanes
// whose root is the seed's root set their bit of the flip mask.
__global__ void __launch_bounds__(256) k_wolff_apply(uint32_t* __restrict__ planes, int L, int Wc,
                                                     const uint32_t* __restrict__ parent,
                                                     WolffCtl* __restrict__ ctl, FastDiv fplane, FastDiv fwc) {
  if (ctl->need_label == 0) return;
  __shared__ uint32_t s_root, s_count;
  if (threadIdx.x == 0) {
    s_root = __ldcg(&parent[__ldcg(&parent[ctl->seed_site])]);
    s_count = 0;
  }
  __syncthreads();
  const uint32_t root = s_root;
  const int n = L / 2;
  const uint32_t words = 2u * (uint32_t)L * (uint32_t)Wc;
  const int lane = threadIdx.x & 31;
  const uint32_t warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  uint32_t count = 0;
  // four words per warp and iteration, their loads in flight together; lanes
  // 0..3 apply the masks of words 0..3
  constexpr int kU = 4;
  for (uint32_t i0 = warp0 * kU; i0 < words; i0 += nwarps * kU) {
    uint32_t p1[kU];
    bool ok[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const uint32_t i = i0 + u < words ? i0 + u : i0;
      const int c = (int)fdiv(i, fplane);
      const uint32_t rem = i - (uint32_t)c * fplane.d;
      const int y = (int)fdiv(rem, fwc), w = (int)(rem - (uint32_t)y * (uint32_t)Wc);
      const int j = 32 * w + lane;
      ok[u] = j < n && i0 + u < words;
      const int x = 2 * (ok[u] ? j : 0) + ((y + c) & 1);
      p1[u] = __ldg(&parent[(size_t)y * L + x]);
    }
    uint32_t mine = 0;
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const bool f = ok[u] && __ldg(&parent[p1[u]]) == root;
      const uint32_t mask = __ballot_sync(0xffffffffu, f);
      if (lane == u) mine = mask;
    }
    if (lane < kU && mine) {
      planes[i0 + lane] ^= mine;
      count += __popc(mine);
    }
  }
  if (count) atomicAdd(&s_count, count);  // lanes 0..3 hold counts
  __syncthreads();
  if (threadIdx.x == 0 && s_count) {
    atomicAdd(&ctl->last_size, s_count);
    atomicAdd(&ctl->flipped, (unsigned long long)s_count);
  }
}

int grid_of(long long items) {
  long long g = (items + 255) / 256;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (int)g;
}

}  // namespace

size_t wolff_grow_smem(int max_sites) {
  return (grow_hash_cap(max_sites) + (size_t)max_sites) * sizeof(uint32_t);
}

cudaError_t launch_wolff_step(const BitsLattice& lat, uint32_t step, uint32_t thr, const RngParams& rng,
                              uint32_t* parent, uint8_t* mark, int max_sites, int max_levels, WolffCtl* ctl,
                              cudaStream_t s) {
  static DeviceCache attr;
  if (!attr.get()) {
    cudaError_t e = cudaFuncSetAttribute(k_wolff_grow, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)wolff_grow_smem(kWolffMaxGrowSites));
    if (e) return e;
    attr.set(1);
  }
  const long long N = (long long)lat.L * lat.L;
  const int ms = max_sites < 1 ? 1 : max_sites;
  const size_t cap = grow_hash_cap(ms);
  uint32_t bits = 0;
  while (((size_t)1 << bits) < cap) ++bits;
  k_wolff_grow<<<1, kGrowThreads, wolff_grow_smem(ms), s>>>(lat.planes, lat.L, lat.Wc, step, thr, rng, max_sites,
                                                            max_levels, bits, ctl, make_fastdiv((uint32_t)lat.L),
                                                            nullptr, 0, 0);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  e = launch_cluster_labels(lat, step, thr, kTagWolffBond, rng, parent, mark, &ctl->need_label, s);
  if (e) return e;
  k_wolff_resolve<<<grid_of(N), 256, 0, s>>>(parent, mark, N, sw_tiled(lat.L), ctl);
  e = cudaGetLastError();
  if (e) return e;
  k_wolff_apply<<<grid_of(2LL * lat.L * lat.Wc * 32), 256, 0, s>>>(
      lat.planes, lat.L, lat.Wc, parent, ctl, make_fastdiv((uint32_t)lat.L * (uint32_t)lat.Wc),
      make_fastdiv((uint32_t)lat.Wc));
  return cudaGetLastError();
}

void wolff_graph_free(WolffGraph* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->exec_unrolled) cudaGraphExecDestroy(g->exec_unrolled);
  if (g->graph_unrolled) cudaGraphDestroy(g->graph_unrolled);
  *g = WolffGraph{};
}

cudaError_t wolff_graph_set_step(WolffCtl* ctl, uint32_t step, cudaStream_t s) {
  k_wolff_set_step<<<1, 1, 0, s>>>(ctl, step);
  return cudaGetLastError();
}

namespace {

// n_steps x [growth -> IF(need_label) { labelling, resolve, apply }] recorded
// into a new graph by stream capture on the private stream cs (capture
// launches nothing), each body straight into its conditional node's graph.
cudaError_t wolff_graph_record(cudaStream_t cs, int n_steps, const BitsLattice& lat, uint32_t thr,
                               const RngParams& rng, uint32_t* parent, uint8_t* mark, int max_sites,
                               int max_levels, WolffCtl* ctl, cudaGraph_t* out) {
  const long long N = (long long)lat.L * lat.L;
  const int ms = max_sites < 1 ? 1 : max_sites;
  const size_t cap = grow_hash_cap(ms);
  uint32_t bits = 0;
  while (((size_t)1 << bits) < cap) ++bits;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaGraphCreate(&graph, 0);
  if (e) return e;
  auto fail = [&](cudaError_t err) {
    cudaGraph_t junk = nullptr;
    cudaStreamEndCapture(cs, &junk);  // closes a capture left open by the failure, if any
    cudaGetLastError();
    cudaGraphDestroy(graph);
    return err;
  };
  cudaGraphNode_t prev = nullptr;  // the previous step's conditional node
  for (int k = 0; k < n_steps; ++k) {
    cudaGraphConditionalHandle cond = 0;
    if ((e = cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault))) return fail(e);
    if ((e = cudaStreamBeginCaptureToGraph(cs, graph, prev ? &prev : nullptr, nullptr, prev ? 1 : 0,
                                           cudaStreamCaptureModeThreadLocal)))
      return fail(e);
    k_wolff_grow<<<1, kGrowThreads, wolff_grow_smem(ms), cs>>>(
        lat.planes, lat.L, lat.Wc, 0u, thr, rng, max_sites, max_levels, bits, ctl,
        make_fastdiv((uint32_t)lat.L), &ctl->step, cond, 1);
    if ((e = cudaGetLastError())) return fail(e);
    // the node the capture just added is the stream's last captured node
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t n_deps = 0;
    if ((e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &n_deps))) return fail(e);
    if (n_deps != 1) return fail(cudaErrorStreamCaptureInvalidated);
    cudaGraphNode_t grow = deps[0];
    if ((e = cudaStreamEndCapture(cs, &graph))) return fail(e);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t cond_node = nullptr;
    if ((e = cudaGraphAddNode(&cond_node, graph, &grow, nullptr, 1, &cp))) return fail(e);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)))
      return fail(e);
    if ((e = launch_cluster_labels(lat, 0u, thr, kTagWolffBond, rng, parent, mark, nullptr, cs,
                                   &ctl->step_body)))
      return fail(e);
    k_wolff_resolve<<<grid_of(N), 256, 0, cs>>>(parent, mark, N, sw_tiled(lat.L), ctl);
    if ((e = cudaGetLastError())) return fail(e);
    k_wolff_apply<<<grid_of(2LL * lat.L * lat.Wc * 32), 256, 0, cs>>>(
        lat.planes, lat.L, lat.Wc, parent, ctl, make_fastdiv((uint32_t)lat.L * (uint32_t)lat.Wc),
        make_fastdiv((uint32_t)lat.Wc));
    if ((e = cudaGetLastError())) return fail(e);
    if ((e = cudaStreamEndCapture(cs, &body))) return fail(e);
    prev = cond_node;
  }
  *out = graph;
  return cudaSuccess;
}

}  // namespace

cudaError_t wolff_graph_build(WolffGraph* g, const BitsLattice& lat, uint32_t thr, const RngParams& rng,
                              uint32_t* parent, uint8_t* mark, int max_sites, int max_levels,
                              WolffCtl* ctl) {
  wolff_graph_free(g);
  static DeviceCache attr;
  cudaError_t e = cudaSuccess;
  if (!attr.get()) {
    e = cudaFuncSetAttribute(k_wolff_grow, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)wolff_grow_smem(kWolffMaxGrowSites));
    if (e) return e;
    attr.set(1);
  }
  cudaStream_t cs = nullptr;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e) return e;
  WolffGraph w;
  e = wolff_graph_record(cs, 1, lat, thr, rng, parent, mark, max_sites, max_levels, ctl, &w.graph);
  if (!e)
    e = wolff_graph_record(cs, kWolffGraphUnroll, lat, thr, rng, parent, mark, max_sites, max_levels, ctl,
                           &w.graph_unrolled);
  if (!e) e = cudaGraphInstantiate(&w.exec, w.graph, 0);
  if (!e) e = cudaGraphInstantiate(&w.exec_unrolled, w.graph_unrolled, 0);
  cudaStreamDestroy(cs);
  if (e) {
    wolff_graph_free(&w);
    return e;
  }
  w.planes = lat.planes;
  w.L = lat.L;
  w.max_sites = max_sites;
  w.max_levels = max_levels;
  w.thr = thr;
  w.replica = rng.replica;
  w.key0 = rng.key0;
  w.key1 = rng.key1;
  w.parent = parent;
  w.mark = mark;
  w.ctl = ctl;
  *g = w;
  return cudaSuccess;
}

}  // namespace ising
