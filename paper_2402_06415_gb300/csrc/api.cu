// C-ABI of libising.so (declarations and contracts in include/ising.h).
//
// Host-side control of the checkerboard Metropolis sweep: argument checks,
// integer thresholds, record bookkeeping, kernel choice and launches on the
// caller's stream.  No arithmetic of the method runs here except the two
// thresholds floor(exp(-beta dE) 2^32), dE = 4, 8 (arXiv 2402.06415,
// Supplementary MC details, step 2), computed once per beta.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "ising.h"

using namespace ising;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int ok() {
  g_err.clear();
  return ISING_OK;
}

// Host-side fault injection for the failure-path tests: ISING_FAULT=alloc
// makes device allocations fail, ISING_FAULT=launch makes sweep launches fail,
// ISING_FAULT=copy makes host<->device copies fail.  Never touches the GPU.
bool fault(const char* what) {
  const char* f = std::getenv("ISING_FAULT");
  return f && std::strstr(f, what) != nullptr;
}

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e__ = (expr);                                                            \
    if (e__ != cudaSuccess)                                                              \
      return fail(ISING_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e__), __FILE__, \
                  __LINE__);                                                             \
  } while (0)

constexpr int64_t kRecCap = 65536;

uint32_t threshold(double beta, int dE) {
  const double p = std::exp(-beta * (double)dE);
  const double t = std::floor(p * 4294967296.0);
  if (t >= 4294967295.0) return 0xffffffffu;
  if (t <= 0.0) return 0u;
  return (uint32_t)t;
}

int words_per_row(int L) { return (L / 2 + 31) / 32; }

}  // namespace

struct ising_ctx {
  int L = 0, layout = 0, dev = 0, sms = 0;
  double beta = 0;
  uint32_t t4 = 0, t8 = 0;
  uint64_t seed = 0;
  uint32_t replica = 0;
  int64_t sweep = 0;
  cudaStream_t stream = nullptr;
  int Wc = 0;
  uint32_t* bits[2] = {nullptr, nullptr};
  int cur = 0;
  int8_t* spins = nullptr;
  unsigned long long* rec = nullptr;  // [kRecCap][2]: anti-bond count, up-spin count
  int64_t rec_count = 0;
  unsigned long long* meas = nullptr;  // [2]
  int kernel = ISING_KERNEL_HALF, k = 1, tile_rows = 1, tile_words = 4, grid = 0, block = 0;
  __nv_bfloat16* nn_w = nullptr;    // BF16 weights of the block proposal
  __nv_bfloat16* nn_w2t = nullptr;
  unsigned long long* blk_stats = nullptr;  // [3] proposed, accepted, device wait time-outs
  int64_t block_passes = 0;
  int proposal = 0;                  // ISING_PROPOSAL_ONESHOT / _STAGED
  int nn_engine = 0;                 // ISING_NN_ENGINE_MMA_SYNC / _TCGEN05 (staged proposal)
  nnc::StagedPlan* plan = nullptr;   // device plan of the staged proposal
  int plan_B = 0;                    // block size the plan was built for
  uint32_t* sw_parent = nullptr;  // Swendsen-Wang scratch
  uint8_t* sw_flip = nullptr;
  int64_t sw_steps = 0;
  WolffCtl* wolff = nullptr;  // Wolff step state (parent / mark scratch shared with Swendsen-Wang)
  int64_t wolff_steps = 0;
  int wolff_max_sites = kWolffMaxGrowSites, wolff_max_levels = 0;
  WolffGraph wolff_graph;           // one Wolff step as a CUDA graph (growth + IF labelling)
  bool wolff_graph_broken = false;  // building it failed once: separate launches from then on
  int cluster_mode = ISING_CLUSTER_AUTO;
  GridCtl* cluster_gctl = nullptr;  // barrier of the persistent cluster kernel
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  int64_t launches = 0;

  int64_t N() const { return (int64_t)L * L; }
  size_t plane_words() const { return (size_t)2 * L * Wc; }
  BitsLattice lat(int which) const { return BitsLattice{bits[which], L, Wc, Wc}; }
  RngParams rng() const { return make_rng(seed, replica, t4, t8); }
};

namespace {

int dev_alloc(void** p, size_t bytes) {
  if (fault("alloc")) return fail(ISING_ENOMEM, "device allocation of %zu bytes failed (injected)", bytes);
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? ISING_ENOMEM : ISING_ECUDA,
                "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  return ISING_OK;
}

void free_all(ising_ctx* c) {
  if (!c) return;
  for (auto e : c->ev) cudaEventDestroy(e);
  c->ev.clear();
  cudaFree(c->bits[0]);
  cudaFree(c->bits[1]);
  cudaFree(c->spins);
  cudaFree(c->rec);
  cudaFree(c->meas);
  cudaFree(c->nn_w);
  cudaFree(c->nn_w2t);
  cudaFree(c->blk_stats);
  cudaFree(c->plan);
  c->plan = nullptr;
  c->plan_B = 0;
  cudaFree(c->sw_parent);
  cudaFree(c->sw_flip);
  wolff_graph_free(&c->wolff_graph);
  cudaFree(c->wolff);
  cudaFree(c->cluster_gctl);
  c->wolff = nullptr;
  c->cluster_gctl = nullptr;
  c->sw_parent = nullptr;
  c->sw_flip = nullptr;
  c->nn_w = c->nn_w2t = nullptr;
  c->blk_stats = nullptr;
  c->bits[0] = c->bits[1] = nullptr;
  c->spins = nullptr;
  c->rec = nullptr;
  c->meas = nullptr;
}

bool beta_ok(double beta) { return std::isfinite(beta) && beta > 0.0; }

int check_ctx(ising_ctx* c) {
  if (!c) return fail(ISING_EINVAL, "null context");
  return ISING_OK;
}

// Kernel configuration validity for this lattice.
int validate_kernel(const ising_ctx* c, int kernel, int k, int tile_rows, int tile_words) {
  if (c->layout == ISING_LAYOUT_BITS) {
    if (kernel == ISING_KERNEL_HALF) return ISING_OK;
    if (kernel == ISING_KERNEL_TILED) {
      if (c->Wc % 4 != 0 || c->L % 64 != 0)
        return fail(ISING_EINVAL, "tiled kernel needs L %% 256 == 0 (L = %d)", c->L);
      if (k < 1 || k > kMaxSweepsPerLaunch)
        return fail(ISING_EINVAL, "sweeps_per_launch must be in 1..%d", kMaxSweepsPerLaunch);
      if (tile_words < 4 || tile_words % 4 != 0 || c->Wc % tile_words != 0)
        return fail(ISING_EINVAL, "tile_words must be a multiple of 4 dividing Wc = %d", c->Wc);
      if (tile_rows < 1 || tile_rows > c->L)
        return fail(ISING_EINVAL, "tile_rows must be in 1..L");
      if (c->L < 4 * k) return fail(ISING_EINVAL, "L must be at least 4 x sweeps_per_launch");
      const size_t smem = (tile_words == 32 || tile_words == 64)
                              ? tiled32_smem_bytes(c->L, k, tile_rows, tile_words)
                              : tiled_smem_bytes(c->L, k, tile_rows, tile_words);
      if (smem > 200 * 1024)
        return fail(ISING_EINVAL, "tile needs %zu bytes of shared memory (> 200 KiB)", smem);
      return ISING_OK;
    }
    return fail(ISING_EINVAL, "kernel %d does not apply to the packed layout", kernel);
  }
  if (kernel == ISING_KERNEL_HALF) return ISING_OK;
  if (kernel == ISING_KERNEL_RESIDENT) {
    if (resident_i8_smem_bytes(c->L) > 200 * 1024)
      return fail(ISING_EINVAL, "resident kernel needs L*L <= 200 KiB (L = %d)", c->L);
    return ISING_OK;
  }
  return fail(ISING_EINVAL, "kernel %d does not apply to the int8 layout", kernel);
}

void resolve_auto(ising_ctx* c) {
  if (c->layout == ISING_LAYOUT_BITS) {
    if (c->Wc % 4 == 0 && c->L % 64 == 0 && c->L >= 256) {
      c->kernel = ISING_KERNEL_TILED;
      c->k = 1;
      int tw = 32;
      while (tw > 4 && c->Wc % tw != 0) tw /= 2;
      c->tile_words = tw;
      // about 108-row strips: for L = 16384 that is 152 strips x 8 tiles,
      // two tiles per resident CTA at 4 CTAs per SM
      c->tile_rows = c->L >= 1024 ? (int)((int64_t)c->L * 152 / 16384) : c->L / 64;
      if (c->tile_rows < 1) c->tile_rows = 1;
    } else {
      c->kernel = ISING_KERNEL_HALF;
    }
  } else {
    c->kernel = resident_i8_smem_bytes(c->L) <= 64 * 1024 ? ISING_KERNEL_RESIDENT
                                                          : ISING_KERNEL_HALF;
  }
  c->grid = 0;
  c->block = 0;
}

int ensure_second_buffer(ising_ctx* c) {
  if (c->bits[1]) return ISING_OK;
  void* p = nullptr;
  int st = dev_alloc(&p, c->plane_words() * sizeof(uint32_t));
  if (st) return st;
  c->bits[1] = (uint32_t*)p;
  cudaError_t e = cudaMemsetAsync(c->bits[1], 0, c->plane_words() * sizeof(uint32_t), c->stream);
  if (e != cudaSuccess) return fail(ISING_ECUDA, "memset: %s", cudaGetErrorString(e));
  return ISING_OK;
}

cudaEvent_t next_event(ising_ctx* c) {
  if (c->ev_used == c->ev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->ev.push_back(e);
  }
  return c->ev[c->ev_used++];
}

// Brackets one sweep-kernel launch with events when timing is on.
struct Timed {
  ising_ctx* c;
  explicit Timed(ising_ctx* cc) : c(cc) {
    if (c->timing) {
      cudaEvent_t e = next_event(c);
      if (e) cudaEventRecord(e, c->stream);
    }
  }
  ~Timed() {
    if (c->timing) {
      cudaEvent_t e = next_event(c);
      if (e) cudaEventRecord(e, c->stream);
    }
  }
};

int zero_records(ising_ctx* c, int64_t first_rec, int64_t n_rec) {
  if (n_rec <= 0) return ISING_OK;
  const int64_t s0 = first_rec % kRecCap;
  const int64_t n1 = std::min<int64_t>(n_rec, kRecCap - s0);
  CUDA_TRY(cudaMemsetAsync(c->rec + 2 * s0, 0, (size_t)n1 * 2 * sizeof(unsigned long long),
                           c->stream));
  if (n_rec > n1)
    CUDA_TRY(cudaMemsetAsync(c->rec, 0, (size_t)(n_rec - n1) * 2 * sizeof(unsigned long long),
                             c->stream));
  return ISING_OK;
}

int launch_result(ising_ctx* c, cudaError_t e, const char* what) {
  ++c->launches;
  if (e != cudaSuccess) return fail(ISING_ECUDA, "%s launch: %s", what, cudaGetErrorString(e));
  return ISING_OK;
}

// Runs sweeps [t0, t0 + n) whose records (if any) all fit in the ring.
int sweep_chunk(ising_ctx* c, int64_t t0, int n, int m) {
  // record bookkeeping: record r of this chunk belongs to sweep t_r
  int64_t first_t = -1, n_rec = 0;
  if (m > 0) {
    for (int64_t t = t0; t < t0 + n; ++t)
      if ((t + 1) % m == 0) {
        if (first_t < 0) first_t = t;
        ++n_rec;
      }
  }
  const int64_t rec0 = c->rec_count;
  if (int st = zero_records(c, rec0, n_rec)) return st;
  auto slot_of = [&](int64_t t) -> int64_t {  // -1 if sweep t is not recorded
    if (m <= 0 || (t + 1) % m != 0) return -1;
    return (rec0 + (t - first_t) / m) % kRecCap;
  };
  const RngParams rng = c->rng();
  if (fault("launch")) return fail(ISING_ECUDA, "sweep launch failed (injected)");

  if (c->layout == ISING_LAYOUT_BITS && c->kernel == ISING_KERNEL_HALF) {
    for (int64_t t = t0; t < t0 + n; ++t) {
      const int64_t sl = slot_of(t);
      for (int col = 0; col < 2; ++col) {
        Timed tm(c);
        cudaError_t e = launch_half_sweep_bits(c->lat(c->cur), rng, col, (uint32_t)t,
                                               (col == 1 && sl >= 0) ? c->rec + 2 * sl : nullptr,
                                               c->grid, c->block, c->stream);
        if (int st = launch_result(c, e, "half sweep")) return st;
      }
    }
  } else if (c->layout == ISING_LAYOUT_BITS && c->kernel == ISING_KERNEL_TILED) {
    for (int64_t t = t0; t < t0 + n; t += c->k) {
      const int kk = (int)std::min<int64_t>(c->k, t0 + n - t);
      RecordSlots slots;
      for (int s = 0; s < kMaxSweepsPerLaunch; ++s)
        slots.slot[s] = s < kk ? (int)slot_of(t + s) : -1;
      Timed tm(c);
      cudaError_t e =
          (c->tile_words == 32 || c->tile_words == 64)
              ? launch_tiled32_sweep_bits(c->lat(c->cur), c->bits[1 - c->cur], rng, (uint32_t)t,
                                          kk, slots, c->rec, c->tile_rows, c->tile_words, c->grid,
                                          c->stream)
              : launch_tiled_sweep_bits(c->lat(c->cur), c->bits[1 - c->cur], rng, (uint32_t)t, kk,
                                        slots, c->rec, c->tile_rows, c->tile_words, c->grid,
                                        c->block, c->stream);
      if (int st = launch_result(c, e, "tiled sweep")) return st;
      c->cur = 1 - c->cur;
    }
  } else if (c->layout == ISING_LAYOUT_I8 && c->kernel == ISING_KERNEL_RESIDENT) {
    Timed tm(c);
    cudaError_t e = launch_resident_sweep_i8(
        c->spins, c->L, rng, (uint32_t)t0, n, m, (uint32_t)(first_t < 0 ? 0 : first_t),
        rec0 % kRecCap, kRecCap, c->rec, c->stream);
    if (int st = launch_result(c, e, "resident sweep")) return st;
  } else {
    for (int64_t t = t0; t < t0 + n; ++t) {
      const int64_t sl = slot_of(t);
      for (int col = 0; col < 2; ++col) {
        Timed tm(c);
        cudaError_t e = launch_half_sweep_i8(c->spins, c->L, rng, col, (uint32_t)t,
                                             (col == 1 && sl >= 0) ? c->rec + 2 * sl : nullptr,
                                             c->stream);
        if (int st = launch_result(c, e, "int8 half sweep")) return st;
      }
    }
  }
  c->rec_count += n_rec;
  return ISING_OK;
}

int to_host_sync(ising_ctx* c, void* dst, const void* src, size_t bytes) {
  if (fault("copy")) return fail(ISING_ECUDA, "device-to-host copy failed (injected)");
  CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (c->cluster_gctl) {
    // a grid barrier of the persistent cluster kernel that gave up stays recorded until the next seed
    int status = 0;
    CUDA_TRY(cudaMemcpy(&status, &c->cluster_gctl->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) return fail(ISING_ETIMEOUT, "grid barrier timed out in the persistent cluster kernel");
  }
  return ISING_OK;
}

int to_device_sync(ising_ctx* c, void* dst, const void* src, size_t bytes) {
  if (fault("copy")) return fail(ISING_ECUDA, "host-to-device copy failed (injected)");
  CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return ISING_OK;
}

}  // namespace

namespace ising {
void set_last_error(const char* msg) { g_err = msg ? msg : ""; }
}  // namespace ising

extern "C" {

const char* ising_last_error(void) { return g_err.c_str(); }

int ising_words_per_row(int L) { return words_per_row(L); }

int ising_thresholds(double beta, uint32_t* t4, uint32_t* t8) {
  if (!beta_ok(beta)) return fail(ISING_EINVAL, "beta must be finite and > 0");
  if (!t4 || !t8) return fail(ISING_EINVAL, "null output pointer");
  *t4 = threshold(beta, 4);
  *t8 = threshold(beta, 8);
  return ok();
}

int ising_create(ising_ctx** out, int L, double beta, int layout, void* stream) {
  if (!out) return fail(ISING_EINVAL, "null output pointer");
  *out = nullptr;
  if (L < 4 || L > 65536 || (L & 1))
    return fail(ISING_EINVAL, "L must be even and in [4, 65536] (got %d)", L);
  if (!beta_ok(beta)) return fail(ISING_EINVAL, "beta must be finite and > 0");
  if (layout != ISING_LAYOUT_I8 && layout != ISING_LAYOUT_BITS)
    return fail(ISING_EINVAL, "unknown layout %d", layout);
  ising_ctx* c = new (std::nothrow) ising_ctx();
  if (!c) return fail(ISING_ENOMEM, "host allocation failed");
  c->L = L;
  c->layout = layout;
  c->beta = beta;
  c->t4 = threshold(beta, 4);
  c->t8 = threshold(beta, 8);
  c->stream = (cudaStream_t)stream;
  c->Wc = words_per_row(L);
  int st = ISING_OK;
  cudaError_t e = cudaGetDevice(&c->dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return fail(ISING_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
  }
  void* p = nullptr;
  if (layout == ISING_LAYOUT_BITS) {
    st = dev_alloc(&p, c->plane_words() * sizeof(uint32_t));
    c->bits[0] = (uint32_t*)p;
  } else {
    st = dev_alloc(&p, (size_t)c->N());
    c->spins = (int8_t*)p;
  }
  if (!st) {
    st = dev_alloc(&p, (size_t)kRecCap * 2 * sizeof(unsigned long long));
    c->rec = (unsigned long long*)p;
  }
  if (!st) {
    st = dev_alloc(&p, 2 * sizeof(unsigned long long));
    c->meas = (unsigned long long*)p;
  }
  if (!st) {
    resolve_auto(c);
    if (c->kernel == ISING_KERNEL_TILED) st = ensure_second_buffer(c);
  }
  if (!st) {
    // all -1 start: zero bits / int8 0xff
    cudaError_t e2 = layout == ISING_LAYOUT_BITS
                         ? cudaMemsetAsync(c->bits[0], 0, c->plane_words() * 4, c->stream)
                         : cudaMemsetAsync(c->spins, 0xff, (size_t)c->N(), c->stream);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(c->stream);
    if (e2 != cudaSuccess) st = fail(ISING_ECUDA, "memset: %s", cudaGetErrorString(e2));
  }
  if (st) {
    std::string msg = g_err;
    free_all(c);
    delete c;
    g_err = msg;
    return st;
  }
  *out = c;
  return ok();
}

int ising_destroy(ising_ctx* c) {
  if (!c) return ok();
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
  return ok();
}

int ising_seed(ising_ctx* c, uint64_t seed) {
  if (int st = check_ctx(c)) return st;
  c->seed = seed;
  c->sweep = 0;
  c->rec_count = 0;
  c->sw_steps = 0;
  c->wolff_steps = 0;
  cudaError_t e;
  if (c->wolff) {
    e = cudaMemsetAsync(c->wolff, 0, sizeof(WolffCtl), c->stream);
    if (e) return fail(ISING_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  }
  if (c->cluster_gctl) {
    e = cudaMemsetAsync(c->cluster_gctl, 0, sizeof(GridCtl), c->stream);
    if (e) return fail(ISING_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  }
  if (c->layout == ISING_LAYOUT_BITS) {
    c->cur = 0;
    e = launch_init_bits(c->lat(0), c->rng(), c->stream);
  } else {
    e = launch_init_i8(c->spins, c->L, c->rng(), c->stream);
  }
  return launch_result(c, e, "init") ? ISING_ECUDA : ok();
}

int ising_set_key(ising_ctx* c, uint64_t seed) {
  if (int st = check_ctx(c)) return st;
  c->seed = seed;
  return ok();
}

int ising_set_replica(ising_ctx* c, uint32_t replica) {
  if (int st = check_ctx(c)) return st;
  c->replica = replica;
  return ok();
}

int ising_set_beta(ising_ctx* c, double beta) {
  if (int st = check_ctx(c)) return st;
  if (!beta_ok(beta)) return fail(ISING_EINVAL, "beta must be finite and > 0");
  c->beta = beta;
  c->t4 = threshold(beta, 4);
  c->t8 = threshold(beta, 8);
  return ok();
}

int ising_set_sweep_counter(ising_ctx* c, int64_t t) {
  if (int st = check_ctx(c)) return st;
  if (t < 0 || t >= (int64_t)1 << 32) return fail(ISING_EINVAL, "sweep counter out of range");
  c->sweep = t;
  return ok();
}

int ising_get_state(ising_ctx* c, uint64_t* seed, uint32_t* replica, int64_t* sweep) {
  if (int st = check_ctx(c)) return st;
  if (seed) *seed = c->seed;
  if (replica) *replica = c->replica;
  if (sweep) *sweep = c->sweep;
  return ok();
}

int ising_sweep(ising_ctx* c, int n_sweeps, int measure_every) {
  if (int st = check_ctx(c)) return st;
  NvtxRange nvtx("ising_sweep");
  if (n_sweeps < 0) return fail(ISING_EINVAL, "n_sweeps must be >= 0");
  if (measure_every < 0) return fail(ISING_EINVAL, "measure_every must be >= 0");
  if (c->sweep + n_sweeps >= ((int64_t)1 << 32))
    return fail(ISING_EINVAL, "sweep counter would exceed 2^32");
  // chunk so that no chunk produces more records than the ring holds
  int64_t t = c->sweep;
  const int64_t end = c->sweep + n_sweeps;
  const int64_t max_chunk = measure_every > 0 ? kRecCap * (int64_t)measure_every : end - t;
  while (t < end) {
    const int64_t n = std::min<int64_t>(end - t, std::max<int64_t>(max_chunk, 1));
    int chunk = (int)std::min<int64_t>(n, 1 << 30);
    if (int st = sweep_chunk(c, t, chunk, measure_every)) return st;
    t += chunk;
    c->sweep = t;
  }
  return ok();
}

int ising_measure(ising_ctx* c, int64_t* E, int64_t* M) {
  if (int st = check_ctx(c)) return st;
  if (!E || !M) return fail(ISING_EINVAL, "null output pointer");
  CUDA_TRY(cudaMemsetAsync(c->meas, 0, 2 * sizeof(unsigned long long), c->stream));
  cudaError_t e = c->layout == ISING_LAYOUT_BITS ? launch_measure_bits(c->lat(c->cur), c->meas, c->stream)
                                                 : launch_measure_i8(c->spins, c->L, c->meas, c->stream);
  if (int st = launch_result(c, e, "measure")) return st;
  unsigned long long h[2];
  if (int st = to_host_sync(c, h, c->meas, sizeof(h))) return st;
  *E = 2 * (int64_t)h[0] - 2 * c->N();
  *M = 2 * (int64_t)h[1] - c->N();
  return ok();
}

int ising_series_count(ising_ctx* c, int64_t* count) {
  if (int st = check_ctx(c)) return st;
  if (!count) return fail(ISING_EINVAL, "null output pointer");
  *count = c->rec_count;
  return ok();
}

int ising_series(ising_ctx* c, int64_t* E_out, int64_t* M_out, int n) {
  if (int st = check_ctx(c)) return st;
  if (n < 0 || n > std::min<int64_t>(c->rec_count, kRecCap))
    return fail(ISING_EINVAL, "n = %d exceeds the available records", n);
  if (n == 0) return ok();
  if (!E_out || !M_out) return fail(ISING_EINVAL, "null output pointer");
  std::vector<unsigned long long> h((size_t)2 * n);
  const int64_t first = c->rec_count - n;
  const int64_t s0 = first % kRecCap;
  const int64_t n1 = std::min<int64_t>(n, kRecCap - s0);
  if (int st = to_host_sync(c, h.data(), c->rec + 2 * s0, (size_t)n1 * 16)) return st;
  if (n > n1)
    if (int st = to_host_sync(c, h.data() + 2 * n1, c->rec, (size_t)(n - n1) * 16)) return st;
  for (int i = 0; i < n; ++i) {
    E_out[i] = 2 * (int64_t)h[2 * i] - 2 * c->N();
    M_out[i] = 2 * (int64_t)h[2 * i + 1] - c->N();
  }
  return ok();
}

static int get_spins_dev(ising_ctx* c, int8_t* dst) {
  if (c->layout == ISING_LAYOUT_I8) {
    CUDA_TRY(cudaMemcpyAsync(dst, c->spins, (size_t)c->N(), cudaMemcpyDeviceToDevice, c->stream));
    return ISING_OK;
  }
  return launch_result(c, launch_unpack_bits(c->lat(c->cur), dst, c->stream), "unpack");
}

static int set_spins_dev(ising_ctx* c, const int8_t* src) {
  if (c->layout == ISING_LAYOUT_I8) {
    CUDA_TRY(cudaMemcpyAsync(c->spins, src, (size_t)c->N(), cudaMemcpyDeviceToDevice, c->stream));
    return ISING_OK;
  }
  return launch_result(c, launch_pack_bits(c->lat(c->cur), src, c->stream), "pack");
}

static int get_bits_dev(ising_ctx* c, uint32_t* dst) {
  if (c->layout == ISING_LAYOUT_BITS) {
    CUDA_TRY(cudaMemcpyAsync(dst, c->bits[c->cur], c->plane_words() * 4, cudaMemcpyDeviceToDevice,
                             c->stream));
    return ISING_OK;
  }
  BitsLattice tmp{dst, c->L, c->Wc, c->Wc};
  return launch_result(c, launch_pack_bits(tmp, c->spins, c->stream), "pack");
}

static int set_bits_dev(ising_ctx* c, const uint32_t* src) {
  if (c->layout == ISING_LAYOUT_BITS) {
    CUDA_TRY(cudaMemcpyAsync(c->bits[c->cur], src, c->plane_words() * 4, cudaMemcpyDeviceToDevice,
                             c->stream));
    return ISING_OK;
  }
  BitsLattice tmp{const_cast<uint32_t*>(src), c->L, c->Wc, c->Wc};
  return launch_result(c, launch_unpack_bits(tmp, c->spins, c->stream), "unpack");
}

int ising_get_spins_device(ising_ctx* c, int8_t* dev_out) {
  if (int st = check_ctx(c)) return st;
  if (!dev_out) return fail(ISING_EINVAL, "null buffer");
  if (int st = get_spins_dev(c, dev_out)) return st;
  return ok();
}

int ising_set_spins_device(ising_ctx* c, const int8_t* dev_in) {
  if (int st = check_ctx(c)) return st;
  if (!dev_in) return fail(ISING_EINVAL, "null buffer");
  if (int st = set_spins_dev(c, dev_in)) return st;
  return ok();
}

int ising_get_bits_device(ising_ctx* c, uint32_t* dev_out) {
  if (int st = check_ctx(c)) return st;
  if (!dev_out) return fail(ISING_EINVAL, "null buffer");
  if (int st = get_bits_dev(c, dev_out)) return st;
  return ok();
}

int ising_set_bits_device(ising_ctx* c, const uint32_t* dev_in) {
  if (int st = check_ctx(c)) return st;
  if (!dev_in) return fail(ISING_EINVAL, "null buffer");
  if (int st = set_bits_dev(c, dev_in)) return st;
  return ok();
}

int ising_get_spins(ising_ctx* c, int8_t* host_out) {
  if (int st = check_ctx(c)) return st;
  if (!host_out) return fail(ISING_EINVAL, "null buffer");
  if (c->layout == ISING_LAYOUT_I8) {
    if (int st = to_host_sync(c, host_out, c->spins, (size_t)c->N())) return st;
    return ok();
  }
  void* tmp = nullptr;
  if (int st = dev_alloc(&tmp, (size_t)c->N())) return st;
  int st = get_spins_dev(c, (int8_t*)tmp);
  if (!st) st = to_host_sync(c, host_out, tmp, (size_t)c->N());
  cudaFree(tmp);
  return st ? st : ok();
}

int ising_set_spins(ising_ctx* c, const int8_t* host_in) {
  if (int st = check_ctx(c)) return st;
  if (!host_in) return fail(ISING_EINVAL, "null buffer");
  for (int64_t i = 0; i < c->N(); ++i)
    if (host_in[i] != 1 && host_in[i] != -1)
      return fail(ISING_EINVAL, "spin %lld is %d, not +-1", (long long)i, (int)host_in[i]);
  if (c->layout == ISING_LAYOUT_I8) {
    if (int st = to_device_sync(c, c->spins, host_in, (size_t)c->N())) return st;
    return ok();
  }
  void* tmp = nullptr;
  if (int st = dev_alloc(&tmp, (size_t)c->N())) return st;
  int st = to_device_sync(c, tmp, host_in, (size_t)c->N());
  if (!st) st = set_spins_dev(c, (const int8_t*)tmp);
  if (!st) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) st = fail(ISING_ECUDA, "sync: %s", cudaGetErrorString(e));
  }
  cudaFree(tmp);
  return st ? st : ok();
}

int ising_get_bits(ising_ctx* c, uint32_t* host_out) {
  if (int st = check_ctx(c)) return st;
  if (!host_out) return fail(ISING_EINVAL, "null buffer");
  if (c->layout == ISING_LAYOUT_BITS) {
    if (int st = to_host_sync(c, host_out, c->bits[c->cur], c->plane_words() * 4)) return st;
    return ok();
  }
  void* tmp = nullptr;
  if (int st = dev_alloc(&tmp, c->plane_words() * 4)) return st;
  int st = get_bits_dev(c, (uint32_t*)tmp);
  if (!st) st = to_host_sync(c, host_out, tmp, c->plane_words() * 4);
  cudaFree(tmp);
  return st ? st : ok();
}

int ising_set_bits(ising_ctx* c, const uint32_t* host_in) {
  if (int st = check_ctx(c)) return st;
  if (!host_in) return fail(ISING_EINVAL, "null buffer");
  // unused lanes of the last word of each row must be zero; copy-and-mask
  // only when such lanes exist (L/2 not a multiple of 32)
  const int nb = c->L / 2 - 32 * (c->Wc - 1);
  std::vector<uint32_t> masked;
  const uint32_t* src = host_in;
  if (nb < 32) {
    masked.assign(host_in, host_in + c->plane_words());
    for (size_t r = 0; r < (size_t)2 * c->L; ++r) masked[r * c->Wc + c->Wc - 1] &= (1u << nb) - 1u;
    src = masked.data();
  }
  if (c->layout == ISING_LAYOUT_BITS) {
    if (int st = to_device_sync(c, c->bits[c->cur], src, c->plane_words() * 4)) return st;
    return ok();
  }
  void* tmp = nullptr;
  if (int st = dev_alloc(&tmp, c->plane_words() * 4)) return st;
  int st = to_device_sync(c, tmp, src, c->plane_words() * 4);
  if (!st) st = set_bits_dev(c, (const uint32_t*)tmp);
  if (!st) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) st = fail(ISING_ECUDA, "sync: %s", cudaGetErrorString(e));
  }
  cudaFree(tmp);
  return st ? st : ok();
}

int ising_set_kernel(ising_ctx* c, int kernel, int k, int tile_rows, int tile_words, int grid,
                     int block) {
  if (int st = check_ctx(c)) return st;
  if (grid < 0 || block < 0 || (block && (block % 32 != 0 || block > 1024)))
    return fail(ISING_EINVAL, "grid must be >= 0 and block a multiple of 32 in [32, 1024]");
  if (kernel == ISING_KERNEL_AUTO) {
    resolve_auto(c);
    if (c->kernel == ISING_KERNEL_TILED)
      if (int st = ensure_second_buffer(c)) return st;
    return ok();
  }
  if (kernel == ISING_KERNEL_TILED && block && block != 256)
    return fail(ISING_EINVAL, "the tiled kernel runs 256 threads per block");
  if (int st = validate_kernel(c, kernel, k, tile_rows, tile_words)) return st;
  if (kernel == ISING_KERNEL_TILED)
    if (int st = ensure_second_buffer(c)) return st;
  c->kernel = kernel;
  c->k = kernel == ISING_KERNEL_TILED ? k : 1;
  c->tile_rows = tile_rows;
  c->tile_words = tile_words;
  c->grid = grid;
  c->block = block;
  return ok();
}

int ising_get_kernel(ising_ctx* c, int* kernel, int* k, int* tile_rows, int* tile_words,
                     int* grid, int* block) {
  if (int st = check_ctx(c)) return st;
  if (kernel) *kernel = c->kernel;
  if (k) *k = c->k;
  if (tile_rows) *tile_rows = c->tile_rows;
  if (tile_words) *tile_words = c->tile_words;
  if (grid) *grid = c->grid;
  if (block) *block = c->block;
  return ok();
}

int ising_set_timing(ising_ctx* c, int enable) {
  if (int st = check_ctx(c)) return st;
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->timing = enable != 0;
  c->ev_used = 0;
  return ok();
}

int ising_kernel_time(ising_ctx* c, double* ms, int64_t* launches) {
  if (int st = check_ctx(c)) return st;
  if (!ms || !launches) return fail(ISING_EINVAL, "null output pointer");
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  double total = 0.0;
  for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
    float f = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&f, c->ev[i], c->ev[i + 1]));
    total += f;
  }
  *ms = total;
  *launches = (int64_t)(c->ev_used / 2);
  return ok();
}

int ising_nn_load(ising_ctx* c, const void* bf16_weights, size_t bytes) {
  if (int st = check_ctx(c)) return st;
  if (!bf16_weights || bytes != nn_blob_bytes())
    return fail(ISING_EINVAL, "weights blob must be %zu bytes of bf16", nn_blob_bytes());
  if (!c->nn_w) {
    cudaError_t e = nn_alloc_weights(&c->nn_w, &c->nn_w2t);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->blk_stats, 3 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->blk_stats, 0, 3 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ISING_ENOMEM, "block-proposal weights: %s", cudaGetErrorString(e));
    }
  }
  CUDA_TRY(nn_load_blob(c->nn_w, c->nn_w2t, bf16_weights, c->stream));
  return ok();
}

int ising_block_pass(ising_ctx* c, int n_passes, int block) {
  if (int st = check_ctx(c)) return st;
  NvtxRange nvtx("ising_block_pass");
  if (!c->nn_w) return fail(ISING_EINVAL, "no network loaded (ising_nn_load)");
  if (c->layout != ISING_LAYOUT_BITS) return fail(ISING_EINVAL, "block passes need the packed layout");
  if (block != 2 && block != 4 && block != 8 && block != 16)
    return fail(ISING_EINVAL, "block must be 2, 4, 8 or 16");
  if (c->L % (2 * block) != 0) return fail(ISING_EINVAL, "L must be a multiple of 2 x block");
  if (n_passes < 0) return fail(ISING_EINVAL, "n_passes must be >= 0");
  if (c->proposal == ISING_PROPOSAL_STAGED && c->plan_B != block) {
    CUDA_TRY(nnc::nn_upload_plan(block, ISING_PROPOSAL_STAGED, &c->plan, nullptr, c->stream));
    c->plan_B = block;
  }
  const RngParams rng = c->rng();
  for (int k = 0; k < n_passes; ++k) {
    for (int col = 0; col < 2; ++col) {
      Timed tm(c);
      cudaError_t e =
          c->proposal == ISING_PROPOSAL_STAGED
              ? nn_staged_block_pass(c->bits[c->cur], c->L, c->Wc, c->plan, block,
                                     (uint32_t)c->block_passes, col, rng, c->beta, c->nn_engine, c->nn_w,
                                     c->nn_w2t, c->blk_stats, c->stream)
              : nn_block_pass(c->bits[c->cur], c->L, c->Wc, block, (uint32_t)c->block_passes, col, rng,
                              c->beta, c->nn_w, c->nn_w2t, c->blk_stats, c->stream);
      if (int st = launch_result(c, e, "block pass")) return st;
    }
    ++c->block_passes;
  }
  return ok();
}

int ising_set_proposal(ising_ctx* c, int kind) {
  if (int st = check_ctx(c)) return st;
  if (kind != ISING_PROPOSAL_ONESHOT && kind != ISING_PROPOSAL_STAGED)
    return fail(ISING_EINVAL, "proposal kind must be ISING_PROPOSAL_ONESHOT or ISING_PROPOSAL_STAGED");
  c->proposal = kind;
  return ok();
}

int ising_set_nn_engine(ising_ctx* c, int engine) {
  if (int st = check_ctx(c)) return st;
  if (engine != ISING_NN_ENGINE_MMA_SYNC && engine != ISING_NN_ENGINE_TCGEN05)
    return fail(ISING_EINVAL, "engine must be ISING_NN_ENGINE_MMA_SYNC or ISING_NN_ENGINE_TCGEN05");
  c->nn_engine = engine;
  return ok();
}

int ising_sweep_blocks(ising_ctx* c, int n_sweeps, int measure_every, int block, int block_every) {
  if (int st = check_ctx(c)) return st;
  if (n_sweeps < 0 || block_every < 0) return fail(ISING_EINVAL, "negative count");
  if (block_every == 0) return ising_sweep(c, n_sweeps, measure_every);
  for (int k = 0; k < n_sweeps; ++k) {
    if (int st = ising_sweep(c, 1, measure_every)) return st;
    if ((c->sweep % block_every) == 0)
      if (int st = ising_block_pass(c, 1, block)) return st;
  }
  return ok();
}

namespace {

// parent (L*L uint32) and mark (L*L bytes) for the cluster steps, on first use
int cluster_scratch(ising_ctx* c) {
  if (c->sw_parent) return ISING_OK;
  void* p = nullptr;
  if (int st = dev_alloc(&p, (size_t)c->N() * sizeof(uint32_t))) return st;
  c->sw_parent = (uint32_t*)p;
  if (int st = dev_alloc(&p, (size_t)c->N())) return st;
  c->sw_flip = (uint8_t*)p;
  return ISING_OK;
}

// floor((1 - e^{-2 beta}) 2^32), clamped: the bond probability of both cluster methods
uint32_t bond_threshold(double beta) {
  const double pb = 1.0 - std::exp(-2.0 * beta);
  const double tf = std::floor(pb * 4294967296.0);
  return tf >= 4294967295.0 ? 0xffffffffu : (tf <= 0.0 ? 0u : (uint32_t)tf);
}

int cluster_checks(ising_ctx* c, int64_t counter, int n_steps, int measure_every) {
  if (c->layout != ISING_LAYOUT_BITS) return fail(ISING_EINVAL, "cluster steps need the packed layout");
  if (n_steps < 0 || measure_every < 0) return fail(ISING_EINVAL, "negative count");
  if (counter + n_steps >= ((int64_t)1 << 32)) return fail(ISING_EINVAL, "step counter overflow");
  if ((int64_t)c->L * c->L >= ((int64_t)1 << 32)) return fail(ISING_EINVAL, "lattice too large");
  return ISING_OK;
}

constexpr int kClusterPersistMaxL = 768;

// Whether cluster steps on this context run as one persistent kernel per call.
bool cluster_persistent(const ising_ctx* c) {
  if (c->cluster_mode == ISING_CLUSTER_PERSISTENT) return true;
  if (c->cluster_mode == ISING_CLUSTER_KERNELS || c->cluster_mode == ISING_CLUSTER_GRAPH) return false;
  // measured on GB300 at beta_c: one launch wins up to L = 512 (70 vs 76 us per
  // step), the kernel-per-phase path at L = 1024 (137 vs 189 us)
  return c->L < kClusterPersistMaxL;
}

// n persistent-kernel cluster steps from step0, records included.
int cluster_persist_run(ising_ctx* c, bool wolff, int64_t step0, int n, int measure_every) {
  if (n <= 0) return ISING_OK;
  if (!c->cluster_gctl) {
    void* p = nullptr;
    if (int st = dev_alloc(&p, sizeof(GridCtl))) return st;
    c->cluster_gctl = (GridCtl*)p;
    CUDA_TRY(cudaMemsetAsync(c->cluster_gctl, 0, sizeof(GridCtl), c->stream));
  }
  Timed tm(c);
  cudaError_t e = launch_cluster_persist(c->lat(c->cur), wolff, (uint32_t)step0, n, measure_every,
                                         bond_threshold(c->beta), c->rng(), c->sw_parent, c->sw_flip, c->rec,
                                         c->rec_count % kRecCap, kRecCap, c->cluster_gctl, c->wolff, c->sms,
                                         c->stream);
  if (int st = launch_result(c, e, "persistent cluster steps")) return st;
  if (measure_every > 0)
    c->rec_count += (step0 + n) / measure_every - step0 / measure_every;
  return ISING_OK;
}

int record_after_step(ising_ctx* c, int64_t t, int measure_every) {
  if (measure_every > 0 && (t + 1) % measure_every == 0) {
    const int64_t slot = c->rec_count % kRecCap;
    if (int st = zero_records(c, c->rec_count, 1)) return st;
    if (int st = launch_result(c, launch_measure_bits(c->lat(c->cur), c->rec + 2 * slot, c->stream), "measure"))
      return st;
    ++c->rec_count;
  }
  return ISING_OK;
}

}  // namespace

int ising_cluster_set_mode(ising_ctx* c, int mode) {
  if (int st = check_ctx(c)) return st;
  if (mode < ISING_CLUSTER_AUTO || mode > ISING_CLUSTER_GRAPH) return fail(ISING_EINVAL, "unknown cluster mode");
  c->cluster_mode = mode;
  return ok();
}

int ising_wolff_set_limits(ising_ctx* c, int max_sites, int max_levels) {
  if (int st = check_ctx(c)) return st;
  if (max_sites < 0 || max_sites > kWolffMaxGrowSites)
    return fail(ISING_EINVAL, "max_sites must be in 0..%d", kWolffMaxGrowSites);
  if (max_levels < 0) return fail(ISING_EINVAL, "max_levels must be >= 0");
  c->wolff_max_sites = max_sites;
  c->wolff_max_levels = max_levels;
  return ok();
}

int ising_wolff_step(ising_ctx* c, int n_steps, int measure_every) {
  if (int st = check_ctx(c)) return st;
  if (int st = cluster_checks(c, c->wolff_steps, n_steps, measure_every)) return st;
  NvtxRange nvtx("ising_wolff_step");
  if (int st = cluster_scratch(c)) return st;
  if (!c->wolff) {
    void* p = nullptr;
    if (int st = dev_alloc(&p, sizeof(WolffCtl))) return st;
    c->wolff = (WolffCtl*)p;
    cudaError_t e = cudaMemsetAsync(c->wolff, 0, sizeof(WolffCtl), c->stream);
    if (e) return fail(ISING_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  }
  if (cluster_persistent(c)) {
    if (int st = cluster_persist_run(c, true, c->wolff_steps, n_steps, measure_every)) return st;
    c->wolff_steps += n_steps;
    return ok();
  }
  const uint32_t thr = bond_threshold(c->beta);
  const RngParams rng = c->rng();
  // default level bound: growth may take about as long as labelling the lattice
  const int levels = c->wolff_max_levels > 0 ? c->wolff_max_levels
                                             : (int)std::min<int64_t>(4096, 32 + (c->N() >> 16));
  if (n_steps > 0 && !c->wolff_graph_broken && c->cluster_mode != ISING_CLUSTER_KERNELS) {
    // graph launches: a step that growth completes runs one kernel
    const BitsLattice lat = c->lat(c->cur);
    WolffGraph& g = c->wolff_graph;
    cudaError_t e = cudaSuccess;
    if (!g.exec || g.planes != lat.planes || g.L != c->L || g.thr != thr || g.replica != rng.replica ||
        g.key0 != rng.key0 || g.key1 != rng.key1 || g.max_sites != c->wolff_max_sites ||
        g.max_levels != levels || g.parent != c->sw_parent || g.mark != c->sw_flip || g.ctl != c->wolff)
      e = wolff_graph_build(&g, lat, thr, rng, c->sw_parent, c->sw_flip, c->wolff_max_sites, levels, c->wolff);
    if (e == cudaSuccess) {
      e = wolff_graph_set_step(c->wolff, (uint32_t)c->wolff_steps, c->stream);
      if (int st = launch_result(c, e, "Wolff step counter")) return st;
      int k = 0;
      if (measure_every == 0)  // no records: kWolffGraphUnroll steps per launch
        for (; k + kWolffGraphUnroll <= n_steps; k += kWolffGraphUnroll) {
          Timed tm(c);
          e = cudaGraphLaunch(g.exec_unrolled, c->stream);
          if (int st = launch_result(c, e, "Wolff step graph")) return st;
          c->launches += kWolffGraphUnroll;  // growth kernels (labelling adds four when it runs)
          c->wolff_steps += kWolffGraphUnroll;
        }
      for (; k < n_steps; ++k) {
        const int64_t t = c->wolff_steps;
        Timed tm(c);
        e = cudaGraphLaunch(g.exec, c->stream);
        if (int st = launch_result(c, e, "Wolff step graph")) return st;
        c->launches += 1;
        if (int st = record_after_step(c, t, measure_every)) return st;
        ++c->wolff_steps;
      }
      return ok();
    }
    cudaGetLastError();
    if (c->cluster_mode == ISING_CLUSTER_GRAPH)
      return fail(ISING_ECUDA, "Wolff step graph: %s", cudaGetErrorString(e));
    c->wolff_graph_broken = true;  // AUTO: separate launches from now on
  }
  for (int k = 0; k < n_steps; ++k) {
    const int64_t t = c->wolff_steps;
    Timed tm(c);
    cudaError_t e = launch_wolff_step(c->lat(c->cur), (uint32_t)t, thr, rng, c->sw_parent, c->sw_flip,
                                      c->wolff_max_sites, levels, c->wolff, c->stream);
    if (int st = launch_result(c, e, "Wolff step")) return st;
    c->launches += 5;  // growth, two labelling kernels, resolve, apply
    if (int st = record_after_step(c, t, measure_every)) return st;
    ++c->wolff_steps;
  }
  return ok();
}

int ising_wolff_stats(ising_ctx* c, int64_t* last_size, int64_t* flipped, int64_t* grown, int64_t* labelled) {
  if (int st = check_ctx(c)) return st;
  WolffCtl h{};
  if (c->wolff)
    if (int st = to_host_sync(c, &h, c->wolff, sizeof(h))) return st;
  if (last_size) *last_size = h.last_size;
  if (flipped) *flipped = (int64_t)h.flipped;
  if (grown) *grown = (int64_t)h.grown;
  if (labelled) *labelled = (int64_t)h.labelled;
  return ok();
}

int ising_sw_step(ising_ctx* c, int n_steps, int measure_every) {
  if (int st = check_ctx(c)) return st;
  if (int st = cluster_checks(c, c->sw_steps, n_steps, measure_every)) return st;
  NvtxRange nvtx("ising_sw_step");
  if (int st = cluster_scratch(c)) return st;
  if (cluster_persistent(c)) {
    if (int st = cluster_persist_run(c, false, c->sw_steps, n_steps, measure_every)) return st;
    c->sw_steps += n_steps;
    return ok();
  }
  const uint32_t thr = bond_threshold(c->beta);
  const RngParams rng = c->rng();
  for (int k = 0; k < n_steps; ++k) {
    const int64_t t = c->sw_steps;
    Timed tm(c);
    cudaError_t e = launch_sw_step(c->lat(c->cur), (uint32_t)t, thr, rng, c->sw_parent, c->sw_flip,
                                   c->stream);
    if (int st = launch_result(c, e, "cluster step")) return st;
    c->launches += 4;  // four kernels per cluster step
    if (int st = record_after_step(c, t, measure_every)) return st;
    ++c->sw_steps;
  }
  return ok();
}

int ising_block_stats(ising_ctx* c, int64_t* proposed, int64_t* accepted) {
  if (int st = check_ctx(c)) return st;
  unsigned long long h[3] = {0, 0, 0};
  if (c->blk_stats)
    if (int st = to_host_sync(c, h, c->blk_stats, sizeof(h))) return st;
  if (proposed) *proposed = (int64_t)h[0];
  if (accepted) *accepted = (int64_t)h[1];
  if (h[2]) return fail(ISING_ETIMEOUT, "a block pass gave up waiting for its tensor-core work");
  return ok();
}

int ising_launch_count(ising_ctx* c, int64_t* launches) {
  if (int st = check_ctx(c)) return st;
  if (!launches) return fail(ISING_EINVAL, "null output pointer");
  *launches = c->launches;
  return ok();
}

}  // extern "C"
