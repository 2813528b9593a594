// Internal launchers shared by the C-ABI layer (api.cu) and the kernel files.
// Every launcher enqueues on `stream` and returns the launch status.
#pragma once
#include <atomic>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>

namespace ising {

// NVTX range for the lifetime of the object (profiler timelines; a no-op when
// no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// Per-sweep record slots for one launch that covers up to kMaxSweepsPerLaunch
// sweeps: slot[s] >= 0 is the index (in units of 2 x u64: anti-bond count,
// up-spin count) where sweep s of the launch adds its observables; -1 = none.
constexpr int kMaxSweepsPerLaunch = 8;
struct RecordSlots {
  int slot[kMaxSweepsPerLaunch];
};

struct BitsLattice {
  uint32_t* planes;  // [2][L][pitch] words; colour c plane at planes + c * L * pitch
  int L;             // even, >= 4
  int Wc;            // words per colour row = ceil(L / 64)
  int pitch;         // row pitch in words (>= Wc)
};

struct RngParams {
  uint32_t key0, key1;  // lo32 / hi32 of the seed
  uint32_t replica;
  uint32_t t4, t8;      // thresholds for dE = 4, 8
  // Philox round keys key0 + r W0, key1 + r W1 (r = 0..9), filled by
  // make_rng(); passed by value so device code reads them as constants
  uint32_t rk0[10], rk1[10];
  // per-plane threshold masks: tm4[k] = all ones iff bit 31 - k of t4 is set
  // (likewise tm8), so the bit-serial compare reads them as constants
  uint32_t tm4[32], tm8[32];
};

// Barrier state of a persistent cooperative kernel (ising_device.cuh's
// grid_sync_bounded): arrival count, generation, time-out status.
struct GridCtl {
  unsigned int count;
  unsigned int gen;
  int status;
  int pad;
};

// Per-device memo for launch settings that CUDA keeps per device (a kernel's
// dynamic shared-memory limit, its occupancy): one slot per device ordinal,
// atomic so concurrent host threads may race on it harmlessly.
struct DeviceCache {
  static constexpr int kMaxDevices = 64;
  std::atomic<long long> v[kMaxDevices];
  DeviceCache() {
    for (auto& x : v) x.store(0);
  }
  static int device() {
    int d = 0;
    cudaGetDevice(&d);
    return d >= 0 && d < kMaxDevices ? d : 0;
  }
  long long get() { return v[device()].load(std::memory_order_relaxed); }
  void set(long long x) { v[device()].store(x, std::memory_order_relaxed); }
};

// Unsigned 32-bit division by a divisor fixed per launch, as a multiply-high, an
// add and a shift (Granlund & Montgomery, PLDI 1994, the round-up method):
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, n / d = (mulhi(m, n) + n) >> l,
// exact for every 32-bit n and d >= 1.
struct FastDiv {
  uint32_t d, m, l;
};

__host__ __device__ inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while (((uint64_t)1 << l) < d) ++l;
  const uint64_t m = ((((uint64_t)1 << l) - d) << 32) / d + 1;
  return FastDiv{d, (uint32_t)m, l};
}

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  return (uint32_t)(((uint64_t)__umulhi(f.m, n) + n) >> f.l);
}
#endif

inline RngParams make_rng(uint64_t seed, uint32_t replica, uint32_t t4, uint32_t t8) {
  RngParams p;
  p.key0 = (uint32_t)(seed & 0xffffffffu);
  p.key1 = (uint32_t)(seed >> 32);
  p.replica = replica;
  p.t4 = t4;
  p.t8 = t8;
  for (int k = 0; k < 32; ++k) {
    p.tm4[k] = ((t4 >> (31 - k)) & 1u) ? 0xffffffffu : 0u;
    p.tm8[k] = ((t8 >> (31 - k)) & 1u) ? 0xffffffffu : 0u;
  }
  for (int r = 0; r < 10; ++r) {
    p.rk0[r] = p.key0 + (uint32_t)r * 0x9E3779B9u;
    p.rk1[r] = p.key1 + (uint32_t)r * 0xBB67AE85u;
  }
  return p;
}

// ---- bit layout (k_bits.cu) ----
cudaError_t launch_init_bits(const BitsLattice& lat, const RngParams& rng, cudaStream_t s);
cudaError_t launch_half_sweep_bits(const BitsLattice& lat, const RngParams& rng, int colour,
                                   uint32_t sweep, unsigned long long* rec /* or null */,
                                   int grid, int block, cudaStream_t s);
// Temporal blocking: k sweeps per launch, shared-memory tile with halo.  Reads
// `in`, writes `out` (must differ).  Requires Wc % tile_words == 0,
// tile_words % 4 == 0, pitch == Wc, L % 2 == 0, tile_rows_count <= L.
cudaError_t launch_tiled_sweep_bits(const BitsLattice& in, uint32_t* out, const RngParams& rng,
                                    uint32_t sweep0, int k, const RecordSlots& slots,
                                    unsigned long long* rec_base, int n_tile_rows,
                                    int tile_words, int grid, int block, cudaStream_t s);
size_t tiled_smem_bytes(int L, int k, int n_tile_rows, int tile_words);
// Same contract as launch_tiled_sweep_bits for tile_words in {32, 64} (faster
// variant: one warp per tile row, compaction of undecided words).  grid <= 0:
// one persistent CTA per resident slot.
cudaError_t launch_tiled32_sweep_bits(const BitsLattice& in, uint32_t* out, const RngParams& rng,
                                      uint32_t sweep0, int k, const RecordSlots& slots,
                                      unsigned long long* rec_base, int n_tile_rows,
                                      int tile_words, int grid, cudaStream_t s);
size_t tiled32_smem_bytes(int L, int k, int n_tile_rows, int tile_words);
cudaError_t launch_measure_bits(const BitsLattice& lat, unsigned long long* out2,
                                cudaStream_t s);
cudaError_t launch_unpack_bits(const BitsLattice& lat, int8_t* spins, cudaStream_t s);
cudaError_t launch_pack_bits(const BitsLattice& lat, const int8_t* spins, cudaStream_t s);

// ---- learned block proposal (nn.cu) ----
}  // namespace ising
#include <cuda_bf16.h>
namespace ising {
cudaError_t nn_alloc_weights(__nv_bfloat16** wbf, __nv_bfloat16** w2t);
cudaError_t nn_load_blob(__nv_bfloat16* wbf, __nv_bfloat16* w2t, const void* host_blob,
                         cudaStream_t s);
size_t nn_blob_bytes();
// One colour of one block pass: every block of that colour (at the pass's
// Philox-drawn offset) gets one exact MH block update, in place.
cudaError_t nn_block_pass(uint32_t* planes, int L, int Wc, int B, uint32_t pass, int colour,
                          const RngParams& rng, double beta, const __nv_bfloat16* wbf,
                          const __nv_bfloat16* w2t, unsigned long long* stats, cudaStream_t s);

// The staged proposal (nn_staged.cu): the same two calls for a proposal
// plan built by nnc::nn_upload_plan (nn_common.cuh).
namespace nnc { struct StagedPlan; }
cudaError_t nn_staged_block_pass(uint32_t* planes, int L, int Wc, const nnc::StagedPlan* d_plan, int B,
                                 uint32_t pass, int colour, const RngParams& rng, double beta, int engine,
                                 const __nv_bfloat16* wbf, const __nv_bfloat16* w2t,
                                 unsigned long long* stats, cudaStream_t s);
cudaError_t nn_batch_staged_block_pass(uint32_t* spins, const long long* off, const int* lad_L,
                                       const int* slot_of, const float* beta_of_slot,
                                       const long long* unit0, long long total_units, int n_rep,
                                       int n_beta, const nnc::StagedPlan* d_plan, int colour,
                                       uint32_t pass, const RngParams& rng, int engine,
                                       const __nv_bfloat16* wbf, const __nv_bfloat16* w2t,
                                       unsigned long long* stats, cudaStream_t s);
namespace nnc {
cudaError_t nn_upload_plan(int B, int kind, StagedPlan** d_plan, int* n_net, cudaStream_t s);
}

// One colour of one block pass over every replica of a batch (see nn.cu).
cudaError_t nn_batch_block_pass(uint32_t* spins, const long long* off, const int* lad_L,
                                const int* slot_of, const float* beta_of_slot,
                                const long long* unit0, long long total_units, int n_rep,
                                int n_beta, int B, int colour, uint32_t pass, const RngParams& rng,
                                const __nv_bfloat16* wbf, const __nv_bfloat16* w2t,
                                unsigned long long* stats, cudaStream_t s);

// One Swendsen-Wang step on a packed lattice (sw.cu); parent: L*L uint32 and
// flip: L*L bytes of scratch.
cudaError_t launch_sw_step(const BitsLattice& lat, uint32_t step, uint32_t thr,
                           const RngParams& rng, uint32_t* parent, uint8_t* flip, cudaStream_t s);

// Connected components of the active bonds (sw.cu): bond b active iff its
// spins agree and word (b & 3) of Philox(b >> 2, step, replica, bond_tag << 16)
// is below thr.  Leaves a forest in parent (tiled path: every site points at a
// local root, mark = 2 at local roots); skipped when gate is non-null and *gate == 0.
// step_ptr non-null: the kernels read the step from that device word instead
// (graph replays of a step whose index lives on the device).
bool sw_tiled(int L);
cudaError_t launch_cluster_labels(const BitsLattice& lat, uint32_t step, uint32_t thr, uint32_t bond_tag,
                                  const RngParams& rng, uint32_t* parent, uint8_t* mark,
                                  const uint32_t* gate, cudaStream_t s, const uint32_t* step_ptr = nullptr);

// Wolff single-cluster step state on the device (wolff.cu).
struct WolffCtl {
  uint32_t need_label;   // 1: growth gave up, the labelling kernels run
  uint32_t seed_site;    // this step's seed
  uint32_t last_size;    // sites flipped by the last step
  uint32_t gave_up_run;  // consecutive steps without a completed growth
  unsigned long long flipped;   // sites flipped, all steps
  unsigned long long grown;     // steps completed by growth
  unsigned long long labelled;  // steps completed by labelling
  uint32_t step;                // graph path: index of the next step (the growth kernel advances it)
  uint32_t step_body;           // graph path: index of the step whose labelling runs
};
constexpr int kWolffMaxGrowSites = 16384;
size_t wolff_grow_smem(int max_sites);
// One Wolff step: growth from the seed bounded by max_sites (0: never grow)
// and max_levels, then (gated on ctl->need_label) labelling and the flip.
cudaError_t launch_wolff_step(const BitsLattice& lat, uint32_t step, uint32_t thr, const RngParams& rng,
                              uint32_t* parent, uint8_t* mark, int max_sites, int max_levels, WolffCtl* ctl,
                              cudaStream_t s);
// The same step as a CUDA graph: the growth kernel sets the condition of an
// IF node whose body holds the labelling, resolve and apply kernels, so a step
// that growth completes launches none of them.  The step index is ctl->step
// (set it with wolff_graph_set_step); the growth kernel advances it.  exec runs
// one step, exec_unrolled kWolffGraphUnroll steps in a row.  Built for one set
// of arguments; the caller rebuilds it when they change.
constexpr int kWolffGraphUnroll = 8;
struct WolffGraph {
  cudaGraph_t graph = nullptr, graph_unrolled = nullptr;
  cudaGraphExec_t exec = nullptr, exec_unrolled = nullptr;
  // the arguments the graph was built for
  const uint32_t* planes = nullptr;
  int L = 0, max_sites = 0, max_levels = 0;
  uint32_t thr = 0, replica = 0, key0 = 0, key1 = 0;
  uint32_t* parent = nullptr;
  uint8_t* mark = nullptr;
  WolffCtl* ctl = nullptr;
};
cudaError_t wolff_graph_build(WolffGraph* g, const BitsLattice& lat, uint32_t thr, const RngParams& rng,
                              uint32_t* parent, uint8_t* mark, int max_sites, int max_levels,
                              WolffCtl* ctl);
void wolff_graph_free(WolffGraph* g);
cudaError_t wolff_graph_set_step(WolffCtl* ctl, uint32_t step, cudaStream_t s);

// Cluster steps as one persistent cooperative kernel (cluster_persist.cu):
// n_steps Swendsen-Wang (wolff = false) or Wolff steps from step0, each a
// connected-component labelling of the whole lattice; records (E, M) after
// step t when (t + 1) % measure_every == 0 into rec slots (rec0 + k) % rec_cap.
// Grid barriers give up after kClusterSpinLimit cycles and set gctl->status.
constexpr long long kClusterSpinLimit = 4000000000LL;  // ~2 s of SM clock per barrier
cudaError_t launch_cluster_persist(const BitsLattice& lat, bool wolff, uint32_t step0, int n_steps,
                                   int measure_every, uint32_t thr, const RngParams& rng, uint32_t* parent,
                                   uint8_t* mark, unsigned long long* rec, long long rec0, long long rec_cap,
                                   GridCtl* gctl,
                                   WolffCtl* wctl, int sms, cudaStream_t s);

// Sets the message returned by ising_last_error() on the calling thread.
void set_last_error(const char* msg);

// ---- int8 layout (k_i8.cu) ----
cudaError_t launch_init_i8(int8_t* s, int L, const RngParams& rng, cudaStream_t st);
// Whole lattice resident in one CTA's shared memory; n sweeps in one launch.
cudaError_t launch_resident_sweep_i8(int8_t* s, int L, const RngParams& rng, uint32_t sweep0,
                                     int n_sweeps, int measure_every, uint32_t rec_first_t,
                                     long long rec_slot0, long long rec_cap,
                                     unsigned long long* rec, cudaStream_t st);
size_t resident_i8_smem_bytes(int L);
cudaError_t launch_half_sweep_i8(int8_t* s, int L, const RngParams& rng, int colour,
                                 uint32_t sweep, unsigned long long* rec, cudaStream_t st);
cudaError_t launch_measure_i8(const int8_t* s, int L, unsigned long long* out2, cudaStream_t st);

}  // namespace ising
