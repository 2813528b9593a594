// Allocation-free variant of the tiled packed sweep: ising_sweep_bits_noalloc.
//
// Who needs it: code that must not call cudaMalloc while it runs -- for
// example a host process that has handed all device memory to its own
// allocator and forbids outside allocations, a real-time loop where an
// allocation (and the implicit device synchronisation cudaMalloc/cudaFree can
// cause) would stall the stream, or a plug-in that is not allowed to own device
// memory.  Such callers own the lattice and the output arrays; this entry point
// brings its own scratch in a statically sized device array instead.
//
// The scratch is one file-scope __device__ array (kScratchBytes, about 8 MiB):
// every GPU that loads libising.so holds it until the process exits.  It is
// shared by all calls on a device and keeps the last call's contents; the parts
// that must start at zero are cleared by every call.  Calls whose work overlaps
// on the GPU (different streams, no ordering between them) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "ising.h"

namespace {

// Scratch layout: [0, kPlaneBytes) second copy of the lattice for the
// ping-pong between launches; then kMaxRecords pairs of u64 accumulators
// (antiparallel bonds, up spins) for the E/M records.
constexpr int kMaxL = 8192;
constexpr size_t kPlaneBytes = (size_t)2 * kMaxL * (kMaxL / 64) * sizeof(uint32_t);  // 8 MiB
constexpr int kMaxRecords = 4096;
constexpr size_t kRecordBytes = (size_t)kMaxRecords * 2 * sizeof(unsigned long long);
constexpr size_t kScratchBytes = kPlaneBytes + kRecordBytes;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up with that device
// current on the first call there and kept for the process.  A cudaDeviceReset
// (or a reset of the primary context) reloads the module and leaves the kept
// address stale; callers that reset a device must not call this entry point on
// it afterwards.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

__global__ void k_records_to_em(const unsigned long long* __restrict__ rec, int n, long long N,
                                int64_t* __restrict__ E, int64_t* __restrict__ M) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    E[i] = 2 * (long long)rec[2 * i] - 2 * N;
    M[i] = 2 * (long long)rec[2 * i + 1] - N;
  }
}

int err(int code, const char* msg) {
  ising::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" int ising_sweep_bits_noalloc(const uint32_t* dev_in, uint32_t* dev_out, int L,
                                        double beta, uint64_t seed, uint32_t replica,
                                        int64_t sweep0, int n_sweeps, int measure_every,
                                        int64_t* dev_E, int64_t* dev_M, int sweeps_per_launch,
                                        void* stream) {
  ising::set_last_error("");
  if (!dev_in || !dev_out) return err(ISING_EINVAL, "null lattice buffer");
  if (L < 256 || L % 256 != 0 || L > kMaxL)
    return err(ISING_EINVAL, "L must be a multiple of 256 and at most 8192 (the static scratch "
                             "holds one 8192 x 8192 packed lattice)");
  if (n_sweeps < 0 || measure_every < 0) return err(ISING_EINVAL, "negative sweep count");
  if (sweep0 < 0 || sweep0 + n_sweeps >= ((int64_t)1 << 32))
    return err(ISING_EINVAL, "sweep counter out of range");
  if (sweeps_per_launch < 1 || sweeps_per_launch > ising::kMaxSweepsPerLaunch)
    return err(ISING_EINVAL, "sweeps_per_launch must be in 1..8");
  uint32_t t4 = 0, t8 = 0;
  if (ising_thresholds(beta, &t4, &t8) != ISING_OK) return err(ISING_EINVAL, "beta must be finite and > 0");
  int n_rec = 0;
  int64_t first_t = -1;
  if (measure_every > 0)
    for (int64_t t = sweep0; t < sweep0 + n_sweeps; ++t)
      if ((t + 1) % measure_every == 0) {
        if (first_t < 0) first_t = t;
        ++n_rec;
      }
  if (n_rec > kMaxRecords) return err(ISING_EINVAL, "more than 4096 records in one call");
  if (n_rec > 0 && (!dev_E || !dev_M)) return err(ISING_EINVAL, "null E/M output arrays");

  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return err(ISING_ECUDA, cudaGetErrorString(e));
  uint32_t* scratch_planes = (uint32_t*)base;
  unsigned long long* rec = (unsigned long long*)((unsigned char*)base + kPlaneBytes);
  cudaStream_t s = (cudaStream_t)stream;
  const int Wc = L / 64;
  const size_t bytes = (size_t)2 * L * Wc * sizeof(uint32_t);

  if (n_rec > 0) {
    e = cudaMemsetAsync(rec, 0, (size_t)n_rec * 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return err(ISING_ECUDA, cudaGetErrorString(e));
  }
  const ising::RngParams rng = ising::make_rng(seed, replica, t4, t8);
  // Tile shape: 64-row strips, 32-word (2048-column) tiles where they divide.
  const int tile_rows = L / 64;
  const int tile_words = Wc % 32 == 0 ? 32 : (Wc % 16 == 0 ? 16 : (Wc % 8 == 0 ? 8 : 4));
  const uint32_t* src = dev_in;
  int launch = 0;
  for (int64_t t = sweep0; t < sweep0 + n_sweeps; t += sweeps_per_launch, ++launch) {
    const int kk = (int)std::min<int64_t>(sweeps_per_launch, sweep0 + n_sweeps - t);
    ising::RecordSlots slots;
    for (int i = 0; i < ising::kMaxSweepsPerLaunch; ++i) {
      const int64_t tt = t + i;
      slots.slot[i] = (i < kk && measure_every > 0 && (tt + 1) % measure_every == 0)
                          ? (int)((tt - first_t) / measure_every)
                          : -1;
    }
    uint32_t* dst = (launch % 2 == 0) ? scratch_planes : dev_out;
    const ising::BitsLattice in{const_cast<uint32_t*>(src), L, Wc, Wc};
    e = ising::launch_tiled_sweep_bits(in, dst, rng, (uint32_t)t, kk, slots, rec, tile_rows,
                                       tile_words, 0, 256, s);
    if (e != cudaSuccess) return err(ISING_ECUDA, cudaGetErrorString(e));
    src = dst;
  }
  if (src != dev_out) {
    e = cudaMemcpyAsync(dev_out, src, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return err(ISING_ECUDA, cudaGetErrorString(e));
  }
  if (n_rec > 0) {
    k_records_to_em<<<(n_rec + 255) / 256, 256, 0, s>>>(rec, n_rec, (long long)L * L, dev_E, dev_M);
    e = cudaGetLastError();
    if (e != cudaSuccess) return err(ISING_ECUDA, cudaGetErrorString(e));
  }
  return ISING_OK;
}
