/*
 * ising.h -- C-ABI of the GB300 checkerboard Metropolis library (libising.so).
 *
 * The library runs the data-parallel hot path of arXiv 2402.06415 ("Many-body
 * computing on Field Programmable Gate Arrays"): the Monte Carlo sweep that the
 * paper splits into two sublattices updated alternately (Results A, Fig. 2),
 * with the three per-site steps of its Supplementary MC details: (1) draw a
 * uniform decision number, (2) compute the local energy change dE and
 * P(dE) = exp(-beta dE), (3) accept iff p < P.  The model is the 2D
 * square-lattice Ising ferromagnet (J = 1, h = 0, periodic boundaries), where
 * dE = 2 s_x sum_n s_n (the integer analogue of the paper's Eq. S1).
 *
 * Conventions for every entry point:
 *  - Return value: an ising_status; ISING_OK (0) on success, a negative code
 *    otherwise.  On error a message is available from ising_last_error() (per
 *    calling thread) and no allocation made by the failing call is leaked.
 *  - Device work is enqueued on the CUDA stream given to ising_create (a
 *    cudaStream_t passed as void*; NULL = the legacy default stream) and calls
 *    return before it finishes, except where a call says it synchronises.
 *  - Host pointers are caller-owned and only read/written during the call.
 *    Device pointers (the *_device variants) must be device memory of the
 *    context's device; they are used asynchronously on the context's stream.
 *  - A context is not thread-safe: serialise calls on one context.
 *  - Spin layouts:
 *      int8 spins:  L*L int8 values +1/-1, row-major, index y*L + x.
 *      packed bits: 2*L*Wc uint32 words, Wc = ceil(L/64); word [c][y][w] holds
 *                   the colour-c sites of row y with colour index
 *                   j = 32w .. 32w+31 (colour c = (x+y)&1, x = 2j + ((y+c)&1)),
 *                   bit (j & 31) set means +1; bits with j >= L/2 are zero.
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = the 64-bit
 *    seed, counter = (group, sweep, replica, tag|colour|block); a site's
 *    uniform u is assembled from bit (j & 31) of 32 plane words (plane k gives
 *    bit 31-k).  The flip rule is: n_anti >= 2 antiparallel neighbours -> flip;
 *    n_anti == 1 -> flip iff u < floor(exp(-4 beta) 2^32);
 *    n_anti == 0 -> flip iff u < floor(exp(-8 beta) 2^32).  Results are
 *    bit-identical across kernels, layouts and launch shapes.
 */
#ifndef ISING_H
#define ISING_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ising_ctx ising_ctx;

typedef enum {
  ISING_OK = 0,
  ISING_EINVAL = -1,    /* bad argument (message says which) */
  ISING_ENOMEM = -2,    /* device or host allocation failed */
  ISING_ECUDA = -3,     /* a CUDA call failed (message has the CUDA error) */
  ISING_ETIMEOUT = -4,  /* a bounded device wait ran out */
  ISING_EINTERNAL = -5  /* internal consistency check failed */
} ising_status;

typedef enum { ISING_LAYOUT_I8 = 0, ISING_LAYOUT_BITS = 1 } ising_layout;

typedef enum {
  ISING_KERNEL_AUTO = 0,     /* pick per lattice (tiled if it applies, else half) */
  ISING_KERNEL_HALF = 1,     /* one launch per half sweep, spins in global memory */
  ISING_KERNEL_TILED = 2,    /* packed layout: shared-memory tile + halo, k sweeps per launch */
  ISING_KERNEL_RESIDENT = 3  /* int8 layout: whole lattice in one CTA's shared memory */
} ising_kernel;

/* Create a context for one L x L lattice (Results A; the sweep of Fig. 2b).
 * L: even, 4 <= L <= 65536.  beta: inverse temperature, finite and > 0.
 * layout: ising_layout.  stream: cudaStream_t (borrowed, may be NULL).
 * The lattice starts all -1 with seed 0, replica 0, sweep counter 0.
 * Allocates the lattice (and, for the tiled kernel, a second ping-pong copy)
 * plus a record ring of 65536 (E, M) entries on the current CUDA device.
 * Errors: EINVAL (arguments), ENOMEM, ECUDA. */
int ising_create(ising_ctx** out, int L, double beta, int layout, void* stream);

/* Seeded random start (independent +-1 with probability 1/2, one Philox bit
 * per site, tag INIT); resets the sweep counter to 0 and clears the records.
 * Async. */
int ising_seed(ising_ctx* ctx, uint64_t seed);

/* Set the Philox key (the seed) without touching the spins, the sweep counter
 * or the records: with ising_set_spins / ising_set_bits and
 * ising_set_sweep_counter this resumes a saved chain bit-exactly. */
int ising_set_key(ising_ctx* ctx, uint64_t seed);

/* Replica id r used in the Philox counter (default 0).  Async-safe (host). */
int ising_set_replica(ising_ctx* ctx, uint32_t replica);

/* Set beta (> 0, finite); recomputes the integer thresholds on the host. */
int ising_set_beta(ising_ctx* ctx, double beta);

/* Set the sweep counter t of the next sweep (for resuming a chain). */
int ising_set_sweep_counter(ising_ctx* ctx, int64_t t);

/* Current seed, replica and sweep counter. */
int ising_get_state(ising_ctx* ctx, uint64_t* seed, uint32_t* replica, int64_t* sweep);

/* Run n_sweeps full sweeps (colour 0 then colour 1; Results A / Fig. 2b)
 * starting at the current sweep counter t.  After every sweep t with
 * (t + 1) % measure_every == 0 the energy E = -sum s s' (2 L^2 bonds) and
 * magnetisation M = sum s are recorded (measure_every = 0: no records).
 * n_sweeps >= 0, measure_every >= 0, t + n_sweeps < 2^32.  Async. */
int ising_sweep(ising_ctx* ctx, int n_sweeps, int measure_every);

/* E and M of the current configuration.  Synchronises the stream. */
int ising_measure(ising_ctx* ctx, int64_t* E, int64_t* M);

/* Number of records taken since the last ising_seed (the ring keeps the last
 * 65536). */
int ising_series_count(ising_ctx* ctx, int64_t* count);

/* Copy the last n records (oldest first) into host arrays E_out[n], M_out[n].
 * 0 <= n <= min(count, 65536).  Synchronises the stream. */
int ising_series(ising_ctx* ctx, int64_t* E_out, int64_t* M_out, int n);

/* int8 spins to/from host memory (layout above).  get synchronises; set
 * copies synchronously from the host buffer and validates +-1 values. */
int ising_get_spins(ising_ctx* ctx, int8_t* host_out);
int ising_set_spins(ising_ctx* ctx, const int8_t* host_in);

/* Packed words to/from host memory (layout above, 2*L*Wc uint32).  get
 * synchronises; set copies synchronously and zeroes unused bits. */
int ising_get_bits(ising_ctx* ctx, uint32_t* host_out);
int ising_set_bits(ising_ctx* ctx, const uint32_t* host_in);

/* Same as get/set_spins / get/set_bits with device buffers, async on the stream. */
int ising_get_spins_device(ising_ctx* ctx, int8_t* dev_out);
int ising_set_spins_device(ising_ctx* ctx, const int8_t* dev_in);
int ising_get_bits_device(ising_ctx* ctx, uint32_t* dev_out);
int ising_set_bits_device(ising_ctx* ctx, const uint32_t* dev_in);

/* Words per colour row for lattice size L (ceil(L/64)). */
int ising_words_per_row(int L);

/* Choose the sweep kernel and its launch shape.  kernel: ising_kernel.
 * sweeps_per_launch k (tiled: 1..8), tile_rows = number of row strips the
 * lattice is cut into (tiled), tile_words = words per tile row (tiled; must
 * divide Wc and be a multiple of 4), grid/block: launch shape (0 = default).
 * The choice never changes results, only speed.  EINVAL if the kernel does
 * not apply to this lattice/layout. */
int ising_set_kernel(ising_ctx* ctx, int kernel, int sweeps_per_launch, int tile_rows,
                     int tile_words, int grid, int block);

/* The kernel configuration in use (after AUTO resolution). */
int ising_get_kernel(ising_ctx* ctx, int* kernel, int* sweeps_per_launch, int* tile_rows,
                     int* tile_words, int* grid, int* block);

/* Integer thresholds floor(exp(-beta dE) 2^32) for dE = 4 and 8 (Supplementary
 * MC step 2), computed in double on the host. */
int ising_thresholds(double beta, uint32_t* t4, uint32_t* t8);

/* Launch accounting and live kernel timing.  With timing enabled, every sweep
 * kernel launch is bracketed by CUDA events on the context's stream;
 * ising_kernel_time synchronises and returns the summed device time (ms) and
 * launch count of the sweep kernels since timing was last enabled.
 * ising_launch_count returns all kernels this context launched so far. */
int ising_set_timing(ising_ctx* ctx, int enable);
int ising_kernel_time(ising_ctx* ctx, double* ms, int64_t* launches);
int ising_launch_count(ising_ctx* ctx, int64_t* launches);

/* Allocation-free sweep (no counterpart in the paper: an interface for
 * callers that may not allocate device memory while they run, e.g. a host
 * application that gives all device memory to its own allocator, a real-time
 * loop where cudaMalloc/cudaFree would stall the stream, or a plug-in that may
 * not own device memory).  Runs n_sweeps sweeps of the packed tiled kernel on
 * a caller-owned lattice: dev_in and dev_out are device buffers in the packed
 * layout (2*L*(L/64) uint32, may be the same buffer), the sweep counter starts
 * at sweep0, and after every sweep t with (t+1) % measure_every == 0 the E and
 * M of that sweep go to the device arrays dev_E[i], dev_M[i] (i = record index
 * in this call; measure_every = 0: no records, dev_E/dev_M may be NULL).
 * sweeps_per_launch: 1..8.  Results are bit-identical to ising_sweep with the
 * tiled kernel.
 * Allocates nothing: scratch (a second lattice copy and the record
 * accumulators) is a static device array of about 8 MiB that every GPU loading
 * libising.so holds until the process exits.  Hence L must be a multiple of
 * 256 and at most 8192, and at most 4096 records per call (EINVAL otherwise).
 * The first call on a device looks up the array's device address (once per
 * device, current device); make that first call before any stream capture.
 * A cudaDeviceReset of that device leaves the kept address stale: do not call
 * this entry point on a device after resetting it.
 * All calls on a device share the array and leave their contents in it (the
 * record accumulators are cleared at the start of every call); calls that
 * overlap on the GPU race on it, so order them on one stream.  Async on
 * `stream`; errors: EINVAL, ECUDA (message from ising_last_error()). */
int ising_sweep_bits_noalloc(const uint32_t* dev_in, uint32_t* dev_out, int L, double beta,
                             uint64_t seed, uint32_t replica, int64_t sweep0, int n_sweeps,
                             int measure_every, int64_t* dev_E, int64_t* dev_M,
                             int sweeps_per_launch, void* stream);

/* ------------------------------------------------------------------------
 * Batched replicas with parallel tempering (no counterpart in the paper,
 * whose MC runs one chain per lattice; the sweep each replica runs is the
 * paper's checkerboard sweep, Results A / Supplementary MC steps 1-3).
 * n_ladders ladders of n_beta replicas each; ladder l has lattice size L[l]
 * (even, 4..1024) and replica i of ladder l uses Philox replica id
 * l * n_beta + i.  betas (ascending, > 0) are the temperature slots shared by
 * all ladders.  Every sweep runs each replica at the beta of its slot; after
 * every sweep t with (t + 1) % pt_every == 0 each ladder performs exchange step
 * n = (t + 1) / pt_every - 1 over the slot pairs (a, a+1), a = n % 2, n % 2 + 2,
 * ...: the two configurations swap slots iff u < floor(min(1,
 * exp[(beta_a - beta_{a+1}) (E_a - E_{a+1})]) 2^32), u = word 0 of Philox
 * counter (a, n, l, PT << 16) under the seed key.  A run is one persistent
 * cooperative kernel launch; the state lives on the device.
 * ------------------------------------------------------------------------ */
typedef struct ising_batch ising_batch;

/* Create (device allocations for all replicas) and seed with 0.  stream:
 * cudaStream_t, borrowed.  Errors: EINVAL, ENOMEM, ECUDA. */
int ising_batch_create(ising_batch** out, int n_ladders, const int* L, int n_beta,
                       const double* betas, int pt_every, void* stream);

/* Seeded random start of every replica (the INIT stream of its replica id),
 * identity slot assignment, zero counters, sweep counter 0.  Synchronises. */
int ising_batch_seed(ising_batch* b, uint64_t seed);

/* Work decomposition: replica words per work item (16..16384, default 512),
 * threads per CTA (32, 64, 128 or 256; 0 = 256), grid (0 = all resident CTAs).
 * Never changes results.  Drops a captured graph. */
int ising_batch_set_kernel(ising_batch* b, int words_per_item, int threads, int grid);

/* Keep E, M and the slot of every replica at each exchange step in a device
 * ring of `capacity` steps (0 = off).  Drops a captured graph. */
int ising_batch_set_series(ising_batch* b, int capacity);

/* Run n_sweeps sweeps (with the exchange steps that fall in them) in one
 * persistent launch, or by replaying the graph captured for this n_sweeps.
 * Async; check ising_batch_status for a barrier timeout. */
int ising_batch_run(ising_batch* b, int n_sweeps);

/* Capture one run of n_sweeps into a CUDA graph; later ising_batch_run(b,
 * n_sweeps) calls replay it (the sweep counter lives on the device, so every
 * replay continues the chain). */
int ising_batch_capture(ising_batch* b, int n_sweeps);

/* Synchronise and read the device status word (0 ok; ETIMEOUT if a grid
 * barrier ran out of its ~2 s budget, EINTERNAL on an impossible energy
 * difference) and the device sweep counter. */
int ising_batch_status(ising_batch* b, int* status, int64_t* sweep);

/* Host copies of the slot assignment perm[l * n_beta + a] (replica index at
 * slot a of ladder l) and of E, M of every replica after its last round. */
int ising_batch_state(ising_batch* b, int32_t* perm, int64_t* E, int64_t* M);

/* Accepted and attempted exchanges of pair (a, a+1) of ladder l at index
 * l * n_beta + a (host arrays of n_ladders * n_beta). */
int ising_batch_swap_counts(ising_batch* b, int64_t* accepts, int64_t* attempts);

/* The last n_steps recorded exchange steps, oldest first: E, M and slot of
 * every replica (host arrays of n_steps * n_ladders * n_beta). */
int ising_batch_series(ising_batch* b, int n_steps, int32_t* E, int32_t* M, int16_t* slot);

/* int8 spins (L*L, row-major) of replica i of ladder l.  Synchronises. */
int ising_batch_get_spins(ising_batch* b, int ladder, int replica, int8_t* host_out);

/* Learned block proposal on every replica of the batch (the same move as
 * ising_block_pass, per replica at the beta of its current slot, Philox replica
 * id = its batch replica id).  Load the BF16 blob first; then each pass updates
 * all squares of colour 0, then colour 1, of every replica.  Async. */
int ising_batch_nn_load(ising_batch* b, const void* bf16_weights, size_t bytes);
int ising_batch_block_pass(ising_batch* b, int n_passes, int block);
int ising_batch_block_stats(ising_batch* b, int64_t* proposed, int64_t* accepted);
/* Proposal family of the batch's block passes (as ising_set_proposal). */
int ising_batch_set_proposal(ising_batch* b, int kind);
/* Layer-2 engine of the batch's staged block passes (as ising_set_nn_engine). */
int ising_batch_set_nn_engine(ising_batch* b, int engine);

/* Failure-path self test (no counterpart in the paper): launches one kernel
 * that waits, with the same bounded spin as the batch grid barrier, on a device
 * flag that nothing sets.  The wait gives up after timeout_s (0 < t <= 10) of
 * SM clock cycles; the call then returns ISING_ETIMEOUT with *device_status = 1,
 * and the CUDA context stays usable.  Synchronises. */
int ising_selftest_wait(double timeout_s, int* device_status);

/* Work items, CTAs used, host-side sweep counter. */
int ising_batch_info(ising_batch* b, int* n_items, int* grid, int64_t* sweep);

/* Free everything (NULL-safe; synchronises). */
int ising_batch_destroy(ising_batch* b);

/* ------------------------------------------------------------------------
 * Learned block proposal (no counterpart in the paper; an extra exact move of
 * the same chain).  A block pass draws an offset (ox, oy) in [0, block)^2 from
 * Philox (tag BLK_OFFSET), tiles the lattice into block x block squares at that
 * offset, and updates all squares of block-colour 0, then of colour 1 (colour =
 * (bx + by) % 2; squares of one colour share no bond).  Each square's interior
 * is resampled from a CNN conditioned on the four edges of the ring around it
 * and accepted with the exact Metropolis-Hastings probability
 * min(1, exp(-beta dE) q(old) / q(new)), q the quantised proposal density.
 * Network: 3 x 3 convolutions 2 -> 32 -> 32 -> 1 channels, ReLU after the first
 * two, zero padding on the (block+2)^2 frame; channel 0 = ring-edge spins,
 * channel 1 = ring-edge mask.  BF16 weights, FP32 accumulation (tensor cores).
 * Weight blob (10145 bf16, this order): W1[32][2][3][3], b1[32],
 * W2[32][32][3][3], b2[32], W3[1][32][3][3], b3[1].
 * ------------------------------------------------------------------------ */

/* Load the BF16 weight blob (bytes = 2 * 10145) into the context.  Synchronises. */
int ising_nn_load(ising_ctx* ctx, const void* bf16_weights, size_t bytes);

/* Proposal family of the block passes (no counterpart in the paper).
 * ONESHOT (default): every interior site drawn at once from the CNN logits
 * conditioned on the ring edges (the description above).
 * STAGED: the interior is drawn site by site in stages, each conditioned on
 * the ring edges and the sites drawn before it (an autoregressive proposal):
 *   site classes local to the square (i = row, j = column, 0-based):
 *   0: i, j even; 1: i, j odd, ((i-1)/2 + (j-1)/2) even; 2: other i, j odd;
 *   3: i + j odd.  Depth d = min(i, j, B-1-i, B-1-j).  For band k = d / 2 =
 *   0, 1, ...: a NETWORK stage with the band's undrawn class-0 sites, one with
 *   its class-1 sites, then repeatedly an EXACT stage with every undrawn site
 *   whose four neighbours are known, else with every undrawn class-2 site whose
 *   unknown neighbours have all their other neighbours known, until neither
 *   applies; a last such closure draws the rest (ising_proposal_schedule).
 *   Network stage: the CNN on channel 0 = known spins (0 elsewhere), channel
 *   1 = known mask.  Exact stage: logit = sum over known neighbours n of
 *   2 beta s_n + sum over unknown neighbours n of
 *   log cosh(beta (h_n + 1)) - log cosh(beta (h_n - 1)), h_n the sum of n's
 *   other neighbours: the exact conditional with n summed out.
 *   Every stage draws s_i = +1 iff u_i < P_i (P_i the quantised sigmoid, same
 *   Philox draws as ONESHOT); q = product over all stages; q(old) by the same
 *   stages on the current interior.  The MH test is unchanged.
 * Applies to later ising_block_pass / ising_sweep_blocks calls. */
enum { ISING_PROPOSAL_ONESHOT = 0, ISING_PROPOSAL_STAGED = 1 };
int ising_set_proposal(ising_ctx* ctx, int kind);

/* Engine of the STAGED proposal's second convolution (32 -> 32 channels, the
 * contraction that dominates its cost); results agree to FP32 rounding order.
 * MMA_SYNC (default): warp-level mma.sync m16n8k16, FP16 operands, FP32
 * accumulators in registers, on exactly the frame positions the stage needs.
 * TCGEN05: tcgen05.mma with M = 128 frame positions x N = 32 channels, FP16
 * operands staged in shared memory, FP32 accumulators in tensor memory (64 of
 * its columns per tile, at most 3 tiles), issued by one thread and completed
 * through an mbarrier whose wait is bounded (about 1 s of SM clock): on a time
 * out the square is rejected and ising_block_stats returns ISING_ETIMEOUT.
 * On the 18 x 18 frames of 16 x 16 squares the tile granularity costs more
 * than the tensor pipe saves (the default is the faster engine there).
 * ISING_EINVAL for other values.  Applies to later block passes. */
enum { ISING_NN_ENGINE_MMA_SYNC = 0, ISING_NN_ENGINE_TCGEN05 = 1 };
int ising_set_nn_engine(ising_ctx* ctx, int engine);

/* The stage schedule of a proposal for squares of side block (2..16, even):
 * stage_of_site[block * block] (row-major interior index -> stage) and
 * stage_exact[n] (1 = exact stage, 0 = network stage), host arrays of at
 * least block^2 and `capacity` entries; *n_stages = number of stages.
 * Host only (no GPU needed).  ISING_EINVAL if capacity is too small. */
int ising_proposal_schedule(int block, int kind, uint8_t* stage_of_site, uint8_t* stage_exact,
                            int capacity, int* n_stages);

/* n_passes block passes with squares of side `block` (2, 4, 8 or 16; L must be
 * a multiple of 2 * block; packed layout).  Async. */
int ising_block_pass(ising_ctx* ctx, int n_passes, int block);

/* Interleaved schedule: n_sweeps plain sweeps (records as in ising_sweep); after
 * every sweep t with (t + 1) % block_every == 0 one block pass with squares of
 * side `block` (block_every = 0: plain sweeps only).  Async. */
int ising_sweep_blocks(ising_ctx* ctx, int n_sweeps, int measure_every, int block, int block_every);

/* Swendsen-Wang cluster steps on the packed lattice (no counterpart in the
 * paper beyond its pointer to cluster methods; Swendsen & Wang 1987).  Step n:
 * bonds between equal spins are active iff u < floor((1 - exp(-2 beta)) 2^32),
 * u = word (b & 3) of Philox(b >> 2, n, replica, SW_BOND << 16) for bond
 * b = 2 (y L + x) + dir (dir 0: to x+1, 1: to y+1); each connected cluster flips
 * iff bit 31 of word (m & 3) of Philox(m >> 2, n, replica, SW_FLIP << 16), m its
 * smallest site index.  Records E, M after every step n with
 * (n + 1) % measure_every == 0 into the same record ring as ising_sweep.  The
 * step counter n is separate from the sweep counter; ising_seed resets it to 0.  Allocates
 * 5 bytes per site of scratch on first use; L = 65536 (2^32 sites) is
 * rejected with ISING_EINVAL.  Async. */
int ising_sw_step(ising_ctx* ctx, int n_steps, int measure_every);

/* How cluster steps (ising_sw_step, ising_wolff_step) run: AUTO = one
 * persistent launch per call for L < 768 (up to 64 x 64 sites one CTA with the
 * lattice in shared memory, else a cooperative grid with three bounded
 * grid-barrier phases per step: runs, unions, flips; a barrier wait gives up
 * after about 2 s and later synchronising calls then fail with ISING_ETIMEOUT;
 * work queued after the timed-out step, sweeps included, ran on a lattice the
 * step left half-updated, so the lattice and its records are undefined until
 * ising_seed, ising_set_spins or ising_set_bits),
 * a few kernels per step from L = 768 (from L = 2048 with tiled labelling in
 * shared memory; Wolff first tries growth from the seed, and its step is one
 * CUDA graph launch (eight steps per launch when nothing is recorded): the
 * growth kernel sets the condition of an IF node that holds the labelling
 * kernels, so a step that growth completes runs one kernel; if the graph
 * cannot be built, AUTO falls back to separate launches
 * whose labelling kernels return at once when growth has completed the step).
 * KERNELS (separate launches) / PERSISTENT / GRAPH (the Wolff graph at any L;
 * Swendsen-Wang steps as KERNELS) force one way.  The chain is the same either
 * way, bit for bit. */
enum { ISING_CLUSTER_AUTO = 0, ISING_CLUSTER_KERNELS = 1, ISING_CLUSTER_PERSISTENT = 2, ISING_CLUSTER_GRAPH = 3 };
int ising_cluster_set_mode(ising_ctx* ctx, int mode);

/* Wolff single-cluster steps (Wolff, PRL 62, 361 (1989)) on the packed layout:
 * the paper's Discussion names cluster algorithms as the next step for its
 * Monte Carlo.  Step n:
 * seed site m = floor(u N / 2^32), u = word 0 of Philox(0, n, replica, 16 << 16);
 * a bond b = 2 (y L + x) + dir between equal spins is active iff
 * u < floor((1 - e^{-2 beta}) 2^32), u = word (b & 3) of
 * Philox(b >> 2, n, replica, 17 << 16); the connected cluster of active bonds
 * holding m flips.  Bit-identical to any sequential growth of the same cluster.
 * The step counter n is separate from the other counters; ising_seed resets it.
 * Shares the 5 bytes per site of scratch of ising_sw_step (allocated on first
 * use); L = 65536 is rejected with ISING_EINVAL.  measure_every > 0 records
 * (E, M) after every such step into the series ring.  Async. */
int ising_wolff_step(ising_ctx* ctx, int n_steps, int measure_every);

/* How a Wolff step of the kernel path (ising_cluster_set_mode) finds its
 * cluster: growth from the seed in one CTA while the cluster has at most
 * max_sites sites (0..16384; 0 = never) and max_levels breadth-first levels
 * (0 = a default that grows with L), otherwise connected components of the
 * whole lattice.  Changes cost only, never the chain. */
int ising_wolff_set_limits(ising_ctx* ctx, int max_sites, int max_levels);

/* Sites flipped by the last Wolff step, by all steps since ising_seed, and how
 * many steps finished by growth and by labelling (synchronises). */
int ising_wolff_stats(ising_ctx* ctx, int64_t* last_size, int64_t* flipped, int64_t* grown,
                      int64_t* labelled);

/* Squares proposed and accepted by this context's block passes (synchronises). */
int ising_block_stats(ising_ctx* ctx, int64_t* proposed, int64_t* accepted);

/* Trainer: FP32 master weights, Adam state and BF16 inference copies of the
 * same network.  Windows are int8 spins of (block+2)^2 sites, row-major: the
 * ring around a block (corners ignored) and its interior (the training target).
 * Loss = mean over windows of sum_i BCE(logit_i, (s_i + 1) / 2). */
typedef struct ising_nn ising_nn;
int ising_nn_param_count(void);
int ising_nn_create(ising_nn** out, int block, int channels, void* stream);
int ising_nn_set_params(ising_nn* nn, const float* host_params, int count);
int ising_nn_get_params(ising_nn* nn, float* host_params, int count);
/* BF16 blob of the current weights, for ising_nn_load (bytes = 2 * 10145). */
int ising_nn_export(ising_nn* nn, void* host_bf16, size_t bytes);
/* Inference logits (BF16 tensor-core path) of count windows on the device:
 * dev_windows [count][(block+2)^2] int8 -> dev_logits [count][block^2] float. */
int ising_nn_logits(ising_nn* nn, const int8_t* dev_windows, int count, float* dev_logits);
/* FP32 loss and gradients (host arrays; grads may be NULL).  Synchronises. */
int ising_nn_loss_grad(ising_nn* nn, const int8_t* dev_windows, int count, float* loss,
                       float* host_grads);
/* One Adam step (lr, betas 0.9 / 0.999, eps 1e-8) on one minibatch. */
int ising_nn_train_step(ising_nn* nn, const int8_t* dev_windows, int count, float lr, float* loss);
/* One Adam step (as ising_nn_train_step) with the caller's gradients
 * (host, count = 10145 floats, C-ABI parameter order) instead of a minibatch's;
 * updates the FP32 master weights and the BF16 inference copy.  Synchronises. */
int ising_nn_apply_grads(ising_nn* nn, const float* host_grads, int count, float lr);
/* Proposal family the trainer fits (default ONESHOT).  STAGED: one training
 * sample per (window, network stage): the stage's known mask on the input,
 * loss terms at the stage's sites; loss = their sum / number of windows
 * (minus the mean log-likelihood of the network stages). */
int ising_nn_set_proposal(ising_nn* nn, int kind);
/* Layer-2 engine of ising_nn_stage_logits / ising_nn_log_q (as
 * ising_set_nn_engine; training keeps its own FP32 path). */
int ising_nn_set_engine(ising_nn* nn, int engine);
/* Training kernel of ising_nn_loss_grad / ising_nn_train_step.
 * FP32 (default): every layer in FP32 on the CUDA cores (gradients to FP32
 * rounding order of the float64 objective).
 * BF16_TC: the 32 -> 32 convolution's forward, input-gradient and
 * weight-gradient contractions on the tensor cores (mma.sync m16n8k16, BF16
 * operands: activations, dL/dz2 and the weights rounded to BF16; FP32
 * accumulation); layers 1 and 3 in FP32.  Same objective, gradients to BF16
 * rounding.  The FP32 master weights and Adam are unchanged.  ISING_EINVAL for
 * other values. */
enum { ISING_NN_TRAIN_FP32 = 0, ISING_NN_TRAIN_BF16_TC = 1 };
int ising_nn_set_train_precision(ising_nn* nn, int precision);
/* Logits of stage `stage` of the trainer's proposal for count windows on the
 * device (BF16 inference path): network stages give the CNN logits, exact
 * stages the exact log-odds at beta, at the stage's sites; other sites 0.
 * dev_windows [count][(block+2)^2] int8 (interior sites drawn after the stage
 * are ignored) -> dev_logits [count][block^2] float.  Async. */
int ising_nn_stage_logits(ising_nn* nn, const int8_t* dev_windows, int count, int stage, double beta,
                          float* dev_logits);
/* Natural log of the quantised proposal density of each window's interior
 * given its ring (the q(old) of a block move), FP32.  Async. */
int ising_nn_log_q(ising_nn* nn, const int8_t* dev_windows, int count, double beta, float* dev_log_q);
int ising_nn_destroy(ising_nn* nn);

/* ------------------------------------------------------------------------
 * 2D XY model: the paper's own Monte Carlo workload (Eq. 1; Supplementary
 * "Detail of the MC calculation for the XY model"; checkerboard of Fig. 2).
 * Spins are unit vectors u = (cos theta, sin theta).  Per site: theta' = 2 pi U1,
 * p = U2 (24-bit uniforms from Philox), dE = -(u' - u) . h, h = sum of the four
 * neighbour vectors (Eq. S1 with its sign corrected), accept iff dE <= 0 or
 * p < exp(-beta dE).  precision: 64 (double, as in the paper) or 32 (float).
 * cos/sin/exp are the library's own Taylor/Cody-Waite routines, so the chain is
 * reproducible bit for bit.  L even, 2..32768.  Records (every measure_every
 * sweeps) hold E = -sum_bonds u.u' and the magnetisation vector, in double.
 * ------------------------------------------------------------------------ */
typedef struct ising_xy ising_xy;
int ising_xy_create(ising_xy** out, int L, double beta, int precision, void* stream);
/* Seeded random start (uniform angles); sweep counter 0; clears records. */
int ising_xy_seed(ising_xy* x, uint64_t seed);
/* n_sweeps sweeps (async). */
int ising_xy_sweep(ising_xy* x, int n_sweeps, int measure_every);
/* Kernel form: 0 automatic (persistent for L <= 256), 1 one launch per half
 * sweep, 2 persistent cooperative kernel (all CTAs co-resident, one launch per
 * ising_xy_sweep call, a bounded grid barrier between half sweeps).  Results
 * are identical in every mode.  If a persistent barrier gives up (after ~2 s)
 * the next synchronising call returns ISING_ETIMEOUT until ising_xy_seed. */
int ising_xy_set_mode(ising_xy* x, int mode);
/* Kernels this context has launched. */
int ising_xy_launch_count(ising_xy* x, int64_t* count);
/* Runs the persistent kernels' grid barrier with one CTA that never arrives;
 * *timed_out = 1 when the others gave up after timeout_s (0 < timeout_s <= 10)
 * as they must.  The context stays usable. */
int ising_selftest_grid_barrier(double timeout_s, int* timed_out);
/* Last n records (oldest first): E, Mx, My (host arrays; any may be NULL). */
int ising_xy_series(ising_xy* x, double* E, double* Mx, double* My, int n);
/* Spins as host [L][L][2] doubles (cos, sin), row-major y*L + x. */
int ising_xy_get_spins(ising_xy* x, double* host_uv);
int ising_xy_set_spins(ising_xy* x, const double* host_uv);
/* Accepted updates since the last seed (synchronises). */
int ising_xy_accepted(ising_xy* x, int64_t* accepted);
int ising_xy_destroy(ising_xy* x);

/* ------------------------------------------------------------------------
 * Fixed-point XY model for the operand-precision study (Supplementary
 * "Operand bit width optimization trial", Tab. S3): spin angles are fixed-point
 * numbers with F = frac_bits fractional bits (the paper's (m, n) types with
 * m - n = F), random words keep 32 bits, all arithmetic is integer.  Angle
 * grid k 2^-F, k in [0, K), K = round(2 pi 2^F); C[k], S[k] = cos, sin of the
 * grid angle rounded to F fractional bits (nearest, ties up); per site of colour
 * c (even x + y first): (hx, hy) = sum of the four neighbours' (C, S);
 * k' = floor(u1 K / 2^32); dE = -round(((C[k'] - C[k]) hx + (S[k'] - S[k]) hy)
 * / 2^F); accept iff dE <= 0 or u2 < floor(exp(-beta dE 2^-F) 2^32).  Words:
 * start k = floor(w K / 2^32), w = word (n & 3) of Philox(n >> 2, 0, 0,
 * XYFIX_INIT << 16), n = y L + x; sweep t: Philox(j >> 1, t, 0, XYFIX_MET << 16
 * | c << 8), j = y (L/2) + (x >> 1), words 2 (j & 1) and 2 (j & 1) + 1 = u1, u2.
 * Records: E2 = sum over bonds of C C' + S S' (energy -E2 2^-2F), Mx = sum C,
 * My = sum S (scale 2^-F).  L even in [2, 32768], frac_bits in [6, 16].
 * flags: ISING_XYFIX_QUANTISE_P holds the acceptance probability in the same
 * fixed-point type too, truncated to F fractional bits: the threshold becomes
 * floor(exp(-beta dE 2^-F) 2^F) 2^(32-F) (clamped to 2^32 - 1).
 * ------------------------------------------------------------------------ */
enum { ISING_XYFIX_QUANTISE_P = 1 };
typedef struct ising_xyfix ising_xyfix;
int ising_xyfix_create(ising_xyfix** out, int L, double beta, int frac_bits, int flags,
                       void* cuda_stream);
/* Seeded random start; sweep counter 0; clears records and the accepted count. */
int ising_xyfix_seed(ising_xyfix* x, uint64_t seed);
/* n_sweeps sweeps (async). */
int ising_xyfix_sweep(ising_xyfix* x, int n_sweeps, int measure_every);
/* Kernel form, as ising_xy_set_mode. */
int ising_xyfix_set_mode(ising_xyfix* x, int mode);
/* Last n records, oldest first (host arrays; any may be NULL).  Synchronises. */
int ising_xyfix_series(ising_xyfix* x, int64_t* E2, int64_t* Mx, int64_t* My, int n);
/* Angle indices as host int32 [L][L], row-major y*L + x.  Synchronise; set
 * rejects indices outside [0, K) with ISING_EINVAL. */
int ising_xyfix_get_angles(ising_xyfix* x, int32_t* host_k);
int ising_xyfix_set_angles(ising_xyfix* x, const int32_t* host_k);
/* K, accepted moves since seeding, kernels launched (any may be NULL). */
int ising_xyfix_info(ising_xyfix* x, int64_t* K, int64_t* accepted, int64_t* launches);
int ising_xyfix_destroy(ising_xyfix* x);

/* ------------------------------------------------------------------------
 * Ising model on lattices with a four-site unit cell, swept by sublattice
 * (the paper's quadripartition: Results "optimising the partition", Fig. 5b/5d,
 * Supplementary Fig. S4a-c).  Lc x Lc periodic cells, 4 Lc^2 sites, spins as
 * s[q][Y][X] (q the sublattice).
 *   ISING_QUAD_SQUARE: square lattice of side 2 Lc, site (2X + i, 2Y + j) in
 *     sublattice q = i + 2j; J1 on nearest, J2 on diagonal (next-nearest)
 *     neighbours (J2 = 0: the plain square lattice).
 *   ISING_QUAD_SQOCT: square-octagon (4.8.8) lattice; cell sites A, B, C, D
 *     (q = 0..3) joined A-B-C-D-A by J1 bonds, octagon bonds J2 between
 *     B(X, Y)-D(X+1, Y) and A(X, Y)-C(X, Y+1).
 * A sweep updates sublattice 0, 1, 2, 3; a site with a1 (a2) antiparallel J1
 * (J2) neighbours out of z1 (z2) flips iff dE = 2 J1 (z1 - 2 a1) +
 * 2 J2 (z2 - 2 a2) <= 0 or u < floor(exp(-beta dE) 2^32), u from Philox planes
 * P_{4m+k} = word k of Philox(g, t, replica, QUAD_MET << 16 | q << 8 | m),
 * g = Y ceil(Lc/32) + (X >> 5), u = sum_k bit_{X & 31}(P_k) 2^(31-k).  Start:
 * s = +1 iff bit X & 31 of word 0 of Philox(g, 0, replica, QUAD_INIT << 16 |
 * q << 8).  Records after sweep t with (t + 1) % measure_every == 0:
 * B1 = sum over J1 bonds of s s', B2 likewise for J2, M = sum s; the energy is
 * -J1 B1 - J2 B2.  Lc in [2, 16384]; beta > 0; finite couplings.
 * ------------------------------------------------------------------------ */
enum { ISING_QUAD_SQUARE = 0, ISING_QUAD_SQOCT = 1 };
typedef struct ising_quad ising_quad;
int ising_quad_create(ising_quad** out, int lattice, int Lc, double beta, double J1, double J2,
                      void* cuda_stream);
/* Seeded random start; sweep counter 0; clears records. */
int ising_quad_seed(ising_quad* x, uint64_t seed);
/* Replica id of the counter map; re-seeds with the current seed. */
int ising_quad_set_replica(ising_quad* x, uint32_t replica);
/* n_sweeps sweeps (async). */
int ising_quad_sweep(ising_quad* x, int n_sweeps, int measure_every);
/* Last n records, oldest first (host arrays; any may be NULL).  Synchronises. */
int ising_quad_series(ising_quad* x, int64_t* B1, int64_t* B2, int64_t* M, int n);
/* Spins as host int8 [4][Lc][Lc] (+1 / -1).  Synchronise. */
int ising_quad_get_spins(ising_quad* x, int8_t* host_out);
int ising_quad_set_spins(ising_quad* x, const int8_t* host_in);
/* Kernels this context has launched. */
int ising_quad_launch_count(ising_quad* x, int64_t* count);
int ising_quad_destroy(ising_quad* x);

/* Free everything the context owns.  NULL-safe.  Synchronises the stream. */
int ising_destroy(ising_ctx* ctx);

/* Message of the last failed call on this thread ("" if none). */
const char* ising_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ISING_H */
