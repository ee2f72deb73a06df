/*
 * su3.h -- C ABI of libsu3: checkerboard heatbath sweeps of pure SU(3)
 * lattice gauge theory with the Wilson action on a periodic 4D lattice, on one
 * NVIDIA GB300 (sm_103a).
 *
 * The operation is the one Berg & Wu time in "Fortran MPI Checkerboard Code
 * for SU(3) Lattice Gauge Theory II" (arXiv:0904.1179):
 *   - MCMC of pure SU(3) LGT with the Wilson action and periodic boundary
 *     conditions (Sec. 1, Introduction);
 *   - checkerboard updating: the links of one direction mu and one site parity
 *     do not share staples and are updated together (Abstract; Sec. 1;
 *     Appendix A, Eq. (mscb18): the checkerboard half-lattice storage);
 *   - every SU(3) matrix update is a one-hit heatbath (Sec. 2.1, remark on
 *     the 97.2% one-hit acceptance at beta = 5.7);
 *   - a timing run performs `nequi` sweeps with no measurement and no I/O, and
 *     the start configuration is created and timed separately (Sec. 2, the
 *     timing programs cbsu3time2mpi{a,b,c}.f and the lswp switch).
 * The paper leaves the update itself to its predecessor; this library reads
 * it as: Wilson action S = beta * sum_P (1 - Re Tr U_P / 3); for each link the
 * staple A (sum of the six three-link paths closing a plaquette with it);
 * Cabibbo-Marinari over the SU(2) subgroups (0,1), (0,2), (1,2) in that order,
 * each with one Kennedy-Pendleton proposal at alpha = 2*beta*k/3 that is
 * accepted or leaves the subgroup unchanged; then Gram-Schmidt
 * reunitarisation.  One sweep = for mu = 0..3: even sites, then odd sites.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = 64-bit seed,
 * counter = (site, mu | subgroup<<2 | call<<4, sweep index low word,
 * tag | (sweep index high word)<<4), tag 0 = update, 1 = hot start.  The
 * sweep index is the only RNG state, so (seed, sweep count, links) is a
 * complete checkpoint and results do not depend on launch configuration.
 *
 * Conventions for every entry point:
 *   - Site x = (x0,x1,x2,x3), canonical index s = x0 + L0*(x1 + L1*(x2 + L2*x3)).
 *   - Canonical host layout of a configuration (links_get/set):
 *       double U[L3][L2][L1][L0][4 mu][3 row][3 col][2 re/im], x0 fastest.
 *     The paper's direction 1 is mu = 0.  n_doubles = V * 4 * 18.
 *   - Extents must be even and >= 2 (the checkerboard with periodic boundaries
 *     needs even extents) and 4*V must fit in 31 bits.
 *   - Every int-returning call returns SU3_OK (0) or a negative SU3_E* code;
 *     su3_last_error() then describes the failure (thread-local, static
 *     storage, valid until the next failing call on the same thread).
 *   - No C++ exception crosses this boundary.  No call traps or asserts on the
 *     device.
 *   - A handle is not re-entrant: calls on one handle must not overlap in time
 *     from several host threads.  Distinct handles are independent.
 *   - The library owns all device memory of a handle (allocated at create,
 *     freed at destroy).  Host pointers passed in stay owned by the caller and
 *     are not retained after the call returns.
 *   - Work is enqueued on the handle's stream.  Calls that return data to the
 *     host (su3_plaquette, su3_links_get, su3_stats, ...) synchronise that
 *     stream; asynchronous failures of earlier work are reported there.
 */
#ifndef SU3_H
#define SU3_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SU3_API __attribute__((visibility("default")))
#else
#define SU3_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct su3_lattice* su3_handle;

enum { SU3_COLD = 0, SU3_HOT = 1 };
enum { SU3_FP64 = 0, SU3_FP32_MIXED = 1, SU3_FP32_EFT = 2 };
enum {
  SU3_OK = 0,
  SU3_EINVAL = -1,   /* bad argument: NULL handle/pointer, odd or too large extent, beta <= 0, bad enum */
  SU3_ENOMEM = -2,   /* device or pinned-host allocation failed */
  SU3_ECUDA = -3,    /* a CUDA runtime call or kernel failed */
  SU3_ETIMEOUT = -4, /* a bounded device-side wait gave up (batched or persistent sweep) */
  SU3_ESIZE = -5     /* caller buffer size does not match the lattice */
};

/* Create a lattice of extents L0..L3 at coupling beta with the given Philox
 * seed and start (SU3_COLD: every link the identity; SU3_HOT: Haar-random
 * SU(3) links drawn from Philox tag 1).  Precision SU3_FP64 stores 18 reals
 * per link in FP64 and computes in FP64.  On success *out receives the
 * handle. */
SU3_API int su3_create(int L0, int L1, int L2, int L3, double beta, uint64_t seed, int start, su3_handle* out);

/* As su3_create, with a precision and a stream.
 * precision SU3_FP32_MIXED: links stored as FP32 rows 0 and 1 (12 reals; row
 *   2 = conj(row0 x row1) is rebuilt on every read), staple and SU(2)
 *   heatbath in FP32, Gram-Schmidt of every updated link in FP64, plaquette
 *   sums in FP64.  Uniforms use 23-bit FP32 draws (one Philox word each).
 * precision SU3_FP32_EFT: as SU3_FP32_MIXED, except that the Gram-Schmidt
 *   coefficients (|row0|^2, |row1|^2, <row0,row1>) are accumulated as
 *   compensated FP32 sums (error-free transformations: TwoProd by FMA,
 *   TwoSum), accurate to about 2^-47 relative, instead of on GB300's FP64
 *   units (1/64 of the FP32 rate).  Same storage, same random numbers; links
 *   agree with SU3_FP32_MIXED to within one FP32 rounding per update.
 * cuda_stream: a cudaStream_t to enqueue all work on (for example PyTorch's
 *   current stream); NULL lets the library create and own a stream.  A
 *   caller-supplied stream must outlive the handle. */
SU3_API int su3_create_ex(int L0, int L1, int L2, int L3, double beta, uint64_t seed, int start, int precision,
                  void* cuda_stream, su3_handle* out);

/* Release the handle and its device memory.  NULL is accepted and ignored. */
SU3_API int su3_destroy(su3_handle h);

/* Perform nsweeps full checkerboard sweeps (nsweeps >= 0).  Asynchronous on
 * the handle's stream: each sweep replays a captured CUDA graph of eight
 * half-sweep kernels, or of one persistent sweep kernel (su3_set_schedule),
 * followed by the sweep-counter increment. */
SU3_API int su3_sweep(su3_handle h, int nsweeps);

/* nsweeps sweeps like su3_sweep, with the mean plaquette after each sweep
 * written to plaq_out[0..nsweeps-1] (the paper leaves measurement routines to
 * the user and asks to evaluate their cost, Sec. 2.2).  The plaquette is fused
 * into the sweep: after the update of U_mu(x) in the odd-site half-sweeps of
 * mu = 1, 2, 3, Re Tr(U_mu(x)_new A_<) -- A_< the staple terms of the
 * directions nu < mu, all already final -- is the sum of the plaquettes of
 * the planes (mu, nu < mu) at x and x - nu-hat; over the three half-sweeps
 * every plaquette of the new configuration is counted once, with no extra
 * pass over the links.  Sums in FP64, fixed-order reduction (reproducible;
 * equal to su3_plaquette up to summation order).  Synchronises once per 4096
 * sweeps.  Acceptance statistics must be off (SU3_EINVAL otherwise). */
SU3_API int su3_sweep_measured(su3_handle h, int nsweeps, double* plaq_out);

/* One checkerboard half-sweep: update every U_mu(x) with parity(x) == parity
 * at the current sweep index, without advancing it.  A full sweep equals the
 * eight calls mu = 0..3, parity 0 then 1, followed by
 * su3_set_sweep_count(h, count + 1).  Asynchronous. */
SU3_API int su3_half_sweep(su3_handle h, int mu, int parity);

/* Mean plaquette (1/(6V)) sum_x sum_{mu<nu} (1/3) Re Tr U_mu(x) U_nu(x+mu)
 * U_mu(x+nu)^+ U_nu(x)^+, products in the storage precision, accumulated in
 * FP64 with a fixed-order reduction (the result is reproducible).
 * Synchronises.  Returns NaN on failure (see su3_last_error). */
SU3_API double su3_plaquette(su3_handle h);

/* Copy the configuration to/from a caller-owned host buffer in the canonical
 * layout (n_doubles must equal V*4*18, else SU3_ESIZE).  Synchronises.
 * For SU3_FP32_MIXED, set rounds rows 0 and 1 to FP32 (round to nearest) and
 * ignores row 2; get returns rows 0 and 1 exactly and row 2 computed in FP64
 * as conj(row0 x row1).  Page-locked buffers transfer fastest.
 * The links set must be SU(3) matrices (to the storage precision): the
 * staple multiplies out rows 0 and 1 of each three-link path and completes
 * row 2 as conj(row0 x row1), which holds for products of SU(3) matrices
 * only.  set does not check; every update reunitarises the link it writes
 * (a link far from unitary, |row|^2 - 1 or <row0,row1> beyond 1e-3, takes a
 * full FP64 Gram-Schmidt in the FP32 paths). */
SU3_API int su3_links_get(su3_handle h, double* host, size_t n_doubles);
SU3_API int su3_links_set(su3_handle h, const double* host, size_t n_doubles);

/* Sweep index (the RNG position).  With the seed and the links it is the full
 * resume state. */
SU3_API int su3_sweep_count(su3_handle h, uint64_t* out);
SU3_API int su3_set_sweep_count(su3_handle h, uint64_t n);

/* Acceptance statistics of the SU(2) proposals (accepted, drawn).  Counting is off by
 * default (it costs a warp reduction and an atomic per warp); enabling resets
 * the counters.  su3_stats synchronises and returns the totals since the last
 * enable or reset. */
SU3_API int su3_set_stats(su3_handle h, int enable);
SU3_API int su3_stats(su3_handle h, uint64_t* accepted, uint64_t* proposed);

/* SU(2) heatbath variant.  max_tries = 1 (the default) is the one-hit
 * heatbath of the paper's MPI code (Sec. 2.1 remark: one proposal, 97.2%
 * accepted at beta = 5.7; a rejected proposal leaves the subgroup unchanged).
 * max_tries > 1 is the repeat-until-accepted heatbath of its non-MPI program:
 * up to max_tries Kennedy-Pendleton proposals per subgroup, proposal n drawn
 * from counter word mu | sub<<2 | call<<4 | n<<6 (proposal 0 is the one-hit
 * draw).  1 <= max_tries <= 2^20.  Valid for single lattices, decomposed
 * lattices and batches. */
SU3_API int su3_set_heatbath(su3_handle h, int max_tries);

/* Lattice properties of a handle. */
SU3_API int su3_info(su3_handle h, int dims[4], double* beta, uint64_t* seed, int* precision);

/* Threads per block of the half-sweep kernels (a multiple of 32 in
 * [32, 256]); 0 restores the default: 128, halved (down to 32) while a
 * half-sweep would have fewer blocks than the GPU has SMs, so that the links
 * of a small lattice spread over as many SMs as possible.  Results do not
 * depend on it: every link update is independent inside a half-sweep and its
 * random numbers are keyed by its site. */
SU3_API int su3_set_block_size(su3_handle h, int threads);

/* Threads per link update of the one-hit half-sweep (an implementation
 * choice; the paper has none): 0 = automatic (the default), 1 = one thread
 * per link (FP64 and single-site FP32 stores) or per pair of links (FP32
 * stores in the site-paired layout, L3 a multiple of 4), 4 = four lanes per
 * link, which share the staple's paths (for small lattices, whose half-sweep
 * leaves the GPU mostly idle).  Results do not depend on it: every form adds
 * the staple in the same order and rounds every step identically.  Phases
 * that measure the plaquette and the repeat-until-accepted heatbath always
 * take the one-thread form.  Not for batch or decomposed handles: SU3_EINVAL. */
SU3_API int su3_set_lanes(su3_handle h, int lanes);

/* How a sweep is scheduled on the GPU (an implementation choice; the paper's
 * sweep is the eight half-sweeps mu = 0..3, even then odd sites, Sec. 1):
 *   SU3_SCHED_PHASES: eight half-sweep kernels, one after the other;
 *   SU3_SCHED_PERSISTENT: one kernel per sweep whose blocks take tiles of
 *     the eight half-sweeps in order from a device counter; a tile starts
 *     once the previous half-sweep has finished the tiles its staples read or
 *     that read its links (the x3 layers of the pair lattice next to its
 *     own), so that one half-sweep's last wave overlaps the next one's first.
 *     Applies to FP32 stores in the site-paired layout (L3 a multiple of 4)
 *     with one thread per pair, at least 4 layers (L3 >= 8), a layer of
 *     L0*L1*L2/2 pairs that is a whole number of blocks, and lattices whose
 *     blocks run in the natural order (an x3 layer of all eight link arrays
 *     of at most 48 MiB: 32^4, 40^4, 48^4; 64^4 keeps the eight kernels and
 *     their tiled block order).  Its waits are bounded in time
 *     (su3_sweep_debug); if one runs out, the sweep stops and the next
 *     synchronising call returns SU3_ETIMEOUT;
 *   SU3_SCHED_PER_DIRECTION: the same tiles in four persistent launches, one
 *     per direction mu with its even and odd half-sweeps, so that each
 *     launch runs the update code of one direction; launches 1-3 are
 *     programmatic dependent launches whose tiles start while the previous
 *     direction drains and wait, as inside a launch, for the layers they
 *     read.  Applies also to FP64 stores (one thread per link, tiles of
 *     sites of one x3 layer: L0*L1*L2/2 a whole number of blocks, L3 >= 4);
 *   SU3_SCHED_CHAINED: eight half-sweep launches chained the same way, a
 *     block's tile given by its index (no counter), each tile waiting only
 *     for the layers of the previous half-sweep it reads (site-paired FP32
 *     stores where SU3_SCHED_PERSISTENT applies, FP64 stores where
 *     SU3_SCHED_PER_DIRECTION does);
 *   SU3_SCHED_AUTO (the default): where they apply, SU3_SCHED_CHAINED for
 *     the site-paired FP32 store when one half-sweep is 1 to 10 waves of the
 *     GPU, w = (V/4 pairs) / (512 x SMs) (24^4: +15 % mixed, +17 % EFT;
 *     32^4: +10 %, +6 %; 40^4: +0.8 %, +0.1 % against eight launches), and
 *     SU3_SCHED_PER_DIRECTION for FP64 when it is 1 to 5 waves,
 *     w = (V/2 links) / (384 x SMs) (24^4: +5 %); else eight half-sweep
 *     kernels (faster at 48^4, and on small lattices whose half-sweep is in
 *     flight at once).
 * su3_sweep_measured always runs the eight kernels (its measuring update
 * variants would make the persistent kernel spill).
 * Results do not depend on it, bit for bit.  SU3_EINVAL for an unknown value,
 * for SU3_SCHED_PERSISTENT where it does not apply, and for batch or
 * decomposed handles. */
enum { SU3_SCHED_AUTO = 0, SU3_SCHED_PHASES = 1, SU3_SCHED_PERSISTENT = 2, SU3_SCHED_PER_DIRECTION = 3, SU3_SCHED_CHAINED = 4 };
SU3_API int su3_set_schedule(su3_handle h, int schedule);

/* The schedule the next sweep runs with (SU3_SCHED_PHASES,
 * SU3_SCHED_PERSISTENT, SU3_SCHED_PER_DIRECTION or SU3_SCHED_CHAINED) into
 * *schedule. */
SU3_API int su3_get_schedule(su3_handle h, int* schedule);

/* Fault-detection hook of the persistent sweep (single lattices), as
 * su3_batch_debug for batches: wait_limit_s (0 < limit <= 60) bounds each
 * wait (default 2 s); withhold_item >= 0 makes that work item of every
 * launch of the sweep (in the launch's dispatch order, from 0: phase *
 * tiles per phase + position for the phases the launch holds; a chained
 * half-sweep's tiles by block index) never report completion, so that the
 * waits on it run out; -1 disables withholding. */
SU3_API int su3_sweep_debug(su3_handle h, double wait_limit_s, int withhold_item);

/* ---------------------------------------------------------------------------
 * Domain decomposition emulated on one device (Sec. 2.1, Eq. (MPInp), Tables
 * 1 and 2): the first ndmpi directions are cut into mpifactor parts each,
 * giving np = mpifactor^ndmpi sublattices (the PBC case nlat = 1; the printed
 * Eq. (MPInp) reads "ndmpi**mpifactor", which Tables 1-3 contradict:
 * np = 1296 for ndmpi 4, mpifactor 6).  Each sublattice keeps its own
 * extended store with one ghost layer on each side of a cut direction; after
 * every checkerboard half-sweep the updated links on the sublattice faces are
 * copied into the ghost cells that the neighbours' staples read (the
 * boundary exchange, Appendix A Eq. (mscb18)), by one gather launch over all
 * sublattices.  lbcex = 0 (only with mpifactor 1) is the paper's "exchange
 * off" run: one sublattice covering the lattice, no direction cut, periodic
 * wrap inside it, no ghost layers and no exchange -- the same sublattice
 * kernel as the cut runs, so it is their like-for-like baseline.  Results are
 * bit for bit those of su3_create_ex with the same arguments: the random
 * numbers are keyed by the global site.
 * ------------------------------------------------------------------------- */

/* Create a decomposed lattice.  Arguments as for su3_create_ex plus
 *   ndmpi: number of cut directions, 1..4 (directions 0..ndmpi-1);
 *   mpifactor: parts per cut direction, >= 1; every cut extent must split
 *     into even parts of at least 2 sites;
 *   lbcex: 1 = boundary exchange on, 0 = off (mpifactor 1 only).
 * The handle accepts every single-lattice call: su3_sweep and su3_half_sweep
 * run the decomposed sweep; su3_sweep_measured fuses the plaquette into the
 * sublattice updates exactly as into the undivided ones; su3_set_heatbath
 * applies to the sublattice updates; su3_plaquette, su3_links_get and
 * su3_links_set first gather the sublattices into (or scatter them from) the
 * handle's global store.  su3_set_lanes is not available on it (SU3_EINVAL).
 * Errors: SU3_EINVAL (arguments), SU3_ENOMEM / SU3_ECUDA (allocation). */
SU3_API int su3_decomp_create(int L0, int L1, int L2, int L3, double beta, uint64_t seed, int start, int precision,
                              int ndmpi, int mpifactor, int lbcex, void* cuda_stream, su3_handle* out);

/* Plan a decomposition without a GPU (host computation only): validates the
 * arguments exactly as su3_decomp_create does and returns the number of
 * sublattices and the links the boundary exchange copies per sweep (every
 * ghost cell a staple reads -- faces of the cut directions and the x + a - b
 * edges -- refreshed for its four directions once per sweep; 0 with the
 * exchange off).  Pointers may be NULL.  Errors: SU3_EINVAL. */
SU3_API int su3_decomp_plan(int L0, int L1, int L2, int L3, int ndmpi, int mpifactor, int lbcex, int* nsub,
                            long long* halo_links_per_sweep);

/* Decomposition of a handle (any pointer may be NULL): ndmpi, mpifactor,
 * lbcex, the number of sublattices, and the links the boundary exchange
 * copies per sweep.  A handle from su3_create reports 0, 1, 0, 1, 0. */
SU3_API int su3_decomp_info(su3_handle h, int* ndmpi, int* mpifactor, int* lbcex, int* nsub,
                            long long* halo_links_per_sweep);

/* ---------------------------------------------------------------------------
 * Batches: n independent replicas, each with its own extents, beta and Philox
 * seed (the same counter layout, keyed by the replica's seed), swept together
 * by four kernel launches per sweep, one per direction mu with the even and
 * odd half-sweeps of every replica (one block per tile of a replica's
 * half-sweep, tiles taken in phase order; launches 1-3 are programmatic
 * dependent launches that start while the one before drains), captured in a
 * CUDA graph.  Each
 * replica performs exactly the single-lattice sweep: replica r after k sweeps
 * equals a lattice created alone with dims[r], betas[r], seeds[r] after k
 * sweeps, bit for bit.
 * ------------------------------------------------------------------------- */

/* Create a batch.  dims[r] = {L0, L1, L2, L3} of replica r (even, >= 2),
 * betas[r] > 0, seeds[r] its Philox key; start and precision as for
 * su3_create_ex (one of each for all replicas); cuda_stream as for
 * su3_create_ex.  The handle is a batch handle: use the su3_batch_* calls,
 * su3_sweep_count/su3_set_sweep_count (one sweep index for all replicas),
 * su3_status and su3_destroy.  Arrays are read during the call only.
 * Errors: SU3_EINVAL (bad n, extent, beta, enum, NULL), SU3_ENOMEM, SU3_ECUDA.
 * The tile and grid configuration comes from an earlier su3_batch_autotune of
 * the same replica set in this process, if there was one. */
SU3_API int su3_batch_create(int n, const int (*dims)[4], const double* betas, const uint64_t* seeds, int start,
                             int precision, void* cuda_stream, su3_handle* out);

/* nsweeps sweeps of every replica; asynchronous, one graph replay (memset of
 * the arrival counters, the four per-direction sweep kernels, the
 * sweep-counter increment) per sweep.  A tile of phase k of replica r
 * waits for all tiles of phase k-1 of r, in its own launch or the one before; the wait is bounded in time and, if
 * it runs out, the sweep stops and the next synchronising call returns
 * SU3_ETIMEOUT (the configuration is then incomplete). */
SU3_API int su3_batch_sweep(su3_handle b, int nsweeps);

/* Mean plaquette of every replica (definition of su3_plaquette) into out_n[0..n-1].
 * Synchronises; SU3_ETIMEOUT if an earlier batched sweep timed out. */
SU3_API int su3_batch_plaquettes(su3_handle b, double* out_n);

/* Copy replica `replica` to/from a host buffer in the canonical layout of
 * su3_links_get/set (n_doubles = V_r * 72).  Synchronises. */
SU3_API int su3_batch_links_get(su3_handle b, int replica, double* host, size_t n_doubles);
SU3_API int su3_batch_links_set(su3_handle b, int replica, const double* host, size_t n_doubles);

/* Number of replicas. */
SU3_API int su3_batch_size(su3_handle b, int* n);

/* Dispatch configuration: threads per block (= half-sites per tile, a multiple
 * of 32 in [32, 256]; 0 = 128), blocks_per_sm (>= 0; accepted and kept, but
 * without effect: the sweep launches one block per work item, and
 * su3_batch_get_config reports the blocks the GPU keeps resident per SM),
 * replicas per L2 window (0 = all: phase-major order over the whole batch).
 * Results do not depend on it. */
SU3_API int su3_batch_config(su3_handle b, int threads, int blocks_per_sm, int window);
SU3_API int su3_batch_get_config(su3_handle b, int* threads, int* blocks_per_sm, int* window);

/* Time every candidate configuration (threads 64/128/256, windows of n, n/2,
 * n/4, ... replicas) on this batch
 * -- one untimed sweep, then the median of three timed sweeps each --,
 * keep the fastest, and remember it for batches of the same replica extents
 * and precision on the same GPU model in this process.  The links and the
 * sweep index are saved before and restored after tuning, so the chain is
 * unchanged.  Outputs (may be NULL) receive the chosen configuration.
 * Allocates a temporary copy of the links. */
SU3_API int su3_batch_autotune(su3_handle b, int* threads, int* blocks_per_sm, int* window);

/* Fault-detection hook.  wait_limit_s (0 < limit <= 60) bounds each wait of
 * the batched sweep (default 2 s); withhold_item >= 0 makes that work item
 * (in the dispatch order of each direction's launch, which numbers its items
 * from 0) never signal its completion, so that the waits on it
 * run out -- the way to test SU3_ETIMEOUT without faulting the GPU.  -1
 * disables withholding. */
SU3_API int su3_batch_debug(su3_handle b, double wait_limit_s, int withhold_item);

/* Synchronise the handle's stream and report asynchronous failures:
 * SU3_ETIMEOUT if a batched or persistent sweep gave up waiting (the status
 * is then cleared),
 * SU3_ECUDA for a CUDA error, else SU3_OK. */
SU3_API int su3_status(su3_handle h);

/* Mean plaquette of a link store held by the caller in device memory,
 * computed without allocating any memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- runtimes that
 * hand out device memory only from their own pool or arena, and plugins or
 * callbacks that must not touch the process allocator.  It performs no
 * cudaMalloc, cudaFree or other allocating call.
 *   links: device pointer to a configuration in the library's device layout,
 *     half-lattice structure of arrays indexed by h = s/2 (s the canonical
 *     site index; each parity holds one site of every pair 2h, 2h+1):
 *       SU3_FP64:       double2 [4 mu][2 parity][9 entries row*3+col][V/2]
 *       SU3_FP32_MIXED, SU3_FP32_EFT (the same store), L3 not a multiple
 *       of 4:           float4  [4 mu][2 parity][3 columns k][V/2], rows 0
 *                       and 1 only: column k = (re u0k, re u1k, im u0k,
 *                       im u1k); row 2 is conj(row0 x row1);
 *       SU3_FP32_MIXED, SU3_FP32_EFT, L3 a multiple of 4 (site pairs x and
 *       x + (L3/2) e3 side by side):
 *                       float4  [4 mu][2 parity][Vp'/32][6 entries e = 3r+k]
 *                       [32], Vp = V/4 pairs per (mu, parity) in tiles of
 *                       32, Vp' = Vp rounded up to a multiple of 32 (the
 *                       padding is never read): pair j is lane j mod 32 of
 *                       tile j / 32, and for rows r = 0, 1 its entry e =
 *                       (re u_rk(x), re u_rk(x'), im u_rk(x), im u_rk(x')),
 *                       where j is the half index of x on the L0 x L1 x L2 x
 *                       L3/2 pair lattice (x3 < L3/2) and x' = x + (L3/2) e3.
 *   out: device pointer to one double that receives the mean plaquette, as
 *     defined for su3_plaquette, when the work enqueued on cuda_stream runs.
 *   cuda_stream: the cudaStream_t to enqueue on (NULL = the default stream).
 * The call is asynchronous and does not synchronise.  Its scratch -- one FP64
 * partial sum per block of 256 sites -- is a fixed 512 KiB device array that
 * every GPU loading libsu3 holds until process exit; lattices of more than
 * 2^24 sites (64^4) are rejected with SU3_ESIZE.  Each call writes every
 * partial it reads, so nothing in the scratch needs to start at zero, but all
 * calls share the one array: calls that overlap on the GPU (on different
 * streams, or from several host threads) race and return wrong results.  The
 * first call on each device looks up the array's device address with that
 * device current (cudaGetSymbolAddress) and caches it.  The cache remembers
 * the CUDA context it was filled in: after the context is destroyed and
 * created again (cudaDeviceReset) the next call looks the address up again.
 * Errors: SU3_EINVAL (NULL pointer, odd or
 * < 2 extent, bad precision), SU3_ESIZE (too many sites), SU3_ECUDA (lookup
 * or launch failed); su3_last_error() describes them. */
SU3_API int su3_plaquette_noalloc(const void* links, int L0, int L1, int L2, int L3, int precision, double* out,
                                  void* cuda_stream);

/* Bounds-checked builds only (libsu3_bounds.so, compiled with
 * -DSU3_BOUNDS_CHECK; an implementation aid, the paper has none): every link
 * load and store of every kernel -- single lattices, batch replicas,
 * sublattices with their ghost layers, the staging copies -- checks its
 * direction, parity and index against the extent of the store it addresses;
 * an access out of range is skipped and recorded, never trapped.  *status
 * receives 0 if no access was out of range since the last clear, else 1;
 * clear != 0 resets it.  Synchronous.  SU3_EINVAL in the product build (no
 * checks compiled in) or for a NULL status. */
SU3_API int su3_bounds_status(unsigned int* status, int clear);

/* Description of the last failure on the calling thread ("" if none). */
SU3_API const char* su3_last_error(void);

/* Library version string. */
SU3_API const char* su3_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SU3_H */
