// su3_kernels.h -- launch interface between the host runtime (su3_api.cu) and
// the sm_103a kernels (su3_kernels.cu).  Internal to libsu3.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "su3_device.cuh"

// Largest block of the half-sweep kernels (their register budget assumes it).
constexpr int kMaxSweepThreads = 256;

struct HalfSweepArgs {
  su3dev::Geometry geom;
  su3dev::PhiloxRoundKeys key;
  int parity;
  double beta;        // FP64 path
  double three_over_beta_f64;  // FP64 path: 3 / beta
  float three_over_beta;       // FP32 path: 3 / beta, so that 1/alpha = 3 / (2 beta k) = three_over_beta / (2k)
  int max_tries;      // SU(2) proposals per subgroup: 1 = one-hit heatbath
  const uint64_t* sweep;  // device sweep counter (RNG position)
  void* links;
  unsigned long long* stats;  // [accepted, proposed], used when counting
  double* meas;               // fused plaquette: per-block partial sums of this phase (nullptr: off)
  int split;                  // FP64 one-hit sweep of a small lattice: four lanes per link (see k_half_sweep_f64_split)
  int pairs;                  // FP32 store in the site-paired layout (L3 a multiple of 4; su3_sitepair.cuh)
  su3dev::Geometry pgeom;     // the pair lattice L0 x L1 x L2 x L3/2 (pairs only)
  int tile2;                  // paired kernel: > 0 runs its blocks in tiles of tile2 x2-lines (su3_kernels_pair.cu)
};

struct InitArgs {
  su3dev::Geometry geom;
  su3dev::PhiloxRoundKeys key;
  int precision;
  void* links;
  int pairs;  // FP32 store in the site-paired layout
};

struct PlaqArgs {
  su3dev::Geometry geom;
  const void* links;
  double* partials;
  int pairs;  // FP32 store in the site-paired layout
};

struct ConvArgs {
  su3dev::Geometry geom;
  int precision;
  long long s_begin, n_sites;
  double* canon;  // device staging buffer, canonical layout of the chunk
  void* links;
  int pairs;  // FP32 store in the site-paired layout
};

// Whether an FP32 store of an L0 x L1 x L2 x L3 lattice uses the site-paired
// layout (su3_sitepair.cuh): L3 a multiple of 4.
inline bool su3_fp32_pairs(int L3) { return L3 % 4 == 0; }

cudaError_t su3k_launch_half_sweep(const HalfSweepArgs& a, int mu, int precision, bool stats, int threads, cudaStream_t s);
// Blocks of one half-sweep launch (the partial sums of the fused plaquette
// come one per block).
int su3k_half_sweep_blocks(const HalfSweepArgs& a, int precision, int threads);
// The site-paired FP32 half-sweep (su3_kernels_pair.cu): one thread per pair
// of links, the staple's loads staged through shared memory.
cudaError_t su3k_launch_half_sweep_pair(const HalfSweepArgs& a, int mu, bool eft, bool stats, int threads, cudaStream_t s);
// Block order of the paired kernel for a pair lattice gp and block size:
// tile2 (> 0: blocks walk tiles of tile2 lines of x2 per step of x3), 0 for
// the natural order.
int su3k_pair_tile2(const su3dev::Geometry& gp, int threads);
// Dynamic shared memory per thread of the site-paired half-sweep, and the
// kernel attributes it needs (set once, before any stream capture).
constexpr int kPairRingBytesPerThread = 3 * 7 * 16;
cudaError_t su3k_prepare();

// The persistent sweeps (su3_sweepq.cuh): the half-sweeps of one sweep as
// tiles of one block each, handed out in order from a device counter; a tile
// of phase q starts once phase q-1 has finished the x3 layers its staples
// reach (its own layer and the two beside it).  Site-paired FP32
// (su3_kernels_pair.cu): x3 layers of the pair lattice, tiles of `threads`
// pairs; FP64 (su3_kernels.cu): x3 layers of the lattice, tiles of `threads`
// sites of one parity.
struct SweepQueue {
  unsigned int* counters;  // [0]: next work item of a one-launch sweep, [mu]: of direction mu's launch;
                           // [kSweepTickets + q * layers + l]: tiles of phase q done in layer l; zeroed before each sweep
  int* status;             // 0, or kSweepTimeout once a bounded wait ran out (then every block stops)
  long long wait_ns;       // bound of one wait
  int withhold;            // fault-injection hook: this work item never reports completion (-1: none)
};
constexpr int kSweepTimeout = 1;
constexpr int kSweepTickets = 4;
// Layers of the pair lattice for the persistent sweep with blocks of
// `threads`, or 0 where it does not apply (a layer is not a whole number of
// tiles, fewer than four layers, or a block order other than the natural
// one); *tiles_per_layer is set with it.
int su3k_pair_sweep_layers(const su3dev::Geometry& gp, int threads, int* tiles_per_layer);
// The same for the FP64 store of lattice g (layers of L0 L1 L2 / 2 sites per
// parity; at least four).
int su3k_f64_sweep_layers(const su3dev::Geometry& g, int threads, int* tiles_per_layer);
// Counter words for a lattice of `layers` layers.
inline int su3k_sweep_words(int layers) { return kSweepTickets + 8 * layers; }
// One sweep of the site-paired FP32 store: one launch (kOneLaunch); four, one
// per direction mu with its two half-sweeps (kPerDirection); or eight, one
// per half-sweep, each block's tile from its index (kChained); the launches
// of a sweep chained by programmatic dependent launch.  a.parity is unused;
// a.meas must be null (sweeps that measure the plaquette run the eight
// half-sweep kernels).
enum class SweepForm { kOneLaunch, kPerDirection, kChained };
cudaError_t su3k_launch_sweep_pair(const HalfSweepArgs& a, const SweepQueue& q, bool eft, bool stats, int threads,
                                   SweepForm form, cudaStream_t s);
// The FP64 sweep as four chained per-direction launches (k_sweep_f64) or,
// with `chained`, eight chained half-sweep launches (k_half_sweep_f64_chain);
// one thread per link, loads through L2 (the links change during the launch).
cudaError_t su3k_launch_sweep_f64(const HalfSweepArgs& a, const SweepQueue& q, bool stats, int threads, bool chained,
                                  cudaStream_t s);

// Status words of the bounds-checked build, one per translation unit with
// kernels (su3_device.cuh, link_ok); 0 in the product build.
cudaError_t su3k_bounds_status_kernels(unsigned int* v, bool clear);
cudaError_t su3k_bounds_status_pair(unsigned int* v, bool clear);
cudaError_t su3k_bounds_status_batch(unsigned int* v, bool clear);
cudaError_t su3k_bounds_status_decomp(unsigned int* v, bool clear);
cudaError_t su3k_launch_increment(uint64_t* counter, uint64_t n, cudaStream_t s);
// Sum the nparts fused-plaquette partials of one sweep (fixed order) into
// out[*sweep % cap] * scale.
cudaError_t su3k_launch_meas_final(const double* parts, int nparts, double scale, const uint64_t* sweep, double* out,
                                   int cap, cudaStream_t s);
cudaError_t su3k_launch_set_counter(uint64_t* counter, uint64_t n, cudaStream_t s);
cudaError_t su3k_launch_init(const InitArgs& a, bool hot, cudaStream_t s);
int su3k_plaquette_blocks(const su3dev::Geometry& g);
cudaError_t su3k_launch_plaquette(const PlaqArgs& a, int precision, double* out, cudaStream_t s);
cudaError_t su3k_launch_conv(const ConvArgs& a, bool to_store, cudaStream_t s);

// Record a failure for su3_last_error() (thread-local); returns code.
int su3_internal_fail(int code, const char* msg);
