// su3_runtime.h -- host-side state shared by the libsu3 runtime files
// (su3_api.cu: single lattices; su3_batch.cu: batches of replicas).  Internal.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "su3.h"
#include "su3_kernels.h"

// Threads per block of the half-sweep kernels unless set otherwise.
constexpr int kSu3DefaultThreads = 128;
// Sites per chunk of the canonical-layout staging buffer (37.7 MB of FP64 links).
constexpr long long kChunkSites = 1LL << 16;

struct su3_batch;
struct su3_decomp;

struct su3_lattice {
  int L[4] = {0, 0, 0, 0};
  long long V = 0;
  double beta = 0.0;
  uint64_t seed = 0;
  int precision = SU3_FP64;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* links = nullptr;
  size_t link_bytes = 0;
  uint64_t* d_sweep = nullptr;
  uint64_t sweep_host = 0;
  unsigned long long* d_stats = nullptr;
  bool stats_on = false;
  double* d_partials = nullptr;
  double* d_plaq = nullptr;
  double* h_plaq = nullptr;               // pinned
  unsigned long long* h_stats = nullptr;  // pinned, 2 words
  double* d_stage = nullptr;   // canonical-layout staging buffers (two, for the
  double* d_stage2 = nullptr;  // copy/convert pipeline of links_get/set)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};
  cudaEvent_t ev_conv[2] = {nullptr, nullptr};
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // indexed by stats_on
  cudaGraphExec_t graph_meas = nullptr;           // sweep with the fused plaquette
  double* d_meas_parts = nullptr;  // fused plaquette: block partials of the 3 measuring phases
  int meas_blocks = 0;             // blocks per phase the partials were sized for
  double* d_meas = nullptr;        // plaquette per sweep, ring of meas_cap entries
  double* h_meas = nullptr;        // pinned copy
  int meas_cap = 0;
  int threads = kSu3DefaultThreads;
  int max_tries = 1;  // SU(2) proposals per subgroup (1: one-hit heatbath)
  bool split = false;  // small FP64 lattice: four lanes per link update
  bool pairs = false;  // FP32 store in the site-paired layout (L3 a multiple of 4)
  su3dev::Geometry geom{};
  su3dev::Geometry pgeom{};  // pair lattice L0 x L1 x L2 x L3/2 (pairs only)
  su3dev::PhiloxKey key{};
  // persistent site-paired FP32 sweep (su3k_launch_sweep_pair)
  int schedule = 0;                  // SU3_SCHED_AUTO, SU3_SCHED_PHASES or SU3_SCHED_PERSISTENT
  unsigned int* d_pq = nullptr;      // its work counter and per-(phase, layer) completion counts
  int pq_words = 0;
  int* d_pstatus = nullptr;          // kSweepTimeout after a wait ran out
  int* h_pstatus = nullptr;          // pinned
  long long pq_wait_ns = 2000000000LL;
  int pq_withhold = -1;
  su3_batch* batch = nullptr;    // non-null for a batch of replicas
  su3_decomp* decomp = nullptr;  // non-null for a decomposed lattice (su3_decomp_create)
};

// Record a failure for su3_last_error(); returns code.
int su3_fail(int code, const char* fmt, ...);
int su3_cuda_fail(cudaError_t e, const char* what);
int su3_sync(su3_lattice* h, const char* what);
// Copy a configuration (geometry g, device store at `links`) to or from a host
// buffer in the canonical layout, chunk by chunk: host<->device copies on a
// second stream overlap the layout conversions on the handle's stream.
// Synchronises.
int su3_transfer(su3_lattice* h, const su3dev::Geometry& g, void* links, bool pairs, double* host, bool get,
                 const char* what);
// Free a handle and everything it owns (batch part included).
void su3_release_handle(su3_lattice* h);
// Free the batch part of a handle (defined in su3_batch.cu).
void su3_batch_release(su3_batch* b);
// Drop the batch's captured sweep graph (its parameters changed).
void su3_batch_invalidate(su3_batch* b);
// Decomposed lattices (defined in su3_decomp.cu).  The handle's global store
// and the sublattice stores are kept in step lazily.
bool su3_decomp_active(const su3_lattice* h);
void su3_decomp_release(su3_decomp* d);
void su3_decomp_invalidate(su3_decomp* d);
int su3_decomp_sweep(su3_lattice* h, int nsweeps);
int su3_decomp_half_sweep(su3_lattice* h, int mu, int parity);
// Partials per phase of the decomposed sweep's fused plaquette, and the graph
// of one measured decomposed sweep (built on first use; it writes the
// handle's d_meas_parts and d_meas ring).
int su3_decomp_meas_blocks(su3_lattice* h);
int su3_decomp_sweep_measured_graph(su3_lattice* h, cudaGraphExec_t* out);
int su3_decomp_sync_global(su3_lattice* h);   // before reading the global store
void su3_decomp_global_written(su3_lattice* h);  // after writing it
// Largest number of SU(2) proposals per subgroup (the try index has 26 bits
// in the Philox counter).
constexpr int kMaxHeatbathTries = 1 << 20;

#define SU3_CUDA(call, what)                               \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return su3_cuda_fail(e_, what); \
  } while (0)
