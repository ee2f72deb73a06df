// su3_batch.cu -- many independent replicas (each with its own extents, beta and
// seed) swept together: four launches per sweep, one per direction, captured
// in a CUDA graph.
//
// Every replica runs the checkerboard sweep of Berg & Wu (arXiv:0904.1179,
// Abstract and Sec. 1): eight dependent half-sweep phases (mu = 0..3, even then
// odd sites).  Small replicas cannot fill a GB300 one phase at a time, so the
// launches interleave all replicas' phases:
//   - the work of a sweep is a list of items (replica, phase, tile of `threads`
//     consecutive half-sites), ordered window by window -- a window is a group of
//     replicas small enough to stay resident in L2 across its eight phases --
//     and within a window phase by phase;
//   - the items are split by direction into four launches (phases 2 mu and
//     2 mu + 1: each launch runs one direction's update code), launches 1-3
//     programmatic dependent launches of the one before;
//   - a launch has one block per item; each block takes its item from the
//     launch's device counter in that order (not from blockIdx), so items go
//     out in order to blocks that are running;
//   - a tile of phase k of replica r starts once all tiles of phase k-1 of r
//     have signalled completion (per-(replica, phase) arrival counters).  Every
//     item a block waits for was taken earlier by a block that is running, so
//     the order cannot deadlock however many blocks are resident; the wait is
//     still bounded in time and, when the bound is hit, sets a status word and
//     makes every block stop (no hang, no trap).
// One item per block, rather than a loop of items per persistent block, keeps
// the compiler from holding loop-invariant values across items: the FP32
// update fits 64 registers (8 blocks of 128 per SM) and runs 3.5 % (mixed)
// and 0.7 % (EFT) faster than the loop at 80 registers; one direction per
// launch takes its spills from 136 to 40 bytes per thread (+3.2 / +2.3 %).
// Links written by other blocks of the same launch are read through L2 only
// (ld.global.cg); producers fence before their arrival, consumers acquire.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "su3_runtime.h"
#include "su3_update.cuh"

using namespace su3dev;

namespace {

constexpr int kBatchMaxThreads = 256;
constexpr int kStatusTimeout = 1;
constexpr long long kDefaultWaitNs = 2000000000LL;  // 2 s: a phase of any replica takes microseconds

struct ReplicaDesc {
  Geometry g;
  PhiloxKey key;
  long long offset;  // first element (double2 or float4) of the replica's link store
  double three_over_beta_f64;
  float three_over_beta;
  int ntiles;  // work items per phase
};

struct BatchArgs {
  const ReplicaDesc* reps;
  const int4* schedule;  // (replica, phase, tile, 0) per work item, in dispatch order
  int n_items;
  unsigned int* queue;   // next work item
  unsigned int* done;    // [replica * 8 + phase]: tiles completed in this sweep
  int* status;           // 0 or kStatusTimeout
  const uint64_t* sweep;
  void* links;
  long long wait_ns;
  int withhold_item;  // fault-injection hook: this item never signals completion (-1: none)
  int max_tries;      // SU(2) proposals per subgroup (1: one-hit heatbath)
};

// The update of link (h, MU) of a replica: one direction per launch (the
// sweep's four launches each run one direction's code).
template <typename T, bool EFT, bool REPEAT, int MU>
__device__ __forceinline__ void update_item(const ReplicaDesc& rd, void* links, int h, int p, uint64_t t, int max_tries) {
  const UpdateConsts uc{rd.three_over_beta_f64, rd.three_over_beta, max_tries};
  if constexpr (std::is_same<T, double>::value)
    update_link_f64<MU, true, REPEAT>(rd.g, (double2*)links + rd.offset, h, p, t, rd.key, uc);
  else
    update_link_f32<MU, true, EFT, REPEAT>(rd.g, (float4*)links + rd.offset, h, p, t, rd.key, uc);
}

// Register budget of the FP32 instances: __launch_bounds__(threads, blocks per SM).
#ifndef SU3_BATCH_LB_THREADS
#define SU3_BATCH_LB_THREADS kBatchMaxThreads
#endif
#ifndef SU3_BATCH_F32_MINBLOCKS
#define SU3_BATCH_F32_MINBLOCKS 4
#endif

// The descriptors of up to kParamReplicas replicas travel in the kernel's
// parameters (the constant bank: 200 x 128 B of the 32 KB parameter limit),
// where the update reads the replica's geometry and key as constant operands
// that the compiler may load again at any point instead of holding them in
// registers: at 64 registers the FP32 update then spills 220 B instead of
// 776 B per thread and runs 10 % faster (GB300, the 96-replica batch, FP32
// mixed and EFT).  Larger batches read them from global memory.
constexpr int kParamReplicas = 200;
struct ParamReplicas {
  ReplicaDesc r[kParamReplicas];
};

// One work item (replica, phase, tile) of direction MU's launch; reps: the
// descriptors (kernel parameters or global memory).  The sweep is four
// launches, one per direction MU with the phases 2 MU (even sites) and
// 2 MU + 1 (odd sites) of every replica; launches 1-3 are programmatic
// dependent launches, scheduled once every block of the launch before has
// started: a tile of phase 2 MU waits for its replica's phase 2 MU - 1 of the
// launch before, as a tile of phase 2 MU + 1 waits for phase 2 MU.  Items go
// out in order within each launch, and a launch's blocks start only when
// every block of the one before is running or done, so no wait can deadlock.
template <typename T, bool EFT, bool REPEAT, bool PARAM, int MU>
__device__ __forceinline__ void batch_item(const BatchArgs& a, const ReplicaDesc* reps) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __shared__ int4 s_item;
  __shared__ int s_stop;
  __shared__ ReplicaDesc s_rep;  // global descriptors: the current item's, copied once per block
  const uint64_t t = *a.sweep;
  int idx = -1;
  if (threadIdx.x == 0) {
    int stop = 0;
    int4 it = make_int4(0, 0, 0, 0);
    idx = (int)atomicAdd(a.queue, 1u);
    if (idx >= a.n_items || ld_relaxed_s32(a.status) != 0) {
      stop = 1;
    } else {
      it = a.schedule[idx];
      if (it.y > 0) {
        // wait until every tile of phase it.y - 1 of this replica is done
        const unsigned need = (unsigned)reps[it.x].ntiles;
        const unsigned* cnt = a.done + it.x * 8 + it.y - 1;
        if (ld_acquire_u32(cnt) < need) {
          const unsigned long long t0 = global_ns();
          while (ld_acquire_u32(cnt) < need) {
            if (ld_relaxed_s32(a.status) != 0) {
              stop = 1;
              break;
            }
            if (global_ns() - t0 > (unsigned long long)a.wait_ns) {
              atomicCAS(a.status, 0, kStatusTimeout);
              stop = 1;
              break;
            }
            __nanosleep(128);
          }
        }
      }
    }
    s_item = it;
    s_stop = stop;
    if (!PARAM && !stop) s_rep = reps[it.x];
  }
  __syncthreads();
  const int4 it = s_item;
  if (s_stop) return;
  const ReplicaDesc& rd = PARAM ? reps[it.x] : s_rep;
  const int h = it.z * (int)blockDim.x + (int)threadIdx.x;
  if (h < rd.g.Vh) update_item<T, EFT, REPEAT, MU>(rd, a.links, h, it.y & 1, t, a.max_tries);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (idx != a.withhold_item) atomicAdd(a.done + it.x * 8 + it.y, 1u);
  }
}

template <typename T, bool EFT, bool REPEAT, int MU>
__global__ void __launch_bounds__(SU3_BATCH_LB_THREADS, std::is_same<T, float>::value ? SU3_BATCH_F32_MINBLOCKS : 1)
    k_batch_sweep(BatchArgs a) {
  batch_item<T, EFT, REPEAT, false, MU>(a, a.reps);
}

template <typename T, bool EFT, bool REPEAT, int MU>
__global__ void __launch_bounds__(SU3_BATCH_LB_THREADS, std::is_same<T, float>::value ? SU3_BATCH_F32_MINBLOCKS : 1)
    k_batch_sweep_c(const __grid_constant__ BatchArgs a, const __grid_constant__ ParamReplicas pr) {
  batch_item<T, EFT, REPEAT, true, MU>(a, pr.r);
}

// Direction MU's launch: a plain launch for MU = 0, a programmatic dependent
// launch of the one before for MU = 1..3.
template <typename T, bool EFT, bool REPEAT, int MU>
cudaError_t launch_mu(const BatchArgs& a, const ParamReplicas* pr, int threads, cudaStream_t s) {
  if (a.n_items == 0) return cudaSuccess;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.n_items);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = MU > 0 ? 1 : 0;
  return pr ? cudaLaunchKernelEx(&cfg, k_batch_sweep_c<T, EFT, REPEAT, MU>, a, *pr)
            : cudaLaunchKernelEx(&cfg, k_batch_sweep<T, EFT, REPEAT, MU>, a);
}

template <typename T, bool EFT, bool REPEAT>
cudaError_t launch_kind(const BatchArgs* a, const ParamReplicas* pr, int threads, cudaStream_t s) {
  cudaError_t e;
  if ((e = launch_mu<T, EFT, REPEAT, 0>(a[0], pr, threads, s)) != cudaSuccess) return e;
  if ((e = launch_mu<T, EFT, REPEAT, 1>(a[1], pr, threads, s)) != cudaSuccess) return e;
  if ((e = launch_mu<T, EFT, REPEAT, 2>(a[2], pr, threads, s)) != cudaSuccess) return e;
  return launch_mu<T, EFT, REPEAT, 3>(a[3], pr, threads, s);
}

// The sweep's four launches, a[mu] holding direction mu's work items; one
// block per work item; pr: the descriptors as kernel parameters (batches of
// at most kParamReplicas replicas), or null.
cudaError_t launch_batch(const BatchArgs* a, const ParamReplicas* pr, int precision, int threads, cudaStream_t s) {
  const bool rep = a[0].max_tries > 1;
  if (precision == SU3_FP64)
    return rep ? launch_kind<double, false, true>(a, pr, threads, s) : launch_kind<double, false, false>(a, pr, threads, s);
  if (precision == SU3_FP32_EFT)
    return rep ? launch_kind<float, true, true>(a, pr, threads, s) : launch_kind<float, true, false>(a, pr, threads, s);
  return rep ? launch_kind<float, false, true>(a, pr, threads, s) : launch_kind<float, false, false>(a, pr, threads, s);
}

int max_blocks_per_sm(int precision, int threads) {
  int n = 0;
  cudaError_t e =
      precision == SU3_FP64
          ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_sweep_c<double, false, false, 0>, threads, 0)
          : precision == SU3_FP32_EFT
                ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_sweep_c<float, true, false, 0>, threads, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_sweep_c<float, false, false, 0>, threads, 0);
  return e == cudaSuccess ? n : 0;
}

std::mutex g_tune_mutex;
std::map<std::string, std::vector<int>> g_tune_cache;  // key -> {threads, blocks per SM, window}

}  // namespace

SU3_BOUNDS_STATUS_FN(su3k_bounds_status_batch)

struct su3_batch {
  int n = 0;
  std::vector<Geometry> geoms;
  std::vector<double> betas;
  std::vector<uint64_t> seeds;
  std::vector<long long> offsets;  // element offsets (double2 or float4)
  size_t elem_bytes = 0;
  ReplicaDesc* d_reps = nullptr;
  std::unique_ptr<ParamReplicas> param_reps;  // the same, as kernel parameters (n <= kParamReplicas)
  int4* d_schedule = nullptr;  // the work items of directions 0..3, one after another
  int n_items_mu[4] = {0, 0, 0, 0};
  unsigned* d_sync = nullptr;  // [mu] queue of direction mu's launch, [4 + 8r + k] arrival counters
  int* d_status = nullptr;
  int* h_status = nullptr;  // pinned
  double* d_plaq_n = nullptr;
  double* h_plaq_n = nullptr;  // pinned
  int threads = 128;
  int blocks_per_sm = 0;  // as given to su3_batch_config; no effect (one block per work item)
  int window = 0;         // replicas per window, 0: all
  int num_sms = 0;
  cudaGraphExec_t graph = nullptr;
  long long wait_ns = kDefaultWaitNs;
  int withhold_item = -1;
  std::string tune_key;
};

void su3_batch_invalidate(su3_batch* b) {
  if (b && b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

void su3_batch_release(su3_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  cudaFree(b->d_reps);
  cudaFree(b->d_schedule);
  cudaFree(b->d_sync);
  cudaFree(b->d_status);
  cudaFree(b->d_plaq_n);
  cudaFreeHost(b->h_status);
  cudaFreeHost(b->h_plaq_n);
  delete b;
}

namespace {

su3_batch* batch_of(su3_handle h) { return h ? h->batch : nullptr; }

int fail(int code, const char* what) { return su3_fail(code, "%s", what); }

void drop_graph(su3_batch* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

int tiles_of(const Geometry& g, int threads) { return (g.Vh + threads - 1) / threads; }

// Upload the replica descriptors and the dispatch order for the current tile
// size and window.
int build_schedule(su3_lattice* h) {
  su3_batch* b = h->batch;
  std::vector<ReplicaDesc> reps(b->n);
  for (int r = 0; r < b->n; ++r) {
    ReplicaDesc d{};
    d.g = b->geoms[r];
    d.key.k0 = (uint32_t)b->seeds[r];
    d.key.k1 = (uint32_t)(b->seeds[r] >> 32);
    d.offset = b->offsets[r];
    d.three_over_beta_f64 = 3.0 / b->betas[r];
    d.three_over_beta = (float)(3.0 / b->betas[r]);
    d.ntiles = tiles_of(d.g, b->threads);
    reps[r] = d;
  }
  // dispatch order: windows of replicas, phase-major inside a window; split
  // by direction (phases 2 mu, 2 mu + 1) into the four launches, each keeping
  // that order
  std::vector<int4> by_mu[4];
  const int w = b->window > 0 ? b->window : b->n;
  for (int r0 = 0; r0 < b->n; r0 += w) {
    const int r1 = std::min(b->n, r0 + w);
    for (int k = 0; k < 8; ++k)
      for (int r = r0; r < r1; ++r)
        for (int tl = 0; tl < reps[r].ntiles; ++tl) by_mu[k >> 1].push_back(make_int4(r, k, tl, 0));
  }
  std::vector<int4> items;
  for (int mu = 0; mu < 4; ++mu) {
    b->n_items_mu[mu] = (int)by_mu[mu].size();
    items.insert(items.end(), by_mu[mu].begin(), by_mu[mu].end());
  }
  cudaFree(b->d_schedule);
  b->d_schedule = nullptr;
  SU3_CUDA(cudaMalloc(&b->d_schedule, items.size() * sizeof(int4)), "batch schedule");
  SU3_CUDA(cudaMemcpy(b->d_schedule, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice), "batch schedule");
  SU3_CUDA(cudaMemcpy(b->d_reps, reps.data(), reps.size() * sizeof(ReplicaDesc), cudaMemcpyHostToDevice),
           "batch descriptors");
  if (b->n <= kParamReplicas) {
    if (!b->param_reps) b->param_reps.reset(new (std::nothrow) ParamReplicas());
    if (!b->param_reps) return fail(SU3_ENOMEM, "batch descriptors: host allocation failed");
    std::copy(reps.begin(), reps.end(), b->param_reps->r);
  }
  return SU3_OK;
}

// Blocks of the sweep kernel the GPU keeps resident per SM (reported by
// su3_batch_get_config; the launch has one block per work item).
int resident_blocks_per_sm(su3_lattice* h) {
  const int fit = max_blocks_per_sm(h->precision, h->batch->threads);
  return fit > 0 ? fit : 1;
}

int enqueue_batch_sweep(su3_lattice* h) {
  su3_batch* b = h->batch;
  SU3_CUDA(cudaMemsetAsync(b->d_sync, 0, (4 + 8 * (size_t)b->n) * sizeof(unsigned), h->stream), "batch counters");
  BatchArgs a[4];
  long long first = 0;
  for (int mu = 0; mu < 4; ++mu) {
    a[mu] = BatchArgs{};
    a[mu].reps = b->d_reps;
    a[mu].schedule = b->d_schedule + first;
    a[mu].n_items = b->n_items_mu[mu];
    a[mu].queue = b->d_sync + mu;
    a[mu].done = b->d_sync + 4;
    a[mu].status = b->d_status;
    a[mu].sweep = h->d_sweep;
    a[mu].links = h->links;
    a[mu].wait_ns = b->wait_ns;
    a[mu].withhold_item = b->withhold_item;
    a[mu].max_tries = h->max_tries;
    first += b->n_items_mu[mu];
  }
  SU3_CUDA(launch_batch(a, b->param_reps.get(), h->precision, b->threads, h->stream), "batch sweep launch");
  SU3_CUDA(su3k_launch_increment(h->d_sweep, 1, h->stream), "sweep counter launch");
  return SU3_OK;
}

int ensure_batch_graph(su3_lattice* h) {
  su3_batch* b = h->batch;
  if (b->graph) return SU3_OK;
  cudaGraph_t graph = nullptr;
  SU3_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "batch graph capture");
  const int rc = enqueue_batch_sweep(h);
  const cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  if (rc != SU3_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return su3_cuda_fail(e, "batch graph capture end");
  const cudaError_t ei = cudaGraphInstantiate(&b->graph, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    b->graph = nullptr;
    return su3_cuda_fail(ei, "batch graph instantiate");
  }
  return SU3_OK;
}

int set_config(su3_lattice* h, int threads, int blocks_per_sm, int window) {
  su3_batch* b = h->batch;
  if (threads == 0) threads = 128;
  if (threads < 32 || threads > SU3_BATCH_LB_THREADS || (threads & 31))
    return su3_fail(SU3_EINVAL, "su3_batch_config: threads %d is not a multiple of 32 in [32, %d]", threads,
                    (int)SU3_BATCH_LB_THREADS);
  if (blocks_per_sm < 0 || window < 0) return fail(SU3_EINVAL, "su3_batch_config: negative argument");
  SU3_CUDA(cudaStreamSynchronize(h->stream), "su3_batch_config");
  const bool resched = threads != b->threads || window != b->window || !b->d_schedule;
  b->threads = threads;
  b->blocks_per_sm = blocks_per_sm;
  b->window = window;
  drop_graph(b);
  return resched ? build_schedule(h) : SU3_OK;
}

int check_status(su3_lattice* h, const char* what) {
  su3_batch* b = h->batch;
  const int rc = su3_sync(h, what);
  if (rc != SU3_OK) return rc;
  SU3_CUDA(cudaMemcpy(b->h_status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost), what);
  if (*b->h_status != 0) {
    SU3_CUDA(cudaMemset(b->d_status, 0, sizeof(int)), what);
    return su3_fail(SU3_ETIMEOUT,
                    "%s: a batched sweep gave up waiting for a phase to complete (bounded wait of %.3f s); the "
                    "configuration of that sweep is incomplete",
                    what, (double)b->wait_ns * 1e-9);
  }
  return SU3_OK;
}

std::string tune_key_of(const su3_lattice* h) {
  std::string k = h->precision == SU3_FP64 ? "f64" : (h->precision == SU3_FP32_EFT ? "f32e" : "f32m");
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p{};
  cudaGetDeviceProperties(&p, dev);
  k += "|sm" + std::to_string(p.major) + std::to_string(p.minor) + "x" + std::to_string(p.multiProcessorCount);
  for (const Geometry& g : h->batch->geoms)
    k += "|" + std::to_string(g.L0) + "," + std::to_string(g.L1) + "," + std::to_string(g.L2) + "," + std::to_string(g.L3);
  return k;
}

}  // namespace

extern "C" {

int su3_batch_create(int n, const int (*dims)[4], const double* betas, const uint64_t* seeds, int start, int precision,
                     void* cuda_stream, su3_handle* out) {
  if (!out) return fail(SU3_EINVAL, "su3_batch_create: out is NULL");
  *out = nullptr;
  if (n < 1 || !dims || !betas || !seeds) return fail(SU3_EINVAL, "su3_batch_create: need n >= 1 and non-NULL arrays");
  if (start != SU3_COLD && start != SU3_HOT) return fail(SU3_EINVAL, "su3_batch_create: bad start");
  if (precision != SU3_FP64 && precision != SU3_FP32_MIXED && precision != SU3_FP32_EFT)
    return fail(SU3_EINVAL, "su3_batch_create: bad precision");
  su3_batch* b = new (std::nothrow) su3_batch;
  su3_lattice* h = b ? new (std::nothrow) su3_lattice : nullptr;
  if (!b || !h) {
    delete b;
    return fail(SU3_ENOMEM, "su3_batch_create: host allocation failed");
  }
  h->batch = b;
  h->precision = precision;
  b->n = n;
  b->elem_bytes = precision == SU3_FP64 ? sizeof(double2) : sizeof(float4);
  const int ncomp = precision == SU3_FP64 ? kEntriesF64 : kGroupsF32;
  long long total = 0, vmax = 0;
  for (int r = 0; r < n; ++r) {
    for (int mu = 0; mu < 4; ++mu)
      if (dims[r][mu] < 2 || (dims[r][mu] & 1)) {
        su3_release_handle(h);
        return su3_fail(SU3_EINVAL, "su3_batch_create: replica %d extent L%d = %d must be even and >= 2", r, mu,
                        dims[r][mu]);
      }
    const long long V = (long long)dims[r][0] * dims[r][1] * dims[r][2] * dims[r][3];
    if (4 * V > 0x7fffffffLL) {
      su3_release_handle(h);
      return su3_fail(SU3_EINVAL, "su3_batch_create: replica %d: 4*V exceeds 2^31-1", r);
    }
    if (!(betas[r] > 0.0) || !std::isfinite(betas[r])) {
      su3_release_handle(h);
      return su3_fail(SU3_EINVAL, "su3_batch_create: replica %d: beta must be finite and > 0", r);
    }
    const Geometry g = make_geometry(dims[r][0], dims[r][1], dims[r][2], dims[r][3]);
    b->geoms.push_back(g);
    b->betas.push_back(betas[r]);
    b->seeds.push_back(seeds[r]);
    b->offsets.push_back(total);
    total += 8LL * ncomp * g.Vh;
    vmax = std::max(vmax, V);
  }
  h->V = vmax;
  h->beta = betas[0];
  h->seed = seeds[0];
  h->link_bytes = (size_t)total * b->elem_bytes;
  cudaError_t e;
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      su3_release_handle(h);
      return su3_cuda_fail(e, "su3_batch_create: stream");
    }
    h->own_stream = true;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
  Geometry gmax{};
  gmax.Vh = (int)(vmax / 2);
  const long long chunk = vmax < kChunkSites ? vmax : kChunkSites;
  if ((e = cudaMalloc(&h->links, h->link_bytes)) != cudaSuccess ||
      (e = cudaMalloc(&h->d_sweep, sizeof(uint64_t))) != cudaSuccess ||
      (e = cudaMalloc(&h->d_stats, 2 * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMalloc(&h->d_partials, (size_t)su3k_plaquette_blocks(gmax) * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&h->d_stage, (size_t)chunk * 72 * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_reps, (size_t)n * sizeof(ReplicaDesc))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_sync, (4 + 8 * (size_t)n) * sizeof(unsigned))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_status, sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_plaq_n, (size_t)n * sizeof(double))) != cudaSuccess ||
      (e = cudaMallocHost(&b->h_status, sizeof(int))) != cudaSuccess ||
      (e = cudaMallocHost(&b->h_plaq_n, (size_t)n * sizeof(double))) != cudaSuccess) {
    const int rc = su3_cuda_fail(e, "su3_batch_create: allocation");
    cudaGetLastError();
    su3_release_handle(h);
    return rc;
  }
  int rc = SU3_OK;
  if ((e = cudaMemsetAsync(h->d_sweep, 0, sizeof(uint64_t), h->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(b->d_status, 0, sizeof(int), h->stream)) != cudaSuccess)
    rc = su3_cuda_fail(e, "su3_batch_create: memset");
  for (int r = 0; r < n && rc == SU3_OK; ++r) {
    PhiloxKey k{(uint32_t)seeds[r], (uint32_t)(seeds[r] >> 32)};
    // replicas keep one site per FP32 column group (the persistent kernel runs the single-site update)
    InitArgs ia{b->geoms[r], philox_round_keys(k), precision, (char*)h->links + b->offsets[r] * b->elem_bytes, 0};
    e = su3k_launch_init(ia, start == SU3_HOT, h->stream);
    if (e != cudaSuccess) rc = su3_cuda_fail(e, "su3_batch_create: start configuration");
  }
  if (rc == SU3_OK) {
    b->tune_key = tune_key_of(h);
    std::vector<int> cfg;
    {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      auto it = g_tune_cache.find(b->tune_key);
      if (it != g_tune_cache.end()) cfg = it->second;
    }
    if (cfg.size() == 3) {
      b->threads = cfg[0];
      b->blocks_per_sm = cfg[1];
      b->window = cfg[2];
    }
    rc = build_schedule(h);
  }
  if (rc == SU3_OK) rc = su3_sync(h, "su3_batch_create");
  if (rc != SU3_OK) {
    su3_release_handle(h);
    return rc;
  }
  *out = h;
  return SU3_OK;
}

int su3_batch_sweep(su3_handle h, int nsweeps) {
  su3_batch* b = batch_of(h);
  if (!b) return fail(SU3_EINVAL, "su3_batch_sweep: not a batch handle");
  if (nsweeps < 0) return fail(SU3_EINVAL, "su3_batch_sweep: nsweeps < 0");
  if (nsweeps == 0) return SU3_OK;
  int rc = ensure_batch_graph(h);
  if (rc != SU3_OK) return rc;
  for (int i = 0; i < nsweeps; ++i) SU3_CUDA(cudaGraphLaunch(b->graph, h->stream), "su3_batch_sweep: graph launch");
  h->sweep_host += (uint64_t)nsweeps;
  return SU3_OK;
}

int su3_batch_plaquettes(su3_handle h, double* out_n) {
  su3_batch* b = batch_of(h);
  if (!b || !out_n) return fail(SU3_EINVAL, "su3_batch_plaquettes: not a batch handle or NULL output");
  for (int r = 0; r < b->n; ++r) {
    PlaqArgs a{b->geoms[r], (const char*)h->links + b->offsets[r] * b->elem_bytes, h->d_partials, 0};
    SU3_CUDA(su3k_launch_plaquette(a, h->precision, b->d_plaq_n + r, h->stream), "su3_batch_plaquettes");
  }
  SU3_CUDA(cudaMemcpyAsync(b->h_plaq_n, b->d_plaq_n, (size_t)b->n * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
           "su3_batch_plaquettes");
  const int rc = check_status(h, "su3_batch_plaquettes");
  if (rc != SU3_OK) return rc;
  memcpy(out_n, b->h_plaq_n, (size_t)b->n * sizeof(double));
  return SU3_OK;
}

static int batch_links(su3_handle h, int replica, double* host, size_t n_doubles, bool get) {
  su3_batch* b = batch_of(h);
  const char* what = get ? "su3_batch_links_get" : "su3_batch_links_set";
  if (!b || !host) return su3_fail(SU3_EINVAL, "%s: not a batch handle or NULL buffer", what);
  if (replica < 0 || replica >= b->n) return su3_fail(SU3_EINVAL, "%s: replica %d out of range", what, replica);
  const Geometry& g = b->geoms[replica];
  const long long V = 2LL * g.Vh;
  if (n_doubles != (size_t)V * 72) return su3_fail(SU3_ESIZE, "%s: n = %zu, expected %lld", what, n_doubles, V * 72);
  void* base = (char*)h->links + b->offsets[replica] * b->elem_bytes;
  const int rc = su3_transfer(h, g, base, false, host, get, what);
  if (rc != SU3_OK) return rc;
  return check_status(h, what);
}

int su3_batch_links_get(su3_handle h, int replica, double* host, size_t n_doubles) {
  return batch_links(h, replica, host, n_doubles, true);
}

int su3_batch_links_set(su3_handle h, int replica, const double* host, size_t n_doubles) {
  return batch_links(h, replica, const_cast<double*>(host), n_doubles, false);
}

int su3_batch_config(su3_handle h, int threads, int blocks_per_sm, int window) {
  if (!batch_of(h)) return fail(SU3_EINVAL, "su3_batch_config: not a batch handle");
  return set_config(h, threads, blocks_per_sm, window);
}

int su3_batch_get_config(su3_handle h, int* threads, int* blocks_per_sm, int* window) {
  su3_batch* b = batch_of(h);
  if (!b) return fail(SU3_EINVAL, "su3_batch_get_config: not a batch handle");
  if (threads) *threads = b->threads;
  if (blocks_per_sm) *blocks_per_sm = resident_blocks_per_sm(h);
  if (window) *window = b->window > 0 ? std::min(b->window, b->n) : b->n;
  return SU3_OK;
}

int su3_batch_autotune(su3_handle h, int* threads, int* blocks_per_sm, int* window) {
  su3_batch* b = batch_of(h);
  if (!b) return fail(SU3_EINVAL, "su3_batch_autotune: not a batch handle");
  // Tuning sweeps advance the chain: save the links and the sweep counter and
  // restore them afterwards, so tuning leaves no trace in the results.
  void* saved = nullptr;
  SU3_CUDA(cudaStreamSynchronize(h->stream), "su3_batch_autotune");
  SU3_CUDA(cudaMalloc(&saved, h->link_bytes), "su3_batch_autotune: save buffer");
  cudaError_t e = cudaMemcpyAsync(saved, h->links, h->link_bytes, cudaMemcpyDeviceToDevice, h->stream);
  const uint64_t count = h->sweep_host;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int best[3] = {b->threads, b->blocks_per_sm, b->window};
  float best_ms = 1e30f;
  int rc = e == cudaSuccess ? SU3_OK : su3_cuda_fail(e, "su3_batch_autotune");
  std::vector<int> windows = {0};
  for (int d = 2; d <= 16 && b->n / d >= 1; d *= 2) windows.push_back((b->n + d - 1) / d);
  for (int thr : {64, 128, 256}) {
    if (thr > SU3_BATCH_LB_THREADS) continue;
    {
      const int bps = 0;  // one block per work item: no blocks-per-SM choice
      for (int w : windows) {
        if (rc != SU3_OK) break;
        rc = set_config(h, thr, bps, w);
        if (rc == SU3_OK) rc = ensure_batch_graph(h);
        if (rc != SU3_OK) break;
        // one untimed sweep, then the median of three timed sweeps (one slow
        // sample -- another context's work, a clock step -- does not decide)
        float t3[3] = {0.f, 0.f, 0.f};
        e = cudaGraphLaunch(b->graph, h->stream);
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
          if ((e = cudaEventRecord(e0, h->stream)) != cudaSuccess ||
              (e = cudaGraphLaunch(b->graph, h->stream)) != cudaSuccess ||
              (e = cudaEventRecord(e1, h->stream)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
              (e = cudaEventElapsedTime(&t3[k], e0, e1)) != cudaSuccess)
            break;
        }
        if (e != cudaSuccess) {
          rc = su3_cuda_fail(e, "su3_batch_autotune: timing");
          break;
        }
        std::sort(t3, t3 + 3);
        const float ms = t3[1];
        if (ms < best_ms) {
          best_ms = ms;
          best[0] = thr;
          best[1] = bps;
          best[2] = w;
        }
      }
    }
  }
  if (rc == SU3_OK) rc = check_status(h, "su3_batch_autotune");
  if (rc == SU3_OK) rc = set_config(h, best[0], best[1], best[2]);
  if (rc == SU3_OK) {
    e = cudaMemcpyAsync(h->links, saved, h->link_bytes, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = su3k_launch_set_counter(h->d_sweep, count, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = su3_cuda_fail(e, "su3_batch_autotune: restore");
    h->sweep_host = count;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(saved);
  if (rc != SU3_OK) return rc;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[b->tune_key] = {best[0], best[1], best[2]};
  }
  return su3_batch_get_config(h, threads, blocks_per_sm, window);
}

int su3_batch_debug(su3_handle h, double wait_limit_s, int withhold_item) {
  su3_batch* b = batch_of(h);
  if (!b) return fail(SU3_EINVAL, "su3_batch_debug: not a batch handle");
  if (!(wait_limit_s > 0.0) || wait_limit_s > 60.0) return fail(SU3_EINVAL, "su3_batch_debug: wait limit not in (0, 60] s");
  if (withhold_item < -1) return fail(SU3_EINVAL, "su3_batch_debug: bad item");
  SU3_CUDA(cudaStreamSynchronize(h->stream), "su3_batch_debug");
  b->wait_ns = (long long)(wait_limit_s * 1e9);
  b->withhold_item = withhold_item;
  drop_graph(b);
  return SU3_OK;
}

int su3_status(su3_handle h) {
  if (!h) return fail(SU3_EINVAL, "su3_status: NULL handle");
  if (!h->batch) return su3_sync(h, "su3_status");
  return check_status(h, "su3_status");
}

int su3_batch_size(su3_handle h, int* n) {
  su3_batch* b = batch_of(h);
  if (!b || !n) return fail(SU3_EINVAL, "su3_batch_size: not a batch handle or NULL output");
  *n = b->n;
  return SU3_OK;
}

}  // extern "C"
