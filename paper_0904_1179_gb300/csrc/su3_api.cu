// su3_api.cu -- host runtime of libsu3 and its C ABI (include/su3.h).
//
// A handle owns the device link store, the sweep counter (the RNG position),
// the plaquette scratch, the acceptance counters, a staging buffer for layout
// conversion and the instantiated CUDA graphs of one sweep.  The timing
// programs of Berg & Wu (Sec. 2) run `nequi` sweeps with nothing else in the
// loop; su3_sweep replays a graph of the eight half-sweeps for each of them.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "su3_runtime.h"

namespace {

thread_local char g_err[512] = "";

}  // namespace

int su3_fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

int su3_cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return su3_fail(SU3_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return su3_fail(SU3_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int su3_sync(su3_lattice* h, const char* what) {
  SU3_CUDA(cudaStreamSynchronize(h->stream), what);
  SU3_CUDA(cudaGetLastError(), what);
  if (h->d_pstatus) {
    SU3_CUDA(cudaMemcpy(h->h_pstatus, h->d_pstatus, sizeof(int), cudaMemcpyDeviceToHost), what);
    if (*h->h_pstatus != 0) {
      SU3_CUDA(cudaMemset(h->d_pstatus, 0, sizeof(int)), what);
      return su3_fail(SU3_ETIMEOUT,
                      "%s: a sweep gave up waiting for tiles of the previous half-sweep (bounded wait of %.3f s); "
                      "the configuration is incomplete",
                      what, (double)h->pq_wait_ns * 1e-9);
    }
  }
  return SU3_OK;
}

namespace {

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return su3_fail(code, "%s", buf);
}

int cuda_fail(cudaError_t e, const char* what) { return su3_cuda_fail(e, what); }

constexpr int kDefaultThreads = kSu3DefaultThreads;

// Default block size for a half-sweep of Vh links: 128 threads, fewer (down
// to one warp) when that would leave SMs idle, so that a small lattice's
// links spread over as many SMs as there are warps (each link's update is a
// long serial chain, and on the FP64 pipe a few warps saturate an SM).
int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms;
}

// Half-sweeps of small lattices run four lanes per link (k_half_sweep_*_split):
// there the latency of one update is the bound.  FP64: when the split still
// gives at most four warps per SM (GB300: 8^4 1.51x, 8^3x16 1.44x faster;
// beyond that the FP64 pipe is loaded and the idle lanes during the heatbath
// cost what the shorter staple chain saves: 10^4 1.04x, 12^4 0.61x).  FP32:
// at most eight warps per SM (8^4 1.35x, 10^4 1.27x; 12^4 would lose: 0.92x).
bool use_split(int Vh, int precision) {
  const int sms = sm_count();
  const long long warps_per_sm = precision == SU3_FP64 ? 4 : 8;
  return sms > 0 && 4LL * Vh <= 32LL * warps_per_sm * sms;
}

int default_threads(int Vh) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0) {
    cudaGetLastError();
    return kDefaultThreads;
  }
  int t = kDefaultThreads;
  while (t > 32 && (Vh + t - 1) / t < sms) t /= 2;
  return t;
}

}  // namespace

namespace {

void drop_graphs(su3_lattice* h) {
  for (auto& g : h->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  if (h->graph_meas) {
    cudaGraphExecDestroy(h->graph_meas);
    h->graph_meas = nullptr;
  }
}

void release(su3_lattice* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  cudaFree(h->d_pq);
  cudaFree(h->d_pstatus);
  cudaFreeHost(h->h_pstatus);
  if (h->batch) su3_batch_release(h->batch);
  if (h->decomp) su3_decomp_release(h->decomp);
  cudaFree(h->links);
  cudaFree(h->d_sweep);
  cudaFree(h->d_stats);
  cudaFree(h->d_partials);
  cudaFree(h->d_plaq);
  cudaFree(h->d_stage);
  cudaFree(h->d_stage2);
  cudaFree(h->d_meas_parts);
  cudaFree(h->d_meas);
  cudaFreeHost(h->h_meas);
  for (int b = 0; b < 2; ++b) {
    if (h->ev_copied[b]) cudaEventDestroy(h->ev_copied[b]);
    if (h->ev_conv[b]) cudaEventDestroy(h->ev_conv[b]);
  }
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  cudaFreeHost(h->h_plaq);
  cudaFreeHost(h->h_stats);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

HalfSweepArgs half_sweep_args(const su3_lattice* h, int parity) {
  HalfSweepArgs a{};
  a.meas = nullptr;
  a.split = h->split;
  a.pairs = h->pairs;
  a.pgeom = h->pgeom;
  a.tile2 = h->pairs ? su3k_pair_tile2(h->pgeom, h->threads) : 0;
  a.geom = h->geom;
  a.key = su3dev::philox_round_keys(h->key);
  a.parity = parity;
  a.beta = h->beta;
  a.three_over_beta = (float)(3.0 / h->beta);
  a.three_over_beta_f64 = 3.0 / h->beta;
  a.max_tries = h->max_tries;
  a.sweep = h->d_sweep;
  a.links = h->links;
  a.stats = h->d_stats;
  return a;
}

// Whether the sweep can run as persistent launches: the site-paired FP32
// store with one lane per link and a pair lattice whose x3 layers are whole
// tiles (one launch per sweep or one per direction, su3k_launch_sweep_pair);
// or the FP64 store with one lane per link and x3 layers of whole tiles (one
// launch per direction, su3k_launch_sweep_f64).
bool pair_persistent_applies(const su3_lattice* h) {
  int tpl = 0;
  return h->pairs && !h->split && su3k_pair_sweep_layers(h->pgeom, h->threads, &tpl) > 0;
}
bool f64_persistent_applies(const su3_lattice* h) {
  int tpl = 0;
  return h->precision == SU3_FP64 && !h->split && su3k_f64_sweep_layers(h->geom, h->threads, &tpl) > 0;
}
bool persistent_applies(const su3_lattice* h) { return pair_persistent_applies(h) || f64_persistent_applies(h); }

// Waves of the GPU in one half-sweep: site pairs at about 512 threads per SM
// (128 registers), FP64 links at 384 (3 warps of 136-142 registers per
// scheduler).
double half_sweep_waves(const su3_lattice* h) {
  const int sms = sm_count();
  if (sms <= 0) return 1e9;
  return h->pairs ? (double)h->pgeom.Vh / (512.0 * sms) : (double)h->geom.Vh / (384.0 * sms);
}

// SU3_SCHED_AUTO by the number of waves of a half-sweep, after measurements
// on GB300 against eight launches.  Site-paired FP32 (mixed / EFT), the eight
// chained half-sweep launches: 24^4 (1.1 waves) +15 / +17 %, 32^4 (3.4 waves)
// +10 / +6 %, 32^3 x 64 (6.7 waves) +3.4 / +0.9 %, 40^4 (8.2 waves) +0.8 /
// +0.1 %, 48^4 (17 waves) -2.4 / -2.4 %: chained below 10 waves.  FP64, one
// launch per direction: 24^4 (2.8 waves) +5.1 %, 32^4 (9 waves), 40^4 and
// 48^4 +0.3 to +0.4 %: per direction below 5 waves.  Under one wave a whole
// half-sweep is in flight at once and the tiles of the next one wait on it
// (FP32 per direction: 24^3 x 16, 0.7 waves, -38 %; 16^4, 0.2 waves, -62 %;
// FP64 16^4, 0.6 waves, -31 %): eight launches.
int auto_schedule(const su3_lattice* h) {
  const double w = half_sweep_waves(h);
  if (h->pairs) return w >= 1.0 && w < 10.0 ? SU3_SCHED_CHAINED : SU3_SCHED_PHASES;
  return w >= 1.0 && w < 5.0 ? SU3_SCHED_PER_DIRECTION : SU3_SCHED_PHASES;
}

// Whether a schedule other than eight independent launches applies to h.
bool schedule_applies(const su3_lattice* h, int schedule) {
  switch (schedule) {
    case SU3_SCHED_PERSISTENT: return pair_persistent_applies(h);
    case SU3_SCHED_CHAINED:
    case SU3_SCHED_PER_DIRECTION: return persistent_applies(h);
    default: return true;
  }
}

// The schedule the next sweep runs with (measuring sweeps: always eight
// launches).
int effective_schedule(const su3_lattice* h, bool measured = false) {
  if (measured || !persistent_applies(h)) return SU3_SCHED_PHASES;
  const int sched = h->schedule == SU3_SCHED_AUTO ? auto_schedule(h) : h->schedule;
  return schedule_applies(h, sched) ? sched : SU3_SCHED_PHASES;
}

bool use_persistent(const su3_lattice* h, bool measured = false) {
  return effective_schedule(h, measured) != SU3_SCHED_PHASES;
}

// Counters and status word of the persistent sweep (allocated on first use,
// outside any stream capture).
int ensure_pair_queue(su3_lattice* h) {
  if (h->d_pq) return SU3_OK;
  const int words = su3k_sweep_words(h->pairs ? h->pgeom.L3 : h->geom.L3);
  cudaError_t e;
  if ((e = cudaMalloc(&h->d_pq, (size_t)words * sizeof(unsigned int))) != cudaSuccess ||
      (e = cudaMalloc(&h->d_pstatus, sizeof(int))) != cudaSuccess ||
      (e = cudaMallocHost(&h->h_pstatus, sizeof(int))) != cudaSuccess ||
      (e = cudaMemsetAsync(h->d_pstatus, 0, sizeof(int), h->stream)) != cudaSuccess) {
    cudaFree(h->d_pq);
    cudaFree(h->d_pstatus);
    cudaFreeHost(h->h_pstatus);
    h->d_pq = nullptr;
    h->d_pstatus = nullptr;
    h->h_pstatus = nullptr;
    return cuda_fail(e, "persistent sweep counters");
  }
  h->pq_words = words;
  return SU3_OK;
}

// One sweep: mu = 0..3, even then odd sites, then the sweep counter.  With
// `measured`, the odd-site phases of mu = 1, 2, 3 also leave block partials of
// Re Tr(U_new A_<) (A_< = staple terms of nu < mu); together they hold every
// plaquette of the updated configuration once, and a last kernel sums them
// into the ring slot of this sweep.
int enqueue_sweep_body(su3_lattice* h, bool measured) {
  const int blocks = su3k_half_sweep_blocks(half_sweep_args(h, 1), h->precision, h->threads);
  if (use_persistent(h, measured)) {
    const HalfSweepArgs a = half_sweep_args(h, 0);
    const SweepQueue q{h->d_pq, h->d_pstatus, h->pq_wait_ns, h->pq_withhold};
    SU3_CUDA(cudaMemsetAsync(h->d_pq, 0, (size_t)h->pq_words * sizeof(unsigned int), h->stream),
             "sweep counters reset");
    if (h->precision == SU3_FP64)
      SU3_CUDA(su3k_launch_sweep_f64(a, q, h->stats_on, h->threads, effective_schedule(h) == SU3_SCHED_CHAINED,
                                     h->stream),
               "persistent sweep launch");
    else
      SU3_CUDA(su3k_launch_sweep_pair(a, q, h->precision == SU3_FP32_EFT, h->stats_on, h->threads,
                                      effective_schedule(h) == SU3_SCHED_CHAINED        ? SweepForm::kChained
                                      : effective_schedule(h) == SU3_SCHED_PER_DIRECTION ? SweepForm::kPerDirection
                                                                                         : SweepForm::kOneLaunch,
                                      h->stream),
               "persistent sweep launch");
  } else {
    for (int mu = 0; mu < 4; ++mu)
      for (int p = 0; p < 2; ++p) {
        HalfSweepArgs a = half_sweep_args(h, p);
        if (measured && p == 1 && mu >= 1) a.meas = h->d_meas_parts + (size_t)(mu - 1) * blocks;
        SU3_CUDA(su3k_launch_half_sweep(a, mu, h->precision, h->stats_on, h->threads, h->stream),
                 "half-sweep launch");
      }
  }
  if (measured)
    SU3_CUDA(su3k_launch_meas_final(h->d_meas_parts, 3 * blocks, 1.0 / (6.0 * (double)h->V), h->d_sweep, h->d_meas,
                                    h->meas_cap, h->stream),
             "plaquette reduction launch");
  SU3_CUDA(su3k_launch_increment(h->d_sweep, 1, h->stream), "sweep counter launch");
  return SU3_OK;
}

int ensure_graph(su3_lattice* h, bool measured = false) {
  cudaGraphExec_t& exec = measured ? h->graph_meas : h->graph[h->stats_on ? 1 : 0];
  if (exec) return SU3_OK;
  if (use_persistent(h, measured)) {
    const int rc = ensure_pair_queue(h);
    if (rc != SU3_OK) return rc;
  }
  cudaGraph_t graph = nullptr;
  SU3_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "graph capture begin");
  const int rc = enqueue_sweep_body(h, measured);
  const cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  if (rc != SU3_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "graph capture end");
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    exec = nullptr;
    return cuda_fail(ei, "graph instantiate");
  }
  return SU3_OK;
}

int sync(su3_lattice* h, const char* what) { return su3_sync(h, what); }

// Single-lattice calls reject batch handles and vice versa.
bool is_batch(const su3_lattice* h) { return h && h->batch; }

}  // namespace

void su3_release_handle(su3_lattice* h) { release(h); }

int su3_internal_fail(int code, const char* msg) { return su3_fail(code, "%s", msg); }

namespace {

// Second staging buffer, copy stream and events of the transfer pipeline,
// created on first use.
int ensure_transfer(su3_lattice* h, const char* what) {
  if (h->copy_stream) return SU3_OK;
  const long long chunk = h->V < kChunkSites ? h->V : kChunkSites;
  SU3_CUDA(cudaMalloc(&h->d_stage2, (size_t)chunk * 72 * sizeof(double)), what);
  for (int b = 0; b < 2; ++b) {
    SU3_CUDA(cudaEventCreateWithFlags(&h->ev_copied[b], cudaEventDisableTiming), what);
    SU3_CUDA(cudaEventCreateWithFlags(&h->ev_conv[b], cudaEventDisableTiming), what);
  }
  SU3_CUDA(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking), what);
  return SU3_OK;
}

}  // namespace

int su3_transfer(su3_lattice* h, const su3dev::Geometry& g, void* links, bool pairs, double* host, bool get,
                 const char* what) {
  int rc = ensure_transfer(h, what);
  if (rc != SU3_OK) return rc;
  const long long V = 2LL * g.Vh;
  double* stage[2] = {h->d_stage, h->d_stage2};
  int i = 0;
  for (long long s0 = 0; s0 < V; s0 += kChunkSites, ++i) {
    const long long n = (V - s0) < kChunkSites ? (V - s0) : kChunkSites;
    const int b = i & 1;
    cudaStream_t cs = h->copy_stream;
    const size_t bytes = (size_t)n * 72 * sizeof(double);
    ConvArgs a{g, h->precision, s0, n, stage[b], links, pairs ? 1 : 0};
    if (get) {
      // stage[b] is free once the copy-out of chunk i-2 has finished
      if (i >= 2) SU3_CUDA(cudaStreamWaitEvent(h->stream, h->ev_copied[b], 0), what);
      SU3_CUDA(su3k_launch_conv(a, false, h->stream), what);
      SU3_CUDA(cudaEventRecord(h->ev_conv[b], h->stream), what);
      SU3_CUDA(cudaStreamWaitEvent(cs, h->ev_conv[b], 0), what);
      SU3_CUDA(cudaMemcpyAsync(host + s0 * 72, stage[b], bytes, cudaMemcpyDeviceToHost, cs), what);
      SU3_CUDA(cudaEventRecord(h->ev_copied[b], cs), what);
    } else {
      // stage[b] is free once the conversion of chunk i-2 has read it
      if (i >= 2) SU3_CUDA(cudaStreamWaitEvent(cs, h->ev_conv[b], 0), what);
      SU3_CUDA(cudaMemcpyAsync(stage[b], host + s0 * 72, bytes, cudaMemcpyHostToDevice, cs), what);
      SU3_CUDA(cudaEventRecord(h->ev_copied[b], cs), what);
      SU3_CUDA(cudaStreamWaitEvent(h->stream, h->ev_copied[b], 0), what);
      SU3_CUDA(su3k_launch_conv(a, true, h->stream), what);
      SU3_CUDA(cudaEventRecord(h->ev_conv[b], h->stream), what);
    }
  }
  SU3_CUDA(cudaStreamSynchronize(h->copy_stream), what);
  return su3_sync(h, what);
}

extern "C" {

const char* su3_last_error(void) { return g_err; }

const char* su3_version(void) { return "libsu3 1.0 (sm_103a)"; }

int su3_create_ex(int L0, int L1, int L2, int L3, double beta, uint64_t seed, int start, int precision, void* cuda_stream,
                  su3_handle* out) {
  if (!out) return fail(SU3_EINVAL, "su3_create: out is NULL");
  *out = nullptr;
  const int L[4] = {L0, L1, L2, L3};
  for (int mu = 0; mu < 4; ++mu)
    if (L[mu] < 2 || (L[mu] & 1))
      return fail(SU3_EINVAL, "su3_create: extent L%d = %d must be even and >= 2", mu, L[mu]);
  const long long V = (long long)L0 * L1 * L2 * L3;
  if (4 * V > 0x7fffffffLL) return fail(SU3_EINVAL, "su3_create: 4*V = %lld exceeds 2^31-1", 4 * V);
  if (!(beta > 0.0) || !std::isfinite(beta)) return fail(SU3_EINVAL, "su3_create: beta must be finite and > 0");
  if (start != SU3_COLD && start != SU3_HOT) return fail(SU3_EINVAL, "su3_create: bad start %d", start);
  if (precision != SU3_FP64 && precision != SU3_FP32_MIXED && precision != SU3_FP32_EFT)
    return fail(SU3_EINVAL, "su3_create: bad precision %d", precision);

  su3_lattice* h = new (std::nothrow) su3_lattice;
  if (!h) return fail(SU3_ENOMEM, "su3_create: host allocation failed");
  for (int mu = 0; mu < 4; ++mu) h->L[mu] = L[mu];
  h->V = V;
  h->beta = beta;
  h->seed = seed;
  h->precision = precision;
  h->geom = su3dev::make_geometry(L0, L1, L2, L3);
  h->pairs = precision != SU3_FP64 && su3_fp32_pairs(L3);
  if (h->pairs) h->pgeom = su3dev::make_geometry(L0, L1, L2, L3 / 2);
  h->key.k0 = (uint32_t)seed;
  h->key.k1 = (uint32_t)(seed >> 32);
  h->threads = default_threads(h->pairs ? h->pgeom.Vh : h->geom.Vh);
  h->split = use_split(h->geom.Vh, precision);
  {
    const cudaError_t ep = su3k_prepare();
    if (ep != cudaSuccess) {
      delete h;
      return cuda_fail(ep, "su3_create: kernel attributes");
    }
  }

  cudaError_t e;
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete h;
      return cuda_fail(e, "su3_create: stream");
    }
    h->own_stream = true;
  }
  // the site-paired FP32 store pads each (mu, parity) array to whole tiles of pairs
  h->link_bytes = h->pairs ? (size_t)8 * 6 * su3dev::pair_padded(V / 4) * sizeof(float4)
                           : (size_t)V * 4 * (precision == SU3_FP64 ? 18 * sizeof(double) : 12 * sizeof(float));
  const int nparts = su3k_plaquette_blocks(h->geom);
  const long long chunk = V < kChunkSites ? V : kChunkSites;
  if ((e = cudaMalloc(&h->links, h->link_bytes)) != cudaSuccess ||
      (e = cudaMalloc(&h->d_sweep, sizeof(uint64_t))) != cudaSuccess ||
      (e = cudaMalloc(&h->d_stats, 2 * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMalloc(&h->d_partials, (size_t)nparts * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&h->d_plaq, sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&h->d_stage, (size_t)chunk * 4 * 18 * sizeof(double))) != cudaSuccess ||
      (e = cudaMallocHost(&h->h_plaq, sizeof(double))) != cudaSuccess ||
      (e = cudaMallocHost(&h->h_stats, 2 * sizeof(unsigned long long))) != cudaSuccess) {
    const int rc = cuda_fail(e, "su3_create: allocation");
    cudaGetLastError();
    release(h);
    return rc;
  }
  int rc = SU3_OK;
  if ((e = cudaMemsetAsync(h->d_sweep, 0, sizeof(uint64_t), h->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(h->d_stats, 0, 2 * sizeof(unsigned long long), h->stream)) != cudaSuccess) {
    rc = cuda_fail(e, "su3_create: memset");
  }
  if (rc == SU3_OK) {
    InitArgs ia{h->geom, su3dev::philox_round_keys(h->key), precision, h->links, h->pairs ? 1 : 0};
    e = su3k_launch_init(ia, start == SU3_HOT, h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "su3_create: start configuration");
  }
  if (rc == SU3_OK) rc = sync(h, "su3_create");
  if (rc != SU3_OK) {
    release(h);
    return rc;
  }
  *out = h;
  return SU3_OK;
}

int su3_create(int L0, int L1, int L2, int L3, double beta, uint64_t seed, int start, su3_handle* out) {
  return su3_create_ex(L0, L1, L2, L3, beta, seed, start, SU3_FP64, nullptr, out);
}

int su3_destroy(su3_handle h) {
  release(h);
  return SU3_OK;
}

int su3_sweep(su3_handle h, int nsweeps) {
  if (!h) return fail(SU3_EINVAL, "su3_sweep: NULL handle");
  if (is_batch(h)) return fail(SU3_EINVAL, "su3_sweep: batch handle (use the su3_batch_* calls)");
  if (nsweeps < 0) return fail(SU3_EINVAL, "su3_sweep: nsweeps < 0");
  if (nsweeps == 0) return SU3_OK;
  if (su3_decomp_active(h)) return su3_decomp_sweep(h, nsweeps);
  int rc = ensure_graph(h);
  if (rc != SU3_OK) return rc;
  cudaGraphExec_t exec = h->graph[h->stats_on ? 1 : 0];
  for (int n = 0; n < nsweeps; ++n) SU3_CUDA(cudaGraphLaunch(exec, h->stream), "su3_sweep: graph launch");
  h->sweep_host += (uint64_t)nsweeps;
  return SU3_OK;
}

int su3_sweep_measured(su3_handle h, int nsweeps, double* plaq_out) {
  if (!h) return fail(SU3_EINVAL, "su3_sweep_measured: NULL handle");
  if (is_batch(h)) return fail(SU3_EINVAL, "su3_sweep_measured: batch handle (use su3_batch_plaquettes)");
  if (nsweeps < 0 || (nsweeps > 0 && !plaq_out)) return fail(SU3_EINVAL, "su3_sweep_measured: bad nsweeps or NULL out");
  if (h->stats_on) return fail(SU3_EINVAL, "su3_sweep_measured: disable acceptance statistics first");
  if (nsweeps == 0) return SU3_OK;
  const bool dec = su3_decomp_active(h);
  const int blocks = dec ? su3_decomp_meas_blocks(h) : su3k_half_sweep_blocks(half_sweep_args(h, 1), h->precision, h->threads);
  if (h->meas_blocks != blocks || !h->d_meas) {
    SU3_CUDA(cudaStreamSynchronize(h->stream), "su3_sweep_measured");
    if (h->graph_meas) {
      cudaGraphExecDestroy(h->graph_meas);
      h->graph_meas = nullptr;
    }
    if (h->decomp) su3_decomp_invalidate(h->decomp);  // its graphs hold the old partials buffer
    cudaFree(h->d_meas_parts);
    h->d_meas_parts = nullptr;
    SU3_CUDA(cudaMalloc(&h->d_meas_parts, (size_t)3 * blocks * sizeof(double)), "su3_sweep_measured: partials");
    h->meas_blocks = blocks;
    if (!h->d_meas) {
      h->meas_cap = 4096;
      SU3_CUDA(cudaMalloc(&h->d_meas, (size_t)h->meas_cap * sizeof(double)), "su3_sweep_measured: ring");
      SU3_CUDA(cudaMallocHost(&h->h_meas, (size_t)h->meas_cap * sizeof(double)), "su3_sweep_measured: ring");
    }
  }
  cudaGraphExec_t exec = nullptr;
  int rc = dec ? su3_decomp_sweep_measured_graph(h, &exec) : ensure_graph(h, true);
  if (rc != SU3_OK) return rc;
  if (!dec) exec = h->graph_meas;
  for (int done = 0; done < nsweeps;) {
    const int n = (nsweeps - done) < h->meas_cap ? (nsweeps - done) : h->meas_cap;
    const uint64_t t0 = h->sweep_host;
    for (int i = 0; i < n; ++i) SU3_CUDA(cudaGraphLaunch(exec, h->stream), "su3_sweep_measured: graph launch");
    h->sweep_host += (uint64_t)n;
    // copy back only the n slots just written (two pieces where they wrap)
    const int first = (int)(t0 % (uint64_t)h->meas_cap);
    const int n1 = n < h->meas_cap - first ? n : h->meas_cap - first;
    SU3_CUDA(cudaMemcpyAsync(h->h_meas + first, h->d_meas + first, (size_t)n1 * sizeof(double),
                             cudaMemcpyDeviceToHost, h->stream),
             "su3_sweep_measured: copy");
    if (n > n1)
      SU3_CUDA(cudaMemcpyAsync(h->h_meas, h->d_meas, (size_t)(n - n1) * sizeof(double), cudaMemcpyDeviceToHost,
                               h->stream),
               "su3_sweep_measured: copy");
    rc = sync(h, "su3_sweep_measured");
    if (rc != SU3_OK) return rc;
    for (int i = 0; i < n; ++i) plaq_out[done + i] = h->h_meas[(t0 + (uint64_t)i) % (uint64_t)h->meas_cap];
    done += n;
  }
  return SU3_OK;
}

int su3_half_sweep(su3_handle h, int mu, int parity) {
  if (!h) return fail(SU3_EINVAL, "su3_half_sweep: NULL handle");
  if (is_batch(h)) return fail(SU3_EINVAL, "su3_half_sweep: batch handle (use the su3_batch_* calls)");
  if (mu < 0 || mu > 3 || parity < 0 || parity > 1) return fail(SU3_EINVAL, "su3_half_sweep: bad mu/parity");
  if (su3_decomp_active(h)) return su3_decomp_half_sweep(h, mu, parity);
  SU3_CUDA(su3k_launch_half_sweep(half_sweep_args(h, parity), mu, h->precision, h->stats_on, h->threads, h->stream),
           "su3_half_sweep");
  return SU3_OK;
}

double su3_plaquette(su3_handle h) {
  if (!h || is_batch(h)) {
    fail(SU3_EINVAL, h ? "su3_plaquette: batch handle (use su3_batch_plaquettes)" : "su3_plaquette: NULL handle");
    return NAN;
  }
  if (su3_decomp_sync_global(h) != SU3_OK) return NAN;
  PlaqArgs a{h->geom, h->links, h->d_partials, h->pairs ? 1 : 0};
  cudaError_t e = su3k_launch_plaquette(a, h->precision, h->d_plaq, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_plaq, h->d_plaq, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    cuda_fail(e, "su3_plaquette");
    return NAN;
  }
  return *h->h_plaq;
}

int su3_links_get(su3_handle h, double* host, size_t n_doubles) {
  if (!h || !host) return fail(SU3_EINVAL, "su3_links_get: NULL argument");
  if (is_batch(h)) return fail(SU3_EINVAL, "su3_links_get: batch handle (use the su3_batch_* calls)");
  if (n_doubles != (size_t)h->V * 72) return fail(SU3_ESIZE, "su3_links_get: n = %zu, expected %lld", n_doubles, h->V * 72);
  const int rc = su3_decomp_sync_global(h);
  if (rc != SU3_OK) return rc;
  return su3_transfer(h, h->geom, h->links, h->pairs, host, true, "su3_links_get");
}

int su3_links_set(su3_handle h, const double* host, size_t n_doubles) {
  if (!h || !host) return fail(SU3_EINVAL, "su3_links_set: NULL argument");
  if (is_batch(h)) return fail(SU3_EINVAL, "su3_links_set: batch handle (use the su3_batch_* calls)");
  if (n_doubles != (size_t)h->V * 72) return fail(SU3_ESIZE, "su3_links_set: n = %zu, expected %lld", n_doubles, h->V * 72);
  const int rc = su3_transfer(h, h->geom, h->links, h->pairs, const_cast<double*>(host), false, "su3_links_set");
  if (rc == SU3_OK) su3_decomp_global_written(h);
  return rc;
}

int su3_sweep_count(su3_handle h, uint64_t* out) {
  if (!h || !out) return fail(SU3_EINVAL, "su3_sweep_count: NULL argument");
  *out = h->sweep_host;
  return SU3_OK;
}

int su3_set_sweep_count(su3_handle h, uint64_t n) {
  if (!h) return fail(SU3_EINVAL, "su3_set_sweep_count: NULL handle");
  SU3_CUDA(su3k_launch_set_counter(h->d_sweep, n, h->stream), "su3_set_sweep_count");
  h->sweep_host = n;
  return SU3_OK;
}

int su3_set_stats(su3_handle h, int enable) {
  if (!h) return fail(SU3_EINVAL, "su3_set_stats: NULL handle");
  if (is_batch(h)) return fail(SU3_EINVAL, "su3_set_stats: batch handle (use the su3_batch_* calls)");
  h->stats_on = enable != 0;
  if (h->stats_on)
    SU3_CUDA(cudaMemsetAsync(h->d_stats, 0, 2 * sizeof(unsigned long long), h->stream), "su3_set_stats");
  return SU3_OK;
}

int su3_stats(su3_handle h, uint64_t* accepted, uint64_t* proposed) {
  if (!h || !accepted || !proposed) return fail(SU3_EINVAL, "su3_stats: NULL argument");
  SU3_CUDA(cudaMemcpyAsync(h->h_stats, h->d_stats, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream),
           "su3_stats");
  const int rc = sync(h, "su3_stats");
  if (rc != SU3_OK) return rc;
  *accepted = h->h_stats[0];
  *proposed = h->h_stats[1];
  return SU3_OK;
}

int su3_info(su3_handle h, int dims[4], double* beta, uint64_t* seed, int* precision) {
  if (!h) return fail(SU3_EINVAL, "su3_info: NULL handle");
  if (dims)
    for (int mu = 0; mu < 4; ++mu) dims[mu] = h->L[mu];
  if (beta) *beta = h->beta;
  if (seed) *seed = h->seed;
  if (precision) *precision = h->precision;
  return SU3_OK;
}

int su3_set_heatbath(su3_handle h, int max_tries) {
  if (!h) return fail(SU3_EINVAL, "su3_set_heatbath: NULL handle");
  if (max_tries < 1 || max_tries > kMaxHeatbathTries)
    return fail(SU3_EINVAL, "su3_set_heatbath: max_tries %d not in [1, %d]", max_tries, kMaxHeatbathTries);
  if (max_tries != h->max_tries) {
    SU3_CUDA(cudaStreamSynchronize(h->stream), "su3_set_heatbath");
    drop_graphs(h);
    if (h->batch) su3_batch_invalidate(h->batch);
    if (h->decomp) su3_decomp_invalidate(h->decomp);
    h->max_tries = max_tries;
  }
  return SU3_OK;
}

int su3_bounds_status(unsigned int* status, int clear) {
  if (!status) return fail(SU3_EINVAL, "su3_bounds_status: NULL status");
  *status = 0u;
#ifdef SU3_BOUNDS_CHECK
  cudaError_t (*const tus[4])(unsigned int*, bool) = {su3k_bounds_status_kernels, su3k_bounds_status_pair,
                                                        su3k_bounds_status_batch, su3k_bounds_status_decomp};
  for (auto f : tus) {
    unsigned int v = 0u;
    SU3_CUDA(f(&v, clear != 0), "su3_bounds_status");
    *status |= v;
  }
  return SU3_OK;
#else
  (void)clear;
  return fail(SU3_EINVAL, "su3_bounds_status: this library was built without bounds checks");
#endif
}

int su3_set_lanes(su3_handle h, int lanes) {
  if (!h) return fail(SU3_EINVAL, "su3_set_lanes: NULL handle");
  if (is_batch(h) || su3_decomp_active(h))
    return fail(SU3_EINVAL, "su3_set_lanes: not for batch or decomposed handles");
  if (lanes != 0 && lanes != 1 && lanes != 4) return fail(SU3_EINVAL, "su3_set_lanes: lanes %d not 0, 1 or 4", lanes);
  const bool split = lanes == 0 ? use_split(h->geom.Vh, h->precision) : lanes == 4;
  if (split != h->split) {
    SU3_CUDA(cudaStreamSynchronize(h->stream), "su3_set_lanes");
    drop_graphs(h);
    h->split = split;
  }
  return SU3_OK;
}

int su3_set_schedule(su3_handle h, int schedule) {
  if (!h) return fail(SU3_EINVAL, "su3_set_schedule: NULL handle");
  if (is_batch(h) || su3_decomp_active(h))
    return fail(SU3_EINVAL, "su3_set_schedule: not for batch or decomposed handles");
  if (schedule != SU3_SCHED_AUTO && schedule != SU3_SCHED_PHASES && schedule != SU3_SCHED_PERSISTENT &&
      schedule != SU3_SCHED_PER_DIRECTION && schedule != SU3_SCHED_CHAINED)
    return fail(SU3_EINVAL, "su3_set_schedule: unknown schedule %d", schedule);
  if (!schedule_applies(h, schedule))
    return fail(SU3_EINVAL,
                "su3_set_schedule: the persistent and chained sweeps need one thread per link (pair) and x3 layers "
                "of whole blocks: the site-paired FP32 store (L3 >= 8, the natural block order; all forms) or the "
                "FP64 store (L3 >= 4; per direction or chained half-sweeps)");
  if (schedule != h->schedule) {
    SU3_CUDA(cudaStreamSynchronize(h->stream), "su3_set_schedule");
    drop_graphs(h);
    h->schedule = schedule;
  }
  return SU3_OK;
}

int su3_get_schedule(su3_handle h, int* schedule) {
  if (!h || !schedule) return fail(SU3_EINVAL, "su3_get_schedule: NULL argument");
  if (is_batch(h)) return fail(SU3_EINVAL, "su3_get_schedule: batch handle");
  *schedule = su3_decomp_active(h) ? SU3_SCHED_PHASES : effective_schedule(h);
  return SU3_OK;
}

int su3_sweep_debug(su3_handle h, double wait_limit_s, int withhold_item) {
  if (!h) return fail(SU3_EINVAL, "su3_sweep_debug: NULL handle");
  if (is_batch(h)) return fail(SU3_EINVAL, "su3_sweep_debug: batch handle (use su3_batch_debug)");
  if (!(wait_limit_s > 0.0) || wait_limit_s > 60.0) return fail(SU3_EINVAL, "su3_sweep_debug: wait limit not in (0, 60] s");
  if (withhold_item < -1) return fail(SU3_EINVAL, "su3_sweep_debug: withhold_item < -1");
  SU3_CUDA(cudaStreamSynchronize(h->stream), "su3_sweep_debug");
  drop_graphs(h);
  h->pq_wait_ns = (long long)(wait_limit_s * 1e9);
  h->pq_withhold = withhold_item;
  return SU3_OK;
}

int su3_set_block_size(su3_handle h, int threads) {
  if (!h) return fail(SU3_EINVAL, "su3_set_block_size: NULL handle");
  if (is_batch(h)) return fail(SU3_EINVAL, "su3_set_block_size: batch handle (use the su3_batch_* calls)");
  if (threads == 0) threads = default_threads(h->pairs ? h->pgeom.Vh : h->geom.Vh);
  if (threads < 32 || threads > kMaxSweepThreads || (threads & 31))
    return fail(SU3_EINVAL, "su3_set_block_size: %d is not a multiple of 32 in [32, %d]", threads, kMaxSweepThreads);
  if (threads != h->threads) {
    SU3_CUDA(cudaStreamSynchronize(h->stream), "su3_set_block_size");
    drop_graphs(h);
    if (h->decomp) su3_decomp_invalidate(h->decomp);
    h->threads = threads;
  }
  return SU3_OK;
}

}  // extern "C"
