// su3_noalloc.cu -- su3_plaquette_noalloc: the mean plaquette of a link store
// that the caller holds in device memory, computed without allocating
// anything.
//
// Some callers cannot call cudaMalloc: runtimes that hand out device memory
// only through their own pool or arena, and callbacks or plugins that must
// not touch the process's allocator.  For them the reduction's scratch -- one
// partial sum per thread block -- lives in a fixed file-scope device array
// instead of a handle's cudaMalloc'd buffer.
// Every GPU that loads libsu3 holds this array (512 KiB) until the process
// exits.  The kernels are the library's plaquette kernels (su3_kernels.cu),
// launched with that array as their partial-sum buffer.
#include <cuda.h>

#include <cstdio>
#include <mutex>

#include "su3.h"
#include "su3_device.cuh"
#include "su3_kernels.h"

using namespace su3dev;

namespace {

// One FP64 partial per block of the plaquette kernel (256 sites): 65,536
// partials cover lattices up to 2^24 sites (64^4).
constexpr int kMaxPartials = 1 << 16;
constexpr long long kMaxSites = (long long)kMaxPartials * 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_plaq_scratch[kMaxPartials];

// Device address of the array per device ordinal, with the identity of the
// CUDA context it was looked up in: a context that was torn down and created
// again (cudaDeviceReset) loads the module afresh, possibly at another
// address, so the address is looked up again when the context changes.
struct ScratchEntry {
  double* addr;
  unsigned long long ctx_id;
  bool ctx_known;
};

std::mutex g_setup_mutex;
ScratchEntry g_scratch[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
bool g_entry_resolved = false;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

int fail(int code, const char* msg) {
  char m[256];
  snprintf(m, sizeof m, "su3_plaquette_noalloc: %s", msg);
  return su3_internal_fail(code, m);
}

// Unique id of the calling thread's current context (false if there is none
// or the driver cannot tell).  The driver calls are resolved through the
// runtime, so libsu3 does not link the driver library.  Called with
// g_setup_mutex held.
bool current_context_id(unsigned long long* id) {
  if (!g_entry_resolved) {
    g_entry_resolved = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_get_current = (CtxGetCurrentFn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_get_id = (CtxGetIdFn)f;
  }
  if (!g_ctx_get_current || !g_ctx_get_id) return false;
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return g_ctx_get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the scratch array on the current device.  The host-side
// name g_plaq_scratch is only a stand-in for the symbol, so the address is
// looked up with the device current (cudaGetSymbolAddress) on the first call
// in each context and cached.
int scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SU3_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(SU3_ECUDA, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  ScratchEntry& ent = g_scratch[dev];
  unsigned long long id = 0;
  const bool have_id = current_context_id(&id);
  if (!ent.addr || (have_id && ent.ctx_known && id != ent.ctx_id)) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_plaq_scratch);
    if (e != cudaSuccess || !p) return fail(SU3_ECUDA, e != cudaSuccess ? cudaGetErrorString(e) : "null symbol address");
    ent.addr = (double*)p;
    // the lookup binds the runtime's context if none was current before
    ent.ctx_known = have_id || current_context_id(&id);
    ent.ctx_id = id;
  }
  *out = ent.addr;
  return SU3_OK;
}

}  // namespace

extern "C" SU3_API int su3_plaquette_noalloc(const void* links, int L0, int L1, int L2, int L3, int precision,
                                             double* out, void* cuda_stream) {
  if (!links || !out) return fail(SU3_EINVAL, "links and out must be device pointers");
  const int L[4] = {L0, L1, L2, L3};
  for (int mu = 0; mu < 4; ++mu)
    if (L[mu] < 2 || (L[mu] & 1)) return fail(SU3_EINVAL, "every extent must be even and >= 2");
  if (precision != SU3_FP64 && precision != SU3_FP32_MIXED && precision != SU3_FP32_EFT)
    return fail(SU3_EINVAL, "bad precision");
  // the site count, one factor at a time, so that no product can overflow
  long long V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    V *= L[mu];
    if (V > kMaxSites) {
      char m[160];
      snprintf(m, sizeof m, "lattice of more than %lld sites exceeds the fixed scratch of %d partial sums (64^4)",
               kMaxSites, kMaxPartials);
      return fail(SU3_ESIZE, m);
    }
  }
  const Geometry g = make_geometry(L0, L1, L2, L3);
  if (su3k_plaquette_blocks(g) > kMaxPartials) return fail(SU3_ESIZE, "more partial sums than the fixed scratch holds");
  double* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != SU3_OK) return rc;
  // SU3_FP32_MIXED and SU3_FP32_EFT share the FP32 two-row store, site-paired when L3 is a multiple of 4
  const int pairs = precision != SU3_FP64 && su3_fp32_pairs(L3) ? 1 : 0;
  const cudaError_t e = su3k_launch_plaquette(PlaqArgs{g, links, scratch, pairs},
                                              precision == SU3_FP64 ? SU3_FP64 : SU3_FP32_MIXED, out,
                                              (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return fail(SU3_ECUDA, cudaGetErrorString(e));
  return SU3_OK;
}
