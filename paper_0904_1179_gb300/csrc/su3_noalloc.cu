// su3_noalloc.cu -- su3_plaquette_noalloc: the mean plaquette of a link store
// that the caller holds in device memory, computed without allocating
// anything.
//
// Some callers cannot call cudaMalloc: code running while a CUDA stream is
// being captured into a graph (allocation is not a capturable operation),
// runtimes that hand out device memory only through their own pool or arena,
// and callbacks or plugins that must not touch the process's allocator.  For
// them the reduction's scratch -- one partial sum per thread block -- lives in
// a fixed file-scope device array instead of a handle's cudaMalloc'd buffer.
// Every GPU that loads libsu3 holds this array (512 KiB) until the process
// exits.
#include <cstdio>
#include <mutex>

#include "su3.h"
#include "su3_device.cuh"
#include "su3_kernels.h"

using namespace su3dev;

namespace {

constexpr int kThreads = 256;  // sites per block of the partial-sum kernel
// One FP64 partial per block: 65,536 blocks of 256 sites covers lattices up to
// 2^24 sites (64^4).
constexpr int kMaxPartials = 1 << 16;
constexpr long long kMaxSites = (long long)kMaxPartials * kThreads;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_plaq_scratch[kMaxPartials];

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};

template <typename T>
__device__ __forceinline__ mat3<T> load_link(const void* U, int mu, int p, int h, int Vh);
template <>
__device__ __forceinline__ mat3<double> load_link<double>(const void* U, int mu, int p, int h, int Vh) {
  return load_f64((const double2*)U, mu, p, h, Vh);
}
template <>
__device__ __forceinline__ mat3<float> load_link<float>(const void* U, int mu, int p, int h, int Vh) {
  return load_f32((const float4*)U, mu, p, h, Vh);
}

// Sum over the six planes at one site of Re Tr(X Y^+), X = U_mu(x) U_nu(x+mu), Y = U_nu(x) U_mu(x+nu).
template <typename T>
__device__ __forceinline__ double site_plaquettes(const Geometry& g, const void* U, const Site& st, int h, int p) {
  const int q = p ^ 1;
  double sum = 0.0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu)
#pragma unroll
    for (int nu = mu + 1; nu < 4; ++nu) {
      const mat3<T> a = load_link<T>(U, mu, p, h, g.Vh);
      const mat3<T> b = load_link<T>(U, nu, q, nb_half(g, st, mu, +1), g.Vh);
      const mat3<T> c = load_link<T>(U, nu, p, h, g.Vh);
      const mat3<T> d = load_link<T>(U, mu, q, nb_half(g, st, nu, +1), g.Vh);
      T tr = T(0);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          cx<T> x = mk(T(0), T(0)), y = x;
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            x = mac(x, a.e[i][j], b.e[j][k]);
            y = mac(y, c.e[i][j], d.e[j][k]);
          }
          tr = fma(x.re, y.re, tr);
          tr = fma(x.im, y.im, tr);
        }
      sum += (double)tr;
    }
  return sum;
}

// Block b writes partials[b]; every entry read by the final kernel is written
// first in the same call, so nothing in the scratch has to start at zero.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_noalloc_partial(Geometry g, const void* U, double* partials) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // over 2 * Vh: (parity, h)
  double v = 0.0;
  if (idx < 2 * g.Vh) {
    const int p = idx >= g.Vh ? 1 : 0;
    const int h = idx - p * g.Vh;
    v = site_plaquettes<T>(g, U, site_of(g, h, p), h, p);
  }
  __shared__ double red[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) partials[blockIdx.x] = w;
  }
}

__global__ void __launch_bounds__(1024) k_noalloc_final(const double* partials, int n, double scale, double* out) {
  __shared__ double red[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += partials[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) *out = w * scale;
  }
}

int fail(int code, const char* msg) {
  char m[256];
  snprintf(m, sizeof m, "su3_plaquette_noalloc: %s", msg);
  return su3_internal_fail(code, m);
}

// Device address of the scratch array on the current device.  The host-side
// name g_plaq_scratch is only a stand-in for the symbol, so the address is
// looked up once per device with that device current and then cached.
int scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SU3_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(SU3_ECUDA, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_plaq_scratch);
    if (e != cudaSuccess || !p) return fail(SU3_ECUDA, e != cudaSuccess ? cudaGetErrorString(e) : "null symbol address");
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return SU3_OK;
}

}  // namespace

extern "C" SU3_API int su3_plaquette_noalloc(const void* links, int L0, int L1, int L2, int L3, int precision,
                                             double* out, void* cuda_stream) {
  if (!links || !out) return fail(SU3_EINVAL, "links and out must be device pointers");
  const int L[4] = {L0, L1, L2, L3};
  for (int mu = 0; mu < 4; ++mu)
    if (L[mu] < 2 || (L[mu] & 1)) return fail(SU3_EINVAL, "every extent must be even and >= 2");
  if (precision != SU3_FP64 && precision != SU3_FP32_MIXED) return fail(SU3_EINVAL, "bad precision");
  const long long V = (long long)L0 * L1 * L2 * L3;
  if (V > kMaxSites) {
    char m[160];
    snprintf(m, sizeof m, "lattice of %lld sites exceeds the fixed scratch of %d partial sums (at most %lld sites, 64^4)",
             V, kMaxPartials, kMaxSites);
    return fail(SU3_ESIZE, m);
  }
  double* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != SU3_OK) return rc;
  const Geometry g = make_geometry(L0, L1, L2, L3);
  const int blocks = (int)((V + kThreads - 1) / kThreads);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (precision == SU3_FP64)
    k_noalloc_partial<double><<<blocks, kThreads, 0, s>>>(g, links, scratch);
  else
    k_noalloc_partial<float><<<blocks, kThreads, 0, s>>>(g, links, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SU3_ECUDA, cudaGetErrorString(e));
  k_noalloc_final<<<1, 1024, 0, s>>>(scratch, blocks, 1.0 / (3.0 * 6.0 * (double)V), out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SU3_ECUDA, cudaGetErrorString(e));
  return SU3_OK;
}
