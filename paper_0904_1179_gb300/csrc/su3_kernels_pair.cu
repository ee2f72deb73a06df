// su3_kernels_pair.cu -- the site-paired FP32 half-sweep for sm_103a.
//
// One thread updates the two links U_mu(x), U_mu(x') of a site pair
// x' = x + (L3/2) e3 on paired FP32 arithmetic (su3_sitepair.cuh): the
// checkerboard (Berg & Wu, arXiv:0904.1179, Abstract and Sec. 1) makes every
// link of the half-sweep (mu, parity) independent, and the two members of a
// pair share all neighbour index arithmetic.  The staple's 18 neighbour link
// pairs stream through a ring of three shared-memory slots per thread
// (cp.async), and the staple's three directions run as a loop that is not
// unrolled, which keeps the instruction stream within the instruction caches.
// The results equal those of the single-site FP32 kernels bit for bit.
#include "su3_kernels.h"

#include "su3_sitepair.cuh"

using namespace su3dev;

namespace {

// Block sum of one value per thread into out[blockIdx.x] (fixed order).
__device__ __forceinline__ void block_partial_pair(double v, double* out) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) out[blockIdx.x] = w;
  }
}

// 128 registers per thread: two blocks of 256 or four of 128 threads per SM.
template <int MU, bool EFT, bool REPEAT, bool MEAS>
__global__ void __launch_bounds__(256, 2) k_half_sweep_f32_pair(HalfSweepArgs args, int stats) {
  extern __shared__ float4 smem[];
  const Geometry& gp = args.pgeom;
  const int j0 = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = j0 < gp.Vh;
  const int j = active ? j0 : gp.Vh - 1;  // every lane takes part; a lane past the end stores nothing
  const UpdateConsts uc{args.three_over_beta_f64, args.three_over_beta, args.max_tries};
  const PairRing rg = pair_ring(smem);
  double2 m = make_double2(0.0, 0.0);
  UpdateCount c = update_pair_f32_rolled<MU, false, EFT, REPEAT, MEAS>(gp, (float4*)args.links, j, args.parity,
                                                                       *args.sweep, args.key, uc, rg, active, &m);
  if (!active) {
    c = UpdateCount{0, 0};
    m = make_double2(0.0, 0.0);
  }
  if (stats) {
    const int acc = __reduce_add_sync(0xffffffffu, c.accepted);
    const int prop = __reduce_add_sync(0xffffffffu, c.proposed);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&args.stats[0], (unsigned long long)acc);
      atomicAdd(&args.stats[1], (unsigned long long)prop);
    }
  }
  if (MEAS) block_partial_pair(m.x + m.y, args.meas);
}

template <int MU, bool EFT, bool REPEAT, bool MEAS>
cudaError_t launch_pair(const HalfSweepArgs& a, bool stats, int threads, cudaStream_t s) {
  const int blocks = (a.pgeom.Vh + threads - 1) / threads;
  k_half_sweep_f32_pair<MU, EFT, REPEAT, MEAS>
      <<<blocks, threads, (size_t)kPairRingBytesPerThread * threads, s>>>(a, stats ? 1 : 0);
  return cudaGetLastError();
}

template <int MU, bool EFT>
cudaError_t launch_pair_mu(const HalfSweepArgs& a, bool stats, int threads, cudaStream_t s) {
  const bool repeat = a.max_tries > 1;
  if (MU > 0 && a.meas)  // fused plaquette (statistics are not counted in these phases)
    return repeat ? launch_pair<MU, EFT, true, (MU > 0)>(a, false, threads, s)
                  : launch_pair<MU, EFT, false, (MU > 0)>(a, false, threads, s);
  return repeat ? launch_pair<MU, EFT, true, false>(a, stats, threads, s)
                : launch_pair<MU, EFT, false, false>(a, stats, threads, s);
}

template <typename F>
cudaError_t set_smem(F f) {
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kPairRingBytesPerThread * 256);
}

template <int MU, bool EFT>
cudaError_t prepare_mu() {
  cudaError_t e;
  if ((e = set_smem(k_half_sweep_f32_pair<MU, EFT, false, false>)) != cudaSuccess) return e;
  if ((e = set_smem(k_half_sweep_f32_pair<MU, EFT, true, false>)) != cudaSuccess) return e;
  if (MU > 0) {
    if ((e = set_smem(k_half_sweep_f32_pair<MU, EFT, false, (MU > 0)>)) != cudaSuccess) return e;
    if ((e = set_smem(k_half_sweep_f32_pair<MU, EFT, true, (MU > 0)>)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <bool EFT>
cudaError_t prepare_all() {
  cudaError_t e;
  if ((e = prepare_mu<0, EFT>()) != cudaSuccess) return e;
  if ((e = prepare_mu<1, EFT>()) != cudaSuccess) return e;
  if ((e = prepare_mu<2, EFT>()) != cudaSuccess) return e;
  return prepare_mu<3, EFT>();
}

}  // namespace

cudaError_t su3k_launch_half_sweep_pair(const HalfSweepArgs& a, int mu, bool eft, bool stats, int threads,
                                        cudaStream_t s) {
  if (eft) {
    switch (mu) {
      case 0: return launch_pair_mu<0, true>(a, stats, threads, s);
      case 1: return launch_pair_mu<1, true>(a, stats, threads, s);
      case 2: return launch_pair_mu<2, true>(a, stats, threads, s);
      default: return launch_pair_mu<3, true>(a, stats, threads, s);
    }
  }
  switch (mu) {
    case 0: return launch_pair_mu<0, false>(a, stats, threads, s);
    case 1: return launch_pair_mu<1, false>(a, stats, threads, s);
    case 2: return launch_pair_mu<2, false>(a, stats, threads, s);
    default: return launch_pair_mu<3, false>(a, stats, threads, s);
  }
}

// The paired kernels take up to 86 KB of dynamic shared memory (256 threads);
// the attribute is a property of the kernel, set once per process and device.
cudaError_t su3k_prepare() {
  cudaError_t e = prepare_all<false>();
  if (e == cudaSuccess) e = prepare_all<true>();
  return e;
}
