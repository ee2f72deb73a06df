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
#include "su3_sweepq.cuh"

using namespace su3dev;

namespace {

// Block sum of one value per thread into *slot (fixed order).
__device__ __forceinline__ void block_partial_pair(double v, double* slot) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) *slot = w;
  }
}

// Order of the blocks.  A line is the hL0 L1 pairs of one (x2, x3) of the
// pair lattice.  In the natural order the x3 neighbours of a line were last
// touched one whole x2 sweep (L2 lines) earlier; when that window of L2 lines
// of all eight (mu, parity) arrays outgrows the L2 cache (a 64^4 lattice: 64
// lines of 1.5 MB), the blocks instead walk the (x2, x3) plane in columns of
// tile2 lines of x2, x3 slower inside a column, so that the x3 neighbours are
// tile2 lines back.  Only the x2 neighbours across a column edge are then
// far away.  The mapping is a permutation of the blocks, each block still one
// contiguous range of pairs inside one line.
__device__ __forceinline__ int pair_block_start(const Geometry& gp, int tile2, int block, int threads) {
  if (tile2 <= 0) return block * threads;
  const int npl = gp.hL0 * gp.L1;  // pairs per line (a multiple of threads when tile2 > 0)
  const int bpl = npl / threads;
  const int line = block / bpl, sub = block - line * bpl;
  const int col = line / (tile2 * gp.L3), r = line - col * tile2 * gp.L3;
  const int x3 = r / tile2, x2 = col * tile2 + (r - x3 * tile2);
  return npl * (x2 + gp.L2 * x3) + sub * threads;
}

// 128 registers per thread: two blocks of 256 or four of 128 threads per SM.
template <int MU, bool EFT, bool REPEAT, bool MEAS>
__global__ void __launch_bounds__(256, 2) k_half_sweep_f32_pair(HalfSweepArgs args, int stats) {
  extern __shared__ float4 smem[];
  const Geometry& gp = args.pgeom;
  const int j0 = pair_block_start(gp, args.tile2, blockIdx.x, blockDim.x) + threadIdx.x;
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
  if (MEAS) block_partial_pair(m.x + m.y, args.meas + blockIdx.x);
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

// ---------------------------------------------------------------------------
// The persistent and chained sweeps.  Each of the eight half-sweep launches
// of a sweep leaves its SMs partly idle while its last blocks drain and the
// next launch ramps up (at 32^4, 3.4 waves of 152 SMs x 4 blocks, the SMs
// hold no warp for about a tenth of each launch).  Here a tile of a
// half-sweep waits only for the x3 layers of the pair lattice that its
// staples read, so the next half-sweep's tiles fill the SMs while the
// previous one drains (su3_sweepq.cuh; on the pair lattice a step across the
// x3 boundary stays in a neighbouring layer): the tiles handed out from a
// device counter in one persistent launch per sweep or per direction
// (k_sweep_f32_pair), or taken by block index in eight chained launches
// (k_half_sweep_f32_chain, the default).
// ---------------------------------------------------------------------------

template <int MU, bool EFT, bool REPEAT>
__device__ __forceinline__ UpdateCount pair_item(const HalfSweepArgs& args, int j, int p, uint64_t t,
                                                 const UpdateConsts& uc, const PairRing& rg) {
  return update_pair_f32_rolled<MU, true, EFT, REPEAT>(args.pgeom, (float4*)args.links, j, p, t, args.key, uc, rg);
}

// One block per tile of the sweep (8 x tiles per phase blocks), its work item
// taken from the queue (su3_sweepq.cuh).  (A loop of items per persistent
// block would let the compiler keep loop-invariant
// values of the four update variants in registers across the loop, and the
// update spills; one item per block keeps the per-phase kernel's registers.)
// Sweeps that measure the plaquette run the eight half-sweep kernels: the
// measuring update variants added to this kernel's four made it spill and
// ran 6 % slower.
// MUSEL = -1: the eight half-sweeps of the sweep in one launch; MUSEL = 0..3:
// the two half-sweeps (even, odd sites) of direction MUSEL, one launch per
// direction, so that a launch runs a single update variant (the code of one
// direction); its first half-sweep waits on the previous launch's last.
template <int MUSEL, bool EFT, bool REPEAT>
__global__ void __launch_bounds__(256, 2)
    k_sweep_f32_pair(HalfSweepArgs args, SweepQueue qa, int tiles_per_layer, int layers, int stats) {
  extern __shared__ float4 smem[];
  __shared__ SweepItem s_item;
  constexpr int kPhases = MUSEL < 0 ? 8 : 2, kFirst = MUSEL < 0 ? 0 : 2 * MUSEL;
  if (MUSEL >= 0) signal_dependents();
  take_sweep_item<kPhases, kFirst>(qa, MUSEL < 0 ? 0 : MUSEL, tiles_per_layer, layers, &s_item);
  __syncthreads();
  const SweepItem it = s_item;
  if (it.phase < 0) return;
  const UpdateConsts uc{args.three_over_beta_f64, args.three_over_beta, args.max_tries};
  const PairRing rg = pair_ring(smem);
  const uint64_t t = *args.sweep;
  const int mu = it.phase >> 1, p = it.phase & 1;
  const int j = it.tile * (int)blockDim.x + (int)threadIdx.x;  // layers are whole tiles: always a pair of the lattice
  UpdateCount c;
  if (MUSEL >= 0) {
    c = pair_item<(MUSEL < 0 ? 0 : MUSEL), EFT, REPEAT>(args, j, p, t, uc, rg);
  } else {
    switch (mu) {
      case 0: c = pair_item<0, EFT, REPEAT>(args, j, p, t, uc, rg); break;
      case 1: c = pair_item<1, EFT, REPEAT>(args, j, p, t, uc, rg); break;
      case 2: c = pair_item<2, EFT, REPEAT>(args, j, p, t, uc, rg); break;
      default: c = pair_item<3, EFT, REPEAT>(args, j, p, t, uc, rg); break;
    }
  }
  if (stats) {
    const int acc = __reduce_add_sync(0xffffffffu, c.accepted);
    const int prop = __reduce_add_sync(0xffffffffu, c.proposed);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&args.stats[0], (unsigned long long)acc);
      atomicAdd(&args.stats[1], (unsigned long long)prop);
    }
  }
  report_sweep_item(qa, layers, it);
}

// One half-sweep (phase 2 MU + parity) of the chained sweep: one block per
// tile, the tile from the block's index (su3_sweepq.cuh), waiting only for the
// layers of the previous launch's half-sweep that its staples read.
template <int MU, bool EFT, bool REPEAT>
__global__ void __launch_bounds__(256, 2)
    k_half_sweep_f32_chain(HalfSweepArgs args, SweepQueue qa, int tiles_per_layer, int layers, int stats, int parity) {
  extern __shared__ float4 smem[];
  __shared__ SweepItem s_item;
  signal_dependents();
  own_sweep_item(qa, 2 * MU + parity, tiles_per_layer, layers, &s_item);
  __syncthreads();
  const SweepItem it = s_item;
  if (it.phase < 0) return;
  const UpdateConsts uc{args.three_over_beta_f64, args.three_over_beta, args.max_tries};
  const PairRing rg = pair_ring(smem);
  const int j = it.tile * (int)blockDim.x + (int)threadIdx.x;  // layers are whole tiles: always a pair of the lattice
  const UpdateCount c = pair_item<MU, EFT, REPEAT>(args, j, parity, *args.sweep, uc, rg);
  if (stats) {
    const int acc = __reduce_add_sync(0xffffffffu, c.accepted);
    const int prop = __reduce_add_sync(0xffffffffu, c.proposed);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&args.stats[0], (unsigned long long)acc);
      atomicAdd(&args.stats[1], (unsigned long long)prop);
    }
  }
  report_sweep_item(qa, layers, it);
}

// The two chained launches of direction MU (the first of the sweep, MU = 0
// even sites, is an ordinary launch).
template <int MU, bool EFT, bool REPEAT>
cudaError_t launch_chain_mu(const HalfSweepArgs& a, const SweepQueue& q, int tpl, int layers, int st, int threads,
                            size_t smem, cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tpl * layers);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  for (int p = 0; p < 2; ++p) {
    cfg.numAttrs = MU == 0 && p == 0 ? 0 : 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_half_sweep_f32_chain<MU, EFT, REPEAT>, a, q, tpl, layers, st, p);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <bool EFT, bool REPEAT>
cudaError_t launch_sweep(const HalfSweepArgs& a, const SweepQueue& q, int tpl, int layers, bool stats, int threads,
                         SweepForm form, cudaStream_t s) {
  const size_t smem = (size_t)kPairRingBytesPerThread * threads;
  const int st = stats ? 1 : 0;
  if (form == SweepForm::kChained) {
    cudaError_t e;
    if ((e = launch_chain_mu<0, EFT, REPEAT>(a, q, tpl, layers, st, threads, smem, s)) != cudaSuccess) return e;
    if ((e = launch_chain_mu<1, EFT, REPEAT>(a, q, tpl, layers, st, threads, smem, s)) != cudaSuccess) return e;
    if ((e = launch_chain_mu<2, EFT, REPEAT>(a, q, tpl, layers, st, threads, smem, s)) != cudaSuccess) return e;
    return launch_chain_mu<3, EFT, REPEAT>(a, q, tpl, layers, st, threads, smem, s);
  }
  if (form == SweepForm::kOneLaunch) {
    k_sweep_f32_pair<-1, EFT, REPEAT><<<8 * tpl * layers, threads, smem, s>>>(a, q, tpl, layers, st);
    return cudaGetLastError();
  }
  const int blocks = 2 * tpl * layers;
  k_sweep_f32_pair<0, EFT, REPEAT><<<blocks, threads, smem, s>>>(a, q, tpl, layers, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // directions 1-3: programmatic dependent launches (su3_sweepq.cuh)
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if ((e = cudaLaunchKernelEx(&cfg, k_sweep_f32_pair<1, EFT, REPEAT>, a, q, tpl, layers, st)) != cudaSuccess) return e;
  if ((e = cudaLaunchKernelEx(&cfg, k_sweep_f32_pair<2, EFT, REPEAT>, a, q, tpl, layers, st)) != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, k_sweep_f32_pair<3, EFT, REPEAT>, a, q, tpl, layers, st);
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
  if ((e = set_smem(k_sweep_f32_pair<-1, EFT, false>)) != cudaSuccess) return e;
  if ((e = set_smem(k_half_sweep_f32_chain<0, EFT, false>)) != cudaSuccess) return e;
  if ((e = set_smem(k_half_sweep_f32_chain<1, EFT, false>)) != cudaSuccess) return e;
  if ((e = set_smem(k_half_sweep_f32_chain<2, EFT, false>)) != cudaSuccess) return e;
  if ((e = set_smem(k_half_sweep_f32_chain<3, EFT, false>)) != cudaSuccess) return e;
  if ((e = set_smem(k_half_sweep_f32_chain<0, EFT, true>)) != cudaSuccess) return e;
  if ((e = set_smem(k_half_sweep_f32_chain<1, EFT, true>)) != cudaSuccess) return e;
  if ((e = set_smem(k_half_sweep_f32_chain<2, EFT, true>)) != cudaSuccess) return e;
  if ((e = set_smem(k_half_sweep_f32_chain<3, EFT, true>)) != cudaSuccess) return e;
  if ((e = set_smem(k_sweep_f32_pair<-1, EFT, true>)) != cudaSuccess) return e;
  if ((e = set_smem(k_sweep_f32_pair<0, EFT, false>)) != cudaSuccess) return e;
  if ((e = set_smem(k_sweep_f32_pair<1, EFT, false>)) != cudaSuccess) return e;
  if ((e = set_smem(k_sweep_f32_pair<2, EFT, false>)) != cudaSuccess) return e;
  if ((e = set_smem(k_sweep_f32_pair<3, EFT, false>)) != cudaSuccess) return e;
  if ((e = set_smem(k_sweep_f32_pair<0, EFT, true>)) != cudaSuccess) return e;
  if ((e = set_smem(k_sweep_f32_pair<1, EFT, true>)) != cudaSuccess) return e;
  if ((e = set_smem(k_sweep_f32_pair<2, EFT, true>)) != cudaSuccess) return e;
  if ((e = set_smem(k_sweep_f32_pair<3, EFT, true>)) != cudaSuccess) return e;
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

SU3_BOUNDS_STATUS_FN(su3k_bounds_status_pair)

int su3k_pair_sweep_layers(const Geometry& gp, int threads, int* tiles_per_layer) {
  const long long per_layer = (long long)gp.hL0 * gp.L1 * gp.L2;  // pairs of one parity in one x3 layer
  if (threads <= 0 || per_layer % threads != 0 || gp.L3 < 4 || su3k_pair_tile2(gp, threads) != 0) return 0;
  *tiles_per_layer = (int)(per_layer / threads);
  return gp.L3;
}

cudaError_t su3k_launch_sweep_pair(const HalfSweepArgs& a, const SweepQueue& q, bool eft, bool stats, int threads,
                                   SweepForm form, cudaStream_t s) {
  int tpl = 0;
  const int layers = su3k_pair_sweep_layers(a.pgeom, threads, &tpl);
  if (layers == 0) return cudaErrorInvalidValue;
  if (a.meas) return cudaErrorInvalidValue;  // measuring sweeps run the eight half-sweep kernels
  const bool rep = a.max_tries > 1;
  if (eft)
    return rep ? launch_sweep<true, true>(a, q, tpl, layers, stats, threads, form, s)
               : launch_sweep<true, false>(a, q, tpl, layers, stats, threads, form, s);
  return rep ? launch_sweep<false, true>(a, q, tpl, layers, stats, threads, form, s)
             : launch_sweep<false, false>(a, q, tpl, layers, stats, threads, form, s);
}

int su3k_pair_tile2(const Geometry& gp, int threads) {
  const long long npl = (long long)gp.hL0 * gp.L1;
  const long long line_bytes = npl * 96 * 8;  // one line of all eight (mu, parity) arrays
  // Tiles only where the natural window exceeds 48 MiB, and then columns
  // whose window stays within 32 MiB.  Measured on GB300: 48^4 (a 40.5 MiB
  // window) runs 0.4-1.8 % faster in the natural order than in columns of 24
  // lines; 64^4 (96 MiB) runs 3-4 % faster in columns of 16 lines (24 MiB)
  // than in the natural order and 4-8 % faster than in columns of 32 lines
  // (48 MiB); 32^4 (12 MiB) runs 2-3 % slower in columns of 8 lines.
  const long long trigger = 48LL << 20, window = 32LL << 20;
  if (npl % threads != 0 || line_bytes * gp.L2 <= trigger) return 0;
  int best = 0;
  for (int t = 2; t < gp.L2; ++t)
    if (gp.L2 % t == 0 && line_bytes * t <= window) best = t;
  return best;
}

// The paired kernels take up to 86 KB of dynamic shared memory (256 threads);
// the attribute is a property of the kernel, set once per process and device.
cudaError_t su3k_prepare() {
  cudaError_t e = prepare_all<false>();
  if (e == cudaSuccess) e = prepare_all<true>();
  return e;
}
