// su3_kernels.cu -- sm_103a kernels of the checkerboard SU(3) heatbath sweep.
//
// One thread updates one link U_mu(x) of the half-sweep (mu, parity): it
// gathers the six-staple sum from the 18 neighbouring links, runs the one-hit
// Kennedy-Pendleton heatbath in the SU(2) subgroups (0,1), (0,2), (1,2)
// (Cabibbo-Marinari), reunitarises in FP64 and stores the link.  Links of one
// (mu, parity) never enter each other's staples (checkerboard updating,
// Abstract and Sec. 1 of Berg & Wu, arXiv:0904.1179), so threads are
// independent; the counter-based Philox stream makes the result independent of
// the launch configuration.  The work is a 4D stencil of 3x3 complex products,
// not a dense contraction, so it runs on the FP32/FP64 CUDA cores.
#include "su3_kernels.h"

#include "su3_device.cuh"
#include "su3_sitepair.cuh"
#include "su3_sweepq.cuh"
#include "su3_update.cuh"

using namespace su3dev;

// Register budget of the FP32-mixed half-sweep: __launch_bounds__(threads,
// min blocks per SM).  The defaults keep every block size up to
// kMaxSweepThreads legal.
#ifndef SU3_F32_LB_THREADS
#define SU3_F32_LB_THREADS kMaxSweepThreads
#endif
#ifndef SU3_F32_MINBLOCKS
#define SU3_F32_MINBLOCKS 4
#endif

namespace {

// ---------------------------------------------------------------------------
// Single-lattice half-sweeps: one thread per link of (mu, parity).
// ---------------------------------------------------------------------------
template <bool STATS>
__device__ __forceinline__ void count_stats(UpdateCount c, unsigned long long* stats) {
  if (STATS) {
    const int acc = __reduce_add_sync(0xffffffffu, c.accepted);
    const int prop = __reduce_add_sync(0xffffffffu, c.proposed);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&stats[0], (unsigned long long)acc);
      atomicAdd(&stats[1], (unsigned long long)prop);
    }
  }
}

// Block sum of one value per thread into out[blockIdx.x] (fixed order).
__device__ __forceinline__ void block_partial(double v, double* out) {
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

template <int MU, bool STATS, bool REPEAT, bool MEAS>
__global__ void __launch_bounds__(kMaxSweepThreads) k_half_sweep_f64(HalfSweepArgs args) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  UpdateCount c{0, 0};
  double m = 0.0;
  if (h < args.geom.Vh) {
    const UpdateConsts uc{args.three_over_beta_f64, args.three_over_beta, args.max_tries};
    c = update_link_f64<MU, false, REPEAT, MEAS>(args.geom, (double2*)args.links, h, args.parity, *args.sweep, args.key,
                                                 uc, &m);
  }
  count_stats<STATS>(c, args.stats);
  if (MEAS) block_partial(m, args.meas);
}

// The FP64 sweep as four persistent launches, one per direction MU with its
// even and odd half-sweeps, chained by programmatic dependent launch
// (su3_sweepq.cuh): a block takes a tile of `threads` sites of one parity in
// one x3 layer of the lattice and waits only for the layers of the previous
// half-sweep that its staples read, so one half-sweep's last wave overlaps
// the next one's first and only one launch tail per sweep remains.  The
// links change while the launch runs, so they are read through L2 (CG); the
// update is that of k_half_sweep_f64, bit for bit.
template <int MU, bool REPEAT>
__global__ void __launch_bounds__(kMaxSweepThreads)
    k_sweep_f64(HalfSweepArgs args, SweepQueue qa, int tiles_per_layer, int layers, int stats) {
  __shared__ SweepItem s_item;
  signal_dependents();
  take_sweep_item<2, 2 * MU>(qa, MU, tiles_per_layer, layers, &s_item);
  __syncthreads();
  const SweepItem it = s_item;
  if (it.phase < 0) return;
  const UpdateConsts uc{args.three_over_beta_f64, args.three_over_beta, args.max_tries};
  const int h = it.tile * (int)blockDim.x + (int)threadIdx.x;  // layers are whole tiles: always a site of the lattice
  const UpdateCount c =
      update_link_f64<MU, true, REPEAT, false>(args.geom, (double2*)args.links, h, it.phase & 1, *args.sweep, args.key, uc);
  if (stats) count_stats<true>(c, args.stats);
  report_sweep_item(qa, layers, it);
}

// One FP64 half-sweep (phase 2 MU + parity) of the chained sweep: one block
// per tile of sites of one x3 layer, the tile from the block's index
// (su3_sweepq.cuh), waiting only for the layers of the previous launch's
// half-sweep that its staples read.
template <int MU, bool REPEAT>
__global__ void __launch_bounds__(kMaxSweepThreads)
    k_half_sweep_f64_chain(HalfSweepArgs args, SweepQueue qa, int tiles_per_layer, int layers, int stats, int parity) {
  __shared__ SweepItem s_item;
  signal_dependents();
  own_sweep_item(qa, 2 * MU + parity, tiles_per_layer, layers, &s_item);
  __syncthreads();
  const SweepItem it = s_item;
  if (it.phase < 0) return;
  const UpdateConsts uc{args.three_over_beta_f64, args.three_over_beta, args.max_tries};
  const int h = it.tile * (int)blockDim.x + (int)threadIdx.x;  // layers are whole tiles: always a site of the lattice
  const UpdateCount c =
      update_link_f64<MU, true, REPEAT, false>(args.geom, (double2*)args.links, h, parity, *args.sweep, args.key, uc);
  if (stats) count_stats<true>(c, args.stats);
  report_sweep_item(qa, layers, it);
}

// A small lattice's half-sweep has too few links to fill the GPU, and each
// link's FP64 update is a long dependent chain: the time is its latency.
// Here four lanes share one link: lanes 0, 1, 2 compute rows 0,1 of the two
// staple paths of the first, second and third direction nu != MU at the same
// time, lane 0 gathers them and adds them up in the single-thread order
// (forward then backward path, nu ascending, row 2 formed in the
// accumulation), so the staple, and everything after it, is bit for bit that
// of k_half_sweep_f64.  Lane 3 only idles.
__device__ __forceinline__ mat3<double> shfl_rows01(const mat3<double>& m, int src) {
  mat3<double> r;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      r.e[i][k].re = __shfl_sync(0xffffffffu, m.e[i][k].re, src);
      r.e[i][k].im = __shfl_sync(0xffffffffu, m.e[i][k].im, src);
    }
  return r;
}

template <int MU, bool STATS>
__global__ void __launch_bounds__(kMaxSweepThreads) k_half_sweep_f64_split(HalfSweepArgs args) {
  const Geometry& g = args.geom;
  const int p = args.parity;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int link = gid >> 2, part = gid & 3;
  const bool active = link < g.Vh;
  const int h = active ? link : 0;  // a group past the end works on site 0 and discards it (shuffles stay converged)
  const Site st = site_of(g, h, p);
  double2* U = (double2*)args.links;
  mat3<double> F = zero3<double>(), B = zero3<double>();
  if (part < 3) {
    const int nu = part < MU ? part : part + 1;
    const int h_pmu = nb_half(g, st, MU, +1);
    F = forward_path<double, false>(g, U, st, h, p, MU, nu, h_pmu, nb_half_rt(g, st, nu, +1));
    B = backward_path<double, false>(g, U, p, MU, nu, nb_half_rt(g, st, nu, -1), nb_half2_rt(g, st, MU, nu));
  }
  const int lane0 = (threadIdx.x & 31) & ~3;
  mat3<double> A;
  init_completed(A, F);
  acc_completed(A, B);
#pragma unroll
  for (int k = 1; k < 3; ++k) {
    acc_completed(A, shfl_rows01(F, lane0 + k));
    acc_completed(A, shfl_rows01(B, lane0 + k));
  }
  UpdateCount c{0, 0};
  if (part == 0 && active) {
    const UpdateConsts uc{args.three_over_beta_f64, args.three_over_beta, 1};
    c = heatbath_f64<MU, false, false, false>(g, U, h, p, *args.sweep, (uint32_t)canon(g, st), args.key, uc, A, A,
                                             nullptr);
  }
  count_stats<STATS>(c, args.stats);
}

// The same four-lane split for FP32 storage: rows 0,1 of the staple paths on
// row pairs (12 floats each) are gathered into lane 0 and added in the
// single-thread order; no register cap (small lattices leave the SMs nearly
// empty).
__device__ __forceinline__ pm3 shfl_pm3_rows01(const pm3& m, int src) {
  pm3 r;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r.re[k].x = __shfl_sync(0xffffffffu, m.re[k].x, src);
    r.re[k].y = __shfl_sync(0xffffffffu, m.re[k].y, src);
    r.im[k].x = __shfl_sync(0xffffffffu, m.im[k].x, src);
    r.im[k].y = __shfl_sync(0xffffffffu, m.im[k].y, src);
  }
  return r;
}

template <int MU, bool STATS, bool EFT, bool PAIRS>
__global__ void __launch_bounds__(kMaxSweepThreads) k_half_sweep_f32_split(HalfSweepArgs args) {
  const Geometry& g = args.geom;
  const int p = args.parity;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int link = gid >> 2, part = gid & 3;
  const bool active = link < g.Vh;
  const int h = active ? link : 0;
  const Site st = site_of(g, h, p);
  float4* U = (float4*)args.links;
  pm3 F = zero_p(), B = zero_p();
  if (part < 3) {
    const int nu = part < MU ? part : part + 1;
    const int h_pmu = nb_half(g, st, MU, +1);
    F = forward_path_p<false, PAIRS>(g, U, h, p, MU, nu, h_pmu, nb_half_rt(g, st, nu, +1));
    B = backward_path_p<false, PAIRS>(g, U, p, MU, nu, nb_half_rt(g, st, nu, -1), nb_half2_rt(g, st, MU, nu));
  }
  const int lane0 = (threadIdx.x & 31) & ~3;
  pm3 A;
  init_completed_p(A, F);
  acc_completed_p(A, B);
#pragma unroll
  for (int k = 1; k < 3; ++k) {
    acc_completed_p(A, shfl_pm3_rows01(F, lane0 + k));
    acc_completed_p(A, shfl_pm3_rows01(B, lane0 + k));
  }
  UpdateCount c{0, 0};
  if (part == 0 && active) {
    const UpdateConsts uc{args.three_over_beta_f64, args.three_over_beta, 1};
    c = heatbath_f32_on<MU, EFT, false, false, PAIRS>(g, U, h, p, *args.sweep, (uint32_t)canon(g, st), args.key, uc, A,
                                                       A, nullptr, load_pm3_l<false, PAIRS>(U, MU, p, h, g.Vh), true);
  }
  count_stats<STATS>(c, args.stats);
}

template <int MU, bool STATS, bool EFT, bool REPEAT, bool MEAS>
__global__ void __launch_bounds__(SU3_F32_LB_THREADS, SU3_F32_MINBLOCKS) k_half_sweep_f32(HalfSweepArgs args) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  UpdateCount c{0, 0};
  double m = 0.0;
  if (h < args.geom.Vh) {
    const UpdateConsts uc{args.three_over_beta_f64, args.three_over_beta, args.max_tries};
    c = update_link_f32<MU, false, EFT, REPEAT, MEAS>(args.geom, (float4*)args.links, h, args.parity, *args.sweep,
                                                      args.key, uc, &m);
  }
  count_stats<STATS>(c, args.stats);
  if (MEAS) block_partial(m, args.meas);
}

__global__ void k_increment(uint64_t* counter, uint64_t n) { *counter += n; }

__global__ void __launch_bounds__(1024) k_meas_final(const double* parts, int n, double scale, const uint64_t* sweep,
                                                     double* out, int cap) {
  __shared__ double red[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += parts[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) out[*sweep % (uint64_t)cap] = w * scale;
  }
}
__global__ void k_set_counter(uint64_t* counter, uint64_t n) { *counter = n; }

// ---------------------------------------------------------------------------
// Start configurations.
// ---------------------------------------------------------------------------
__global__ void k_cold_start(InitArgs args) {
  const Geometry g = args.geom;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // over 8 * Vh (mu, parity, h)
  if (idx >= 8 * g.Vh) return;
  const int mp = idx / g.Vh, h = idx - mp * g.Vh;
  const int mu = mp >> 1, p = mp & 1;
  if (args.precision == 0) {
    mat3<double> m = zero3<double>();
    m.e[0][0] = m.e[1][1] = m.e[2][2] = mk(1.0, 0.0);
    store_f64((double2*)args.links, mu, p, h, g.Vh, m);
  } else {
    float o[12] = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f};
    store_f32_rows01_any((float4*)args.links, mu, p, h, g.Vh, args.pairs, o);
  }
}

// Haar SU(3): two complex Gaussian rows (Box-Muller on Philox tag 1 words,
// counter (s, mu | call<<4, 0, 1), call = 0..5), Gram-Schmidt, row 2 completed.
__global__ void k_hot_start(InitArgs args) {
  const Geometry g = args.geom;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 8 * g.Vh) return;
  const int mp = idx / g.Vh, h = idx - mp * g.Vh;
  const int mu = mp >> 1, p = mp & 1;
  const Site st = site_of(g, h, p);
  const uint32_t s = (uint32_t)canon(g, st);
  double gz[12];
#pragma unroll
  for (int call = 0; call < 6; ++call) {
    const uint4 w = philox4x32_10(rng_counter(s, (uint32_t)(mu | (call << 4)), 0, kTagHotStart), args.key);
    const double ua = u01_f64(w.x, w.y), ub = u01_f64(w.z, w.w);
    const double rad = sqrt(-2.0 * log(ua));
    double sn, cs;
    sincos(kTwoPi * ub, &sn, &cs);
    gz[2 * call] = rad * cs;
    gz[2 * call + 1] = rad * sn;
  }
  cx<double> r0[3], r1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r0[k] = mk(gz[2 * k], gz[2 * k + 1]);
    r1[k] = mk(gz[6 + 2 * k], gz[6 + 2 * k + 1]);
  }
  gram_schmidt_rows01(r0, r1);
  if (args.precision == 0) {
    mat3<double> m;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      m.e[0][k] = r0[k];
      m.e[1][k] = r1[k];
    }
    complete_row2(m);
    store_f64((double2*)args.links, mu, p, h, g.Vh, m);
  } else {
    float o[12];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      o[2 * k] = (float)r0[k].re;
      o[2 * k + 1] = (float)r0[k].im;
      o[6 + 2 * k] = (float)r1[k].re;
      o[6 + 2 * k + 1] = (float)r1[k].im;
    }
    store_f32_rows01_any((float4*)args.links, mu, p, h, g.Vh, args.pairs, o);
  }
}

// ---------------------------------------------------------------------------
// Plaquette: one thread per site, six planes, FP64 accumulation, fixed-order
// block reduction into partials[blockIdx.x], then one block sums the partials.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ mat3<T> load_any(const void* U, int mu, int p, int h, int Vh, bool pairs);
template <>
__device__ __forceinline__ mat3<double> load_any<double>(const void* U, int mu, int p, int h, int Vh, bool) {
  return load_f64((const double2*)U, mu, p, h, Vh);
}
template <>
__device__ __forceinline__ mat3<float> load_any<float>(const void* U, int mu, int p, int h, int Vh, bool pairs) {
  return load_f32_any((const float4*)U, mu, p, h, Vh, pairs);
}

// Re Tr(X Y^+) with X = U_mu(x) U_nu(x+mu), Y = U_nu(x) U_mu(x+nu).
template <typename T>
__device__ __forceinline__ double plaq_site(const Geometry& g, const void* U, const Site& st, int h, int p, bool pairs) {
  const int q = p ^ 1;
  double sum = 0.0;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu)
#pragma unroll
    for (int nu = mu + 1; nu < 4; ++nu) {
      const mat3<T> a = load_any<T>(U, mu, p, h, g.Vh, pairs);
      const mat3<T> b = load_any<T>(U, nu, q, nb_half(g, st, mu, +1), g.Vh, pairs);
      const mat3<T> c = load_any<T>(U, nu, p, h, g.Vh, pairs);
      const mat3<T> d = load_any<T>(U, mu, q, nb_half(g, st, nu, +1), g.Vh, pairs);
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

template <typename T>
__global__ void __launch_bounds__(256) k_plaquette_partial(PlaqArgs args) {
  const Geometry g = args.geom;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // over 2 * Vh: (parity, h)
  double v = 0.0;
  if (idx < 2 * g.Vh) {
    const int p = idx >= g.Vh ? 1 : 0;
    const int h = idx - p * g.Vh;
    const Site st = site_of(g, h, p);
    v = plaq_site<T>(g, args.links, st, h, p, args.pairs != 0);
  }
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x >> 5;
    double w = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) args.partials[blockIdx.x] = w;
  }
}

__global__ void __launch_bounds__(1024) k_plaquette_final(const double* partials, int n, double scale, double* out) {
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

// ---------------------------------------------------------------------------
// Canonical host layout <-> device store, for a chunk of sites [s_begin, s_begin + n).
// Canonical: double[s][mu][row][col][re/im].
// ---------------------------------------------------------------------------
// Row 2 from FP32 rows 0,1 in FP64 with every product and sum rounded
// separately (no contraction): conj(row0 x row1).
__device__ __forceinline__ cx<double> cmul_rn(cx<double> a, cx<double> b) {
  return mk(__dsub_rn(__dmul_rn(a.re, b.re), __dmul_rn(a.im, b.im)), __dadd_rn(__dmul_rn(a.re, b.im), __dmul_rn(a.im, b.re)));
}

__global__ void k_canon_to_store(ConvArgs args) {
  const Geometry g = args.geom;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4LL * args.n_sites) return;
  const int mu = (int)(idx / args.n_sites);
  const long long i = idx - (long long)mu * args.n_sites;
  const long long s = args.s_begin + i;
  const int h = (int)(s >> 1);
  const int x0 = (int)(s % g.L0);
  const int r = (int)(s / g.L0);
  const int x1 = r % g.L1, x2 = (r / g.L1) % g.L2, x3 = r / (g.L1 * g.L2);
  const int p = (x0 + x1 + x2 + x3) & 1;
  const double* src = args.canon + (i * 4 + mu) * 18;
  if (args.precision == 0) {
    mat3<double> m;
#pragma unroll
    for (int c = 0; c < 9; ++c) m.e[c / 3][c % 3] = mk(src[2 * c], src[2 * c + 1]);
    store_f64((double2*)args.links, mu, p, h, g.Vh, m);
  } else {
    float o[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) o[c] = (float)src[c];
    store_f32_rows01_any((float4*)args.links, mu, p, h, g.Vh, args.pairs, o);
  }
}

__global__ void k_store_to_canon(ConvArgs args) {
  const Geometry g = args.geom;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4LL * args.n_sites) return;
  const int mu = (int)(idx / args.n_sites);
  const long long i = idx - (long long)mu * args.n_sites;
  const long long s = args.s_begin + i;
  const int h = (int)(s >> 1);
  const int x0 = (int)(s % g.L0);
  const int r = (int)(s / g.L0);
  const int x1 = r % g.L1, x2 = (r / g.L1) % g.L2, x3 = r / (g.L1 * g.L2);
  const int p = (x0 + x1 + x2 + x3) & 1;
  double* dst = args.canon + (i * 4 + mu) * 18;
  if (args.precision == 0) {
    const mat3<double> m = load_f64((const double2*)args.links, mu, p, h, g.Vh);
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      dst[2 * c] = m.e[c / 3][c % 3].re;
      dst[2 * c + 1] = m.e[c / 3][c % 3].im;
    }
  } else {
    const mat3<float> m = load_f32_rows01_any((const float4*)args.links, mu, p, h, g.Vh, args.pairs);
    cx<double> a[3], b[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      a[k] = mk((double)m.e[0][k].re, (double)m.e[0][k].im);
      b[k] = mk((double)m.e[1][k].re, (double)m.e[1][k].im);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dst[2 * k] = a[k].re;
      dst[2 * k + 1] = a[k].im;
      dst[6 + 2 * k] = b[k].re;
      dst[6 + 2 * k + 1] = b[k].im;
    }
    const cx<double> x = cmul_rn(a[1], b[2]), y = cmul_rn(a[2], b[1]);
    const cx<double> z0 = mk(__dsub_rn(x.re, y.re), __dsub_rn(x.im, y.im));
    const cx<double> x1c = cmul_rn(a[2], b[0]), y1 = cmul_rn(a[0], b[2]);
    const cx<double> z1 = mk(__dsub_rn(x1c.re, y1.re), __dsub_rn(x1c.im, y1.im));
    const cx<double> x2c = cmul_rn(a[0], b[1]), y2 = cmul_rn(a[1], b[0]);
    const cx<double> z2 = mk(__dsub_rn(x2c.re, y2.re), __dsub_rn(x2c.im, y2.im));
    dst[12] = z0.re;
    dst[13] = -z0.im;
    dst[14] = z1.re;
    dst[15] = -z1.im;
    dst[16] = z2.re;
    dst[17] = -z2.im;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
template <int MU, bool REPEAT>
static cudaError_t launch_chain_f64_mu(const HalfSweepArgs& a, const SweepQueue& q, int tpl, int layers, int st,
                                       int threads, cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tpl * layers);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = attr;
  for (int p = 0; p < 2; ++p) {
    cfg.numAttrs = MU == 0 && p == 0 ? 0 : 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_half_sweep_f64_chain<MU, REPEAT>, a, q, tpl, layers, st, p);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <bool REPEAT>
static cudaError_t launch_sweep_f64(const HalfSweepArgs& a, const SweepQueue& q, int tpl, int layers, bool stats,
                                    int threads, bool chained, cudaStream_t s) {
  const int blocks = 2 * tpl * layers, st = stats ? 1 : 0;
  if (chained) {
    cudaError_t e;
    if ((e = launch_chain_f64_mu<0, REPEAT>(a, q, tpl, layers, st, threads, s)) != cudaSuccess) return e;
    if ((e = launch_chain_f64_mu<1, REPEAT>(a, q, tpl, layers, st, threads, s)) != cudaSuccess) return e;
    if ((e = launch_chain_f64_mu<2, REPEAT>(a, q, tpl, layers, st, threads, s)) != cudaSuccess) return e;
    return launch_chain_f64_mu<3, REPEAT>(a, q, tpl, layers, st, threads, s);
  }
  k_sweep_f64<0, REPEAT><<<blocks, threads, 0, s>>>(a, q, tpl, layers, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // directions 1-3: programmatic dependent launches (su3_sweepq.cuh)
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if ((e = cudaLaunchKernelEx(&cfg, k_sweep_f64<1, REPEAT>, a, q, tpl, layers, st)) != cudaSuccess) return e;
  if ((e = cudaLaunchKernelEx(&cfg, k_sweep_f64<2, REPEAT>, a, q, tpl, layers, st)) != cudaSuccess) return e;
  return cudaLaunchKernelEx(&cfg, k_sweep_f64<3, REPEAT>, a, q, tpl, layers, st);
}

template <int MU, bool STATS, bool EFT, bool REPEAT, bool MEAS>
static cudaError_t launch_f32(const HalfSweepArgs& a, int blocks, int threads, cudaStream_t s) {
  k_half_sweep_f32<MU, STATS, EFT, REPEAT, MEAS><<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

template <int MU, bool STATS, bool REPEAT, bool MEAS>
static cudaError_t launch_prec(const HalfSweepArgs& a, int precision, int blocks, int threads, cudaStream_t s) {
  if (precision == 0) {
    k_half_sweep_f64<MU, STATS, REPEAT, MEAS><<<blocks, threads, 0, s>>>(a);
    return cudaGetLastError();
  }
  if (precision == 2) return launch_f32<MU, STATS, true, REPEAT, MEAS>(a, blocks, threads, s);
  return launch_f32<MU, STATS, false, REPEAT, MEAS>(a, blocks, threads, s);
}

template <int MU, bool STATS, bool EFT>
static void launch_f32_split(const HalfSweepArgs& a, int blocks, int threads, cudaStream_t s) {
  if (a.pairs)
    k_half_sweep_f32_split<MU, STATS, EFT, true><<<blocks, threads, 0, s>>>(a);
  else
    k_half_sweep_f32_split<MU, STATS, EFT, false><<<blocks, threads, 0, s>>>(a);
}

template <int MU>
static cudaError_t launch_half_sweep_mu(const HalfSweepArgs& a, int precision, bool stats, int threads, cudaStream_t s) {
  const int blocks = (a.geom.Vh + threads - 1) / threads;
  const bool repeat = a.max_tries > 1;
  // FP32 in the site-paired layout: the paired kernel, except for the
  // four-lane form of small lattices
  if (precision != 0 && a.pairs && !(a.split && !repeat && !(MU > 0 && a.meas)))
    return su3k_launch_half_sweep_pair(a, MU, precision == 2, stats, threads, s);
  if (MU > 0 && a.meas) {  // fused plaquette (statistics are not counted in these phases)
    return repeat ? launch_prec<MU, false, true, (MU > 0)>(a, precision, blocks, threads, s)
                  : launch_prec<MU, false, false, (MU > 0)>(a, precision, blocks, threads, s);
  }
  if (a.split && !repeat) {
    const int sblocks = (4 * a.geom.Vh + threads - 1) / threads;
    if (precision == 0) {
      if (stats)
        k_half_sweep_f64_split<MU, true><<<sblocks, threads, 0, s>>>(a);
      else
        k_half_sweep_f64_split<MU, false><<<sblocks, threads, 0, s>>>(a);
    } else if (precision == 2) {
      if (stats)
        launch_f32_split<MU, true, true>(a, sblocks, threads, s);
      else
        launch_f32_split<MU, false, true>(a, sblocks, threads, s);
    } else {
      if (stats)
        launch_f32_split<MU, true, false>(a, sblocks, threads, s);
      else
        launch_f32_split<MU, false, false>(a, sblocks, threads, s);
    }
    return cudaGetLastError();
  }
  if (stats)
    return repeat ? launch_prec<MU, true, true, false>(a, precision, blocks, threads, s)
                  : launch_prec<MU, true, false, false>(a, precision, blocks, threads, s);
  return repeat ? launch_prec<MU, false, true, false>(a, precision, blocks, threads, s)
                : launch_prec<MU, false, false, false>(a, precision, blocks, threads, s);
}

int su3k_f64_sweep_layers(const Geometry& g, int threads, int* tiles_per_layer) {
  const long long per_layer = (long long)g.hL0 * g.L1 * g.L2;  // sites of one parity in one x3 layer
  if (threads <= 0 || threads > kMaxSweepThreads || per_layer % threads != 0 || g.L3 < 4) return 0;
  *tiles_per_layer = (int)(per_layer / threads);
  return g.L3;
}

cudaError_t su3k_launch_sweep_f64(const HalfSweepArgs& a, const SweepQueue& q, bool stats, int threads, bool chained,
                                  cudaStream_t s) {
  int tpl = 0;
  const int layers = su3k_f64_sweep_layers(a.geom, threads, &tpl);
  if (layers == 0 || a.meas || a.split) return cudaErrorInvalidValue;
  return a.max_tries > 1 ? launch_sweep_f64<true>(a, q, tpl, layers, stats, threads, chained, s)
                         : launch_sweep_f64<false>(a, q, tpl, layers, stats, threads, chained, s);
}

cudaError_t su3k_launch_half_sweep(const HalfSweepArgs& a, int mu, int precision, bool stats, int threads, cudaStream_t s) {
  switch (mu) {
    case 0: return launch_half_sweep_mu<0>(a, precision, stats, threads, s);
    case 1: return launch_half_sweep_mu<1>(a, precision, stats, threads, s);
    case 2: return launch_half_sweep_mu<2>(a, precision, stats, threads, s);
    default: return launch_half_sweep_mu<3>(a, precision, stats, threads, s);
  }
}

SU3_BOUNDS_STATUS_FN(su3k_bounds_status_kernels)

int su3k_half_sweep_blocks(const HalfSweepArgs& a, int precision, int threads) {
  const int n = (precision != 0 && a.pairs) ? a.pgeom.Vh : a.geom.Vh;
  return (n + threads - 1) / threads;
}

cudaError_t su3k_launch_increment(uint64_t* counter, uint64_t n, cudaStream_t s) {
  k_increment<<<1, 1, 0, s>>>(counter, n);
  return cudaGetLastError();
}

cudaError_t su3k_launch_meas_final(const double* parts, int nparts, double scale, const uint64_t* sweep, double* out,
                                   int cap, cudaStream_t s) {
  k_meas_final<<<1, 1024, 0, s>>>(parts, nparts, scale, sweep, out, cap);
  return cudaGetLastError();
}

cudaError_t su3k_launch_set_counter(uint64_t* counter, uint64_t n, cudaStream_t s) {
  k_set_counter<<<1, 1, 0, s>>>(counter, n);
  return cudaGetLastError();
}

cudaError_t su3k_launch_init(const InitArgs& a, bool hot, cudaStream_t s) {
  const long long n = 8LL * a.geom.Vh;
  const int threads = 128;
  const int blocks = (int)((n + threads - 1) / threads);
  if (hot)
    k_hot_start<<<blocks, threads, 0, s>>>(a);
  else
    k_cold_start<<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

int su3k_plaquette_blocks(const Geometry& g) { return (2 * g.Vh + 255) / 256; }

cudaError_t su3k_launch_plaquette(const PlaqArgs& a, int precision, double* out, cudaStream_t s) {
  const int blocks = su3k_plaquette_blocks(a.geom);
  if (precision == 0)
    k_plaquette_partial<double><<<blocks, 256, 0, s>>>(a);
  else
    k_plaquette_partial<float><<<blocks, 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const double V = 2.0 * (double)a.geom.Vh;
  k_plaquette_final<<<1, 1024, 0, s>>>(a.partials, blocks, 1.0 / (3.0 * 6.0 * V), out);
  return cudaGetLastError();
}

cudaError_t su3k_launch_conv(const ConvArgs& a, bool to_store, cudaStream_t s) {
  const long long n = 4LL * a.n_sites;
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  const long long blocks = (n + threads - 1) / threads;
  if (to_store)
    k_canon_to_store<<<(unsigned)blocks, threads, 0, s>>>(a);
  else
    k_store_to_canon<<<(unsigned)blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}
