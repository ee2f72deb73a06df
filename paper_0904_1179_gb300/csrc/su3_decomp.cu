// su3_decomp.cu -- the paper's domain decomposition emulated on one device.
//
// Berg & Wu (arXiv:0904.1179, Sec. 2.1) cut the first ndmpi directions of the
// lattice into mpifactor parts each; every sublattice lives in its own MPI
// process and, between checkerboard steps, sends the boundary links its
// neighbours need (Appendix A: the checkerboard link storage of a face,
// Eq. (mscb18)).  With np = 1 the switch lbcex turns that exchange off (one
// sublattice with periodic wrap inside it) or on (the sublattice exchanges
// with itself), the "1F" and "1" rows of Tables 1 and 2.
//
// Here all np sublattices live on one GPU, each in its own extended-box store
// with a ghost layer on both sides of every cut direction.  One sweep is, for
// mu = 0..3 and parity even then odd:
//   1. one launch updating the (mu, parity) links of every sublattice (the
//      same per-link code as the single lattice, on the sublattice geometry);
//   2. one launch of the boundary exchange: the updated (mu, parity) links on
//      the sublattice faces are copied into the ghost cells that read them
//      (faces, and the edges x + a - b that the staples' corner paths reach),
//      from gather lists built once on the host.
// The random numbers are keyed by the global site, so every link comes out
// bit for bit as in the undivided lattice; what the emulation adds is the
// measured cost of the exchange on a GB300.
#include <new>
#include <vector>

#include "su3_device.cuh"
#include "su3_kernels.h"
#include "su3_runtime.h"
#include "su3_update.cuh"

using namespace su3dev;

struct su3_decomp {
  int ndmpi = 0, nf = 1, np = 1, lbcex = 1;
  bool active = false;         // true once the sublattice stores exist
  SubGeometry geo{};           // sublattice geometry, origin 0
  size_t sub_elems = 0;        // double2 (FP64) or float4 (FP32) elements per sublattice store
  void* d_sub = nullptr;       // np stores
  int4* d_ghost[2] = {nullptr, nullptr};  // gather lists per parity: {dst sub, dst half, src sub, src half}
  int nghost[2] = {0, 0};
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // indexed by stats_on
  cudaGraphExec_t graph_meas = nullptr;            // sweep with the fused plaquette
  bool subs_current = false;   // sublattice stores hold the configuration
  bool global_current = true;  // the handle's global store holds it
};

namespace {

struct DecompArgs {
  SubGeometry g;
  int nf, ndmpi;
  PhiloxRoundKeys key;
  int parity;
  double three_over_beta_f64;
  float three_over_beta;
  const uint64_t* sweep;
  void* subs;
  size_t sub_elems;
  unsigned long long* stats;
  int count_stats;   // accumulate acceptance statistics
  int max_tries;     // SU(2) proposals per subgroup (1: one-hit heatbath)
  double* meas;      // fused plaquette: one partial per block of this phase (nullptr: off)
};

// Origin of sublattice k (index k = k0 + nf*(k1 + nf*...) over the cut directions).
__device__ __forceinline__ SubGeometry sub_geometry(const SubGeometry& base, int nf, int ndmpi, int k) {
  SubGeometry g = base;
  const int l[4] = {base.in.L0, base.in.L1, base.in.L2, base.in.L3};
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    g.o[d] = d < ndmpi ? (k % nf) * l[d] : 0;
    if (d < ndmpi) k /= nf;
  }
  return g;
}

__device__ __forceinline__ void count_stats_d(UpdateCount c, unsigned long long* stats) {
  const int acc = __reduce_add_sync(0xffffffffu, c.accepted);
  const int prop = __reduce_add_sync(0xffffffffu, c.proposed);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&stats[0], (unsigned long long)acc);
    atomicAdd(&stats[1], (unsigned long long)prop);
  }
}

// Block sum of one value per thread into out[block index over the 2D grid], fixed order.
__device__ __forceinline__ void block_partial_d(double v, double* out) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) out[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = w;
  }
}

// REPEAT: repeat-until-accepted heatbath (a.max_tries proposals at most).
// MEAS: the fused plaquette of the odd-site phases of mu = 1, 2, 3, as in the
// undivided kernels (every link of A_< is final; the ghosts were refreshed by
// the exchanges after the phases before).
template <int MU, bool REPEAT, bool MEAS>
__global__ void __launch_bounds__(kMaxSweepThreads) k_decomp_half_sweep_f64(DecompArgs a) {
  const int k = blockIdx.y;
  const SubGeometry g = sub_geometry(a.g, a.nf, a.ndmpi, k);
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  UpdateCount c{0, 0};
  double m = 0.0;
  if (h < g.in.Vh) {
    const UpdateConsts uc{a.three_over_beta_f64, a.three_over_beta, a.max_tries};
    double2* U = (double2*)a.subs + (size_t)k * a.sub_elems;
    c = update_link_f64<MU, false, REPEAT, MEAS>(g, U, h, a.parity, *a.sweep, a.key, uc, &m);
  }
  if (a.count_stats) count_stats_d(c, a.stats);
  if (MEAS) block_partial_d(m, a.meas);
}

template <int MU, bool EFT, bool REPEAT, bool MEAS>
__global__ void __launch_bounds__(kMaxSweepThreads, 4) k_decomp_half_sweep_f32(DecompArgs a) {
  const int k = blockIdx.y;
  const SubGeometry g = sub_geometry(a.g, a.nf, a.ndmpi, k);
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  UpdateCount c{0, 0};
  double m = 0.0;
  if (h < g.in.Vh) {
    const UpdateConsts uc{a.three_over_beta_f64, a.three_over_beta, a.max_tries};
    float4* U = (float4*)a.subs + (size_t)k * a.sub_elems;
    c = update_link_f32<MU, false, EFT, REPEAT, MEAS>(g, U, h, a.parity, *a.sweep, a.key, uc, &m);
  }
  if (a.count_stats) count_stats_d(c, a.stats);
  if (MEAS) block_partial_d(m, a.meas);
}

// Boundary exchange of the (mu, parity) links: one thread per ghost cell.
template <typename E, int NC>
__global__ void k_decomp_exchange(const int4* __restrict__ list, int n, int mu, int parity, E* subs,
                                  size_t sub_elems, int Vh, int nsub) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int4 e = list[i];
  if (!link_ok(mu, parity, e.y, Vh) || !link_ok(mu, parity, e.w, Vh) || !link_ok(0, 0, e.x, nsub) ||
      !link_ok(0, 0, e.z, nsub))
    return;
  const size_t off = link_base(mu, parity, Vh, NC);
  const E* src = subs + (size_t)e.z * sub_elems + off + e.w;
  E* dst = subs + (size_t)e.x * sub_elems + off + e.y;
#pragma unroll
  for (int c = 0; c < NC; ++c) dst[(size_t)c * Vh] = src[(size_t)c * Vh];
}

// Global store <-> sublattice interiors, all four directions of each site.
template <typename E, int NC, bool TO_SUBS>
__global__ void k_decomp_move(SubGeometry base, int nf, int ndmpi, E* global, int Vh_global, E* subs,
                              size_t sub_elems) {
  const int k = blockIdx.y, p = blockIdx.z;
  const SubGeometry g = sub_geometry(base, nf, ndmpi, k);
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= g.in.Vh) return;
  const SubSite st = site_of(g, h, p);
  const int hg = st.s >> 1;
  const int hs = store_index(g, st, h);
  if (!link_ok(0, p, hg, Vh_global) || !link_ok(0, p, hs, g.Vh)) return;
  E* sub = subs + (size_t)k * sub_elems;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    E* a = global + link_base(mu, p, Vh_global, NC) + hg;
    E* b = sub + link_base(mu, p, g.Vh, NC) + hs;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (TO_SUBS)
        b[(size_t)c * g.Vh] = a[(size_t)c * Vh_global];
      else
        a[(size_t)c * Vh_global] = b[(size_t)c * g.Vh];
    }
  }
}

// The same move for an FP32 global store in the site-paired layout
// (su3_sitepair.cuh; the sublattice stores keep one site per column group).
template <bool TO_SUBS>
__global__ void k_decomp_move_f32_pairs(SubGeometry base, int nf, int ndmpi, float4* global, int Vh_global,
                                        float4* subs, size_t sub_elems) {
  const int k = blockIdx.y, p = blockIdx.z;
  const SubGeometry g = sub_geometry(base, nf, ndmpi, k);
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= g.in.Vh) return;
  const SubSite st = site_of(g, h, p);
  const int hg = st.s >> 1;
  const int hs = store_index(g, st, h);
  float4* sub = subs + (size_t)k * sub_elems;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    float r[12];
    if (TO_SUBS) {
      load_pair_site(global, mu, p, hg, Vh_global / 2, r);
      store_f32_rows01(sub, mu, p, hs, g.Vh, r);
    } else {
      const mat3<float> m = load_f32_rows01(sub, mu, p, hs, g.Vh);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        r[2 * c] = m.e[0][c].re;
        r[2 * c + 1] = m.e[0][c].im;
        r[6 + 2 * c] = m.e[1][c].re;
        r[6 + 2 * c + 1] = m.e[1][c].im;
      }
      store_pair_site(global, mu, p, hg, Vh_global / 2, r);
    }
  }
}

template <int MU, bool REPEAT, bool MEAS>
cudaError_t launch_update_form(const DecompArgs& a, int precision, const dim3& grid, int threads, cudaStream_t s) {
  if (precision == SU3_FP64)
    k_decomp_half_sweep_f64<MU, REPEAT, MEAS><<<grid, threads, 0, s>>>(a);
  else if (precision == SU3_FP32_EFT)
    k_decomp_half_sweep_f32<MU, true, REPEAT, MEAS><<<grid, threads, 0, s>>>(a);
  else
    k_decomp_half_sweep_f32<MU, false, REPEAT, MEAS><<<grid, threads, 0, s>>>(a);
  return cudaGetLastError();
}

template <int MU>
cudaError_t launch_update_mu(const DecompArgs& a, int precision, bool stats, int threads, int np, cudaStream_t s) {
  const dim3 grid((a.g.in.Vh + threads - 1) / threads, np);
  DecompArgs b = a;
  b.count_stats = stats ? 1 : 0;
  const bool repeat = a.max_tries > 1;
  if (MU > 0 && a.meas) {  // fused plaquette (statistics are not counted in these phases)
    b.count_stats = 0;
    return repeat ? launch_update_form<MU, true, (MU > 0)>(b, precision, grid, threads, s)
                  : launch_update_form<MU, false, (MU > 0)>(b, precision, grid, threads, s);
  }
  return repeat ? launch_update_form<MU, true, false>(b, precision, grid, threads, s)
                : launch_update_form<MU, false, false>(b, precision, grid, threads, s);
}

cudaError_t launch_update(const DecompArgs& a, int mu, int precision, bool stats, int threads, int np, cudaStream_t s) {
  switch (mu) {
    case 0: return launch_update_mu<0>(a, precision, stats, threads, np, s);
    case 1: return launch_update_mu<1>(a, precision, stats, threads, np, s);
    case 2: return launch_update_mu<2>(a, precision, stats, threads, np, s);
    default: return launch_update_mu<3>(a, precision, stats, threads, np, s);
  }
}

cudaError_t launch_exchange(const su3_decomp* d, int precision, int mu, int parity, cudaStream_t s) {
  const int n = d->nghost[parity];
  if (n == 0) return cudaSuccess;
  const int threads = 256, blocks = (n + threads - 1) / threads;
  if (precision == SU3_FP64)
    k_decomp_exchange<double2, kEntriesF64><<<blocks, threads, 0, s>>>(d->d_ghost[parity], n, mu, parity,
                                                                       (double2*)d->d_sub, d->sub_elems, d->geo.Vh,
                                                                       d->np);
  else
    k_decomp_exchange<float4, kGroupsF32><<<blocks, threads, 0, s>>>(d->d_ghost[parity], n, mu, parity,
                                                                     (float4*)d->d_sub, d->sub_elems, d->geo.Vh,
                                                                     d->np);
  return cudaGetLastError();
}

cudaError_t launch_move(const su3_lattice* h, bool to_subs) {
  const su3_decomp* d = h->decomp;
  const int threads = 256;
  const dim3 grid((d->geo.in.Vh + threads - 1) / threads, d->np, 2);
  if (h->precision == SU3_FP64) {
    if (to_subs)
      k_decomp_move<double2, kEntriesF64, true><<<grid, threads, 0, h->stream>>>(
          d->geo, d->nf, d->ndmpi, (double2*)h->links, h->geom.Vh, (double2*)d->d_sub, d->sub_elems);
    else
      k_decomp_move<double2, kEntriesF64, false><<<grid, threads, 0, h->stream>>>(
          d->geo, d->nf, d->ndmpi, (double2*)h->links, h->geom.Vh, (double2*)d->d_sub, d->sub_elems);
  } else if (h->pairs) {
    if (to_subs)
      k_decomp_move_f32_pairs<true><<<grid, threads, 0, h->stream>>>(d->geo, d->nf, d->ndmpi, (float4*)h->links,
                                                                      h->geom.Vh, (float4*)d->d_sub, d->sub_elems);
    else
      k_decomp_move_f32_pairs<false><<<grid, threads, 0, h->stream>>>(d->geo, d->nf, d->ndmpi, (float4*)h->links,
                                                                       h->geom.Vh, (float4*)d->d_sub, d->sub_elems);
  } else {
    if (to_subs)
      k_decomp_move<float4, kGroupsF32, true><<<grid, threads, 0, h->stream>>>(
          d->geo, d->nf, d->ndmpi, (float4*)h->links, h->geom.Vh, (float4*)d->d_sub, d->sub_elems);
    else
      k_decomp_move<float4, kGroupsF32, false><<<grid, threads, 0, h->stream>>>(
          d->geo, d->nf, d->ndmpi, (float4*)h->links, h->geom.Vh, (float4*)d->d_sub, d->sub_elems);
  }
  return cudaGetLastError();
}

DecompArgs decomp_args(const su3_lattice* h, int parity) {
  const su3_decomp* d = h->decomp;
  DecompArgs a{};
  a.g = d->geo;
  a.nf = d->nf;
  a.ndmpi = d->ndmpi;
  a.key = philox_round_keys(h->key);
  a.parity = parity;
  a.three_over_beta_f64 = 3.0 / h->beta;
  a.three_over_beta = (float)(3.0 / h->beta);
  a.sweep = h->d_sweep;
  a.subs = d->d_sub;
  a.sub_elems = d->sub_elems;
  a.stats = h->d_stats;
  a.max_tries = h->max_tries;
  a.meas = nullptr;
  return a;
}

// Blocks of one decomposed half-sweep launch (the fused plaquette leaves one
// partial per block).
int phase_blocks(const su3_lattice* h) {
  const su3_decomp* d = h->decomp;
  return (d->geo.in.Vh + h->threads - 1) / h->threads * d->np;
}

int enqueue_phase(su3_lattice* h, int mu, int parity, double* meas = nullptr) {
  su3_decomp* d = h->decomp;
  DecompArgs a = decomp_args(h, parity);
  a.meas = meas;
  SU3_CUDA(launch_update(a, mu, h->precision, h->stats_on, h->threads, d->np, h->stream),
           "decomposed half-sweep launch");
  SU3_CUDA(launch_exchange(d, h->precision, mu, parity, h->stream), "boundary exchange launch");
  return SU3_OK;
}

// Bring the sublattice stores up to date from the global store (after a start
// configuration or su3_links_set): scatter the interiors, then fill every ghost.
int ensure_subs(su3_lattice* h) {
  su3_decomp* d = h->decomp;
  if (d->subs_current) return SU3_OK;
  SU3_CUDA(launch_move(h, true), "decomposition scatter");
  for (int mu = 0; mu < 4; ++mu)
    for (int p = 0; p < 2; ++p) SU3_CUDA(launch_exchange(d, h->precision, mu, p, h->stream), "ghost fill");
  d->subs_current = true;
  return SU3_OK;
}

// With `measured`, the odd-site phases of mu = 1, 2, 3 leave block partials of
// the fused plaquette in h->d_meas_parts and a last kernel sums them into the
// ring slot of this sweep (as in the undivided sweep).
int ensure_decomp_graph(su3_lattice* h, bool measured = false) {
  su3_decomp* d = h->decomp;
  cudaGraphExec_t& exec = measured ? d->graph_meas : d->graph[h->stats_on ? 1 : 0];
  if (exec) return SU3_OK;
  const int blocks = phase_blocks(h);
  cudaGraph_t graph = nullptr;
  SU3_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "graph capture begin");
  int rc = SU3_OK;
  for (int mu = 0; mu < 4 && rc == SU3_OK; ++mu)
    for (int p = 0; p < 2 && rc == SU3_OK; ++p)
      rc = enqueue_phase(h, mu, p, measured && p == 1 && mu >= 1 ? h->d_meas_parts + (size_t)(mu - 1) * blocks : nullptr);
  if (rc == SU3_OK && measured) {
    const cudaError_t e = su3k_launch_meas_final(h->d_meas_parts, 3 * blocks, 1.0 / (6.0 * (double)h->V), h->d_sweep,
                                                 h->d_meas, h->meas_cap, h->stream);
    if (e != cudaSuccess) rc = su3_cuda_fail(e, "plaquette reduction launch");
  }
  if (rc == SU3_OK) {
    const cudaError_t e = su3k_launch_increment(h->d_sweep, 1, h->stream);
    if (e != cudaSuccess) rc = su3_cuda_fail(e, "sweep counter launch");
  }
  const cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  if (rc != SU3_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  SU3_CUDA(e, "graph capture end");
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  SU3_CUDA(ei, "graph instantiate");
  return SU3_OK;
}

// Gather lists of the boundary exchange.  A ghost cell is read by a staple if
// exactly one cut coordinate lies outside the interior (a face: x +- nu), or
// two do with one above and one below (an edge: x + mu - nu).
void build_ghost_lists(const int L[4], int ndmpi, int nf, int np, const SubGeometry& g, std::vector<int4> lists[2]) {
  const int* e = g.e;
  const int l[4] = {g.in.L0, g.in.L1, g.in.L2, g.in.L3};
  for (int k = 0; k < np; ++k) {
    int o[4] = {0, 0, 0, 0}, kk = k;
    for (int dd = 0; dd < ndmpi; ++dd) {
      o[dd] = (kk % nf) * l[dd];
      kk /= nf;
    }
    for (int y3 = 0; y3 < e[3]; ++y3)
      for (int y2 = 0; y2 < e[2]; ++y2)
        for (int y1 = 0; y1 < e[1]; ++y1)
          for (int y0 = 0; y0 < e[0]; ++y0) {
            const int y[4] = {y0, y1, y2, y3};
            int below = 0, above = 0;
            for (int dd = 0; dd < 4; ++dd) {
              if (!((g.cut >> dd) & 1)) continue;
              if (y[dd] == 0) ++below;
              if (y[dd] == e[dd] - 1) ++above;
            }
            const int out = below + above;
            if (out == 0 || out > 2 || (out == 2 && (below != 1 || above != 1))) continue;
            int x[4], ys[4], ksrc = 0, mul = 1, par = 0;
            for (int dd = 0; dd < 4; ++dd) {
              const int c = (g.cut >> dd) & 1;
              x[dd] = ((y[dd] - c + o[dd]) % L[dd] + L[dd]) % L[dd];
              par += x[dd];
              if (c) {
                ksrc += (x[dd] / l[dd]) * mul;
                mul *= nf;
                ys[dd] = x[dd] % l[dd] + 1;
              } else {
                ys[dd] = x[dd];
              }
            }
            const int dst = (y[0] >> 1) + g.he0 * (y[1] + e[1] * (y[2] + e[2] * y[3]));
            const int src = (ys[0] >> 1) + g.he0 * (ys[1] + e[1] * (ys[2] + e[2] * ys[3]));
            lists[par & 1].push_back(make_int4(k, dst, ksrc, src));
          }
  }
}

int check_decomposition(const char* fn, const int L[4], int ndmpi, int mpifactor, int lbcex, long long* np) {
  if (ndmpi < 1 || ndmpi > 4) return su3_fail(SU3_EINVAL, "%s: ndmpi %d not in [1, 4]", fn, ndmpi);
  if (mpifactor < 1) return su3_fail(SU3_EINVAL, "%s: mpifactor %d < 1", fn, mpifactor);
  if (lbcex != 0 && lbcex != 1) return su3_fail(SU3_EINVAL, "%s: lbcex must be 0 or 1", fn);
  if (!lbcex && mpifactor > 1)
    return su3_fail(SU3_EINVAL, "%s: the exchange can be off only for one sublattice (mpifactor 1)", fn);
  for (int d = 0; d < 4; ++d)
    if (L[d] < 2 || (L[d] & 1)) return su3_fail(SU3_EINVAL, "%s: extent L%d = %d must be even and >= 2", fn, d, L[d]);
  if (4LL * L[0] * L[1] * L[2] * L[3] > 0x7fffffffLL) return su3_fail(SU3_EINVAL, "%s: 4*V exceeds 2^31-1", fn);
  for (int d = 0; d < ndmpi; ++d)
    if (L[d] % mpifactor || (L[d] / mpifactor) % 2 || L[d] / mpifactor < 2)
      return su3_fail(SU3_EINVAL, "%s: L%d = %d does not split into %d even parts >= 2", fn, d, L[d], mpifactor);
  *np = 1;
  for (int d = 0; d < ndmpi; ++d) *np *= mpifactor;
  if (*np > 65535) return su3_fail(SU3_EINVAL, "%s: %lld sublattices (at most 65535)", fn, *np);
  return SU3_OK;
}

// Sublattice geometry (origin 0): interior extents L/mpifactor in the cut
// directions, one ghost layer on each side of them.
void host_sub_geometry(const int L[4], int ndmpi, int mpifactor, SubGeometry& g) {
  int l[4];
  long long ext = 1;
  g.cut = 0;
  for (int dd = 0; dd < 4; ++dd) {
    const bool cut = dd < ndmpi;
    l[dd] = cut ? L[dd] / mpifactor : L[dd];
    g.e[dd] = l[dd] + (cut ? 2 : 0);
    g.o[dd] = 0;
    if (cut) g.cut |= 1 << dd;
    ext *= g.e[dd];
  }
  g.in = make_geometry(l[0], l[1], l[2], l[3]);
  g.he0 = g.e[0] / 2;
  g.L0 = L[0];
  g.L1 = L[1];
  g.L2 = L[2];
  g.Vh = (int)(ext / 2);
}

}  // namespace

// ---------------------------------------------------------------------------
// Hooks for su3_api.cu.
// ---------------------------------------------------------------------------
bool su3_decomp_active(const su3_lattice* h) { return h && h->decomp && h->decomp->active; }

SU3_BOUNDS_STATUS_FN(su3k_bounds_status_decomp)

void su3_decomp_invalidate(su3_decomp* d) {
  for (auto& g : d->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  if (d->graph_meas) {
    cudaGraphExecDestroy(d->graph_meas);
    d->graph_meas = nullptr;
  }
}

void su3_decomp_release(su3_decomp* d) {
  if (!d) return;
  su3_decomp_invalidate(d);
  cudaFree(d->d_sub);
  cudaFree(d->d_ghost[0]);
  cudaFree(d->d_ghost[1]);
  delete d;
}

int su3_decomp_sweep(su3_lattice* h, int nsweeps) {
  int rc = ensure_subs(h);
  if (rc != SU3_OK) return rc;
  rc = ensure_decomp_graph(h);
  if (rc != SU3_OK) return rc;
  cudaGraphExec_t exec = h->decomp->graph[h->stats_on ? 1 : 0];
  for (int n = 0; n < nsweeps; ++n) SU3_CUDA(cudaGraphLaunch(exec, h->stream), "su3_sweep: graph launch");
  h->sweep_host += (uint64_t)nsweeps;
  h->decomp->global_current = false;
  return SU3_OK;
}

int su3_decomp_meas_blocks(su3_lattice* h) { return phase_blocks(h); }

int su3_decomp_sweep_measured_graph(su3_lattice* h, cudaGraphExec_t* out) {
  int rc = ensure_subs(h);
  if (rc != SU3_OK) return rc;
  rc = ensure_decomp_graph(h, true);
  if (rc != SU3_OK) return rc;
  *out = h->decomp->graph_meas;
  h->decomp->global_current = false;
  return SU3_OK;
}

int su3_decomp_half_sweep(su3_lattice* h, int mu, int parity) {
  int rc = ensure_subs(h);
  if (rc != SU3_OK) return rc;
  rc = enqueue_phase(h, mu, parity);
  if (rc != SU3_OK) return rc;
  h->decomp->global_current = false;
  return SU3_OK;
}

// Before anything reads the handle's global store.
int su3_decomp_sync_global(su3_lattice* h) {
  if (!su3_decomp_active(h) || h->decomp->global_current) return SU3_OK;
  SU3_CUDA(launch_move(h, false), "decomposition gather");
  h->decomp->global_current = true;
  return SU3_OK;
}

// After the global store was written (su3_links_set).
void su3_decomp_global_written(su3_lattice* h) {
  if (!su3_decomp_active(h)) return;
  h->decomp->global_current = true;
  h->decomp->subs_current = false;
}

extern "C" {

int su3_decomp_create(int L0, int L1, int L2, int L3, double beta, uint64_t seed, int start, int precision,
                      int ndmpi, int mpifactor, int lbcex, void* cuda_stream, su3_handle* out) {
  if (!out) return su3_fail(SU3_EINVAL, "su3_decomp_create: out is NULL");
  *out = nullptr;
  const int L[4] = {L0, L1, L2, L3};
  long long np = 1;
  int rc = check_decomposition("su3_decomp_create", L, ndmpi, mpifactor, lbcex, &np);
  if (rc != SU3_OK) return rc;

  su3_handle h = nullptr;
  rc = su3_create_ex(L0, L1, L2, L3, beta, seed, start, precision, cuda_stream, &h);
  if (rc != SU3_OK) return rc;
  su3_decomp* d = new (std::nothrow) su3_decomp;
  if (!d) {
    su3_release_handle(h);
    return su3_fail(SU3_ENOMEM, "su3_decomp_create: host allocation failed");
  }
  h->decomp = d;
  d->ndmpi = ndmpi;
  d->nf = mpifactor;
  d->np = (int)np;
  d->lbcex = lbcex;
  d->active = true;
  // lbcex = 0 (np = 1): one sublattice covering the lattice, no direction
  // cut, periodic wrap inside it and no exchange -- the sublattice kernel
  // without ghost layers, the like-for-like baseline of the cut runs
  const int ncut = lbcex ? ndmpi : 0;
  SubGeometry& g = d->geo;
  host_sub_geometry(L, ncut, mpifactor, g);
  const int ncomp = precision == SU3_FP64 ? kEntriesF64 : kGroupsF32;
  const size_t elem = precision == SU3_FP64 ? sizeof(double2) : sizeof(float4);
  d->sub_elems = (size_t)8 * ncomp * g.Vh;
  std::vector<int4> lists[2];
  build_ghost_lists(L, ncut, mpifactor, d->np, g, lists);
  cudaError_t e = cudaMalloc(&d->d_sub, d->sub_elems * elem * np);
  for (int p = 0; p < 2 && e == cudaSuccess; ++p) {
    d->nghost[p] = (int)lists[p].size();
    if (d->nghost[p] == 0) continue;
    e = cudaMalloc(&d->d_ghost[p], lists[p].size() * sizeof(int4));
    if (e == cudaSuccess)
      e = cudaMemcpy(d->d_ghost[p], lists[p].data(), lists[p].size() * sizeof(int4), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    rc = su3_cuda_fail(e, "su3_decomp_create: allocation");
    cudaGetLastError();
    su3_release_handle(h);
    return rc;
  }
  // the sublattices need no zero fill: every interior cell is scattered and
  // every ghost cell a staple reads is filled before the first sweep
  d->subs_current = false;
  d->global_current = true;
  *out = h;
  return SU3_OK;
}

int su3_decomp_plan(int L0, int L1, int L2, int L3, int ndmpi, int mpifactor, int lbcex, int* nsub,
                    long long* halo_links_per_sweep) {
  const int L[4] = {L0, L1, L2, L3};
  long long np = 1;
  const int rc = check_decomposition("su3_decomp_plan", L, ndmpi, mpifactor, lbcex, &np);
  if (rc != SU3_OK) return rc;
  long long halo = 0;
  if (lbcex) {
    SubGeometry g{};
    host_sub_geometry(L, ndmpi, mpifactor, g);
    std::vector<int4> lists[2];
    build_ghost_lists(L, ndmpi, mpifactor, (int)np, g, lists);
    halo = 4LL * (long long)(lists[0].size() + lists[1].size());
  }
  if (nsub) *nsub = (int)np;
  if (halo_links_per_sweep) *halo_links_per_sweep = halo;
  return SU3_OK;
}

int su3_decomp_info(su3_handle h, int* ndmpi, int* mpifactor, int* lbcex, int* nsub, long long* halo_links_per_sweep) {
  if (!h) return su3_fail(SU3_EINVAL, "su3_decomp_info: NULL handle");
  const su3_decomp* d = h->decomp;
  if (ndmpi) *ndmpi = d ? d->ndmpi : 0;
  if (mpifactor) *mpifactor = d ? d->nf : 1;
  if (lbcex) *lbcex = d ? d->lbcex : 0;
  if (nsub) *nsub = d ? d->np : 1;
  if (halo_links_per_sweep) *halo_links_per_sweep = d ? 4LL * ((long long)d->nghost[0] + d->nghost[1]) : 0;
  return SU3_OK;
}

}  // extern "C"
