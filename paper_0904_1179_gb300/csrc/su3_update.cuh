// su3_update.cuh -- one checkerboard link update on sm_103a CUDA cores, shared
// by the single-lattice half-sweep kernels (one launch per (mu, parity)) and
// the persistent batched sweep.
//
// A link U_mu(x) gathers its six-staple sum from the 18 neighbouring links,
// runs the one-hit Kennedy-Pendleton heatbath in the SU(2) subgroups (0,1),
// (0,2), (1,2) (Cabibbo-Marinari), is reunitarised and stored.  Links of one
// (mu, parity) never enter each other's staples (checkerboard updating,
// Abstract and Sec. 1 of Berg & Wu, arXiv:0904.1179); every update draws its
// random numbers from Philox counters keyed by its site, so the result does
// not depend on which thread, block or launch performs it.  The work is a 4D
// stencil of 3x3 complex products, not a dense contraction: CUDA cores, no
// tensor cores.
#pragma once

#include "su3_device.cuh"
#include "su3_pair.cuh"

namespace su3dev {

constexpr double kTwoPi = 6.283185307179586476925286766559;

template <typename T>
__device__ __forceinline__ mat3<T> zero3() {
  mat3<T> m;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) m.e[i][k] = mk(T(0), T(0));
  return m;
}

// Link loader for the two storage forms.  CG = true reads through L2 only
// (ld.global.cg): required where other thread blocks of the same launch have
// written the links (the persistent batched sweep); otherwise the read-only
// path (ld.global.nc) is used.
template <typename T, bool CG>
struct Store;

template <bool CG>
struct Store<double, CG> {
  __device__ __forceinline__ static mat3<double> load(const void* U, int mu, int p, int h, int Vh) {
    return load_f64<CG>((const double2*)U, mu, p, h, Vh);
  }
};

template <bool CG>
struct Store<float, CG> {
  __device__ __forceinline__ static mat3<float> load(const void* U, int mu, int p, int h, int Vh) {
    return load_f32<CG>((const float4*)U, mu, p, h, Vh);
  }
};

// The FP32 stores come in two layouts: one site per float4 column group (the
// single-site layout) and the site-paired layout of su3_sitepair.cuh, which
// stores the sites x and x + (L3/2) e3 of a lattice whose L3 is a multiple of
// 4 side by side.  Single-site code reads and writes the latter one site at a
// time (PAIRS = true); Vh is the full lattice's half volume in both.
template <bool CG, bool PAIRS>
__device__ __forceinline__ pm3 load_pm3_l(const float4* __restrict__ U, int mu, int p, int h, int Vh) {
  if constexpr (PAIRS) {
    const int Vp = Vh / 2;
    const int half = h >= Vp ? 1 : 0;
    pm3 m;
    if (!link_ok(mu, p, h, Vh)) {
#pragma unroll
      for (int k = 0; k < 3; ++k) m.re[k] = m.im[k] = make_float2(0.f, 0.f);
      return m;
    }
    const float* b = (const float*)(U + pair_offset(mu, p, h - half * Vp, Vp)) + half;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float* e0 = b + 4 * kPairTile * k;        // entry (row 0, column k)
      const float* e1 = b + 4 * kPairTile * (3 + k);  // entry (row 1, column k)
      m.re[k] = make_float2(CG ? __ldcg(e0) : __ldg(e0), CG ? __ldcg(e1) : __ldg(e1));
      m.im[k] = make_float2(CG ? __ldcg(e0 + 2) : __ldg(e0 + 2), CG ? __ldcg(e1 + 2) : __ldg(e1 + 2));
    }
    return m;
  } else {
    return load_pm3<CG>(U, mu, p, h, Vh);
  }
}

// Single-site access to a site-paired store: rows 0,1 of site h's link (mu, p)
// as 12 floats, row 0 then row 1, (re, im) per column (as store_f32_rows01
// takes them); Vp = V/4 pairs per (mu, parity), pair h mod Vp, member h / Vp.
__device__ __forceinline__ void load_pair_site(const float4* __restrict__ U, int mu, int p, int h, int Vp, float r[12]) {
  if (!link_ok(mu, p, h, 2LL * Vp)) {
#pragma unroll
    for (int c = 0; c < 12; ++c) r[c] = 0.f;
    return;
  }
  const int half = h >= Vp ? 1 : 0;
  const float* b = (const float*)(U + pair_offset(mu, p, h - half * Vp, Vp)) + half;
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    r[6 * (e / 3) + 2 * (e % 3)] = __ldg(b + 4 * kPairTile * e);
    r[6 * (e / 3) + 2 * (e % 3) + 1] = __ldg(b + 4 * kPairTile * e + 2);
  }
}

__device__ __forceinline__ void store_pair_site(float4* U, int mu, int p, int h, int Vp, const float r[12]) {
  if (!link_ok(mu, p, h, 2LL * Vp)) return;
  const int half = h >= Vp ? 1 : 0;
  float* b = (float*)(U + pair_offset(mu, p, h - half * Vp, Vp)) + half;
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    b[4 * kPairTile * e] = r[6 * (e / 3) + 2 * (e % 3)];
    b[4 * kPairTile * e + 2] = r[6 * (e / 3) + 2 * (e % 3) + 1];
  }
}

// Six-staple sum A for U_mu(x), x = st of parity p:
//   sum_{nu != mu} U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu).
// Each three-link path is an SU(3) matrix, so only its rows 0 and 1 are
// multiplied out; its row 2, conj(row0 x row1), is formed inside the
// accumulation of A's row 2 (acc_completed).  The paths are added in the
// order forward, backward for nu ascending; every kernel that forms a staple
// keeps this order, so their results agree bit for bit.
// Apart (optional): receives the sum of the terms with nu < MU.  After the
// update, Re Tr(U_new Apart) is the sum of the plaquettes of the planes
// (MU, nu < MU) at x and at x - nu-hat.
// The two three-link paths of direction nu (nu != mu), rows 0,1:
//   forward  F = U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+,
//   backward B = U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu).
// h_pmu is the half index of x + mu-hat.
template <typename T, bool CG, typename G, typename S>
__device__ __forceinline__ mat3<T> forward_path(const G& g, const void* U, const S& st, int h, int p, int mu, int nu,
                                                int h_pmu, int h_pnu) {
  const int q = p ^ 1;
  const mat3<T> a = Store<T, CG>::load(U, nu, q, h_pmu, g.Vh);  // U_nu(x+mu)
  const mat3<T> b = Store<T, CG>::load(U, mu, q, h_pnu, g.Vh);  // U_mu(x+nu)
  mat3<T> t;
  mul_nd_rows01(a, b, t);
  const mat3<T> c = Store<T, CG>::load(U, nu, p, h, g.Vh);  // U_nu(x)
  mat3<T> f;
  mul_nd_rows01(t, c, f);
  return f;
}

template <typename T, bool CG, typename G>
__device__ __forceinline__ mat3<T> backward_path(const G& g, const void* U, int p, int mu, int nu, int h_mnu,
                                                 int h_pmu_mnu) {
  const int q = p ^ 1;
  const mat3<T> d = Store<T, CG>::load(U, nu, p, h_pmu_mnu, g.Vh);  // U_nu(x+mu-nu)
  const mat3<T> e = Store<T, CG>::load(U, mu, q, h_mnu, g.Vh);      // U_mu(x-nu)
  // Rows 0,1 of d^+ e^+ = (e d)^+ are the conjugated columns 0,1 of e d, which
  // need all three rows of e (stored in full here) but no row-2 completion.
  mat3<T> hm;
  mul_nn_cols01(e, d, hm);
  const mat3<T> f = Store<T, CG>::load(U, nu, q, h_mnu, g.Vh);  // U_nu(x-nu)
  mat3<T> b;
  mul_dn_rows01(hm, f, b);
  return b;
}

// A = F (rows 0,1 given, row 2 completed): the first term of a staple.
template <typename T>
__device__ __forceinline__ void init_completed(mat3<T>& A, const mat3<T>& F) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    A.e[0][k] = F.e[0][k];
    A.e[1][k] = F.e[1][k];
  }
  complete_row2(A);
}

template <typename T, int MU, bool CG, typename G, typename S>
__device__ __forceinline__ mat3<T> staple(const G& g, const void* U, const S& st, int h, int p,
                                          mat3<T>* Apart = nullptr) {
  mat3<T> A;
  const int h_pmu = nb_half(g, st, MU, +1);
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == MU) continue;
    const int h_pnu = nb_half(g, st, nu, +1);
    const int h_mnu = nb_half(g, st, nu, -1);
    const int h_pmu_mnu = nb_half2(g, st, MU, nu);
    const mat3<T> F = forward_path<T, CG>(g, U, st, h, p, MU, nu, h_pmu, h_pnu);
    if (nu == (MU == 0 ? 1 : 0)) {
      init_completed(A, F);
    } else {
      acc_completed(A, F);
    }
    acc_completed(A, backward_path<T, CG>(g, U, p, MU, nu, h_mnu, h_pmu_mnu));
    if (Apart && nu == MU - 1) *Apart = A;
  }
  return A;
}


// 2x2 block of W = U A in rows/columns (i, j), projected on the SU(2) direction,
// returned as 2r = (Re(W_ii+W_jj), Im(W_ij+W_ji), Re(W_ij-W_ji), Im(W_ii-W_jj)):
// the factor 1/2 of r cancels in r/|r| and is folded into 1/alpha.
template <typename T>
__device__ __forceinline__ void su2_projection(const mat3<T>& u, const mat3<T>& A, int i, int j, T r[4]) {
  cx<T> wii = mk(T(0), T(0)), wij = wii, wji = wii, wjj = wii;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    wii = mac(wii, u.e[i][c], A.e[c][i]);
    wij = mac(wij, u.e[i][c], A.e[c][j]);
    wji = mac(wji, u.e[j][c], A.e[c][i]);
    wjj = mac(wjj, u.e[j][c], A.e[c][j]);
  }
  r[0] = wii.re + wjj.re;
  r[1] = wij.im + wji.im;
  r[2] = wij.re - wji.re;
  r[3] = wii.im - wjj.im;
}

// rows (i, j) of u <- R rows (i, j), R = Y V^+ with Y = m(a), V = m(v),
// m(q) = [[q0 + i q3, q2 + i q1], [-q2 + i q1, q0 - i q3]].
// rows_j = false leaves row j unchanged (its new value is not needed).
template <typename T>
__device__ __forceinline__ void apply_su2(mat3<T>& u, int i, int j, const T a[4], const T v[4], bool rows_j = true) {
  const cx<T> y00 = mk(a[0], a[3]), y01 = mk(a[2], a[1]);
  const cx<T> v00 = mk(v[0], v[3]), v01 = mk(v[2], v[1]), v10 = mk(-v[2], v[1]), v11 = mk(v[0], -v[3]);
  // (V^+)_{pq} = conj(V_{qp}); a product of two matrices of this SU(2) form
  // has the form again, so R10 = -conj(R01) and R11 = conj(R00).
  const cx<T> R00 = mac_cb(mac_cb(mk(T(0), T(0)), y00, v00), y01, v01);
  const cx<T> R01 = mac_cb(mac_cb(mk(T(0), T(0)), y00, v10), y01, v11);
  const cx<T> R10 = mk(-R01.re, R01.im);
  const cx<T> R11 = mk(R00.re, -R00.im);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cx<T> ui = u.e[i][c], uj = u.e[j][c];
    u.e[i][c] = mac(mul(R00, ui), R01, uj);
    if (rows_j) u.e[j][c] = mac(mul(R10, ui), R11, uj);
  }
}

__device__ __forceinline__ int subrow_i(int sub) { return sub == 2 ? 1 : 0; }
__device__ __forceinline__ int subrow_j(int sub) { return sub == 0 ? 1 : 2; }


// Parameters of one link update that do not vary across the links of a lattice.
struct UpdateConsts {
  double three_over_beta_f64;  // 3 / beta: 1/alpha = 3 / (2 beta k) = three_over_beta / (2k)
  float three_over_beta;
  int max_tries;  // 1: one-hit heatbath; > 1: repeat until accepted, at most this many proposals
};

// Accepted and drawn SU(2) proposals of one link update (a degenerate
// subgroup counts as one proposal).
struct UpdateCount {
  int accepted, proposed;
};

// ---------------------------------------------------------------------------
// One FP64 link update: staple, three one-hit SU(2) heatbath steps, FP64
// Gram-Schmidt, store.  Returns the number of accepted SU(2) proposals.
// ---------------------------------------------------------------------------
// MEAS: also return in *meas (1/3) Re Tr(U_new A_<), A_< the staple terms of
// the directions nu < MU (see staple()).
// G: Geometry (periodic lattice) or SubGeometry (sublattice with ghost
// layers); h enumerates the sites of parity p, hs is where the site is stored.
template <int MU, bool CG, bool REPEAT, bool MEAS, typename KEY, typename G>
__device__ __forceinline__ UpdateCount heatbath_f64(const G& g, double2* U, int h, int p, uint64_t t, uint32_t s,
                                                    const KEY& key, const UpdateConsts& uc, const mat3<double>& A,
                                                    const mat3<double>& Apart, double* meas);

template <int MU, bool CG, bool REPEAT, bool MEAS = false, typename KEY, typename G>
__device__ __forceinline__ UpdateCount update_link_f64(const G& g, double2* U, int h, int p, uint64_t t,
                                                       const KEY& key, const UpdateConsts& uc, double* meas = nullptr) {
  const auto st = site_of(g, h, p);
  const uint32_t s = (uint32_t)canon(g, st);
  h = store_index(g, st, h);
  mat3<double> Apart;
  const mat3<double> A = staple<double, MU, CG>(g, U, st, h, p, MEAS ? &Apart : nullptr);
  return heatbath_f64<MU, CG, REPEAT, MEAS>(g, U, h, p, t, s, key, uc, A, Apart, meas);
}

// Everything after the staple: three SU(2) heatbath steps, Gram-Schmidt and
// the store of link (s, MU) at storage half index h.
template <int MU, bool CG, bool REPEAT, bool MEAS, typename KEY, typename G>
__device__ __forceinline__ UpdateCount heatbath_f64(const G& g, double2* U, int h, int p, uint64_t t, uint32_t s,
                                                    const KEY& key, const UpdateConsts& uc, const mat3<double>& A,
                                                    const mat3<double>& Apart, double* meas) {
  UpdateCount cnt{0, 0};
  mat3<double> u = load_f64<CG>(U, MU, p, h, g.Vh);
#pragma unroll
  for (int sub = 0; sub < 3; ++sub) {
    const int i = subrow_i(sub), j = subrow_j(sub);
    double r[4];  // 2r
    su2_projection(u, A, i, j, r);
    const double kk = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3];  // (2k)^2
    if (!(kk > 0.0)) {  // k = 0: degenerate staple (measure zero), leave the subgroup
      ++cnt.proposed;
      continue;
    }
    const double ik = rsqrt(kk);                           // 1 / (2k)
    const double inv_alpha = uc.three_over_beta_f64 * ik;  // 1/alpha = 3 / (2 beta k)
    const int ntries = REPEAT ? uc.max_tries : 1;
    for (int tr = 0; tr < ntries; ++tr) {
      double uu[6];
#pragma unroll
      for (int call = 0; call < 3; ++call) {
        const uint32_t w1 = (uint32_t)(MU | (sub << 2) | (call << 4)) | ((uint32_t)tr << 6);
        const uint4 w = philox4x32_10(rng_counter(s, w1, t, kTagUpdate), key);
        uu[2 * call] = u01_f64(w.x, w.y);
        uu[2 * call + 1] = u01_f64(w.z, w.w);
      }
      ++cnt.proposed;
      const double c = cospi(2.0 * uu[1]);  // cos(2 pi u1)
      const double delta = -(log_u01(uu[0]) + c * c * log_u01(uu[2])) * inv_alpha;
      if (uu[3] * uu[3] > 1.0 - 0.5 * delta) continue;
      const double a0 = 1.0 - delta;
      double rho = 1.0 - a0 * a0;
      rho = rho > 0.0 ? sqrt(rho) : 0.0;
      const double ct = 1.0 - 2.0 * uu[4];
      double sn = 1.0 - ct * ct;
      sn = sn > 0.0 ? sqrt(sn) : 0.0;
      double sphi, cphi;
      sincospi(2.0 * uu[5], &sphi, &cphi);  // angle 2 pi u5
      const double a[4] = {a0, rho * sn * cphi, rho * sn * sphi, rho * ct};
      const double v[4] = {r[0] * ik, r[1] * ik, r[2] * ik, r[3] * ik};  // r / k
      // Row 2 leaves the last subgroup unused: reunitarisation rebuilds it.
      apply_su2(u, i, j, a, v, sub < 2);
      ++cnt.accepted;
      break;
    }
  }
  cx<double> r0[3] = {u.e[0][0], u.e[0][1], u.e[0][2]};
  cx<double> r1[3] = {u.e[1][0], u.e[1][1], u.e[1][2]};
  gram_schmidt_rows01(r0, r1);
  mat3<double> out;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    out.e[0][k] = r0[k];
    out.e[1][k] = r1[k];
  }
  complete_row2(out);
  store_f64(U, MU, p, h, g.Vh, out);
  if (MEAS) {
    double tr = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) tr = fma(out.e[i][k].re, Apart.e[k][i].re, fma(-out.e[i][k].im, Apart.e[k][i].im, tr));
    *meas = tr * (1.0 / 3.0);
  }
  return cnt;
}

// ---------------------------------------------------------------------------
// FP32-mixed staple on row pairs (su3_pair.cuh): every three-link path is an
// SU(3) matrix, so rows 0,1 are multiplied out two rows at a time and row 2
// is completed.
// ---------------------------------------------------------------------------
// The two paths of direction nu on row pairs, rows 0,1 (as forward_path and
// backward_path above), added to the staple in the same order.
template <bool CG, bool PAIRS = false, typename G>
__device__ __forceinline__ pm3 forward_path_p(const G& g, const float4* U, int h, int p, int mu, int nu, int h_pmu,
                                              int h_pnu) {
  const int q = p ^ 1;
  const pm3 a = load_pm3_l<CG, PAIRS>(U, nu, q, h_pmu, g.Vh);  // U_nu(x+mu)
  pm3 b = load_pm3_l<CG, PAIRS>(U, mu, q, h_pnu, g.Vh);        // U_mu(x+nu)
  complete_row2_p(b);
  pm3 t;
  mul_nd_p(a, b, t);
  pm3 c = load_pm3_l<CG, PAIRS>(U, nu, p, h, g.Vh);  // U_nu(x)
  complete_row2_p(c);
  pm3 f;
  mul_nd_p(t, c, f);
  return f;
}

template <bool CG, bool PAIRS = false, typename G>
__device__ __forceinline__ pm3 backward_path_p(const G& g, const float4* U, int p, int mu, int nu, int h_mnu,
                                               int h_pmu_mnu) {
  const int q = p ^ 1;
  pm3 d = load_pm3_l<CG, PAIRS>(U, nu, p, h_pmu_mnu, g.Vh);  // U_nu(x+mu-nu)
  complete_row2_p(d);
  const pm3 e = load_pm3_l<CG, PAIRS>(U, mu, q, h_mnu, g.Vh);  // U_mu(x-nu)
  pm3 hm;
  mul_nn_p(e, d, hm);
  complete_row2_p(hm);
  pm3 f = load_pm3_l<CG, PAIRS>(U, nu, q, h_mnu, g.Vh);  // U_nu(x-nu)
  complete_row2_p(f);
  pm3 b;
  mul_dn_p(hm, f, b);
  return b;
}

// A = F (rows 0,1 given, row 2 completed): the first term of a staple.
__device__ __forceinline__ void init_completed_p(pm3& A, const pm3& F) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    A.re[k] = F.re[k];
    A.im[k] = F.im[k];
  }
  complete_row2_p(A);
}

template <int MU, bool CG, typename G, typename S>
__device__ __forceinline__ pm3 staple_p(const G& g, const float4* U, const S& st, int h, int p,
                                        pm3* Apart = nullptr) {
  pm3 A;
  const int h_pmu = nb_half(g, st, MU, +1);
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == MU) continue;
    const int h_pnu = nb_half(g, st, nu, +1);
    const int h_mnu = nb_half(g, st, nu, -1);
    const int h_pmu_mnu = nb_half2(g, st, MU, nu);
    const pm3 F = forward_path_p<CG>(g, U, h, p, MU, nu, h_pmu, h_pnu);
    if (nu == (MU == 0 ? 1 : 0)) {
      init_completed_p(A, F);
    } else {
      acc_completed_p(A, F);
    }
    acc_completed_p(A, backward_path_p<CG>(g, U, p, MU, nu, h_mnu, h_pmu_mnu));
    if (Apart && nu == MU - 1) *Apart = A;
  }
  return A;
}

// ---------------------------------------------------------------------------
// cp.async: 16-byte copies from global to shared memory that do not pass
// through registers, tracked in commit groups per thread.
// ---------------------------------------------------------------------------
// Both forms copy through L1 (.ca): cache operators are performance hints
// and do not change the memory-consistency behaviour, so links written by
// other blocks of a persistent launch are seen once the block has acquired
// their completion counts; and on GB300 the L1-bypassing cp.async.cg made the
// site-paired sweep 1.7 times slower.
template <bool CG>
__device__ __forceinline__ void cp_async16(uint32_t saddr, const float4* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The hardware square root (about 1 ulp): the FP32 heatbath needs no
// correctly rounded one.
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------------------
// One FP32-mixed link update: FP32 storage (rows 0,1), FP32 staple and
// heatbath, Gram-Schmidt coefficients in FP64 (EFT = false) or as
// compensated FP32 sums of FP64-class accuracy (EFT = true).  REPEAT = false
// compiles the one-hit heatbath without the retry loop.
// ---------------------------------------------------------------------------
template <int MU, bool CG, bool EFT, bool REPEAT, bool MEAS, typename KEY, typename G>
__device__ __forceinline__ UpdateCount heatbath_f32(const G& g, float4* U, int h, int p, uint64_t t, uint32_t s,
                                                    const KEY& key, const UpdateConsts& uc, const pm3& A,
                                                    const pm3& Apart, double* meas);

template <int MU, bool CG, bool EFT, bool REPEAT, bool MEAS = false, typename KEY, typename G>
__device__ __forceinline__ UpdateCount update_link_f32(const G& g, float4* U, int h, int p, uint64_t t,
                                                       const KEY& key, const UpdateConsts& uc, double* meas = nullptr) {
  const auto st = site_of(g, h, p);
  const uint32_t s = (uint32_t)canon(g, st);
  h = store_index(g, st, h);
  pm3 Apart;
  const pm3 A = staple_p<MU, CG>(g, U, st, h, p, MEAS ? &Apart : nullptr);
  return heatbath_f32<MU, CG, EFT, REPEAT, MEAS>(g, U, h, p, t, s, key, uc, A, Apart, meas);
}

// Everything after the staple (FP32 storage): three SU(2) heatbath steps,
// reunitarisation, store.
template <int MU, bool EFT, bool REPEAT, bool MEAS, bool PAIRS = false, typename KEY, typename G>
__device__ __forceinline__ UpdateCount heatbath_f32_on(const G& g, float4* U, int h, int p, uint64_t t, uint32_t s,
                                                       const KEY& key, const UpdateConsts& uc, const pm3& A,
                                                       const pm3& Apart, double* meas, pm3 u, bool store);

template <int MU, bool CG, bool EFT, bool REPEAT, bool MEAS, typename KEY, typename G>
__device__ __forceinline__ UpdateCount heatbath_f32(const G& g, float4* U, int h, int p, uint64_t t, uint32_t s,
                                                    const KEY& key, const UpdateConsts& uc, const pm3& A,
                                                    const pm3& Apart, double* meas) {
  return heatbath_f32_on<MU, EFT, REPEAT, MEAS>(g, U, h, p, t, s, key, uc, A, Apart, meas,
                                                 load_pm3<CG>(U, MU, p, h, g.Vh), true);
}

// The same with the link's own rows 0,1 given (u); store = false computes
// everything but writes nothing (a lane that only keeps its warp converged).
template <int MU, bool EFT, bool REPEAT, bool MEAS, bool PAIRS, typename KEY, typename G>
__device__ __forceinline__ UpdateCount heatbath_f32_on(const G& g, float4* U, int h, int p, uint64_t t, uint32_t s,
                                                       const KEY& key, const UpdateConsts& uc, const pm3& A,
                                                       const pm3& Apart, double* meas, pm3 u, bool store) {
  UpdateCount cnt{0, 0};
  complete_row2_p(u);
  const float three_over_beta = uc.three_over_beta;
#pragma unroll
  for (int sub = 0; sub < 3; ++sub) {
    const int i = subrow_i(sub), j = subrow_j(sub);
    // 2x2 block (i, j) of W = U A
    cx<float> wii, wij, wji, wjj;
    if (sub == 0) {
      // rows 0 and 1 as one pair: (W_0b, W_1b) = sum_c (U_0c, U_1c) A_cb
      float2 wr[2], wi[2];
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        float2 zr = make_float2(0.f, 0.f), zi = zr;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float ar = pre(A, c, b), ai = pim(A, c, b);
          zr = fma2(u.re[c], bc2(ar), zr);
          zr = fma2(u.im[c], bc2(-ai), zr);
          zi = fma2(u.re[c], bc2(ai), zi);
          zi = fma2(u.im[c], bc2(ar), zi);
        }
        wr[b] = zr;
        wi[b] = zi;
      }
      wii = mk(wr[0].x, wi[0].x);
      wji = mk(wr[0].y, wi[0].y);
      wij = mk(wr[1].x, wi[1].x);
      wjj = mk(wr[1].y, wi[1].y);
    } else {
      wii = mk(0.f, 0.f);
      wij = wii;
      wji = wii;
      wjj = wii;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        wii = mac(wii, pget(u, i, c), pget(A, c, i));
        wij = mac(wij, pget(u, i, c), pget(A, c, j));
        wji = mac(wji, pget(u, j, c), pget(A, c, i));
        wjj = mac(wjj, pget(u, j, c), pget(A, c, j));
      }
    }
    // 2r, as in su2_projection
    const float r[4] = {wii.re + wjj.re, wij.im + wji.im, wij.re - wji.re, wii.im - wjj.im};
    const float kk = __fmaf_rn(r[3], r[3], __fmaf_rn(r[2], r[2], __fmaf_rn(r[1], r[1], __fmul_rn(r[0], r[0]))));  // (2k)^2
    if (!(kk > 4e-30f)) {  // degenerate staple (measure zero): leave the subgroup
      ++cnt.proposed;
      continue;
    }
    const float ik = rsqrtf(kk);             // 1 / (2k)
    const float ia = three_over_beta * ik;  // 1/alpha = 3 / (2 beta k)
    bool acc = false;
    float a[4];
    const int ntries = REPEAT ? uc.max_tries : 1;
    for (int tr = 0; tr < ntries; ++tr) {
      const uint32_t w1b = (uint32_t)(MU | (sub << 2)) | ((uint32_t)tr << 6);
      const uint4 w0 = philox4x32_10(rng_counter(s, w1b, t, kTagUpdate), key);
      const uint4 w1 = philox4x32_10(rng_counter(s, w1b | (1u << 4), t, kTagUpdate), key);
      ++cnt.proposed;
      const float u0 = u01_f32(w0.x), u1 = u01_f32(w0.y), u2 = u01_f32(w0.z), u3 = u01_f32(w0.w);
      const float cc = __cosf(fmaf(6.2831853f, u1, -3.14159265f));  // -cos(2 pi u1); only its square is used
      const float delta = __fmul_rn(-__fmaf_rn(__fmul_rn(cc, cc), __logf(u2), __logf(u0)), ia);
      if (__fmul_rn(u3, u3) > __fmaf_rn(-0.5f, delta, 1.0f)) continue;
      const float u4 = u01_f32(w1.x), u5 = u01_f32(w1.y);
      const float rho = sqrt_approx(fmaxf(0.0f, delta * (2.0f - delta)));  // sqrt(1 - a0^2)
      const float ct = __fmaf_rn(-2.0f, u4, 1.0f);
      const float sn = 2.0f * sqrt_approx(u4 * (1.0f - u4));  // sqrt(1 - ct^2)
      float sphi, cphi;
      __sincosf(fmaf(6.2831853f, u5, -3.14159265f), &sphi, &cphi);  // angle 2 pi u5 - pi
      const float rs = -rho * sn;                                     // undo the shift by pi
      a[0] = 1.0f - delta;
      a[1] = rs * cphi;
      a[2] = rs * sphi;
      a[3] = rho * ct;
      acc = true;
      break;
    }
    if (!acc) continue;
    const float v[4] = {r[0] * ik, r[1] * ik, r[2] * ik, r[3] * ik};
    // R = Y V^+ with Y = m(a), V = m(v), m(q) = [[q0 + i q3, q2 + i q1], [-q2 + i q1, q0 - i q3]]
    const cx<float> y00 = mk(a[0], a[3]), y01 = mk(a[2], a[1]);
    const cx<float> v00 = mk(v[0], v[3]), v01 = mk(v[2], v[1]), v10 = mk(-v[2], v[1]), v11 = mk(v[0], -v[3]);
    const cx<float> R00 = mac_cb(mac_cb(mk(0.f, 0.f), y00, v00), y01, v01);
    const cx<float> R01 = mac_cb(mac_cb(mk(0.f, 0.f), y00, v10), y01, v11);
    const cx<float> R10 = mk(-R01.re, R01.im);  // R keeps the SU(2) form
    const cx<float> R11 = mk(R00.re, -R00.im);
    if (sub == 0) {
      rotate01_p(u, R00, R01, R10, R11);
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const cx<float> ui = pget(u, i, c), uj = pget(u, j, c);
        pset(u, i, c, mac(mul(R00, ui), R01, uj));
        // row 2 leaves the last subgroup unused: reunitarisation rebuilds it
        if (sub < 2) pset(u, j, c, mac(mul(R10, ui), R11, uj));
      }
    }
    ++cnt.accepted;
  }
  cx<float> r0[3], r1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r0[k] = pget(u, 0, k);
    r1[k] = pget(u, 1, k);
  }
  float o[12];
  reunitarise_f32<EFT>(r0, r1, o);
  if (store) {
    if (PAIRS)
      store_pair_site(U, MU, p, h, g.Vh / 2, o);
    else
      store_f32_rows01(U, MU, p, h, g.Vh, o);
  }
  if (MEAS) {
    // the stored link, row 2 completed, against A_<
    mat3<float> un;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      un.e[0][k] = mk(o[2 * k], o[2 * k + 1]);
      un.e[1][k] = mk(o[6 + 2 * k], o[6 + 2 * k + 1]);
    }
    complete_row2(un);
    float tr = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const cx<float> ak = pget(Apart, k, i);
        tr = fmaf(un.e[i][k].re, ak.re, fmaf(-un.e[i][k].im, ak.im, tr));
      }
    *meas = (double)tr * (1.0 / 3.0);
  }
  return cnt;
}

}  // namespace su3dev
