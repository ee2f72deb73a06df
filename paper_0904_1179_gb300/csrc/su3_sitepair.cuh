// su3_sitepair.cuh -- the FP32 link update of two sites at once, on paired
// FP32 arithmetic (fma.rn.f32x2, mul.rn.f32x2, add.rn.f32x2).
//
// Checkerboard updating (Berg & Wu, arXiv:0904.1179, Abstract and Sec. 1)
// makes the links of one (mu, parity) half-sweep independent, so one thread
// may update two of them with the same instruction stream.  The two sites of a
// pair are x = (x0, x1, x2, x3) and x' = x + (L3/2) e3 (L3 a multiple of 4, so
// that x and x' have the same parity and the same x0): every neighbour of x'
// is the neighbour of x moved by the same half period, so the pair shares all
// index arithmetic, and every floating-point operation of the update -- the
// staple's products and row completions, the SU(2) steps, the
// reunitarisation -- runs on (site, site') in one paired instruction.
//
// The pairs live on the "pair lattice" L0 x L1 x L2 x L3/2 (geometry gp,
// pair index j = the half index on that lattice).  Stepping across the x3
// boundary of the pair lattice exchanges the two members: from x3 = L3/2 - 1
// the +x3 neighbour of x is x3 = L3/2, the second member of pair x3 = 0, and
// that of x' wraps to x3 = 0, its first member.  Such a neighbour pair is
// loaded and its two halves exchanged.
//
// Every rounding step is written out and taken in the order of the
// single-site FP32 update (su3_update.cuh, su3_pair.cuh), so both produce
// the same bits.
#pragma once

#include "su3_update.cuh"

namespace su3dev {

// ---------------------------------------------------------------------------
// Site-paired FP32 store: float4 [4 mu][2 parity][Vp' / 32 tiles][6 entries
// e = 3 r + k][32 pairs] for rows r = 0, 1 and columns k, Vp = V/4 pairs per
// (mu, parity), Vp' = Vp rounded up to a multiple of 32 (pair_offset in
// su3_device.cuh); entry e of pair j holds (re u_rk(x), re u_rk(x'),
// im u_rk(x), im u_rk(x')).  Row 2 is conj(row0 x row1), as in the
// single-site store.  A single site h of the full lattice (half index,
// h < V/2) is pair j = h mod Vp, member h / Vp.
// ---------------------------------------------------------------------------

// Whether an FP32 store of a lattice with these extents uses the site-paired
// layout: L3 divisible by 4 (the two members of a pair then share parity and x0).
__host__ __device__ __forceinline__ bool pair_layout(int L3) { return L3 % 4 == 0; }

// The pair lattice of a periodic lattice whose L3 is a multiple of 4.
__host__ inline Geometry make_pair_geometry(const Geometry& g) { return make_geometry(g.L0, g.L1, g.L2, g.L3 / 2); }

// Rows 0,1 of site h's link from an FP32 store in either layout (pairs: the
// site-paired layout, Vh = V/2 of the full lattice), as mat3 rows.
__device__ __forceinline__ mat3<float> load_f32_rows01_any(const float4* __restrict__ U, int mu, int p, int h, int Vh,
                                                           bool pairs) {
  if (!pairs) return load_f32_rows01(U, mu, p, h, Vh);
  float r[12];
  load_pair_site(U, mu, p, h, Vh / 2, r);
  mat3<float> m;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    m.e[0][k] = mk(r[2 * k], r[2 * k + 1]);
    m.e[1][k] = mk(r[6 + 2 * k], r[6 + 2 * k + 1]);
  }
  return m;
}

__device__ __forceinline__ mat3<float> load_f32_any(const float4* __restrict__ U, int mu, int p, int h, int Vh, bool pairs) {
  mat3<float> m = load_f32_rows01_any(U, mu, p, h, Vh, pairs);
  complete_row2(m);
  return m;
}

__device__ __forceinline__ void store_f32_rows01_any(float4* U, int mu, int p, int h, int Vh, bool pairs, const float r[12]) {
  if (pairs)
    store_pair_site(U, mu, p, h, Vh / 2, r);
  else
    store_f32_rows01(U, mu, p, h, Vh, r);
}

// ---------------------------------------------------------------------------
// Paired arithmetic: lane .x belongs to x, lane .y to x'.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 qfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 qmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 qadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 qneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 qsub(float2 a, float2 b) { return __fadd2_rn(a, qneg(b)); }
__device__ __forceinline__ float2 qzero() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ float2 qsel(bool ax, bool ay, float2 a, float2 b) {
  return make_float2(ax ? a.x : b.x, ay ? a.y : b.y);
}

struct qcx {
  float2 re, im;
};
__device__ __forceinline__ qcx qmk(float2 re, float2 im) {
  qcx c;
  c.re = re;
  c.im = im;
  return c;
}
// a b, as mul(cx<float>, cx<float>)
__device__ __forceinline__ qcx qcmul(qcx a, qcx b) {
  return qmk(qfma(qneg(a.im), b.im, qmul(a.re, b.re)), qfma(a.im, b.re, qmul(a.re, b.im)));
}
// acc + a b, as mac
__device__ __forceinline__ qcx qcmac(qcx acc, qcx a, qcx b) {
  acc.re = qfma(a.re, b.re, acc.re);
  acc.re = qfma(qneg(a.im), b.im, acc.re);
  acc.im = qfma(a.re, b.im, acc.im);
  acc.im = qfma(a.im, b.re, acc.im);
  return acc;
}
// acc + a conj(b), as mac_cb
__device__ __forceinline__ qcx qcmac_cb(qcx acc, qcx a, qcx b) {
  acc.re = qfma(a.re, b.re, acc.re);
  acc.re = qfma(a.im, b.im, acc.re);
  acc.im = qfma(qneg(a.re), b.im, acc.im);
  acc.im = qfma(a.im, b.re, acc.im);
  return acc;
}

// A pair of SU(3) matrices; row 2 is valid once completed.
struct PM {
  float2 re[3][3], im[3][3];
};

__device__ __forceinline__ qcx qget(const PM& m, int i, int k) { return qmk(m.re[i][k], m.im[i][k]); }

// Exchange the two members of a loaded pair (a neighbour across the x3
// boundary of the pair lattice).  `sw` is usually the same for the whole warp;
// the vote keeps the exchange off the path of the warps that need none.
__device__ __forceinline__ void swap_halves(PM& m, bool sw) {
  if (__any_sync(0xffffffffu, sw)) {
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const float2 r = m.re[e / 3][e % 3], i = m.im[e / 3][e % 3];
      m.re[e / 3][e % 3] = sw ? make_float2(r.y, r.x) : r;
      m.im[e / 3][e % 3] = sw ? make_float2(i.y, i.x) : i;
    }
  }
}

__device__ __forceinline__ void store_pm_rows01(float4* U, int mu, int p, int j, int Vp, const float2 re[2][3],
                                                const float2 im[2][3]) {
  if (!link_ok(mu, p, j, Vp)) return;
  float4* b = U + pair_offset(mu, p, j, Vp);
#pragma unroll
  for (int e = 0; e < 6; ++e)
    b[kPairTile * e] = make_float4(re[e / 3][e % 3].x, re[e / 3][e % 3].y, im[e / 3][e % 3].x, im[e / 3][e % 3].y);
}

// Row 2 = conj(row0 x row1), in the order of complete_row2_p.
__device__ __forceinline__ void complete_row2_q(PM& m) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int a = (k + 1) % 3, b = (k + 2) % 3;
    qcx v = qcmul(qget(m, 0, a), qget(m, 1, b));
    v = qcmac(v, qmk(qneg(m.re[0][b]), qneg(m.im[0][b])), qget(m, 1, a));
    m.re[2][k] = v.re;
    m.im[2][k] = qneg(v.im);
  }
}

// Rows 0,1 of X Y^+ (Y complete), in the order of mul_nd_p.
__device__ __forceinline__ void mul_nd_q(const PM& X, const PM& Y, PM& Z) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float2 zr = qzero(), zi = qzero();
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        zr = qfma(X.re[i][j], Y.re[k][j], zr);
        zr = qfma(X.im[i][j], Y.im[k][j], zr);
        zi = qfma(X.im[i][j], Y.re[k][j], zi);
        zi = qfma(X.re[i][j], qneg(Y.im[k][j]), zi);
      }
      Z.re[i][k] = zr;
      Z.im[i][k] = zi;
    }
}

// Rows 0,1 of X Y (Y complete), in the order of mul_nn_p.
__device__ __forceinline__ void mul_nn_q(const PM& X, const PM& Y, PM& Z) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float2 zr = qzero(), zi = qzero();
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        zr = qfma(X.re[i][j], Y.re[j][k], zr);
        zr = qfma(X.im[i][j], qneg(Y.im[j][k]), zr);
        zi = qfma(X.re[i][j], Y.im[j][k], zi);
        zi = qfma(X.im[i][j], Y.re[j][k], zi);
      }
      Z.re[i][k] = zr;
      Z.im[i][k] = zi;
    }
}

// Rows 0,1 of H^+ F (H, F complete), in the order of mul_dn_p.
__device__ __forceinline__ void mul_dn_q(const PM& H, const PM& F, PM& Z) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float2 zr = qzero(), zi = qzero();
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        zr = qfma(H.re[j][i], F.re[j][k], zr);
        zr = qfma(H.im[j][i], F.im[j][k], zr);
        zi = qfma(H.re[j][i], F.im[j][k], zi);
        zi = qfma(H.im[j][i], qneg(F.re[j][k]), zi);
      }
      Z.re[i][k] = zr;
      Z.im[i][k] = zi;
    }
}

// A += B, B given by rows 0,1 (its row 2 formed in the accumulation), in the
// order of acc_completed_p.
__device__ __forceinline__ void acc_completed_q(PM& A, const PM& B) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      A.re[i][k] = qadd(A.re[i][k], B.re[i][k]);
      A.im[i][k] = qadd(A.im[i][k], B.im[i][k]);
    }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int a = (k + 1) % 3, b = (k + 2) % 3;
    qcx v = qcmac(qmk(A.re[2][k], qneg(A.im[2][k])), qget(B, 0, a), qget(B, 1, b));
    v = qcmac(v, qmk(qneg(B.re[0][b]), qneg(B.im[0][b])), qget(B, 1, a));
    A.re[2][k] = v.re;
    A.im[2][k] = qneg(v.im);
  }
}

__device__ __forceinline__ void init_completed_q(PM& A, const PM& F) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      A.re[i][k] = F.re[i][k];
      A.im[i][k] = F.im[i][k];
    }
  complete_row2_q(A);
}

// ---------------------------------------------------------------------------
// Pair-lattice neighbours: half index on the pair lattice, and whether the
// step crosses its x3 boundary (the neighbour pair then has its members
// exchanged).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool pair_swap(const Geometry& gp, const Site& s, int nu, int d) {
  return nu == 3 && (d > 0 ? s.x3 == gp.L3 - 1 : s.x3 == 0);
}

// ---------------------------------------------------------------------------
// The staple of a link pair, its 18 neighbour link pairs and then the link
// pair being updated streamed through a ring of three shared-memory slots per
// thread by cp.async: link K + 3 is requested when link K is read, so three
// loads are in flight while the arithmetic of the links before them runs.
// Slot r of thread t is 7 float4 (6 used) at 7 (r blockDim.x + t): 112-byte
// steps between lanes, an odd multiple of 16 bytes, so the 16-byte accesses
// of a quarter warp meet no bank twice.  All lanes of a warp must take part
// (a lane past the end works on a valid pair and stores nothing): a slot is
// refilled after a __syncwarp that orders every lane's read of it before the
// new copies.
//
// The staple's three directions run as a loop that is not unrolled: one copy
// of the loop body instead of three keeps the kernel's instruction stream
// within the instruction caches.  With three slots, link K = 6 i + c of
// direction index i sits in slot c mod 3 whatever i is.
// ---------------------------------------------------------------------------
struct PairRing {
  float4* ptr;  // slot 0 of this thread; slot r at ptr + r step
  uint32_t sa;  // the same as a shared-window address
  int step;     // 7 blockDim.x float4
};

__device__ __forceinline__ PairRing pair_ring(float4* smem) {
  PairRing r;
  r.ptr = smem + 7 * (int)threadIdx.x;
  r.sa = (uint32_t)__cvta_generic_to_shared(r.ptr);
  r.step = 7 * (int)blockDim.x;
  return r;
}

struct RolledLink {
  int mu, par, idx;
  bool sw;
};

// Forward links (c = 0, 1, 2) of direction nu, and backward links (c = 3, 4, 5).
template <int MU>
__device__ __forceinline__ RolledLink rolled_link(const Geometry& gp, const Site& st, int j, int p, int nu, int c) {
  const int q = p ^ 1;
  RolledLink l;
  switch (c) {
    case 0: l = {nu, q, nb_half(gp, st, MU, +1), pair_swap(gp, st, MU, +1)}; break;           // U_nu(x+mu)
    case 1: l = {MU, q, nb_half(gp, st, nu, +1), pair_swap(gp, st, nu, +1)}; break;           // U_mu(x+nu)
    case 2: l = {nu, p, j, false}; break;                                                       // U_nu(x)
    case 3: l = {nu, p, nb_half2(gp, st, MU, nu),                                               // U_nu(x+mu-nu)
                 pair_swap(gp, st, MU, +1) != pair_swap(gp, st, nu, -1)}; break;
    case 4: l = {MU, q, nb_half(gp, st, nu, -1), pair_swap(gp, st, nu, -1)}; break;           // U_mu(x-nu)
    default: l = {nu, q, nb_half(gp, st, nu, -1), pair_swap(gp, st, nu, -1)}; break;          // U_nu(x-nu)
  }
  return l;
}

template <bool CG>
__device__ __forceinline__ void rolled_issue(const Geometry& gp, const float4* U, const RolledLink& l,
                                             const PairRing& rg, int slot) {
  if (!link_ok(l.mu, l.par, l.idx, gp.Vh)) return;
  const float4* b = U + pair_offset(l.mu, l.par, l.idx, gp.Vh);
  const uint32_t sa = rg.sa + (uint32_t)(16 * slot * rg.step);
#pragma unroll
  for (int e = 0; e < 6; ++e) cp_async16<CG>(sa + 16 * e, b + kPairTile * e);
}

// Take link c (0..5) of direction index i (direction nu) and request the link
// three places further on: link c + 3 of the same direction, the first links
// of the next direction, or the updated link pair itself after the last.
template <int MU, int C, bool CG>
__device__ __forceinline__ PM rolled_take(const Geometry& gp, const float4* U, const Site& st, int j, int p, int i,
                                          int nu, const PairRing& rg) {
  cp_async_wait<2>();
  const float4* slot = rg.ptr + (C % 3) * rg.step;
  PM m;
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const float4 c = slot[e];
    m.re[e / 3][e % 3] = make_float2(c.x, c.y);
    m.im[e / 3][e % 3] = make_float2(c.z, c.w);
  }
  __syncwarp();
  if (C < 3) {
    rolled_issue<CG>(gp, U, rolled_link<MU>(gp, st, j, p, nu, C + 3), rg, C % 3);
  } else if (i < 2) {
    const int nx = i + 1 < MU ? i + 1 : i + 2;  // next direction != MU
    rolled_issue<CG>(gp, U, rolled_link<MU>(gp, st, j, p, nx, C - 3), rg, C % 3);
  } else if (C == 3) {
    rolled_issue<CG>(gp, U, RolledLink{MU, p, j, false}, rg, 0);  // the updated link pair
  }
  cp_async_commit();
  swap_halves(m, rolled_link<MU>(gp, st, j, p, nu, C).sw);
  return m;
}

template <int MU, bool CG>
__device__ __forceinline__ PM staple_q_rolled(const Geometry& gp, const float4* U, const Site& st, int j, int p,
                                              const PairRing& rg, PM* own, PM* Apart = nullptr) {
  const int nu0 = MU == 0 ? 1 : 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    rolled_issue<CG>(gp, U, rolled_link<MU>(gp, st, j, p, nu0, c), rg, c);
    cp_async_commit();
  }
  PM A;
#pragma unroll 1
  for (int i = 0; i < 3; ++i) {
    const int nu = i < MU ? i : i + 1;
    {
      // F = U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
      const PM a = rolled_take<MU, 0, CG>(gp, U, st, j, p, i, nu, rg);
      PM b = rolled_take<MU, 1, CG>(gp, U, st, j, p, i, nu, rg);
      complete_row2_q(b);
      PM t;
      mul_nd_q(a, b, t);
      PM c = rolled_take<MU, 2, CG>(gp, U, st, j, p, i, nu, rg);
      complete_row2_q(c);
      PM f;
      mul_nd_q(t, c, f);
      if (i == 0)
        init_completed_q(A, f);
      else
        acc_completed_q(A, f);
    }
    {
      // B = U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)
      PM d = rolled_take<MU, 3, CG>(gp, U, st, j, p, i, nu, rg);
      complete_row2_q(d);
      const PM e = rolled_take<MU, 4, CG>(gp, U, st, j, p, i, nu, rg);
      PM hm;
      mul_nn_q(e, d, hm);
      complete_row2_q(hm);
      PM f = rolled_take<MU, 5, CG>(gp, U, st, j, p, i, nu, rg);
      complete_row2_q(f);
      PM b;
      mul_dn_q(hm, f, b);
      acc_completed_q(A, b);
    }
    if (Apart && nu == MU - 1) *Apart = A;
  }
  cp_async_wait<2>();  // the updated link pair (requested by the last direction's link 3)
  const float4* slot = rg.ptr;
  PM m;
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const float4 c = slot[e];
    m.re[e / 3][e % 3] = make_float2(c.x, c.y);
    m.im[e / 3][e % 3] = make_float2(c.z, c.w);
  }
  *own = m;
  return A;
}

// ---------------------------------------------------------------------------
// Reunitarisation of a link pair, as reunitarise_f32 for each member.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum_q(float2 a, float2 b, float2& s, float2& e) {
  s = qadd(a, b);
  const float2 bb = qsub(s, a);
  e = qadd(qsub(a, qsub(s, bb)), qsub(b, bb));
}

// sum_k x_k y_k as hi + lo (compensated), as dot2
__device__ __forceinline__ void dot2_q(const float2* x, const float2* y, int n, float2& hi, float2& lo) {
  hi = qmul(x[0], y[0]);
  lo = qfma(x[0], y[0], qneg(hi));
  for (int k = 1; k < n; ++k) {
    const float2 p = qmul(x[k], y[k]);
    const float2 pe = qfma(x[k], y[k], qneg(p));
    float2 s, se;
    two_sum_q(hi, p, s, se);
    hi = s;
    lo = qadd(lo, qadd(pe, se));
  }
}

// One member's full FP64 Gram-Schmidt (rows far from orthonormal).
__device__ __forceinline__ void gs_full_member(const float2 a_re[3], const float2 a_im[3], const float2 b_re[3],
                                               const float2 b_im[3], int m, float out[12]) {
  cx<double> r0[3], r1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r0[k] = mk((double)(m ? a_re[k].y : a_re[k].x), (double)(m ? a_im[k].y : a_im[k].x));
    r1[k] = mk((double)(m ? b_re[k].y : b_re[k].x), (double)(m ? b_im[k].y : b_im[k].x));
  }
  gram_schmidt_rows01(r0, r1);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    out[2 * k] = (float)r0[k].re;
    out[2 * k + 1] = (float)r0[k].im;
    out[6 + 2 * k] = (float)r1[k].re;
    out[6 + 2 * k + 1] = (float)r1[k].im;
  }
}

// Rows a (row 0) and b (row 1) of a link pair, reunitarised into ore/oim.
template <bool EFT>
__device__ __forceinline__ void reunitarise_q(const float2 a_re[3], const float2 a_im[3], const float2 b_re[3],
                                              const float2 b_im[3], float2 ore[2][3], float2 oim[2][3]) {
  float2 e0, dr, di, cr, ci, e1;
  if (EFT) {
    float2 ar[6], br[6], bx[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ar[2 * k] = a_re[k];
      ar[2 * k + 1] = a_im[k];
      br[2 * k] = b_re[k];
      br[2 * k + 1] = b_im[k];
      bx[2 * k] = b_im[k];
      bx[2 * k + 1] = qneg(b_re[k]);
    }
    float2 h0, l0, h1, l1, hr, lr, hi_, li;
    dot2_q(ar, ar, 6, h0, l0);
    dot2_q(br, br, 6, h1, l1);
    dot2_q(ar, br, 6, hr, lr);
    dot2_q(ar, bx, 6, hi_, li);
    const float2 one = make_float2(1.0f, 1.0f);
    e0 = qadd(qsub(h0, one), l0);
    dr = qadd(hr, lr);
    di = qadd(hi_, li);
    const float2 inv_n0 = qsub(one, e0);
    cr = qmul(dr, inv_n0);
    ci = qmul(di, inv_n0);
    e1 = qsub(qadd(qsub(h1, one), l1), qfma(ci, di, qmul(cr, dr)));
  } else {
    double n0[2], n1[2], dre[2], dim[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      n0[m] = n1[m] = dre[m] = dim[m] = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double ar = f32_to_f64_bits(m ? a_re[k].y : a_re[k].x), ai = f32_to_f64_bits(m ? a_im[k].y : a_im[k].x);
        const double br = f32_to_f64_bits(m ? b_re[k].y : b_re[k].x), bi = f32_to_f64_bits(m ? b_im[k].y : b_im[k].x);
        n0[m] = fma(ar, ar, fma(ai, ai, n0[m]));
        n1[m] = fma(br, br, fma(bi, bi, n1[m]));
        dre[m] = fma(ar, br, fma(ai, bi, dre[m]));
        dim[m] = fma(ar, bi, fma(-ai, br, dim[m]));
      }
    }
    e0 = make_float2((float)(n0[0] - 1.0), (float)(n0[1] - 1.0));
    dr = make_float2((float)dre[0], (float)dre[1]);
    di = make_float2((float)dim[0], (float)dim[1]);
    const float2 inv_n0 = qsub(make_float2(1.0f, 1.0f), e0);
    cr = qmul(dr, inv_n0);
    ci = qmul(di, inv_n0);
    e1 = qsub(make_float2((float)(n1[0] - 1.0), (float)(n1[1] - 1.0)), qfma(ci, di, qmul(cr, dr)));
  }
  const bool okx = fabsf(e0.x) < 1e-3f && fabsf(e1.x) < 1e-3f && fabsf(dr.x) < 1e-3f && fabsf(di.x) < 1e-3f;
  const bool oky = fabsf(e0.y) < 1e-3f && fabsf(e1.y) < 1e-3f && fabsf(dr.y) < 1e-3f && fabsf(di.y) < 1e-3f;
  const float2 s0 = qmul(e0, qfma(make_float2(0.375f, 0.375f), e0, make_float2(-0.5f, -0.5f)));
  const float2 s1 = qmul(e1, qfma(make_float2(0.375f, 0.375f), e1, make_float2(-0.5f, -0.5f)));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ore[0][k] = qfma(a_re[k], s0, a_re[k]);
    oim[0][k] = qfma(a_im[k], s0, a_im[k]);
    // r1 - c r0
    const float2 tr = qfma(qneg(cr), a_re[k], qfma(ci, a_im[k], b_re[k]));
    const float2 ti = qfma(qneg(cr), a_im[k], qfma(qneg(ci), a_re[k], b_im[k]));
    ore[1][k] = qfma(tr, s1, tr);
    oim[1][k] = qfma(ti, s1, ti);
  }
  if (!(okx && oky)) {  // a member far from unitary: full FP64 Gram-Schmidt for it
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      if (m ? oky : okx) continue;
      float o[12];
      gs_full_member(a_re, a_im, b_re, b_im, m, o);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (m) {
          ore[0][k].y = o[2 * k];
          oim[0][k].y = o[2 * k + 1];
          ore[1][k].y = o[6 + 2 * k];
          oim[1][k].y = o[6 + 2 * k + 1];
        } else {
          ore[0][k].x = o[2 * k];
          oim[0][k].x = o[2 * k + 1];
          ore[1][k].x = o[6 + 2 * k];
          oim[1][k].x = o[6 + 2 * k + 1];
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The heatbath of a link pair after its staple: three SU(2) steps, each member
// drawing its own random numbers (its own site's Philox counters) and taking
// its own accept decision, then reunitarisation and the store.  In the order
// of heatbath_f32_on.  s0 is the canonical index of the first member; the
// second is s0 + V/2.
// ---------------------------------------------------------------------------
template <bool REPEAT, typename KEY>
__device__ __forceinline__ bool kp_member(float ia, uint32_t s, uint32_t w1base, uint64_t t, const KEY& key,
                                          int ntries, int& proposed, float a[4]) {
  for (int tr = 0; tr < ntries; ++tr) {
    const uint32_t w1b = w1base | ((uint32_t)tr << 6);
    const uint4 w0 = philox4x32_10(rng_counter(s, w1b, t, kTagUpdate), key);
    const uint4 w1 = philox4x32_10(rng_counter(s, w1b | (1u << 4), t, kTagUpdate), key);
    ++proposed;
    const float u0 = u01_f32(w0.x), u1 = u01_f32(w0.y), u2 = u01_f32(w0.z), u3 = u01_f32(w0.w);
    const float cc = __cosf(fmaf(6.2831853f, u1, -3.14159265f));
    const float delta = __fmul_rn(-__fmaf_rn(__fmul_rn(cc, cc), __logf(u2), __logf(u0)), ia);
    if (__fmul_rn(u3, u3) > __fmaf_rn(-0.5f, delta, 1.0f)) continue;
    const float u4 = u01_f32(w1.x), u5 = u01_f32(w1.y);
    const float rho = sqrt_approx(fmaxf(0.0f, delta * (2.0f - delta)));
    const float ct = __fmaf_rn(-2.0f, u4, 1.0f);
    const float sn = 2.0f * sqrt_approx(u4 * (1.0f - u4));
    float sphi, cphi;
    __sincosf(fmaf(6.2831853f, u5, -3.14159265f), &sphi, &cphi);
    const float rs = -rho * sn;
    a[0] = 1.0f - delta;
    a[1] = rs * cphi;
    a[2] = rs * sphi;
    a[3] = rho * ct;
    return true;
  }
  return false;
}

// Both members' one-hit proposals at once, without branches (the accept
// decisions are returned, the proposals computed whatever they are): each
// member draws from its own site's counters (s0, s1), and the FP32
// arithmetic of kp_member's first try runs on paired instructions, lane by
// lane the same roundings (the transcendentals stay one per lane).
__device__ __forceinline__ float2 u01_q(uint32_t a, uint32_t b) {
  return qsub(make_float2(__int_as_float((int)(0x3F800000u | (a >> 9))), __int_as_float((int)(0x3F800000u | (b >> 9)))),
              make_float2(1.0f - 0x1p-24f, 1.0f - 0x1p-24f));
}
__device__ __forceinline__ float2 qconst(float c) { return make_float2(c, c); }

template <typename KEY>
__device__ __forceinline__ void kp_pair_1hit(float2 ia, uint32_t s0, uint32_t s1, uint32_t w1base, uint64_t t,
                                             const KEY& key, bool& accx, bool& accy, float2 a[4]) {
  const uint4 x0 = philox4x32_10(rng_counter(s0, w1base, t, kTagUpdate), key);
  const uint4 y0 = philox4x32_10(rng_counter(s1, w1base, t, kTagUpdate), key);
  const uint4 x1 = philox4x32_10(rng_counter(s0, w1base | (1u << 4), t, kTagUpdate), key);
  const uint4 y1 = philox4x32_10(rng_counter(s1, w1base | (1u << 4), t, kTagUpdate), key);
  const float2 u0 = u01_q(x0.x, y0.x), u1 = u01_q(x0.y, y0.y), u2 = u01_q(x0.z, y0.z), u3 = u01_q(x0.w, y0.w);
  const float2 ph = qfma(qconst(6.2831853f), u1, qconst(-3.14159265f));
  const float2 cc = make_float2(__cosf(ph.x), __cosf(ph.y));
  const float2 l0 = make_float2(__logf(u0.x), __logf(u0.y)), l2 = make_float2(__logf(u2.x), __logf(u2.y));
  const float2 delta = qmul(qneg(qfma(qmul(cc, cc), l2, l0)), ia);
  const float2 lhs = qmul(u3, u3), rhs = qfma(qconst(-0.5f), delta, qconst(1.0f));
  accx = !(lhs.x > rhs.x);
  accy = !(lhs.y > rhs.y);
  const float2 u4 = u01_q(x1.x, y1.x), u5 = u01_q(x1.y, y1.y);
  const float2 q = qmul(delta, qsub(qconst(2.0f), delta));
  const float2 rho = make_float2(sqrt_approx(fmaxf(0.0f, q.x)), sqrt_approx(fmaxf(0.0f, q.y)));
  const float2 ct = qfma(qconst(-2.0f), u4, qconst(1.0f));
  const float2 w = qmul(u4, qsub(qconst(1.0f), u4));
  const float2 sn = qmul(qconst(2.0f), make_float2(sqrt_approx(w.x), sqrt_approx(w.y)));
  const float2 pf = qfma(qconst(6.2831853f), u5, qconst(-3.14159265f));
  float2 sphi, cphi;
  __sincosf(pf.x, &sphi.x, &cphi.x);
  __sincosf(pf.y, &sphi.y, &cphi.y);
  const float2 rs = qmul(qneg(rho), sn);
  a[0] = qsub(qconst(1.0f), delta);
  a[1] = qmul(rs, cphi);
  a[2] = qmul(rs, sphi);
  a[3] = qmul(rho, ct);
}

template <int MU, bool EFT, bool REPEAT, bool MEAS, typename KEY>
__device__ __forceinline__ UpdateCount heatbath_q(const Geometry& gp, float4* U, int j, int p, uint64_t t, uint32_t s0,
                                                  uint32_t s1, const KEY& key, const UpdateConsts& uc, const PM& A,
                                                  const PM& Apart, double2* meas, PM u, bool store) {
  UpdateCount cnt{0, 0};
  complete_row2_q(u);
  const float2 tob = make_float2(uc.three_over_beta, uc.three_over_beta);
#pragma unroll
  for (int sub = 0; sub < 3; ++sub) {
    const int i = subrow_i(sub), jj = subrow_j(sub);
    // 2x2 block (i, jj) of W = U A, as mac over c from 0
    qcx wii = qmk(qzero(), qzero()), wij = wii, wji = wii, wjj = wii;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      wii = qcmac(wii, qget(u, i, c), qget(A, c, i));
      wij = qcmac(wij, qget(u, i, c), qget(A, c, jj));
      wji = qcmac(wji, qget(u, jj, c), qget(A, c, i));
      wjj = qcmac(wjj, qget(u, jj, c), qget(A, c, jj));
    }
    const float2 r0 = qadd(wii.re, wjj.re), r1 = qadd(wij.im, wji.im);
    const float2 r2 = qsub(wij.re, wji.re), r3 = qsub(wii.im, wjj.im);
    const float2 kk = qfma(r3, r3, qfma(r2, r2, qfma(r1, r1, qmul(r0, r0))));
    const bool degx = !(kk.x > 4e-30f), degy = !(kk.y > 4e-30f);
    const float2 ik = make_float2(rsqrtf(kk.x), rsqrtf(kk.y));
    const float2 ia = qmul(tob, ik);
    const int ntries = REPEAT ? uc.max_tries : 1;
    const uint32_t w1base = (uint32_t)(MU | (sub << 2));
    bool accx = false, accy = false;
    float2 a0, a1, a2, a3;
    if (REPEAT) {
      float ax[4] = {1.f, 0.f, 0.f, 0.f}, ay[4] = {1.f, 0.f, 0.f, 0.f};
      if (degx)
        ++cnt.proposed;
      else
        accx = kp_member<REPEAT>(ia.x, s0, w1base, t, key, ntries, cnt.proposed, ax);
      if (degy)
        ++cnt.proposed;
      else
        accy = kp_member<REPEAT>(ia.y, s1, w1base, t, key, ntries, cnt.proposed, ay);
      if (!(accx || accy)) continue;
      a0 = make_float2(ax[0], ay[0]);
      a1 = make_float2(ax[1], ay[1]);
      a2 = make_float2(ax[2], ay[2]);
      a3 = make_float2(ax[3], ay[3]);
    } else {
      // a degenerate member draws nothing in the single-site update; here its
      // draws are made and thrown away, which changes no other number
      float2 a[4];
      kp_pair_1hit(ia, s0, s1, w1base, t, key, accx, accy, a);
      accx = accx && !degx;
      accy = accy && !degy;
      cnt.proposed += 2;
      a0 = a[0];
      a1 = a[1];
      a2 = a[2];
      a3 = a[3];
    }
    cnt.accepted += (int)accx + (int)accy;
    const float2 v0 = qmul(r0, ik), v1 = qmul(r1, ik), v2 = qmul(r2, ik), v3 = qmul(r3, ik);
    // R = Y V^+, Y = m(a), V = m(v), m(q) = [[q0 + i q3, q2 + i q1], [-q2 + i q1, q0 - i q3]]
    const qcx y00 = qmk(a0, a3), y01 = qmk(a2, a1);
    const qcx v00 = qmk(v0, v3), v01 = qmk(v2, v1), v10 = qmk(qneg(v2), v1), v11 = qmk(v0, qneg(v3));
    const qcx z = qmk(qzero(), qzero());
    const qcx R00 = qcmac_cb(qcmac_cb(z, y00, v00), y01, v01);
    const qcx R01 = qcmac_cb(qcmac_cb(z, y00, v10), y01, v11);
    const qcx R10 = qmk(qneg(R01.re), R01.im);
    const qcx R11 = qmk(R00.re, qneg(R00.im));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const qcx ui = qget(u, i, c), uj = qget(u, jj, c);
      const qcx ni = qcmac(qcmul(R00, ui), R01, uj);
      u.re[i][c] = qsel(accx, accy, ni.re, ui.re);
      u.im[i][c] = qsel(accx, accy, ni.im, ui.im);
      // row 2 leaves the last subgroup unused: reunitarisation rebuilds it
      if (sub < 2) {
        const qcx nj = qcmac(qcmul(R10, ui), R11, uj);
        u.re[jj][c] = qsel(accx, accy, nj.re, uj.re);
        u.im[jj][c] = qsel(accx, accy, nj.im, uj.im);
      }
    }
  }
  float2 ore[2][3], oim[2][3];
  reunitarise_q<EFT>(u.re[0], u.im[0], u.re[1], u.im[1], ore, oim);
  if (store) store_pm_rows01(U, MU, p, j, gp.Vh, ore, oim);
  if (MEAS) {
    // the stored link pair, row 2 completed, against A_<
    PM un;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        un.re[r][k] = ore[r][k];
        un.im[r][k] = oim[r][k];
      }
    complete_row2_q(un);
    float2 tr = qzero();
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) tr = qfma(un.re[i][k], Apart.re[k][i], qfma(qneg(un.im[i][k]), Apart.im[k][i], tr));
    *meas = make_double2((double)tr.x * (1.0 / 3.0), (double)tr.y * (1.0 / 3.0));
  }
  return cnt;
}

// One link-pair update: the staged staple, the heatbath, the store.  j: the
// pair index (a clamped lane passes a valid index and store = false); meas:
// with MEAS, (1/3) Re Tr(U_new A_<) of both members.
template <int MU, bool CG, bool EFT, bool REPEAT, bool MEAS = false, typename KEY>
__device__ __forceinline__ UpdateCount update_pair_f32_rolled(const Geometry& gp, float4* U, int j, int p, uint64_t t,
                                                              const KEY& key, const UpdateConsts& uc,
                                                              const PairRing& rg, bool store = true,
                                                              double2* meas = nullptr) {
  const Site st = site_of(gp, j, p);
  const uint32_t s0 = (uint32_t)canon(gp, st);
  const uint32_t s1 = s0 + (uint32_t)(2 * gp.Vh);
  PM Apart, own;
  const PM A = staple_q_rolled<MU, CG>(gp, U, st, j, p, rg, &own, MEAS ? &Apart : nullptr);
  return heatbath_q<MU, EFT, REPEAT, MEAS>(gp, U, j, p, t, s0, s1, key, uc, A, Apart, meas, own, store);
}

}  // namespace su3dev
