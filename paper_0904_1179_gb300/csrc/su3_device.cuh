// su3_device.cuh -- device building blocks of the checkerboard SU(3) heatbath
// sweep for sm_103a: complex 3x3 algebra on CUDA cores, Philox4x32-10, the
// uniform maps, checkerboard index arithmetic and the link store.
//
// The method is the pure SU(3) Wilson-action checkerboard update of Berg & Wu
// (arXiv:0904.1179, Abstract and Sec. 1): the links of one direction mu and one
// site parity never share a staple, so each (mu, parity) half-sweep updates
// all of its links in parallel, one thread per link.  Each update is a
// one-hit heatbath (Sec. 2.1) built as Cabibbo-Marinari over the SU(2)
// subgroups (0,1), (0,2), (1,2) with the Kennedy-Pendleton sampler, followed
// by Gram-Schmidt reunitarisation.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "su3_log_table.cuh"

namespace su3dev {

// ---------------------------------------------------------------------------
// Link store.  Half-lattice structure of arrays, one array per (mu, parity,
// component group), indexed by the checkerboard half index h = s / 2 where
// s = x0 + L0*(x1 + L1*(x2 + L2*x3)) and L0 is even, so each parity holds
// exactly one site of every pair (2h, 2h+1).
//   FP64:       double2 [4 mu][2 parity][9 entries (row*3+col)][Vh]
//   FP32-mixed: float4  [4 mu][2 parity][3 columns][Vh], rows 0 and 1 only:
//               column k holds (re u0k, re u1k, im u0k, im u1k), so one load
//               gives the row pairs (u0k, u1k) of real and of imaginary parts
//               that the paired FP32 arithmetic (fma.rn.f32x2) works on.
// ---------------------------------------------------------------------------
constexpr int kEntriesF64 = 9;
constexpr int kGroupsF32 = 3;

// Philox4x32-10 constants (Salmon, Moraes, Dror, Shaw, SC'11).
constexpr uint32_t kPhiloxMulA = 0xD2511F53u;
constexpr uint32_t kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kPhiloxWeylA = 0x9E3779B9u;
constexpr uint32_t kPhiloxWeylB = 0xBB67AE85u;

// RNG stream tags (fourth counter word, low 4 bits).
constexpr uint32_t kTagUpdate = 0u;
constexpr uint32_t kTagHotStart = 1u;

// Division of n in [0, 2^31) by a fixed d >= 1 as a multiply and a shift:
// with s = ceil(log2 d) and m = ceil(2^(31+s) / d) < 2^32,
// floor(n m / 2^(31+s)) = floor(n / d) exactly, because the excess
// n (m d - 2^(31+s)) / (d 2^(31+s)) is below 2^-s <= 1/d (Granlund and
// Montgomery, PLDI 1994).
struct Divisor {
  uint32_t m;
  int shift;  // 31 + s
};

__host__ inline Divisor make_divisor(uint32_t d) {
  int s = 0;
  while ((1ull << s) < d) ++s;
  const unsigned long long two = 1ull << (31 + s);
  return Divisor{(uint32_t)((two + d - 1) / d), 31 + s};
}

__host__ __device__ __forceinline__ int udiv(int n, const Divisor& d) {
  return (int)(((unsigned long long)(uint32_t)n * d.m) >> d.shift);
}

struct Geometry {
  int L0, L1, L2, L3;
  int hL0;      // L0 / 2
  int Vh;       // V / 2
  int s1, s2, s3;  // strides of x1, x2, x3 in the canonical index: L0, L0*L1, L0*L1*L2
  Divisor div_hL0, div_L1, div_L2;
  // Half-index steps: hs[nu] = change of h for x_nu + 1 (nu >= 1), and
  // wrap[nu] = (L_nu - 1) hs[nu], the change when x_nu wraps from L_nu - 1 to
  // 0 (with the sign reversed); wrap[0] = L0/2 - 1 for x0.
  int hs[4], wrap[4];
};

// Geometry of a periodic L0 x L1 x L2 x L3 lattice (L0 even, V/2 < 2^31).
__host__ inline Geometry make_geometry(int L0, int L1, int L2, int L3) {
  Geometry g{};
  g.L0 = L0;
  g.L1 = L1;
  g.L2 = L2;
  g.L3 = L3;
  g.hL0 = L0 / 2;
  g.Vh = (int)((long long)L0 * L1 * L2 * L3 / 2);
  g.s1 = L0;
  g.s2 = L0 * L1;
  g.s3 = L0 * L1 * L2;
  g.div_hL0 = make_divisor((uint32_t)g.hL0);
  g.div_L1 = make_divisor((uint32_t)L1);
  g.div_L2 = make_divisor((uint32_t)L2);
  g.hs[0] = 0;
  g.hs[1] = g.hL0;
  g.hs[2] = g.hL0 * L1;
  g.hs[3] = g.hL0 * L1 * L2;
  g.wrap[0] = g.hL0 - 1;
  g.wrap[1] = (L1 - 1) * g.hs[1];
  g.wrap[2] = (L2 - 1) * g.hs[2];
  g.wrap[3] = (L3 - 1) * g.hs[3];
  return g;
}

struct PhiloxKey {
  uint32_t k0, k1;
};

// The ten round keys of one seed (key, key + W, ..., key + 9W), computed once
// on the host so that each round reads them from the kernel's parameter bank.
struct PhiloxRoundKeys {
  uint32_t k[10][2];
};

__host__ __device__ inline PhiloxRoundKeys philox_round_keys(PhiloxKey key) {
  PhiloxRoundKeys rk;
  uint32_t k0 = key.k0, k1 = key.k1;
  for (int r = 0; r < 10; ++r) {
    rk.k[r][0] = k0;
    rk.k[r][1] = k1;
    k0 += kPhiloxWeylA;
    k1 += kPhiloxWeylB;
  }
  return rk;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 block function: ten rounds, each two 32x32->64-bit products
// and a xor with the round key.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxRoundKeys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo_a = kPhiloxMulA * c.x;
    const uint32_t hi_a = __umulhi(kPhiloxMulA, c.x);
    const uint32_t lo_b = kPhiloxMulB * c.z;
    const uint32_t hi_b = __umulhi(kPhiloxMulB, c.z);
    c = make_uint4(hi_b ^ c.y ^ rk.k[r][0], lo_b, hi_a ^ c.w ^ rk.k[r][1], lo_a);
  }
  return c;
}

// Same block function with the round keys derived on the fly from the seed
// (used where the key differs between work items, e.g. per replica).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, PhiloxKey key) {
  uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo_a = kPhiloxMulA * c.x;
    const uint32_t hi_a = __umulhi(kPhiloxMulA, c.x);
    const uint32_t lo_b = kPhiloxMulB * c.z;
    const uint32_t hi_b = __umulhi(kPhiloxMulB, c.z);
    c = make_uint4(hi_b ^ c.y ^ k0, lo_b, hi_a ^ c.w ^ k1, lo_a);
    k0 += kPhiloxWeylA;
    k1 += kPhiloxWeylB;
  }
  return c;
}

// Counter of draw `w1` (= mu | sub<<2 | call<<4) of site s at sweep t.
__device__ __forceinline__ uint4 rng_counter(uint32_t site, uint32_t w1, uint64_t t, uint32_t tag) {
  return make_uint4(site, w1, (uint32_t)t, tag | ((uint32_t)(t >> 32) << 4));
}

// Uniform in [2^-53, 1-2^-53]: 52 bits (a<<20 | b>>12) centred in its bin.
// Built from the bits: 1 + x 2^-52 is exact, and subtracting 1 - 2^-53 leaves
// (x + 1/2) 2^-52 exactly (Sterbenz), without an integer-to-FP64 conversion.
__device__ __forceinline__ double u01_f64(uint32_t a, uint32_t b) {
  const uint64_t x = ((uint64_t)a << 20) | (uint64_t)(b >> 12);
  return __longlong_as_double((long long)(0x3FF0000000000000ull | x)) - (1.0 - 0x1p-53);
}

// Natural logarithm of a uniform u in (0, 1) (a normal double, as u01_f64
// makes them), by table-driven argument reduction (P. T. P. Tang, ACM TOMS 16
// (1990) 378): u = m 2^e with m in [1, 2), F = 1 + j/64 the table point
// nearest m, r = (m - F)/F with |r| <= 2^-7, and
//     log u = e ln 2 + log F + log(1 + r),
// log(1 + r) from its Taylor series to r^7 (truncation 2^-52 relative).  The
// table (su3_log_table.cuh) holds log F and 1/F rounded to double; the result
// is within a few ulp of the exact logarithm.  Eleven FP64 operations.
__device__ __forceinline__ double log_u01(double u) {
  const long long b = __double_as_longlong(u);
  const int e = (int)(b >> 52) - 1023;  // u in (0, 1): e in [-53, -1]
  const long long mb = b & 0x000FFFFFFFFFFFFFLL;
  const double m = __longlong_as_double(mb | 0x3FF0000000000000LL);             // [1, 2)
  const int j = (int)((mb + (1LL << 45)) >> 46);                                 // round(64 (m - 1)), 0..64
  const double F = __longlong_as_double(0x3FF0000000000000LL + ((long long)j << 46));  // 1 + j/64 (2 for j = 64)
  const double r = (m - F) * __ldg(&kInvF[j]);
  double p = 1.0 / 7.0;
  p = fma(p, r, -1.0 / 6.0);
  p = fma(p, r, 1.0 / 5.0);
  p = fma(p, r, -1.0 / 4.0);
  p = fma(p, r, 1.0 / 3.0);
  p = fma(p, r, -0.5);
  p = fma(p, r, 1.0);
  // e as a double without a conversion: 2^52 + 1024 + e from its bits, minus 2^52 + 1024
  const double ed = __longlong_as_double(0x4330000000000000LL + (long long)(e + 1024)) - 4503599627371520.0;
  return fma(ed, 0x1.62e42fefa39efp-1, __ldg(&kLogF[j])) + r * p;
}

// Uniform in [2^-24, 1-2^-24]: 23 bits centred in the bin, exact in float.
__device__ __forceinline__ float u01_f32(uint32_t a) {
  return __int_as_float((int)(0x3F800000u | (a >> 9))) - (1.0f - 0x1p-24f);  // (m + 1/2) 2^-23, exact
}

// ---------------------------------------------------------------------------
// Complex numbers and 3x3 matrices held in registers.
// ---------------------------------------------------------------------------
template <typename T>
struct cx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T re, T im) {
  cx<T> r;
  r.re = re;
  r.im = im;
  return r;
}
template <typename T>
__device__ __forceinline__ cx<T> conj(cx<T> a) {
  return mk(a.re, -a.im);
}
template <typename T>
__device__ __forceinline__ cx<T> add(cx<T> a, cx<T> b) {
  return mk(a.re + b.re, a.im + b.im);
}
template <typename T>
__device__ __forceinline__ cx<T> mul(cx<T> a, cx<T> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// FP32 product with every rounding step written out (no contraction left to
// the compiler), so that the single-site and the site-paired FP32 updates
// (su3_sitepair.cuh) round identically: re = fma(-a.im, b.im, a.re b.re),
// im = fma(a.im, b.re, a.re b.im).
__device__ __forceinline__ cx<float> mul(cx<float> a, cx<float> b) {
  return mk(__fmaf_rn(-a.im, b.im, __fmul_rn(a.re, b.re)), __fmaf_rn(a.im, b.re, __fmul_rn(a.re, b.im)));
}
// acc + a*b
template <typename T>
__device__ __forceinline__ cx<T> mac(cx<T> acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + a*conj(b)
template <typename T>
__device__ __forceinline__ cx<T> mac_cb(cx<T> acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(-a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + conj(a)*b
template <typename T>
__device__ __forceinline__ cx<T> mac_ca(cx<T> acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}

template <typename T>
struct mat3 {
  cx<T> e[3][3];
};

// Row 2 of an SU(3) matrix from rows 0 and 1: conj(row0 x row1).
template <typename T>
__device__ __forceinline__ void complete_row2(mat3<T>& m) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int a = (k + 1) % 3, b = (k + 2) % 3;
    cx<T> v = mul(m.e[0][a], m.e[1][b]);
    v = mac(v, mk(-m.e[0][b].re, -m.e[0][b].im), m.e[1][a]);
    m.e[2][k] = conj(v);
  }
}

// Rows 0,1 of X * Y^+ (Y complete).
template <typename T>
__device__ __forceinline__ void mul_nd_rows01(const mat3<T>& X, const mat3<T>& Y, mat3<T>& Z) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cx<T> s = mk(T(0), T(0));
#pragma unroll
      for (int j = 0; j < 3; ++j) s = mac_cb(s, X.e[i][j], Y.e[k][j]);
      Z.e[i][k] = s;
    }
}

// Columns 0,1 of X * Y (X complete, Y's columns 0,1 used); column 2 of Z is
// left unset.
template <typename T>
__device__ __forceinline__ void mul_nn_cols01(const mat3<T>& X, const mat3<T>& Y, mat3<T>& Z) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      cx<T> s = mk(T(0), T(0));
#pragma unroll
      for (int j = 0; j < 3; ++j) s = mac(s, X.e[i][j], Y.e[j][k]);
      Z.e[i][k] = s;
    }
}

// Rows 0,1 of X^+ * Y (X's columns 0,1 used, Y complete).
template <typename T>
__device__ __forceinline__ void mul_dn_rows01(const mat3<T>& X, const mat3<T>& Y, mat3<T>& Z) {
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cx<T> s = mk(T(0), T(0));
#pragma unroll
      for (int j = 0; j < 3; ++j) s = mac_ca(s, X.e[j][i], Y.e[j][k]);
      Z.e[i][k] = s;
    }
}

// A += B for an SU(3) matrix B of which only rows 0,1 are set: row 2 of B is
// formed as conj(row0 x row1) inside the accumulation of A's row 2.
template <typename T>
__device__ __forceinline__ void acc_completed(mat3<T>& A, const mat3<T>& B) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    A.e[0][k] = add(A.e[0][k], B.e[0][k]);
    A.e[1][k] = add(A.e[1][k], B.e[1][k]);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int a = (k + 1) % 3, b = (k + 2) % 3;
    // A_2k + conj(v) = conj(conj(A_2k) + v), v = B_0a B_1b - B_0b B_1a
    cx<T> v = mac(conj(A.e[2][k]), B.e[0][a], B.e[1][b]);
    v = mac(v, mk(-B.e[0][b].re, -B.e[0][b].im), B.e[1][a]);
    A.e[2][k] = conj(v);
  }
}

// ---------------------------------------------------------------------------
// Checkerboard geometry.  A thread owns half index h and parity p; its site
// has x0 = 2*(h mod hL0) + ((p + x1 + x2 + x3) & 1).
// ---------------------------------------------------------------------------
struct Site {
  int x0, x1, x2, x3;
  int r;  // x1 + L1*(x2 + L2*x3)
  int h;  // half index (x0 >> 1) + hL0 * r
};

__host__ __device__ __forceinline__ Site site_of(const Geometry& g, int h, int p) {
  Site st;
  const int r = udiv(h, g.div_hL0);
  const int x0e = 2 * (h - r * g.hL0);
  st.r = r;
  const int q = udiv(r, g.div_L1);
  st.x1 = r - q * g.L1;
  st.x3 = udiv(q, g.div_L2);
  st.x2 = q - st.x3 * g.L2;
  st.x0 = x0e + ((p + st.x1 + st.x2 + st.x3) & 1);
  st.h = h;
  return st;
}

__host__ __device__ __forceinline__ int canon(const Geometry& g, const Site& s) { return s.x0 + g.L0 * s.r; }

// The half index is separable, h = (x0 >> 1) + hs1 x1 + hs2 x2 + hs3 x3, so
// a step of d = +1 or -1 along nu changes it by an offset that depends only
// on x_nu: +-hs[nu], or the wrap offset at the boundary; along x0 the step
// changes x0 >> 1 by 0 or d, depending on the parity of x0.
__host__ __device__ __forceinline__ int nb_offset(const Geometry& g, const Site& s, int nu, int d) {
  if (nu == 0) {
    if (d > 0) return s.x0 == g.L0 - 1 ? -g.wrap[0] : (s.x0 & 1);
    return s.x0 == 0 ? g.wrap[0] : (s.x0 & 1) - 1;
  }
  const int x = nu == 1 ? s.x1 : (nu == 2 ? s.x2 : s.x3);
  const int L = nu == 1 ? g.L1 : (nu == 2 ? g.L2 : g.L3);
  if (d > 0) return x == L - 1 ? -g.wrap[nu] : g.hs[nu];
  return x == 0 ? g.wrap[nu] : -g.hs[nu];
}

// Half index of the neighbour x + d*nu-hat (d = +1 or -1), periodic.
__host__ __device__ __forceinline__ int nb_half(const Geometry& g, const Site& s, int nu, int d) {
  return s.h + nb_offset(g, s, nu, d);
}

__device__ __forceinline__ int wrap_coord(int x, int L) { return x < 0 ? x + L : (x >= L ? x - L : x); }

// nb_half and nb_half2 for a direction known only at run time (it differs
// between the lanes that share one link update): selects, no indexed arrays.
__device__ __forceinline__ int nb_half_rt(const Geometry& g, const Site& s, int nu, int d) {
  const int x0 = nu == 0 ? wrap_coord(s.x0 + d, g.L0) : s.x0;
  const int x1 = nu == 1 ? wrap_coord(s.x1 + d, g.L1) : s.x1;
  const int x2 = nu == 2 ? wrap_coord(s.x2 + d, g.L2) : s.x2;
  const int x3 = nu == 3 ? wrap_coord(s.x3 + d, g.L3) : s.x3;
  return (x0 >> 1) + g.hL0 * (x1 + g.L1 * (x2 + g.L2 * x3));
}

__device__ __forceinline__ int nb_half2_rt(const Geometry& g, const Site& s, int nu, int rho) {
  const int x0 = wrap_coord(s.x0 + (nu == 0) - (rho == 0), g.L0);
  const int x1 = wrap_coord(s.x1 + (nu == 1) - (rho == 1), g.L1);
  const int x2 = wrap_coord(s.x2 + (nu == 2) - (rho == 2), g.L2);
  const int x3 = wrap_coord(s.x3 + (nu == 3) - (rho == 3), g.L3);
  return (x0 >> 1) + g.hL0 * (x1 + g.L1 * (x2 + g.L2 * x3));
}

// Half index of x + nu-hat - rho-hat for nu != rho.
__host__ __device__ __forceinline__ int nb_half2(const Geometry& g, const Site& s, int nu, int rho) {
  return s.h + nb_offset(g, s, nu, +1) + nb_offset(g, s, rho, -1);
}

// Storage half index of the thread's own site (the plain lattice stores the
// site where it enumerates it).
__device__ __forceinline__ int store_index(const Geometry&, const Site&, int h) { return h; }

// ---------------------------------------------------------------------------
// Sublattice with ghost layers: the paper's domain decomposition (Sec. 2.1:
// the first ndmpi directions cut into mpifactor parts each) emulated on one
// device.  A sublattice stores an extended box: extent l_d + 2 in a cut
// direction (one ghost layer on each side, filled by the boundary exchange),
// l_d = L_d otherwise (periodic wrap inside the sublattice).  Threads
// enumerate the interior sites of one parity with the plain rule on the
// interior extents; the global site (for the random numbers) is the
// interior coordinate plus the sublattice origin.  Interior extents in cut
// directions are even, so origins are even and local parity is global
// parity.
// ---------------------------------------------------------------------------
struct SubGeometry {
  Geometry in;         // interior extents (thread enumeration)
  int e[4];            // extended extents
  int he0;             // e0 / 2
  int Vh;              // extended sites / 2: the storage stride
  int cut;             // bit d set: direction d is cut (ghost layers)
  int o[4];            // global coordinate of the interior origin
  int L0, L1, L2;      // global extents for the canonical index
};

struct SubSite {
  int y0, y1, y2, y3;  // extended-box coordinates
  int r;               // y1 + e1*(y2 + e2*y3)
  int s;               // global canonical index
};

__device__ __forceinline__ SubSite site_of(const SubGeometry& g, int h, int p) {
  const Site t = site_of(g.in, h, p);
  SubSite st;
  const int c0 = g.cut & 1, c1 = (g.cut >> 1) & 1, c2 = (g.cut >> 2) & 1, c3 = (g.cut >> 3) & 1;
  st.y0 = t.x0 + c0;
  st.y1 = t.x1 + c1;
  st.y2 = t.x2 + c2;
  st.y3 = t.x3 + c3;
  st.r = st.y1 + g.e[1] * (st.y2 + g.e[2] * st.y3);
  st.s = (t.x0 + g.o[0]) + g.L0 * ((t.x1 + g.o[1]) + g.L1 * ((t.x2 + g.o[2]) + g.L2 * (t.x3 + g.o[3])));
  return st;
}

__device__ __forceinline__ int canon(const SubGeometry&, const SubSite& s) { return s.s; }

__device__ __forceinline__ int store_index(const SubGeometry& g, const SubSite& st, int) {
  return (st.y0 >> 1) + g.he0 * st.r;
}

// Step d (+1 or -1) along nu: into the ghost layer in a cut direction,
// periodic inside the sublattice otherwise.
__device__ __forceinline__ int sub_step(const SubGeometry& g, int y, int nu, int d) {
  y += d;
  if (!((g.cut >> nu) & 1)) y = y < 0 ? y + g.e[nu] : (y >= g.e[nu] ? y - g.e[nu] : y);
  return y;
}

__device__ __forceinline__ int sub_half(const SubGeometry& g, int y0, int y1, int y2, int y3) {
  return (y0 >> 1) + g.he0 * (y1 + g.e[1] * (y2 + g.e[2] * y3));
}

__device__ __forceinline__ int nb_half(const SubGeometry& g, const SubSite& s, int nu, int d) {
  int y[4] = {s.y0, s.y1, s.y2, s.y3};
  y[nu] = sub_step(g, y[nu], nu, d);
  return sub_half(g, y[0], y[1], y[2], y[3]);
}

__device__ __forceinline__ int nb_half2(const SubGeometry& g, const SubSite& s, int nu, int rho) {
  int y[4] = {s.y0, s.y1, s.y2, s.y3};
  y[nu] = sub_step(g, y[nu], nu, +1);
  y[rho] = sub_step(g, y[rho], rho, -1);
  return sub_half(g, y[0], y[1], y[2], y[3]);
}

// ---------------------------------------------------------------------------
// Bounds-checked build (compiled with -DSU3_BOUNDS_CHECK; the product build
// has no checks): every link access checks its direction, parity and index
// against the extent of the store it addresses -- a single lattice, one
// replica of a batch, one sublattice's extended box.  An access out of range
// is skipped (a load yields zeros) and bit 0 of the status word of its
// translation unit is set; nothing traps.  su3_bounds_status() reads and
// clears the words.
// ---------------------------------------------------------------------------
#ifdef SU3_BOUNDS_CHECK
static __device__ unsigned int g_su3_bounds_status = 0u;
#endif

__device__ __forceinline__ bool link_ok(int mu, int p, long long h, long long n) {
#ifdef SU3_BOUNDS_CHECK
  if ((unsigned)mu >= 4u || (unsigned)p >= 2u || (unsigned long long)h >= (unsigned long long)n) {
    atomicOr(&g_su3_bounds_status, 1u);
    return false;
  }
#endif
  return true;
}

// Host side: this translation unit's status word (0 and no error in a build
// without checks).
#ifdef SU3_BOUNDS_CHECK
#define SU3_BOUNDS_STATUS_FN(name)                                                             \
  cudaError_t name(unsigned int* v, bool clear) {                                               \
    cudaError_t e = cudaMemcpyFromSymbol(v, g_su3_bounds_status, sizeof(unsigned int));         \
    if (e == cudaSuccess && clear) {                                                            \
      const unsigned int z = 0u;                                                                \
      e = cudaMemcpyToSymbol(g_su3_bounds_status, &z, sizeof(unsigned int));                    \
    }                                                                                           \
    return e;                                                                                   \
  }
#else
#define SU3_BOUNDS_STATUS_FN(name) \
  cudaError_t name(unsigned int* v, bool) { \
    *v = 0u;                                \
    return cudaSuccess;                     \
  }
#endif

// ---------------------------------------------------------------------------
// Ordering between thread blocks of one persistent launch (the batched sweep
// and the persistent site-paired sweep): a block that finished a work item
// releases its count, a block that depends on it reads the count and
// acquires, under a time bound.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// Link loads and stores.
// ---------------------------------------------------------------------------
__device__ __forceinline__ size_t link_base(int mu, int p, int Vh, int ncomp) {
  return ((size_t)(mu * 2 + p) * ncomp) * (size_t)Vh;
}

// Site-paired FP32 store (su3_sitepair.cuh): the Vp pairs of one (mu, parity)
// come in tiles of kPairTile, the last one padded; a tile holds its six
// entries one after another, kPairTile float4 each.  Entry e of pair j sits
// at pair_offset(mu, p, j, Vp) + kPairTile e: the six entries of a link pair
// lie in one 3 KB block, and a warp's 32 consecutive pairs read 512
// contiguous bytes per entry.
constexpr int kPairTile = 32;
__host__ __device__ __forceinline__ long long pair_padded(long long Vp) {
  return (Vp + kPairTile - 1) / kPairTile * kPairTile;
}
__device__ __forceinline__ size_t pair_offset(int mu, int p, int j, int Vp) {
  return (size_t)(mu * 2 + p) * 6 * (size_t)pair_padded(Vp) + (size_t)(j / kPairTile) * (6 * kPairTile) +
         (size_t)(j % kPairTile);
}

template <bool CG>
__device__ __forceinline__ double2 ld_link(const double2* p) {
  return CG ? __ldcg(p) : __ldg(p);
}
template <bool CG>
__device__ __forceinline__ float4 ld_link(const float4* p) {
  return CG ? __ldcg(p) : __ldg(p);
}

template <bool CG = false>
__device__ __forceinline__ mat3<double> load_f64(const double2* __restrict__ U, int mu, int p, int h, int Vh) {
  mat3<double> m;
  if (!link_ok(mu, p, h, Vh)) {
#pragma unroll
    for (int c = 0; c < 9; ++c) m.e[c / 3][c % 3] = mk(0.0, 0.0);
    return m;
  }
  const double2* b = U + link_base(mu, p, Vh, kEntriesF64) + h;
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const double2 v = ld_link<CG>(b + (size_t)c * Vh);
    m.e[c / 3][c % 3] = mk(v.x, v.y);
  }
  return m;
}

__device__ __forceinline__ void store_f64(double2* U, int mu, int p, int h, int Vh, const mat3<double>& m) {
  if (!link_ok(mu, p, h, Vh)) return;
  double2* b = U + link_base(mu, p, Vh, kEntriesF64) + h;
#pragma unroll
  for (int c = 0; c < 9; ++c) b[(size_t)c * Vh] = make_double2(m.e[c / 3][c % 3].re, m.e[c / 3][c % 3].im);
}

// Rows 0 and 1 only; the caller completes row 2 when it needs it.
template <bool CG = false>
__device__ __forceinline__ mat3<float> load_f32_rows01(const float4* __restrict__ U, int mu, int p, int h, int Vh) {
  mat3<float> m;
  if (!link_ok(mu, p, h, Vh)) {
#pragma unroll
    for (int k = 0; k < 3; ++k) m.e[0][k] = m.e[1][k] = mk(0.f, 0.f);
    return m;
  }
  const float4* b = U + link_base(mu, p, Vh, kGroupsF32) + h;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 c = ld_link<CG>(b + (size_t)k * Vh);
    m.e[0][k] = mk(c.x, c.z);
    m.e[1][k] = mk(c.y, c.w);
  }
  return m;
}

template <bool CG = false>
__device__ __forceinline__ mat3<float> load_f32(const float4* __restrict__ U, int mu, int p, int h, int Vh) {
  mat3<float> m = load_f32_rows01<CG>(U, mu, p, h, Vh);
  complete_row2(m);
  return m;
}

// r = row 0 (re, im) x 3 columns, then row 1 (re, im) x 3 columns.
__device__ __forceinline__ void store_f32_rows01(float4* U, int mu, int p, int h, int Vh, const float r[12]) {
  if (!link_ok(mu, p, h, Vh)) return;
  float4* b = U + link_base(mu, p, Vh, kGroupsF32) + h;
#pragma unroll
  for (int k = 0; k < 3; ++k) b[(size_t)k * Vh] = make_float4(r[2 * k], r[6 + 2 * k], r[2 * k + 1], r[6 + 2 * k + 1]);
}

// ---------------------------------------------------------------------------
// Gram-Schmidt reunitarisation in FP64 of rows 0 and 1 (row 2 follows as
// conj(row0 x row1)).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void gram_schmidt_rows01(cx<double> r0[3], cx<double> r1[3]) {
  double n0 = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) n0 = fma(r0[k].re, r0[k].re, fma(r0[k].im, r0[k].im, n0));
  const double i0 = rsqrt(n0);
#pragma unroll
  for (int k = 0; k < 3; ++k) r0[k] = mk(r0[k].re * i0, r0[k].im * i0);
  cx<double> d = mk(0.0, 0.0);
#pragma unroll
  for (int k = 0; k < 3; ++k) d = mac_ca(d, r0[k], r1[k]);
#pragma unroll
  for (int k = 0; k < 3; ++k) r1[k] = mac(r1[k], mk(-d.re, -d.im), r0[k]);
  double n1 = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) n1 = fma(r1[k].re, r1[k].re, fma(r1[k].im, r1[k].im, n1));
  const double i1 = rsqrt(n1);
#pragma unroll
  for (int k = 0; k < 3; ++k) r1[k] = mk(r1[k].re * i1, r1[k].im * i1);
}

// ---------------------------------------------------------------------------
// Reunitarisation of an FP32 link (rows 0, 1) for FP32 storage.
//
// The Gram-Schmidt coefficients -- the norms n0 = |r0|^2, n1 = |r1|^2 and the
// overlap d = <r0, r1> -- are accumulated in FP64 from the exact products of
// the FP32 entries; these sums are where cancellation needs the precision.
// For a link that is unitary to within e = n - 1 = O(1e-6) (every link after
// a heatbath step), the exact Gram-Schmidt result is then applied in FP32 as
//   r0' = r0 (1 + s0),           s0 = 1/sqrt(1 + e0) - 1 = -e0/2 + 3 e0^2/8
//   r1' = (r1 - c r0)(1 + s1),   c = d / n0,  e1 = n1 - |d|^2/n0 - 1,
// each entry by one FMA, i.e. within one FP32 rounding of the FP64
// Gram-Schmidt followed by rounding to FP32 (the series remainder is below
// |e|^3 < 1e-9).  Links far from unitary (|e| or |d| >= 1e-3, e.g. arbitrary
// input from links_set) take the full FP64 Gram-Schmidt instead.
// ---------------------------------------------------------------------------
// Error-free transformations (Knuth TwoSum; TwoProd by FMA): a*b = p + e and
// a + b = s + e exactly in FP32.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// sum_k x_k y_k as hi + lo to about 2^-47 relative (compensated dot product).
__device__ __forceinline__ void dot2(const float* x, const float* y, int n, float& hi, float& lo) {
  hi = x[0] * y[0];
  lo = fmaf(x[0], y[0], -hi);
  for (int k = 1; k < n; ++k) {
    const float p = x[k] * y[k];
    const float pe = fmaf(x[k], y[k], -p);
    float s, se;
    two_sum(hi, p, s, se);
    hi = s;
    lo += pe + se;
  }
}

// The FP64 value of an FP32 number, built from its bits on the integer pipe
// (the FP64 pipe, 1/64 of the FP32 rate on this GPU, is kept for the sums):
// sign, exponent rebiased by 1023 - 127 = 896, the 23 mantissa bits moved to
// the top of the 52.  Exact for every finite x: a subnormal is first scaled
// by 2^64 in FP32 (exact) and the scale taken off the exponent; zero keeps
// its sign.
__device__ __forceinline__ double f32_to_f64_bits(float x) {
  const uint32_t ux = (uint32_t)__float_as_int(x);
  const bool sub = (ux & 0x7F800000u) == 0u;
  const uint32_t u = sub ? (uint32_t)__float_as_int(x * 0x1p64f) : ux;
  const uint32_t mag = u & 0x7FFFFFFFu;
  const uint32_t ebias = sub ? (896u - 64u) << 20 : 896u << 20;
  const uint32_t hi = (u & 0x80000000u) | (mag == 0u ? 0u : (mag >> 3) + ebias);
  const uint32_t lo = u << 29;
  return __hiloint2double((int)hi, (int)lo);
}

// EFT = false: the coefficients n0, n1, d are FP64 sums of the exact FP32
// products (FP64 pipe).  EFT = true: the same sums as compensated FP32 dot
// products (TwoProd by FMA, TwoSum), about 2^-47 relative -- FP64-class
// accuracy on the FP32 pipe, which GB300 runs 64x faster than FP64.
template <bool EFT>
__device__ __forceinline__ void reunitarise_f32(const cx<float> a[3], const cx<float> b[3], float out[12]) {
  float e0, dr, di, cr, ci, e1;
  if (EFT) {
    float ar[6], br[6], bx[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ar[2 * k] = a[k].re;
      ar[2 * k + 1] = a[k].im;
      br[2 * k] = b[k].re;
      br[2 * k + 1] = b[k].im;
      bx[2 * k] = b[k].im;  // Im <a, b> = sum a.re b.im - a.im b.re
      bx[2 * k + 1] = -b[k].re;
    }
    float h0, l0, h1, l1, hr, lr, hi_, li;
    dot2(ar, ar, 6, h0, l0);
    dot2(br, br, 6, h1, l1);
    dot2(ar, br, 6, hr, lr);
    dot2(ar, bx, 6, hi_, li);
    e0 = (h0 - 1.0f) + l0;  // h0 - 1 is exact (Sterbenz)
    dr = hr + lr;
    di = hi_ + li;
    const float inv_n0 = 1.0f - e0;  // 1/n0 to O(e0^2)
    cr = dr * inv_n0;
    ci = di * inv_n0;
    e1 = ((h1 - 1.0f) + l1) - __fmaf_rn(ci, di, __fmul_rn(cr, dr));
  } else {
    double n0 = 0.0, n1 = 0.0, dre = 0.0, dim = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double ar = f32_to_f64_bits(a[k].re), ai = f32_to_f64_bits(a[k].im);
      const double br = f32_to_f64_bits(b[k].re), bi = f32_to_f64_bits(b[k].im);
      n0 = fma(ar, ar, fma(ai, ai, n0));
      n1 = fma(br, br, fma(bi, bi, n1));
      dre = fma(ar, br, fma(ai, bi, dre));
      dim = fma(ar, bi, fma(-ai, br, dim));
    }
    e0 = (float)(n0 - 1.0);
    dr = (float)dre;
    di = (float)dim;
    const float inv_n0 = 1.0f - e0;  // 1/n0 to O(e0^2)
    cr = dr * inv_n0;
    ci = di * inv_n0;
    e1 = (float)(n1 - 1.0) - __fmaf_rn(ci, di, __fmul_rn(cr, dr));
  }
  if (fabsf(e0) < 1e-3f && fabsf(e1) < 1e-3f && fabsf(dr) < 1e-3f && fabsf(di) < 1e-3f) {
    const float s0 = e0 * fmaf(0.375f, e0, -0.5f);
    const float s1 = e1 * fmaf(0.375f, e1, -0.5f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      out[2 * k] = fmaf(a[k].re, s0, a[k].re);
      out[2 * k + 1] = fmaf(a[k].im, s0, a[k].im);
      // r1 - c r0
      const float tr = fmaf(-cr, a[k].re, fmaf(ci, a[k].im, b[k].re));
      const float ti = fmaf(-cr, a[k].im, fmaf(-ci, a[k].re, b[k].im));
      out[6 + 2 * k] = fmaf(tr, s1, tr);
      out[6 + 2 * k + 1] = fmaf(ti, s1, ti);
    }
  } else {
    cx<double> r0[3], r1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      r0[k] = mk((double)a[k].re, (double)a[k].im);
      r1[k] = mk((double)b[k].re, (double)b[k].im);
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
}

}  // namespace su3dev
