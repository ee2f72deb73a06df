// su3_pair.cuh -- FP32 SU(3) algebra on row pairs with fma.rn.f32x2.
//
// An FP32-mixed link is stored column by column as (re u0k, re u1k, im u0k,
// im u1k): a single 16-byte load yields, for column k, the pair of real parts
// and the pair of imaginary parts of rows 0 and 1.  Products X*Y whose left
// factor is held as such row pairs are computed two rows at a time by the
// paired FMA (one instruction, two independent round-to-nearest FMAs), with
// the entries of the right factor broadcast; this halves the instructions of
// the staple's matrix products.  Row 2 is kept as scalars.
#pragma once

#include "su3_device.cuh"

namespace su3dev {

struct pm3 {
  float2 re[3], im[3];     // column k: (row 0, row 1) real parts, imaginary parts
  float r2re[3], r2im[3];  // row 2
};

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Entry (i, k) as a scalar complex number (i, k compile-time after unrolling).
__device__ __forceinline__ float pre(const pm3& m, int i, int k) { return i == 0 ? m.re[k].x : (i == 1 ? m.re[k].y : m.r2re[k]); }
__device__ __forceinline__ float pim(const pm3& m, int i, int k) { return i == 0 ? m.im[k].x : (i == 1 ? m.im[k].y : m.r2im[k]); }
__device__ __forceinline__ cx<float> pget(const pm3& m, int i, int k) { return mk(pre(m, i, k), pim(m, i, k)); }
__device__ __forceinline__ void pset(pm3& m, int i, int k, cx<float> v) {
  if (i == 0) {
    m.re[k].x = v.re;
    m.im[k].x = v.im;
  } else if (i == 1) {
    m.re[k].y = v.re;
    m.im[k].y = v.im;
  } else {
    m.r2re[k] = v.re;
    m.r2im[k] = v.im;
  }
}

template <bool CG>
__device__ __forceinline__ pm3 load_pm3(const float4* __restrict__ U, int mu, int p, int h, int Vh) {
  pm3 m;
  if (!link_ok(mu, p, h, Vh)) {
#pragma unroll
    for (int k = 0; k < 3; ++k) m.re[k] = m.im[k] = make_float2(0.f, 0.f);
    return m;
  }
  const float4* b = U + link_base(mu, p, Vh, kGroupsF32) + h;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 c = ld_link<CG>(b + (size_t)k * Vh);
    m.re[k] = make_float2(c.x, c.y);
    m.im[k] = make_float2(c.z, c.w);
  }
  return m;
}

// Row 2 = conj(row0 x row1).
__device__ __forceinline__ void complete_row2_p(pm3& m) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int a = (k + 1) % 3, b = (k + 2) % 3;
    cx<float> v = mul(pget(m, 0, a), pget(m, 1, b));
    v = mac(v, mk(-pre(m, 0, b), -pim(m, 0, b)), pget(m, 1, a));
    m.r2re[k] = v.re;
    m.r2im[k] = -v.im;
  }
}

// Rows 0,1 of X * Y^+ (Y complete): Z_ik = sum_j X_ij conj(Y_kj).
__device__ __forceinline__ void mul_nd_p(const pm3& X, const pm3& Y, pm3& Z) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float2 zr = make_float2(0.f, 0.f), zi = zr;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float yr = pre(Y, k, j), yi = pim(Y, k, j);
      zr = fma2(X.re[j], bc2(yr), zr);
      zr = fma2(X.im[j], bc2(yi), zr);
      zi = fma2(X.im[j], bc2(yr), zi);
      zi = fma2(X.re[j], bc2(-yi), zi);
    }
    Z.re[k] = zr;
    Z.im[k] = zi;
  }
}

// Rows 0,1 of X * Y (Y complete): Z_ik = sum_j X_ij Y_jk.
__device__ __forceinline__ void mul_nn_p(const pm3& X, const pm3& Y, pm3& Z) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float2 zr = make_float2(0.f, 0.f), zi = zr;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float yr = pre(Y, j, k), yi = pim(Y, j, k);
      zr = fma2(X.re[j], bc2(yr), zr);
      zr = fma2(X.im[j], bc2(-yi), zr);
      zi = fma2(X.re[j], bc2(yi), zi);
      zi = fma2(X.im[j], bc2(yr), zi);
    }
    Z.re[k] = zr;
    Z.im[k] = zi;
  }
}

// Rows 0,1 of H^+ * F (H, F complete): Z_ik = sum_j conj(H_ji) F_jk.  The
// left factor is paired by columns (H_j0, H_j1) of each row j.
__device__ __forceinline__ void mul_dn_p(const pm3& H, const pm3& F, pm3& Z) {
  float2 hr[3], hi[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    hr[j] = make_float2(pre(H, j, 0), pre(H, j, 1));
    hi[j] = make_float2(pim(H, j, 0), pim(H, j, 1));
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float2 zr = make_float2(0.f, 0.f), zi = zr;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float fr = pre(F, j, k), fi = pim(F, j, k);
      zr = fma2(hr[j], bc2(fr), zr);
      zr = fma2(hi[j], bc2(fi), zr);
      zi = fma2(hr[j], bc2(fi), zi);
      zi = fma2(hi[j], bc2(-fr), zi);
    }
    Z.re[k] = zr;
    Z.im[k] = zi;
  }
}

// A += B for an SU(3) matrix B of which only rows 0,1 are set: row 2 of B,
// conj(row0 x row1), is formed inside the accumulation of A's row 2.
__device__ __forceinline__ void acc_completed_p(pm3& A, const pm3& B) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    A.re[k] = add2(A.re[k], B.re[k]);
    A.im[k] = add2(A.im[k], B.im[k]);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int a = (k + 1) % 3, b = (k + 2) % 3;
    // A_2k + conj(v) = conj(conj(A_2k) + v), v = B_0a B_1b - B_0b B_1a
    cx<float> v = mac(mk(A.r2re[k], -A.r2im[k]), pget(B, 0, a), pget(B, 1, b));
    v = mac(v, mk(-pre(B, 0, b), -pim(B, 0, b)), pget(B, 1, a));
    A.r2re[k] = v.re;
    A.r2im[k] = -v.im;
  }
}

__device__ __forceinline__ pm3 zero_p() {
  pm3 m;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    m.re[k] = make_float2(0.f, 0.f);
    m.im[k] = make_float2(0.f, 0.f);
    m.r2re[k] = 0.f;
    m.r2im[k] = 0.f;
  }
  return m;
}

// rows (0, 1) <- R rows (0, 1) for R = [[R00, R01], [R10, R11]]: per column
// (u0c', u1c') = (R00, R10) u0c + (R01, R11) u1c, the two rows in one pair.
__device__ __forceinline__ void rotate01_p(pm3& u, cx<float> R00, cx<float> R01, cx<float> R10, cx<float> R11) {
  const float2 ar = make_float2(R00.re, R10.re), ai = make_float2(R00.im, R10.im);
  const float2 br = make_float2(R01.re, R11.re), bi = make_float2(R01.im, R11.im);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float x0r = u.re[c].x, x0i = u.im[c].x, x1r = u.re[c].y, x1i = u.im[c].y;
    float2 nr = mul2(ar, bc2(x0r));
    nr = fma2(ai, bc2(-x0i), nr);
    nr = fma2(br, bc2(x1r), nr);
    nr = fma2(bi, bc2(-x1i), nr);
    float2 ni = mul2(ar, bc2(x0i));
    ni = fma2(ai, bc2(x0r), ni);
    ni = fma2(br, bc2(x1i), ni);
    ni = fma2(bi, bc2(x1r), ni);
    u.re[c] = nr;
    u.im[c] = ni;
  }
}

}  // namespace su3dev
