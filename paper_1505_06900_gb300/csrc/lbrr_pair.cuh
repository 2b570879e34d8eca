// Paired form of the recursive-regularized collision for the 16-bit stores:
// every value is a float2 holding the same quantity of two neighbouring cells,
// and every operation is one packed FP32x2 instruction (FFMA2 / FADD2 / FMUL2
// of sm_100-family GPUs), which halves the instructions the collision issues
// per cell. The arithmetic is that of lbrr_device.cuh in its weight-scaled
// (G) form: populations are g = (f - w) / w, the D1Q3 weights enter the
// separable moment passes as the integer ratios 1 : 4 : 1 and are divided out
// of the synthesis T/w = (c0 - 3/2 c2, c0 +- 3 c1 + 3 c2).
//
// Coefficient tensor (Sec. 3.5 with eq_rel_a1 in closed form): the
// coefficient of x^a y^b z^c of f0 + om1 f1 is rho ux^a uy^b uz^c plus om1
// times the pair sum of a1^(2) over the index pairs of x^a y^b z^c; it is
// written out below per (b, c) with the products by 0 and 1 removed, since
// packed instructions are not folded by the compiler. The conserved
// coefficients (rho - 1, rho u) are the moments themselves.
#pragma once

#include <cuda_runtime.h>

#include "lbrr_device.cuh"

namespace lbrr {

// FP16 / BF16 values of the 16-bit stores, singly and as packed pairs.
template <int S>
struct Half;
template <>
struct Half<1> {
  using T2 = __half2;
  __device__ __forceinline__ static float to_f(__half v) { return __half2float(v); }
  __device__ __forceinline__ static __half from_f(float v) { return __float2half_rn(v); }
  __device__ __forceinline__ static float2 to_f2(__half2 v) { return __half22float2(v); }
  __device__ __forceinline__ static __half2 from_f2(float2 v) { return __float22half2_rn(v); }
};
template <>
struct Half<2> {
  using T2 = __nv_bfloat162;
  __device__ __forceinline__ static float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ __forceinline__ static __nv_bfloat16 from_f(float v) {
    return __float2bfloat16_rn(v);
  }
  __device__ __forceinline__ static float2 to_f2(__nv_bfloat162 v) {
    return __bfloat1622float2(v);
  }
  __device__ __forceinline__ static __nv_bfloat162 from_f2(float2 v) {
    return __float22bfloat162_rn(v);
  }
};

namespace pair {

using V = float2;

__device__ __forceinline__ V bc(float s) { return make_float2(s, s); }
__device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
// a - b exactly rounded once (b * -1 is exact)
__device__ __forceinline__ V sub(V a, V b) { return __ffma2_rn(b, bc(-1.0f), a); }
__device__ __forceinline__ V scale(float s, V a) { return __fmul2_rn(bc(s), a); }
__device__ __forceinline__ V fmas(float s, V b, V c) { return __ffma2_rn(bc(s), b, c); }

// Macroscopic values of two cells; P = om1 * Pi1 (the only form the
// regularized reconstructions use).
struct Macro2 {
  V drho, rho, jx, jy, jz, ux, uy, uz;
  V pxx, pxy, pxz, pyy, pyz, pzz;
};

// one 1 : 4 : 1 weighted moment pass over a line of three values
__device__ __forceinline__ void mom3(V a, V b, V c, V &s0, V &s1, V &s2) {
  s2 = add(a, c);
  s0 = fmas(4.0f, b, s2);
  s1 = sub(c, a);
}

// x / KDEN for the conserved moments: x k_hi + x k_lo, with k_hi the float32
// rounding of 1 / KDEN and k_lo that of the remainder. The product with k_hi
// alone would scale rho - 1 and rho u by k_hi KDEN = 1 + 7.5e-9 (KDEN = 36,
// 216) at every update, a drift of mass and momentum that adds up over long
// runs; the two-term form leaves one rounding and no systematic factor.
template <int KDEN>
__device__ __forceinline__ V div_k(V x) {
  constexpr float hi = 1.0f / KDEN;
  constexpr float lo = (float)(1.0 / KDEN - (double)hi);
  return fma(x, bc(lo), scale(hi, x));
}

// rho, rho u, u and om1 * Pi1 from the raw weighted moments (KDEN times the
// moments: 36 for D2Q9 and D3Q19, 216 for D3Q27) of g.
template <int KDEN>
__device__ __forceinline__ Macro2 macro(float om1, V m0r, V jxr, V jyr, V jzr, V pxxr, V pyyr,
                                        V pzzr, V pxyr, V pxzr, V pyzr, bool three_d) {
  constexpr float k = 1.0f / KDEN;
  Macro2 m;
  m.drho = div_k<KDEN>(m0r);
  m.jx = div_k<KDEN>(jxr);
  m.jy = div_k<KDEN>(jyr);
  m.rho = add(bc(1.0f), m.drho);
  // u = j / rho correctly rounded, lane by lane (as the scalar form does)
  m.ux = make_float2(m.jx.x / m.rho.x, m.jx.y / m.rho.y);
  m.uy = make_float2(m.jy.x / m.rho.x, m.jy.y / m.rho.y);
  // om1 Pi_ab = om1 k m_ab - om1 (j_a u_b + cs2 (rho - 1) delta_ab)
  const float ok = om1 * k, no = -om1;
  const V c0 = scale(kCs2, m.drho);
  m.pxx = fmas(ok, pxxr, scale(no, fma(m.jx, m.ux, c0)));
  m.pyy = fmas(ok, pyyr, scale(no, fma(m.jy, m.uy, c0)));
  m.pxy = fmas(ok, pxyr, scale(no, mul(m.jx, m.uy)));
  if (three_d) {
    m.jz = div_k<KDEN>(jzr);
    m.uz = make_float2(m.jz.x / m.rho.x, m.jz.y / m.rho.y);
    m.pzz = fmas(ok, pzzr, scale(no, fma(m.jz, m.uz, c0)));
    m.pxz = fmas(ok, pxzr, scale(no, mul(m.jx, m.uz)));
    m.pyz = fmas(ok, pyzr, scale(no, mul(m.jy, m.uz)));
  } else {
    m.jz = m.uz = m.pzz = m.pxz = m.pyz = bc(0.0f);
  }
  return m;
}

// ------------------------------------------------------------------ D2Q9 --
__device__ __forceinline__ Macro2 moments9(const V (&f)[9], float om1) {
  V s0[3], s1[3], s2[3];
#pragma unroll
  for (int l = 0; l < 3; ++l) mom3(f[3 * l], f[3 * l + 1], f[3 * l + 2], s0[l], s1[l], s2[l]);
  V m00, m01, m02, m10, m11, m12, m20, m21, m22;
  mom3(s0[0], s0[1], s0[2], m00, m01, m02);
  mom3(s1[0], s1[1], s1[2], m10, m11, m12);
  mom3(s2[0], s2[1], s2[2], m20, m21, m22);
  const V z = bc(0.0f);
  return macro<36>(om1, m00, m10, m01, z, m20, m02, z, m11, z, z, false);
}

// one-dimensional synthesis with the weight divided out
__device__ __forceinline__ void synth1(V c0, V c1, V c2, V &om, V &oz, V &op) {
  oz = fmas(-1.5f, c2, c0);
  const V p = fmas(3.0f, c2, c0);
  op = fmas(3.0f, c1, p);
  om = fmas(-3.0f, c1, p);
}

__device__ __forceinline__ void synth9(const V (&c)[3][3], V (&f)[9]) {
  V s[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b) synth1(c[0][b], c[1][b], c[2][b], s[0][b], s[1][b], s[2][b]);
#pragma unroll
  for (int ix = 0; ix < 3; ++ix) synth1(s[ix][0], s[ix][1], s[ix][2], f[ix], f[ix + 3], f[ix + 6]);
}

// RR coefficients of x^a y^b (P = om1 Pi): with q1 = (rho, rho uy,
// rho uy^2 + Pyy), q2 = Pxx (1, uy, uy^2), q3 = Pxy (0, 1, 2 uy):
// c0 = q1, c1 = ux q1 + q3, c2 = ux^2 q1 + 2 ux q3 + q2.
__device__ __forceinline__ void coeffs9(const Macro2 &m, V (&c)[3][3]) {
  const V uy2 = add(m.uy, m.uy), uxx = mul(m.ux, m.ux), ux2 = add(m.ux, m.ux);
  const V q1_1 = mul(m.rho, m.uy);
  const V q1_2 = fma(q1_1, m.uy, m.pyy);
  const V q2_1 = mul(m.pxx, m.uy), q2_2 = mul(q2_1, m.uy);
  const V q3_2 = mul(m.pxy, uy2);
  c[0][0] = m.drho;
  c[0][1] = m.jy;
  c[0][2] = q1_2;
  c[1][0] = m.jx;
  c[1][1] = fma(m.ux, q1_1, m.pxy);
  c[1][2] = fma(m.ux, q1_2, q3_2);
  c[2][0] = fma(uxx, m.rho, m.pxx);
  c[2][1] = fma(uxx, q1_1, fma(ux2, m.pxy, q2_1));
  c[2][2] = fma(uxx, q1_2, fma(ux2, q3_2, q2_2));
}

// equilibrium coefficients rho ux^a uy^b (om1 = 0)
__device__ __forceinline__ void coeffs9_eq(const Macro2 &m, V (&c)[3][3]) {
  const V q1_1 = mul(m.rho, m.uy), q1_2 = mul(q1_1, m.uy);
  const V uxx = mul(m.ux, m.ux);
  c[0][0] = m.drho;
  c[0][1] = m.jy;
  c[0][2] = q1_2;
  c[1][0] = m.jx;
  c[1][1] = mul(m.ux, q1_1);
  c[1][2] = mul(m.ux, q1_2);
  c[2][0] = mul(uxx, m.rho);
  c[2][1] = mul(uxx, q1_1);
  c[2][2] = mul(uxx, q1_2);
}

// ----------------------------------------------------------------- D3Q27 --
__device__ __forceinline__ Macro2 moments27(const V (&f)[27], float om1) {
  V x0[9], x1[9], x2[9];
#pragma unroll
  for (int l = 0; l < 9; ++l) mom3(f[3 * l], f[3 * l + 1], f[3 * l + 2], x0[l], x1[l], x2[l]);
  V y00[3], y01[3], y02[3], y10[3], y11[3], y20[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int l = 3 * k;
    V t0, t1, t2;
    mom3(x0[l], x0[l + 1], x0[l + 2], y00[k], y01[k], y02[k]);
    mom3(x1[l], x1[l + 1], x1[l + 2], y10[k], y11[k], t2);
    mom3(x2[l], x2[l + 1], x2[l + 2], y20[k], t1, t0);
  }
  V m000, m001, m002, m010, m011, m020, m100, m101, m110, m200, t[8];
  mom3(y00[0], y00[1], y00[2], m000, m001, m002);
  mom3(y01[0], y01[1], y01[2], m010, m011, t[0]);
  mom3(y02[0], y02[1], y02[2], m020, t[1], t[2]);
  mom3(y10[0], y10[1], y10[2], m100, m101, t[3]);
  mom3(y11[0], y11[1], y11[2], m110, t[4], t[5]);
  mom3(y20[0], y20[1], y20[2], m200, t[6], t[7]);
  return macro<216>(om1, m000, m100, m010, m001, m200, m020, m002, m110, m101, m011, true);
}

__device__ __forceinline__ void synth27(const V (&c)[3][3][3], V (&f)[27]) {
  V sx[3][3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
      synth1(c[0][b][cc], c[1][b][cc], c[2][b][cc], sx[0][b][cc], sx[1][b][cc], sx[2][b][cc]);
#pragma unroll
  for (int ix = 0; ix < 3; ++ix) {
    V sy[3][3];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
      synth1(sx[ix][0][cc], sx[ix][1][cc], sx[ix][2][cc], sy[0][cc], sy[1][cc], sy[2][cc]);
#pragma unroll
    for (int iy = 0; iy < 3; ++iy)
      synth1(sy[iy][0], sy[iy][1], sy[iy][2], f[ix + 3 * iy], f[ix + 3 * iy + 9],
             f[ix + 3 * iy + 18]);
  }
}

// RR coefficients of x^a y^b z^c. The (y, z) matrices
//   Q1 = rho py pz + Pyy h_y pz + Pzz py h_z + Pyz dy dz,
//   Q2 = Pxx py pz,   Q3 = Pxy dy pz + Pxz py dz
// (py = (1, uy, uy^2), h = (0, 0, 1), dy = (0, 1, 2 uy), likewise in z) give
// c0 = Q1, c1 = ux Q1 + Q3, c2 = ux^2 Q1 + 2 ux Q3 + Q2.
__device__ __forceinline__ void coeffs27(const Macro2 &m, V (&c)[3][3][3]) {
  const V uy = m.uy, uz = m.uz;
  const V uyy = mul(uy, uy), uzz = mul(uz, uz), uyz = mul(uy, uz);
  const V uy2 = add(uy, uy), uz2 = add(uz, uz);
  // py[b] pz[c]
  V pp[3][3];
  pp[0][0] = bc(1.0f);
  pp[1][0] = uy;
  pp[2][0] = uyy;
  pp[0][1] = uz;
  pp[0][2] = uzz;
  pp[1][1] = uyz;
  pp[1][2] = mul(uy, uzz);
  pp[2][1] = mul(uyy, uz);
  pp[2][2] = mul(uyy, uzz);
  V q1[3][3], q2[3][3], q3[3][3];
  // rho py pz
  q1[0][0] = m.rho;
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
      if (b + cc > 0) q1[b][cc] = mul(m.rho, pp[b][cc]);
  // + Pyy pz[c] (b = 2), + Pzz py[b] (c = 2)
  q1[2][0] = add(q1[2][0], m.pyy);
  q1[2][1] = fma(m.pyy, uz, q1[2][1]);
  q1[2][2] = fma(m.pyy, uzz, q1[2][2]);
  q1[0][2] = add(q1[0][2], m.pzz);
  q1[1][2] = fma(m.pzz, uy, q1[1][2]);
  q1[2][2] = fma(m.pzz, uyy, q1[2][2]);
  // + Pyz dy dz (b, c > 0): dy dz = 1, 2uz, 2uy, 4 uy uz
  q1[1][1] = add(q1[1][1], m.pyz);
  const V pyz2 = add(m.pyz, m.pyz);
  q1[1][2] = fma(pyz2, uz, q1[1][2]);
  q1[2][1] = fma(pyz2, uy, q1[2][1]);
  q1[2][2] = fma(add(pyz2, pyz2), uyz, q1[2][2]);
  // Q2 = Pxx py pz
  q2[0][0] = m.pxx;
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
      if (b + cc > 0) q2[b][cc] = mul(m.pxx, pp[b][cc]);
  // Q3 = Pxy dy pz + Pxz py dz; dy pz: (1,c) = pz[c], (2,c) = 2 uy pz[c];
  // py dz: (b,1) = py[b], (b,2) = 2 uz py[b]
  q3[0][0] = bc(0.0f);
  const V pxy2 = mul(m.pxy, uy2), pxz2 = mul(m.pxz, uz2);
  q3[1][0] = m.pxy;
  q3[2][0] = pxy2;
  q3[0][1] = m.pxz;
  q3[0][2] = pxz2;
  q3[1][1] = fma(m.pxy, uz, mul(m.pxz, uy));
  q3[1][2] = fma(m.pxy, uzz, mul(pxz2, uy));
  q3[2][1] = fma(pxy2, uz, mul(m.pxz, uyy));
  q3[2][2] = fma(pxy2, uzz, mul(pxz2, uyy));
  const V uxx = mul(m.ux, m.ux), ux2 = add(m.ux, m.ux);
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      c[0][b][cc] = q1[b][cc];
      c[1][b][cc] = (b + cc == 0) ? mul(m.ux, q1[b][cc]) : fma(m.ux, q1[b][cc], q3[b][cc]);
      c[2][b][cc] = (b + cc == 0) ? fma(uxx, q1[b][cc], q2[b][cc])
                                  : fma(uxx, q1[b][cc], fma(ux2, q3[b][cc], q2[b][cc]));
    }
  c[0][0][0] = m.drho;
  c[1][0][0] = m.jx;
  c[0][1][0] = m.jy;
  c[0][0][1] = m.jz;
}

// equilibrium coefficients rho ux^a uy^b uz^c
__device__ __forceinline__ void coeffs27_eq(const Macro2 &m, V (&c)[3][3][3]) {
  const V uy = m.uy, uz = m.uz;
  const V q1_10 = mul(m.rho, uy), q1_20 = mul(q1_10, uy);
  const V q1_01 = mul(m.rho, uz), q1_02 = mul(q1_01, uz);
  V q1[3][3];
  q1[0][0] = m.rho;
  q1[1][0] = q1_10;
  q1[2][0] = q1_20;
  q1[0][1] = q1_01;
  q1[0][2] = q1_02;
  q1[1][1] = mul(q1_10, uz);
  q1[1][2] = mul(q1_10, mul(uz, uz));
  q1[2][1] = mul(q1_20, uz);
  q1[2][2] = mul(q1_20, mul(uz, uz));
  const V uxx = mul(m.ux, m.ux);
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      c[0][b][cc] = q1[b][cc];
      c[1][b][cc] = mul(m.ux, q1[b][cc]);
      c[2][b][cc] = mul(uxx, q1[b][cc]);
    }
  c[0][0][0] = m.drho;
  c[1][0][0] = m.jx;
  c[0][1][0] = m.jy;
  c[0][0][1] = m.jz;
}

// Order-2 regularized coefficients (Sec. 3.8.1): total order <= 2 only.
__device__ __forceinline__ void coeffs_reg2_9(const Macro2 &m, V (&c)[3][3]) {
  const V z = bc(0.0f);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) c[a][b] = z;
  c[0][0] = m.drho;
  c[1][0] = m.jx;
  c[0][1] = m.jy;
  c[2][0] = fma(m.jx, m.ux, m.pxx);
  c[0][2] = fma(m.jy, m.uy, m.pyy);
  c[1][1] = fma(m.jx, m.uy, m.pxy);
}
__device__ __forceinline__ void coeffs_reg2_27(const Macro2 &m, V (&c)[3][3][3]) {
  const V z = bc(0.0f);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) c[a][b][cc] = z;
  c[0][0][0] = m.drho;
  c[1][0][0] = m.jx;
  c[0][1][0] = m.jy;
  c[0][0][1] = m.jz;
  c[2][0][0] = fma(m.jx, m.ux, m.pxx);
  c[0][2][0] = fma(m.jy, m.uy, m.pyy);
  c[0][0][2] = fma(m.jz, m.uz, m.pzz);
  c[1][1][0] = fma(m.jx, m.uy, m.pxy);
  c[1][0][1] = fma(m.jx, m.uz, m.pxz);
  c[0][1][1] = fma(m.jy, m.uz, m.pyz);
}

// ----------------------------------------------------------------- D3Q19 --
// Direction order of q19_to_q27: planes z = -1 (0..4) and z = +1 (14..18)
// hold the crosses (0,-1), (-1,0), (0,0), (1,0), (0,1) (edges and one
// face), plane z = 0 (5..13) the full 3x3 set. With g = df / w the weights
// 1/3 : 1/18 : 1/36 enter the sums as 12 : 2 : 1, so the moments come out
// multiplied by 36.
__device__ __forceinline__ Macro2 moments19(const V (&f)[19], float om1) {
  const V mxx = add(f[1], f[3]), myy = add(f[0], f[4]);
  const V m0 = fmas(2.0f, f[2], add(mxx, myy));
  const V mx = sub(f[3], f[1]), my = sub(f[4], f[0]);
  const V pxx = add(f[15], f[17]), pyy = add(f[14], f[18]);
  const V p0 = fmas(2.0f, f[16], add(pxx, pyy));
  const V px = sub(f[17], f[15]), py = sub(f[18], f[14]);
  // plane z = 0: edges 5, 7, 11, 13; faces 8, 10 (x) and 6, 12 (y); rest 9
  const V e57 = add(f[5], f[7]), e1113 = add(f[11], f[13]);
  const V ee = add(e57, e1113);
  const V fxx = add(f[8], f[10]), fyy = add(f[6], f[12]);
  const V cxx = fmas(2.0f, fxx, ee), cyy = fmas(2.0f, fyy, ee);
  const V c00 = fmas(12.0f, f[9], fmas(2.0f, fyy, cxx));
  const V cx = fmas(2.0f, sub(f[10], f[8]), sub(add(f[7], f[13]), add(f[5], f[11])));
  const V cy = fmas(2.0f, sub(f[12], f[6]), sub(e1113, e57));
  const V cxy = sub(add(f[5], f[13]), add(f[7], f[11]));
  return macro<36>(om1, add(c00, add(m0, p0)), add(cx, add(mx, px)), add(cy, add(my, py)),
                   sub(p0, m0), add(cxx, add(mxx, pxx)), add(cyy, add(myy, pyy)), add(p0, m0),
                   cxy, sub(px, mx), sub(py, my), true);
}

// Post-collision g of a D3Q19 pair on the kept basis (orders 0-2 and the
// sums / differences H_aab +- H_bcc of order 3), as synth_d3q19 of
// lbrr_device.cuh with the weights divided out: A_ab = j_a u_b + P_ab,
// A_abb = u_a A_bb + 2 u_b P_ab (P = om1 Pi), and per class of velocity
//   rest  base = drho - 3/2 tr A
//   face  base + 9/2 A_aa + s (3 j_a - 9 (A_abb + A_acc))
//   edge  base + 9/2 (A_aa + A_bb) + 9 s t A_ab + s (3 j_a + 9 A_abb)
//              + t (3 j_b + 9 A_aab).
// ORDER3 = false: the order-2 regularized comparator. EQ: P = 0 (the
// equilibrium), whose products by zero are left out.
template <bool ORDER3, bool EQ>
__device__ __forceinline__ void synth19(const Macro2 &m, V (&f)[19]) {
  const V ux = m.ux, uy = m.uy, uz = m.uz;
  V axx, ayy, azz, axy, axz, ayz;
  if (EQ) {
    axx = mul(m.jx, ux);
    ayy = mul(m.jy, uy);
    azz = mul(m.jz, uz);
    axy = mul(m.jx, uy);
    axz = mul(m.jx, uz);
    ayz = mul(m.jy, uz);
  } else {
    axx = fma(m.jx, ux, m.pxx);
    ayy = fma(m.jy, uy, m.pyy);
    azz = fma(m.jz, uz, m.pzz);
    axy = fma(m.jx, uy, m.pxy);
    axz = fma(m.jx, uz, m.pxz);
    ayz = fma(m.jy, uz, m.pyz);
  }
  const V jx3 = scale(3.0f, m.jx), jy3 = scale(3.0f, m.jy), jz3 = scale(3.0f, m.jz);
  V ux_ = jx3, uy_ = jy3, uz_ = jz3;              // 3 j_a - 9 (A_abb + A_acc) (faces)
  V exy_x = jx3, exy_y = jy3, exz_x = jx3, exz_z = jz3, eyz_y = jy3, eyz_z = jz3;
  if (ORDER3) {
    V axyy, axzz, axxy, ayzz, axxz, ayyz;
    if (EQ) {
      axyy = mul(ux, ayy);
      axzz = mul(ux, azz);
      axxy = mul(uy, axx);
      ayzz = mul(uy, azz);
      axxz = mul(uz, axx);
      ayyz = mul(uz, ayy);
    } else {
      const V ux2 = add(ux, ux), uy2 = add(uy, uy), uz2 = add(uz, uz);
      axyy = fma(ux, ayy, mul(uy2, m.pxy));
      axzz = fma(ux, azz, mul(uz2, m.pxz));
      axxy = fma(uy, axx, mul(ux2, m.pxy));
      ayzz = fma(uy, azz, mul(uz2, m.pyz));
      axxz = fma(uz, axx, mul(ux2, m.pxz));
      ayyz = fma(uz, ayy, mul(uy2, m.pyz));
    }
    ux_ = fmas(-9.0f, add(axyy, axzz), jx3);
    uy_ = fmas(-9.0f, add(axxy, ayzz), jy3);
    uz_ = fmas(-9.0f, add(axxz, ayyz), jz3);
    exy_x = fmas(9.0f, axyy, jx3);
    exy_y = fmas(9.0f, axxy, jy3);
    exz_x = fmas(9.0f, axzz, jx3);
    exz_z = fmas(9.0f, axxz, jz3);
    eyz_y = fmas(9.0f, ayzz, jy3);
    eyz_z = fmas(9.0f, ayyz, jz3);
  }
  const V base = fmas(-1.5f, add(add(axx, ayy), azz), m.drho);
  f[9] = base;
  const V fx = fmas(4.5f, axx, base), fy = fmas(4.5f, ayy, base), fz = fmas(4.5f, azz, base);
  f[10] = add(fx, ux_);
  f[8] = sub(fx, ux_);
  f[12] = add(fy, uy_);
  f[6] = sub(fy, uy_);
  f[16] = add(fz, uz_);
  f[2] = sub(fz, uz_);
  // edges of the plane (a, b): (+,+), (+,-), (-,+), (-,-)
  auto edges = [](V e, V ab, V U, V W, V &pp, V &pm, V &mp, V &mm) {
    const V ep = fmas(9.0f, ab, e), em = fmas(-9.0f, ab, e);
    const V s = add(U, W), d = sub(U, W);
    pp = add(ep, s);
    mm = sub(ep, s);
    pm = add(em, d);
    mp = sub(em, d);
  };
  edges(fmas(4.5f, add(axx, ayy), base), axy, exy_x, exy_y, f[13], f[7], f[11], f[5]);
  edges(fmas(4.5f, add(axx, azz), base), axz, exz_x, exz_z, f[17], f[3], f[15], f[1]);
  edges(fmas(4.5f, add(ayy, azz), base), ayz, eyz_y, eyz_z, f[18], f[4], f[14], f[0]);
}

// Post-collision g of two cells in place. MODEL 0: RR, 1: order-2
// regularized, 2: BGK g + (1 - om1)(g_eq - g).
template <int Q, int MODEL>
__device__ __forceinline__ void collide(V (&f)[Q], float om1);

template <>
__device__ __forceinline__ void collide<9, 0>(V (&f)[9], float om1) {
  V c[3][3];
  coeffs9(moments9(f, om1), c);
  synth9(c, f);
}
template <>
__device__ __forceinline__ void collide<9, 1>(V (&f)[9], float om1) {
  V c[3][3];
  coeffs_reg2_9(moments9(f, om1), c);
  synth9(c, f);
}
template <>
__device__ __forceinline__ void collide<9, 2>(V (&f)[9], float om1) {
  V c[3][3], eq[9];
  coeffs9_eq(moments9(f, 0.0f), c);
  synth9(c, eq);
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i] = fmas(1.0f - om1, sub(eq[i], f[i]), f[i]);
}
template <>
__device__ __forceinline__ void collide<27, 0>(V (&f)[27], float om1) {
  V c[3][3][3];
  coeffs27(moments27(f, om1), c);
  synth27(c, f);
}
template <>
__device__ __forceinline__ void collide<27, 1>(V (&f)[27], float om1) {
  V c[3][3][3];
  coeffs_reg2_27(moments27(f, om1), c);
  synth27(c, f);
}
template <>
__device__ __forceinline__ void collide<27, 2>(V (&f)[27], float om1) {
  V c[3][3][3], eq[27];
  coeffs27_eq(moments27(f, 0.0f), c);
  synth27(c, eq);
#pragma unroll
  for (int i = 0; i < 27; ++i) f[i] = fmas(1.0f - om1, sub(eq[i], f[i]), f[i]);
}

template <>
__device__ __forceinline__ void collide<19, 0>(V (&f)[19], float om1) {
  synth19<true, false>(moments19(f, om1), f);
}
template <>
__device__ __forceinline__ void collide<19, 1>(V (&f)[19], float om1) {
  synth19<false, false>(moments19(f, om1), f);
}
template <>
__device__ __forceinline__ void collide<19, 2>(V (&f)[19], float om1) {
  V eq[19];
  synth19<true, true>(moments19(f, 0.0f), eq);
#pragma unroll
  for (int i = 0; i < 19; ++i) f[i] = fmas(1.0f - om1, sub(eq[i], f[i]), f[i]);
}

}  // namespace pair
}  // namespace lbrr
