// Device-side building blocks of the recursive-regularized (RR) BGK step
// (arXiv:1505.06900): storage conversion, moments, and the reconstruction
// f_post = f0 + (1 - 1/tau) f1 of Sec. 3.5 on the D2Q9 / D3Q27 Hermite bases.
//
// The kernel does not evaluate the paper's Hermite sums term by term. Both
// lattices are tensor products of the D1Q3 rule, so their Hermite bases are
// tensor products of the 1-D set {1, xi, xi^2 - c_s^2}. On that basis:
//  * the equilibrium coefficient of x^a y^b z^c (a, b, c in {0, 1, 2}) is
//    rho ux^a uy^b uz^c (Sec. 2, a0^(n) = a0^(n-1) u of Sec. 3.1);
//  * the off-equilibrium coefficients given by the recursion eq_rel_a1
//    (Appendix B, starred terms dropped) equal, in closed form, the sum over
//    index pairs of a1^(2) times the velocity components of the other indices,
//    i.e. C1 = 1/2 sum_ab Pi_ab d^2/du_a du_b (ux^a uy^b uz^c);
//  * the population of velocity (xi_x, xi_y, xi_z) is the separable synthesis
//    f = (T (x) T (x) T) C with the 1-D map
//      T(c0, c1, c2)(xi) = w_xi (c0 + 3 xi c1 + 9/2 (xi^2 - 1/3) c2).
// The coefficient tensor of f0 + (1 - 1/tau) f1 is a sum of three rank-one
// terms along x (u_x powers, their second and first u_x derivatives), which
// is how it is assembled; T is then applied along x, y and z.
// All values carried are shifted by the rest state (df = f - w), which keeps
// float32 round-off relative to the deviations rather than to w, and the
// conserved coefficients (rho - 1 and rho u) are the moments themselves, so
// that round-off does not make mass or momentum drift from step to step.
//
// D3Q19 (named in Sec. 5 as the cheaper 3-D quadrature whose recursion the
// paper leaves open) is not a tensor product. It is read as the D3Q27
// velocities without the eight corners, weights 1/3, 1/18, 1/36. Its
// quadrature is exact only to total degree five, so at order three it keeps,
// for each odd index b with even pair (a, c), the sum and the difference
// H_aab +- H_bcc, which it holds orthogonal to each other and to orders 0-2;
// the populations are synthesised from those coefficients directly
// (Lattice<19> below).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbrr {

constexpr float kCs2 = 1.0f / 3.0f;

// D1Q3 weight of xi = k - 1 (k = 0, 1, 2)
__host__ __device__ constexpr float w1(int k) { return k == 1 ? 2.0f / 3.0f : 1.0f / 6.0f; }
// T(0, 0, 1) at xi = k - 1: the second u-derivative factor (1/2, -1, 1/2)
__host__ __device__ constexpr float hh1(int k) { return k == 1 ? -1.0f : 0.5f; }

// velocity component a of direction i of D2Q9 / D3Q27
__host__ __device__ constexpr int vel(int i, int a) {
  return a == 0 ? i % 3 - 1 : (a == 1 ? (i / 3) % 3 - 1 : i / 9 - 1);
}

// D3Q27 index of D3Q19 direction k: the D3Q27 order with the corners left
// out (five directions in each of the planes z = -1 and z = +1, nine in
// z = 0), so that the opposite of k is again 18 - k.
__host__ __device__ constexpr int q19_to_q27(int k) {
  return k < 5 ? k + 1 + (k >= 1) + (k >= 4)
               : (k < 14 ? k + 4 : 19 + (k - 14) + (k >= 15) + (k >= 18));
}

// velocity component a of direction i of the Q-velocity lattice
template <int Q>
__host__ __device__ constexpr int vel_q(int i, int a) {
  return vel(Q == 19 ? q19_to_q27(i) : i, a);
}

// weight of velocity i of a D-dimensional tensor-product lattice
template <int D>
__host__ __device__ constexpr float weight(int i) {
  return D == 2 ? w1(i % 3) * w1((i / 3) % 3) : w1(i % 3) * w1((i / 3) % 3) * w1(i / 9);
}
// 1 / w_i (exact in float32: products of 6 and 3/2)
template <int D>
__host__ __device__ constexpr float inv_weight(int i) {
  return D == 2 ? (1.0f / w1(i % 3)) * (1.0f / w1((i / 3) % 3))
                : (1.0f / w1(i % 3)) * (1.0f / w1((i / 3) % 3)) * (1.0f / w1(i / 9));
}

// weight of velocity i of the Q-velocity lattice and its inverse (D3Q19:
// 1/3 at rest, 1/18 on the faces, 1/36 on the edges; inverses exact)
template <int Q>
__host__ __device__ constexpr float weight_q(int i) {
  if (Q != 19) return weight<Q == 9 ? 2 : 3>(i);
  const int j = q19_to_q27(i);
  const int m = (vel(j, 0) != 0) + (vel(j, 1) != 0) + (vel(j, 2) != 0);
  return m == 0 ? 1.0f / 3.0f : (m == 1 ? 1.0f / 18.0f : 1.0f / 36.0f);
}
template <int Q>
__host__ __device__ constexpr float inv_weight_q(int i) {
  if (Q != 19) return inv_weight<Q == 9 ? 2 : 3>(i);
  const int j = q19_to_q27(i);
  const int m = (vel(j, 0) != 0) + (vel(j, 1) != 0) + (vel(j, 2) != 0);
  return m == 0 ? 3.0f : (m == 1 ? 18.0f : 36.0f);
}

// ---------------------------------------------------------------- storage --
// LB_STORE_F32: df_i as float. LB_STORE_F16 / LB_STORE_BF16: df_i / w_i in
// 16 bits, round to nearest even. load<Q> / store<Q> take the direction i of
// the Q-velocity lattice.
template <int S>
struct Storage;

template <>
struct Storage<0> {
  using T = float;
  template <int Q>
  __device__ __forceinline__ static float load(const T *p, int i) {
    return *p;
  }
  template <int Q>
  __device__ __forceinline__ static void store(T *p, int i, float v) {
    *p = v;
  }
};

template <>
struct Storage<1> {
  using T = __half;
  template <int Q>
  __device__ __forceinline__ static float load(const T *p, int i) {
    return __half2float(*p) * weight_q<Q>(i);
  }
  template <int Q>
  __device__ __forceinline__ static void store(T *p, int i, float v) {
    *p = __float2half_rn(v * inv_weight_q<Q>(i));
  }
};

template <>
struct Storage<2> {
  using T = __nv_bfloat16;
  template <int Q>
  __device__ __forceinline__ static float load(const T *p, int i) {
    return __bfloat162float(*p) * weight_q<Q>(i);
  }
  template <int Q>
  __device__ __forceinline__ static void store(T *p, int i, float v) {
    *p = __float2bfloat16_rn(v * inv_weight_q<Q>(i));
  }
};

// ---------------------------------------------------------------- moments --
// rho, u and a1^(2) = Pi1 = sum xi xi f - rho cs2 I - rho u u (Sec. 2) from
// shifted populations: rho - 1 = sum df, rho u = sum xi df, and
// sum xi xi f = sum xi xi df + cs2 I (the rest state's second moment).
struct Macro {
  float drho, rho;          // rho - 1 and rho
  float jx, jy, jz;         // momentum rho u (the first moments themselves)
  float ux, uy, uz;
  float pxx, pxy, pxz, pyy, pyz, pzz;
};

// One separable moment pass over a line of three values at xi = -1, 0, +1:
// s0 = sum, s1 = first moment, s2 = second moment. With G (populations held
// as g = df / w) the D1Q3 weights are applied as the integer ratios 1 : 4 : 1,
// so every pass multiplies the moments by 6 (undone once at the end).
template <bool G>
__device__ __forceinline__ void mom3(float a, float b, float c, float &s0, float &s1, float &s2) {
  s2 = a + c;
  s0 = G ? fmaf(4.0f, b, s2) : s2 + b;
  s1 = c - a;
}

// rho, rho u and Pi1 from the raw moments m000 (= rho - 1), first moments j
// and second moments p_ab of df.
__device__ __forceinline__ Macro macro_from_moments(float m0, float jx, float jy, float jz,
                                                    float pxx, float pyy, float pzz, float pxy,
                                                    float pxz, float pyz) {
  Macro m;
  m.drho = m0;
  m.rho = 1.0f + m0;
  m.jx = jx;
  m.jy = jy;
  m.jz = jz;
  m.ux = jx / m.rho;
  m.uy = jy / m.rho;
  m.uz = jz / m.rho;
  m.pxx = pxx - kCs2 * m0 - jx * m.ux;
  m.pyy = pyy - kCs2 * m0 - jy * m.uy;
  m.pzz = pzz - kCs2 * m0 - jz * m.uz;
  m.pxy = pxy - jx * m.uy;
  m.pxz = pxz - jx * m.uz;
  m.pyz = pyz - jy * m.uz;
  return m;
}

// Moments of a D2Q9 cell, separable sums over x then y. G: inputs are g.
template <bool G>
__device__ __forceinline__ Macro moments_d2q9(const float (&f)[9]) {
  float s0[3], s1[3], s2[3];  // per y-line: sum, first and second x-moment
#pragma unroll
  for (int l = 0; l < 3; ++l) mom3<G>(f[3 * l], f[3 * l + 1], f[3 * l + 2], s0[l], s1[l], s2[l]);
  float m00, m01, m02, m10, m11, m12, m20, m21, m22;
  mom3<G>(s0[0], s0[1], s0[2], m00, m01, m02);
  mom3<G>(s1[0], s1[1], s1[2], m10, m11, m12);
  mom3<G>(s2[0], s2[1], s2[2], m20, m21, m22);
  const float k = G ? 1.0f / 36.0f : 1.0f;
  return macro_from_moments(k * m00, k * m10, k * m01, 0.0f, k * m20, k * m02, 0.0f, k * m11,
                            0.0f, 0.0f);
}

// Moments of a D3Q27 cell, separable sums over x, then y, then z.
template <bool G>
__device__ __forceinline__ Macro moments_d3q27(const float (&f)[27]) {
  float x0[9], x1[9], x2[9];
#pragma unroll
  for (int l = 0; l < 9; ++l) mom3<G>(f[3 * l], f[3 * l + 1], f[3 * l + 2], x0[l], x1[l], x2[l]);
  // y-pass per z-plane k: moments (x-power p, y-power q) with p + q <= 2
  float y00[3], y01[3], y02[3], y10[3], y11[3], y20[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int l = 3 * k;
    float t0, t1, t2;
    mom3<G>(x0[l], x0[l + 1], x0[l + 2], y00[k], y01[k], y02[k]);
    mom3<G>(x1[l], x1[l + 1], x1[l + 2], y10[k], y11[k], t2);
    mom3<G>(x2[l], x2[l + 1], x2[l + 2], y20[k], t1, t0);
  }
  float m000, m001, m002, m010, m011, m020, m100, m101, m110, m200, t0, t1, t2, t3, t4, t5;
  mom3<G>(y00[0], y00[1], y00[2], m000, m001, m002);
  mom3<G>(y01[0], y01[1], y01[2], m010, m011, t0);
  mom3<G>(y02[0], y02[1], y02[2], m020, t1, t2);
  mom3<G>(y10[0], y10[1], y10[2], m100, m101, t3);
  mom3<G>(y11[0], y11[1], y11[2], m110, t4, t5);
  float t6, t7;
  mom3<G>(y20[0], y20[1], y20[2], m200, t6, t7);
  const float k = G ? 1.0f / 216.0f : 1.0f;
  return macro_from_moments(k * m000, k * m100, k * m010, k * m001, k * m200, k * m020, k * m002,
                            k * m110, k * m101, k * m011);
}

// ------------------------------------------------------------- synthesis --
// 1-D synthesis T of coefficients (c0, c1, c2) at xi = -1, 0, +1; with G the
// weight is divided out: T/w = (c0 - 3/2 c2, c0 +- 3 c1 + 3 c2).
template <bool G>
__device__ __forceinline__ void synth1(float c0, float c1, float c2, float &om, float &oz,
                                       float &op) {
  if (G) {
    oz = fmaf(-1.5f, c2, c0);
    const float p = fmaf(3.0f, c2, c0);
    op = fmaf(3.0f, c1, p);
    om = fmaf(-3.0f, c1, p);
  } else {
    const float q = fmaf(c0, kCs2, c2);
    oz = c0 - q;
    op = 0.5f * (q + c1);
    om = 0.5f * (q - c1);
  }
}

// Coefficients of the shifted post-collision populations of a D2Q9 cell
// (RR, Sec. 3.5): df_post = f0 + om1 f1 - w with om1 = 1 - 1/tau (om1 = 1
// rebuilds f0 + f1). Coefficient of x^a y^b: C = px[a] Q1[b] + h[a] Q2[b] +
// dx[a] Q3[b] with px = (1, ux, ux^2), h = (0, 0, 1), dx = (0, 1, 2 ux) (powers
// of ux and their second and first ux-derivatives) and the y-vectors
//   Q1 = rho (1, uy, uy^2) + om1 Pi_yy (0, 0, 1)
//   Q2 = om1 Pi_xx (1, uy, uy^2),   Q3 = om1 Pi_xy (0, 1, 2 uy).
// The conserved coefficients are then set from the moments themselves
// (C_00 = rho - 1, C_10 = rho ux, C_01 = rho uy), so that mass and momentum
// pass through the update with no other rounding than the synthesis'.
__device__ __forceinline__ void coeffs_rr_d2q9(const Macro &m, float om1, float (&c)[3][3]) {
  const float ux = m.ux, uy = m.uy, uyy = uy * uy;
  const float pxx = om1 * m.pxx, pyy = om1 * m.pyy, pxy = om1 * m.pxy;
  const float q1[3] = {m.rho, m.rho * uy, fmaf(m.rho, uyy, pyy)};
  const float q2[3] = {pxx, pxx * uy, pxx * uyy};
  const float q3[3] = {0.0f, pxy, 2.0f * pxy * uy};
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    c[0][b] = q1[b];
    c[1][b] = fmaf(ux, q1[b], q3[b]);
    c[2][b] = fmaf(ux * ux, q1[b], fmaf(2.0f * ux, q3[b], q2[b]));
  }
  c[0][0] = m.drho;
  c[1][0] = m.jx;
  c[0][1] = m.jy;
}

// Order-2 regularized comparator (Sec. 3.8.1, eq_feq_2): only the
// coefficients of total Hermite order <= 2 are kept, for f0 and for f1.
__device__ __forceinline__ void coeffs_reg2_d2q9(const Macro &m, float om1, float (&c)[3][3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) c[a][b] = 0.0f;
  c[0][0] = m.drho;
  c[1][0] = m.jx;
  c[0][1] = m.jy;
  c[2][0] = fmaf(om1, m.pxx, m.jx * m.ux);
  c[0][2] = fmaf(om1, m.pyy, m.jy * m.uy);
  c[1][1] = fmaf(om1, m.pxy, m.jx * m.uy);
}

// Separable synthesis of a 3x3 coefficient matrix c[a][b] into the nine
// populations, i = ix + 3 iy.
template <bool G>
__device__ __forceinline__ void synth_tensor_d2q9(const float (&c)[3][3], float (&f)[9]) {
  float s[3][3];  // [ix][b]
#pragma unroll
  for (int b = 0; b < 3; ++b) synth1<G>(c[0][b], c[1][b], c[2][b], s[0][b], s[1][b], s[2][b]);
#pragma unroll
  for (int ix = 0; ix < 3; ++ix)
    synth1<G>(s[ix][0], s[ix][1], s[ix][2], f[ix], f[ix + 3], f[ix + 6]);
}

// Separable synthesis of a 3x3x3 coefficient tensor c[a][b][c] (x, y, z
// powers) into the 27 populations, i = ix + 3 iy + 9 iz.
template <bool G>
__device__ __forceinline__ void synth_tensor_d3q27(const float (&c)[3][3][3], float (&f)[27]) {
  float sx[3][3][3];  // [ix][b][c]
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
      synth1<G>(c[0][b][cc], c[1][b][cc], c[2][b][cc], sx[0][b][cc], sx[1][b][cc],
                sx[2][b][cc]);
#pragma unroll
  for (int ix = 0; ix < 3; ++ix) {
    float sy[3][3];  // [iy][c]
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
      synth1<G>(sx[ix][0][cc], sx[ix][1][cc], sx[ix][2][cc], sy[0][cc], sy[1][cc], sy[2][cc]);
#pragma unroll
    for (int iy = 0; iy < 3; ++iy)
      synth1<G>(sy[iy][0], sy[iy][1], sy[iy][2], f[ix + 3 * iy], f[ix + 3 * iy + 9],
                f[ix + 3 * iy + 18]);
  }
}

// Coefficients of the shifted post-collision populations of a D3Q27 cell
// (RR, Sec. 3.5). The coefficient of x^a y^b z^c is C = px[a] Q1[b][c] +
// h[a] Q2[b][c] + dx[a] Q3[b][c] (px, h, dx as in 2D) with the (y, z) matrices
//   Q1 = rho py pz + om1 (Pi_yy h_y pz + Pi_zz py h_z + Pi_yz dy dz)
//   Q2 = om1 Pi_xx py pz,   Q3 = om1 (Pi_xy dy pz + Pi_xz py dz),
// i.e. f0's coefficients rho ux^a uy^b uz^c plus om1 times the recursion's
// pair sums; the conserved coefficients come from the moments directly.
__device__ __forceinline__ void coeffs_rr_d3q27(const Macro &m, float om1, float (&c)[3][3][3]) {
  const float ux = m.ux, uy = m.uy, uz = m.uz;
  const float py[3] = {1.0f, uy, uy * uy}, pz[3] = {1.0f, uz, uz * uz};
  const float dy[3] = {0.0f, 1.0f, 2.0f * uy}, dz[3] = {0.0f, 1.0f, 2.0f * uz};
  const float pxx = om1 * m.pxx, pyy = om1 * m.pyy, pzz = om1 * m.pzz;
  const float pxy = om1 * m.pxy, pxz = om1 * m.pxz, pyz = om1 * m.pyz;
  const float uxx = ux * ux, ux2 = 2.0f * ux;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      const float pp = py[b] * pz[cc];
      float q1 = m.rho * pp;
      if (b == 2) q1 = fmaf(pyy, pz[cc], q1);
      if (cc == 2) q1 = fmaf(pzz, py[b], q1);
      if (b > 0 && cc > 0) q1 = fmaf(pyz, dy[b] * dz[cc], q1);
      const float q2 = pxx * pp;
      float q3 = 0.0f;
      if (b > 0) q3 = fmaf(pxy, dy[b] * pz[cc], q3);
      if (cc > 0) q3 = fmaf(pxz, py[b] * dz[cc], q3);
      c[0][b][cc] = q1;
      c[1][b][cc] = fmaf(ux, q1, q3);
      c[2][b][cc] = fmaf(uxx, q1, fmaf(ux2, q3, q2));
    }
  }
  c[0][0][0] = m.drho;
  c[1][0][0] = m.jx;
  c[0][1][0] = m.jy;
  c[0][0][1] = m.jz;
}

__device__ __forceinline__ void coeffs_reg2_d3q27(const Macro &m, float om1,
                                                  float (&c)[3][3][3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) c[a][b][cc] = 0.0f;
  c[0][0][0] = m.drho;
  c[1][0][0] = m.jx;
  c[0][1][0] = m.jy;
  c[0][0][1] = m.jz;
  c[2][0][0] = fmaf(om1, m.pxx, m.jx * m.ux);
  c[0][2][0] = fmaf(om1, m.pyy, m.jy * m.uy);
  c[0][0][2] = fmaf(om1, m.pzz, m.jz * m.uz);
  c[1][1][0] = fmaf(om1, m.pxy, m.jx * m.uy);
  c[1][0][1] = fmaf(om1, m.pxz, m.jx * m.uz);
  c[0][1][1] = fmaf(om1, m.pyz, m.jy * m.uz);
}

// moments<G>(f): macroscopic moments of one cell (G: f holds g = df / w).
// synth<MODEL, G>(m, om1, f): post-collision populations (MODEL 0: RR,
// 1: order-2 regularized, 2: plain BGK f - (f - f0)/tau, for which f holds the
// pre-collision populations on entry) as df, or as g with G.
template <int Q>
struct Lattice;
template <>
struct Lattice<9> {
  static constexpr int D = 2;
  template <bool G = false>
  __device__ __forceinline__ static Macro moments(const float (&f)[9]) {
    return moments_d2q9<G>(f);
  }
  template <int MODEL, bool G = false>
  __device__ __forceinline__ static void synth(const Macro &m, float om1, float (&f)[9]) {
    float c[3][3];
    if (MODEL == 2) {  // equilibrium coefficients only, then relax
      coeffs_rr_d2q9(m, 0.0f, c);
      float eq[9];
      synth_tensor_d2q9<G>(c, eq);
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i] = fmaf(1.0f - om1, eq[i] - f[i], f[i]);
      return;
    }
    if (MODEL == 0)
      coeffs_rr_d2q9(m, om1, c);
    else
      coeffs_reg2_d2q9(m, om1, c);
    synth_tensor_d2q9<G>(c, f);
  }
};
template <>
struct Lattice<27> {
  static constexpr int D = 3;
  template <bool G = false>
  __device__ __forceinline__ static Macro moments(const float (&f)[27]) {
    return moments_d3q27<G>(f);
  }
  template <int MODEL, bool G = false>
  __device__ __forceinline__ static void synth(const Macro &m, float om1, float (&f)[27]) {
    float c[3][3][3];
    if (MODEL == 2) {  // equilibrium coefficients only, then relax
      coeffs_rr_d3q27(m, 0.0f, c);
      float eq[27];
      synth_tensor_d3q27<G>(c, eq);
#pragma unroll
      for (int i = 0; i < 27; ++i) f[i] = fmaf(1.0f - om1, eq[i] - f[i], f[i]);
      return;
    }
    if (MODEL == 0)
      coeffs_rr_d3q27(m, om1, c);
    else
      coeffs_reg2_d3q27(m, om1, c);
    synth_tensor_d3q27<G>(c, f);
  }
};

// ----------------------------------------------------------------- D3Q19 --
// Moments of a D3Q19 cell (direction order of q19_to_q27): the z = 0 plane is
// a full 3x3 set and takes the separable 2-D sums; the planes z = -1 and
// z = +1 hold the five-velocity crosses (0,-1), (-1,0), (0,0), (1,0), (0,1);
// the three plane sums are then combined along z.
__device__ __forceinline__ Macro moments_d3q19(const float (&f)[19]) {
  // cross of plane z = -1 (f[0..4]) and z = +1 (f[14..18])
  const float mxx = f[1] + f[3], myy = f[0] + f[4];
  const float m0 = (mxx + myy) + f[2], mx = f[3] - f[1], my = f[4] - f[0];
  const float pxx = f[15] + f[17], pyy = f[14] + f[18];
  const float p0 = (pxx + pyy) + f[16], px = f[17] - f[15], py = f[18] - f[14];
  // plane z = 0 (f[5..13], 5 + ix + 3 iy)
  float s0[3], s1[3], s2[3];
#pragma unroll
  for (int l = 0; l < 3; ++l)
    mom3<false>(f[5 + 3 * l], f[6 + 3 * l], f[7 + 3 * l], s0[l], s1[l], s2[l]);
  float c00, c01, c02, c10, c11, c20, t0, t1, t2;
  mom3<false>(s0[0], s0[1], s0[2], c00, c01, c02);
  mom3<false>(s1[0], s1[1], s1[2], c10, c11, t0);
  mom3<false>(s2[0], s2[1], s2[2], c20, t1, t2);
  return macro_from_moments(c00 + (m0 + p0), c10 + (mx + px), c01 + (my + py), p0 - m0,
                            c20 + (mxx + pxx), c02 + (myy + pyy), p0 + m0, c11, px - mx,
                            py - my);
}

// Shifted post-collision populations df = f0 + om1 f1 - w of a D3Q19 cell on
// the kept basis. A_ab = rho u_a u_b + om1 Pi_ab is the order-2 coefficient;
// the order-3 Hermite coefficients are A_abb = rho u_a u_b^2 + om1 (Pi_bb u_a
// + 2 Pi_ab u_b) (f0's rho u u u plus om1 times the recursion eq_rel_a1),
// i.e. u_a A_bb + 2 u_b om1 Pi_ab. On the kept order-3 members (sum and
// difference of H_aab and H_bcc) the expansion of f/w reduces, per class of
// velocity, to
//   rest:                    drho - 3/2 tr A
//   face  xi_a = s:          ... + 9/2 A_aa + s (3 j_a - 9 (A_abb + A_acc))
//   edge  xi_a = s, xi_b = t: ... + 9/2 (A_aa + A_bb) + 9 s t A_ab
//                                 + s (3 j_a + 9 A_abb) + t (3 j_b + 9 A_aab)
// with "..." the rest value. The weights 1/3, 1/18, 1/36 are not float32
// numbers, and multiplying by their roundings would scale mass and momentum
// by 1 + O(1e-8) at every update, a drift that adds up over thousands of
// updates. So the edges are formed from the expression above, and the
// conserved moments close the rest: the odd part of the face pair of axis a
// is j_a minus the a-momentum of the edges (in exact arithmetic this is
// w_face 2 (3 j_a - 9 (A_abb + A_acc))), and the rest population is
// rho - 1 minus the other eighteen. ORDER3 = false drops the order-3
// members (the order-2 regularized comparator). om1 = 0 gives f0 - w.
template <bool ORDER3>
__device__ __forceinline__ void synth_d3q19(const Macro &m, float om1, float (&f)[19]) {
  const float ux = m.ux, uy = m.uy, uz = m.uz;
  const float qxy = om1 * m.pxy, qxz = om1 * m.pxz, qyz = om1 * m.pyz;
  const float axx = fmaf(om1, m.pxx, m.jx * ux), ayy = fmaf(om1, m.pyy, m.jy * uy);
  const float azz = fmaf(om1, m.pzz, m.jz * uz);
  const float axy = fmaf(m.jx, uy, qxy), axz = fmaf(m.jx, uz, qxz), ayz = fmaf(m.jy, uz, qyz);
  float axyy = 0.f, axzz = 0.f, axxy = 0.f, ayzz = 0.f, axxz = 0.f, ayyz = 0.f;
  if (ORDER3) {
    axyy = fmaf(ux, ayy, 2.0f * uy * qxy);
    axzz = fmaf(ux, azz, 2.0f * uz * qxz);
    axxy = fmaf(uy, axx, 2.0f * ux * qxy);
    ayzz = fmaf(uy, azz, 2.0f * uz * qyz);
    axxz = fmaf(uz, axx, 2.0f * ux * qxz);
    ayyz = fmaf(uz, ayy, 2.0f * uy * qyz);
  }
  const float base = fmaf(-1.5f, (axx + ayy) + azz, m.drho);
  const float jx3 = 3.0f * m.jx, jy3 = 3.0f * m.jy, jz3 = 3.0f * m.jz;
  // edges of the plane (a, b): w_edge (e + 9 s t A_ab + s U + t V)
  auto edges = [](float e, float ab9, float U, float V, float &pp, float &pm, float &mp,
                  float &mm) {
    constexpr float w2 = 1.0f / 36.0f;
    const float ep = e + ab9, em = e - ab9;
    pp = w2 * (ep + (U + V));
    mm = w2 * (ep - (U + V));
    pm = w2 * (em + (U - V));
    mp = w2 * (em - (U - V));
  };
  // (x, y): (+,+) 13, (+,-) 7, (-,+) 11, (-,-) 5
  edges(fmaf(4.5f, axx + ayy, base), 9.0f * axy,
        fmaf(9.0f, axyy, jx3), fmaf(9.0f, axxy, jy3),
        f[13], f[7], f[11], f[5]);
  // (x, z): (+,+) 17, (+,-) 3, (-,+) 15, (-,-) 1
  edges(fmaf(4.5f, axx + azz, base), 9.0f * axz,
        fmaf(9.0f, axzz, jx3), fmaf(9.0f, axxz, jz3),
        f[17], f[3], f[15], f[1]);
  // (y, z): (+,+) 18, (+,-) 4, (-,+) 14, (-,-) 0
  edges(fmaf(4.5f, ayy + azz, base), 9.0f * ayz,
        fmaf(9.0f, ayzz, jy3), fmaf(9.0f, ayyz, jz3),
        f[18], f[4], f[14], f[0]);
  // faces: even part w_face (base + 9/2 A_aa), odd part closing j_a
  constexpr float w1 = 1.0f / 18.0f;
  const float ex = ((f[13] + f[7]) + (f[17] + f[3])) - ((f[11] + f[5]) + (f[15] + f[1]));
  const float ey = ((f[13] + f[11]) + (f[18] + f[4])) - ((f[7] + f[5]) + (f[14] + f[0]));
  const float ez = ((f[17] + f[15]) + (f[18] + f[14])) - ((f[3] + f[1]) + (f[4] + f[0]));
  const float sx = w1 * fmaf(4.5f, axx, base), hx = 0.5f * (m.jx - ex);
  const float sy = w1 * fmaf(4.5f, ayy, base), hy = 0.5f * (m.jy - ey);
  const float sz = w1 * fmaf(4.5f, azz, base), hz = 0.5f * (m.jz - ez);
  f[10] = sx + hx;
  f[8] = sx - hx;
  f[12] = sy + hy;
  f[6] = sy - hy;
  f[16] = sz + hz;
  f[2] = sz - hz;
  // rest: closes the mass
  const float e4 = ((f[0] + f[1]) + (f[3] + f[4])) + ((f[14] + f[15]) + (f[17] + f[18]));
  const float e8 = e4 + ((f[5] + f[7]) + (f[11] + f[13]));
  const float fa = ((f[2] + f[6]) + (f[8] + f[10])) + (f[12] + f[16]);
  f[9] = m.drho - (e8 + fa);
}

template <>
struct Lattice<19> {
  static constexpr int D = 3;
  template <bool G = false>
  __device__ __forceinline__ static Macro moments(const float (&f)[19]) {
    static_assert(!G, "D3Q19 runs on shifted populations df only");
    return moments_d3q19(f);
  }
  template <int MODEL, bool G = false>
  __device__ __forceinline__ static void synth(const Macro &m, float om1, float (&f)[19]) {
    static_assert(!G, "D3Q19 runs on shifted populations df only");
    if (MODEL == 2) {  // the model's full equilibrium, then relax
      float eq[19];
      synth_d3q19<true>(m, 0.0f, eq);
#pragma unroll
      for (int i = 0; i < 19; ++i) f[i] = fmaf(1.0f - om1, eq[i] - f[i], f[i]);
      return;
    }
    synth_d3q19<MODEL == 0>(m, om1, f);
  }
};

// Grid geometry passed by value to every kernel. walls: bit a set = axis a
// is bounded by no-slip walls through its first and last node planes
// (Sec. 3.7, boundary conditions); other axes are periodic.
struct Grid {
  int nx, ny, nz;
  long long n;  // nx * ny * nz (cells per population slot)
  int walls = 0;
};

// Periodic neighbour coordinate c + d, d in {-1, 0, 1}.
__device__ __forceinline__ int wrap_add(int c, int d, int n) {
  int r = c + d;
  r = (r < 0) ? r + n : r;
  return (r >= n) ? r - n : r;
}

// ---------------------------------------------------------------- walls --
// Populations whose velocity component along axis a equals s (+1 or -1).
template <int Q>
__host__ __device__ constexpr uint32_t vel_mask(int a, int s) {
  uint32_t m = 0;
  for (int i = 0; i < Q; ++i)
    if (vel_q<Q>(i, a) == s) m |= 1u << i;
  return m;
}

// Populations of node (x, y, z) that stream in from outside the domain
// (x - xi_i beyond a wall plane): c_a = +1 on the first plane of a walled
// axis a, c_a = -1 on the last. Zero off the walls.
template <int Q>
__device__ __forceinline__ uint32_t unknown_mask(const Grid &g, int x, int y, int z) {
  constexpr int D = Lattice<Q>::D;
  uint32_t m = 0;
  if (g.walls & 1) {
    if (x == 0) m |= vel_mask<Q>(0, 1);
    if (x == g.nx - 1) m |= vel_mask<Q>(0, -1);
  }
  if (g.walls & 2) {
    if (y == 0) m |= vel_mask<Q>(1, 1);
    if (y == g.ny - 1) m |= vel_mask<Q>(1, -1);
  }
  if (D == 3 && (g.walls & 4)) {
    if (z == 0) m |= vel_mask<Q>(2, 1);
    if (z == g.nz - 1) m |= vel_mask<Q>(2, -1);
  }
  return m;
}

// bit i set <-> bit opp(i) = Q - 1 - i of m set
template <int Q>
__device__ __forceinline__ uint32_t opposite_mask(uint32_t m) {
  return __brev(m) >> (32 - Q);
}

// Zero-velocity no-slip closure of a boundary node (the regularized
// Dirichlet procedure of Sec. 3.7 with u_bc = 0), on shifted populations:
// with u_bc = 0 the equilibrium is the same for a population and its
// opposite, so giving an unknown population the value of its known opposite
// is the off-equilibrium bounce-back from which the lattice symmetries give
// rho and Pi^(1). A buried link (population and opposite both unknown) is
// set to equilibrium, w_i (rho - 1), with rho closing the mass balance.
template <int Q>
__device__ __forceinline__ void wall_fill(uint32_t unknown, float (&df)[Q]) {
  const uint32_t buried = unknown & opposite_mask<Q>(unknown);
#pragma unroll
  for (int i = 0; i < Q; ++i)
    if (((unknown & ~buried) >> i) & 1u) df[i] = df[Q - 1 - i];
  if (buried) {
    float s = 0.f, wb = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if ((buried >> i) & 1u)
        wb += weight_q<Q>(i);
      else
        s += df[i];
    }
    const float drho = s / (1.f - wb);
#pragma unroll
    for (int i = 0; i < Q; ++i)
      if ((buried >> i) & 1u) df[i] = weight_q<Q>(i) * drho;
  }
}

// Impose u = u_bc = 0 on the moments of a filled boundary node: Pi^(1) is
// then sum xi xi df - c_s^2 (rho - 1) I without the rho u u term.
__device__ __forceinline__ void wall_macro(Macro &m) {
  m.pxx += m.jx * m.ux;
  m.pyy += m.jy * m.uy;
  m.pzz += m.jz * m.uz;
  m.pxy += m.jx * m.uy;
  m.pxz += m.jx * m.uz;
  m.pyz += m.jy * m.uz;
  m.jx = m.jy = m.jz = 0.f;
  m.ux = m.uy = m.uz = 0.f;
}

// Logical (natural-order, pre-collision) shifted populations of cell (x, y, z)
// from an AA store of the given parity (AA parity as in lbrr_step.cu).
template <int Q, int S>
__device__ __forceinline__ void load_logical(const typename Storage<S>::T *__restrict__ f,
                                             const Grid &g, int parity, int x, int y, int z,
                                             float (&df)[Q]) {
  constexpr int D = Lattice<Q>::D;
  const long long n = g.n;
  if (parity == 0) {
    const long long cell = ((long long)z * g.ny + y) * g.nx + x;
#pragma unroll
    for (int i = 0; i < Q; ++i) df[i] = Storage<S>::template load<Q>(f + i * n + cell, i);
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int xs = wrap_add(x, -vel_q<Q>(i, 0), g.nx), ys = wrap_add(y, -vel_q<Q>(i, 1), g.ny);
      const int zs = D == 3 ? wrap_add(z, -vel_q<Q>(i, 2), g.nz) : 0;
      const long long src = ((long long)zs * g.ny + ys) * g.nx + xs;
      df[i] = Storage<S>::template load<Q>(f + (Q - 1 - i) * n + src, i);
    }
  }
}

__device__ __forceinline__ void cell_coords(long long cell, const Grid &g, int &x, int &y,
                                            int &z) {
  x = (int)(cell % g.nx);
  const long long r = cell / g.nx;
  y = (int)(r % g.ny);
  z = (int)(r / g.ny);
}

}  // namespace lbrr
