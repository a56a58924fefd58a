// Per-pair device arithmetic of the NEP descriptor: radial basis (App. A),
// real solid harmonics on the unit sphere (App. B) and the 4-body invariant.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>

namespace gnep {

constexpr int NLM = 24;  // (l, m) components for l = 1..4

// C_lm of Eq. 7: addition-theorem normalisation, sum_m C_lm B_lm(u) B_lm(v) = P_l(u.v).
__device__ __constant__ static const float kClm[NLM] = {
    1.f, 1.f, 1.f,
    0.25f, 3.f, 3.f, 0.75f, 0.75f,
    0.25f, 0.375f, 0.375f, 3.75f, 3.75f, 0.625f, 0.625f,
    0.015625f, 0.625f, 0.625f, 0.3125f, 0.3125f, 4.375f, 4.375f, 0.546875f, 0.546875f};

__host__ __device__ constexpr int lm_l(int lm) { return lm < 3 ? 1 : lm < 8 ? 2 : lm < 15 ? 3 : 4; }

// Basis f_k = (T_k(xi) + 1)/2 f_c(r) of Eq. 6, xi = 2 (r/rc - 1)^2 - 1 (A1.2),
// Chebyshev recursion A1.1, cosine cut-off A2.1.  Listed pairs have r < rc.
template <int K>
__device__ __forceinline__ void radial_basis(float r, float rc_inv, float (&f)[K]) {
  const float x = r * rc_inv;
  const float t = x - 1.f;
  const float xi = 2.f * t * t - 1.f;
  float s, c;
  sincospif(x, &s, &c);
  const float hfc = 0.25f + 0.25f * c;  // f_c / 2
  float tm2 = 1.f, tm1 = xi;
  f[0] = 2.f * hfc;
  if (K > 1) f[1] = (xi + 1.f) * hfc;
#pragma unroll
  for (int k = 2; k < K; ++k) {
    const float tk = 2.f * xi * tm1 - tm2;
    f[k] = (tk + 1.f) * hfc;
    tm2 = tm1;
    tm1 = tk;
  }
}

// Basis and its r-derivative: df_k/dr = 1/2 T_k'(xi) xi' f_c + 1/2 (T_k + 1) f_c'
// with T_k' from the derivative recursion A1.3-A1.5 and f_c' from A2.2.
template <int K>
__device__ __forceinline__ void radial_basis_d(float r, float rc_inv, float (&f)[K], float (&fp)[K]) {
  const float x = r * rc_inv;
  const float t = x - 1.f;
  const float xi = 2.f * t * t - 1.f;
  const float dxi = 4.f * t * rc_inv;
  float s, c;
  sincospif(x, &s, &c);
  const float hfc = 0.25f + 0.25f * c;                 // f_c / 2
  const float hfcp = -0.25f * CUDART_PI_F * rc_inv * s;  // f_c' / 2
  const float a = dxi * hfc;                           // xi' f_c / 2
  float tm2 = 1.f, tm1 = xi, dm2 = 0.f, dm1 = 1.f;
  f[0] = 2.f * hfc;
  fp[0] = 2.f * hfcp;
  if (K > 1) {
    f[1] = (xi + 1.f) * hfc;
    fp[1] = a + (xi + 1.f) * hfcp;
  }
#pragma unroll
  for (int k = 2; k < K; ++k) {
    const float tk = 2.f * xi * tm1 - tm2;
    const float dk = 2.f * tm1 + 2.f * xi * dm1 - dm2;
    f[k] = (tk + 1.f) * hfc;
    fp[k] = dk * a + (tk + 1.f) * hfcp;
    tm2 = tm1; tm1 = tk;
    dm2 = dm1; dm1 = dk;
  }
}

// B_lm(u) = b_lm(u) / r^l evaluated on the unit vector u (B1.1-B4.9 with r = 1).
__device__ __forceinline__ void harmonics(float x, float y, float z, float (&B)[NLM]) {
  const float x2 = x * x, y2 = y * y, z2 = z * z;
  B[0] = z; B[1] = x; B[2] = y;
  B[3] = 3.f * z2 - 1.f; B[4] = x * z; B[5] = y * z; B[6] = x2 - y2; B[7] = 2.f * x * y;
  const float p3 = 5.f * z2 - 1.f;
  B[8] = (5.f * z2 - 3.f) * z; B[9] = p3 * x; B[10] = p3 * y; B[11] = (x2 - y2) * z;
  B[12] = 2.f * x * y * z; B[13] = (x2 - 3.f * y2) * x; B[14] = (3.f * x2 - y2) * y;
  const float w4 = (7.f * z2 - 3.f) * z, p4 = 7.f * z2 - 1.f;
  B[15] = (35.f * z2 - 30.f) * z2 + 3.f; B[16] = w4 * x; B[17] = w4 * y;
  B[18] = p4 * (x2 - y2); B[19] = p4 * 2.f * x * y;
  B[20] = (x2 - 3.f * y2) * x * z; B[21] = (3.f * x2 - y2) * y * z;
  B[22] = x2 * x2 - 6.f * x2 * y2 + y2 * y2; B[23] = 4.f * x * y * (x2 - y2);
}

// Harmonics and their gradients w.r.t. the bond vector d (B9.2).  On the unit
// sphere B(d) = p(d/|d|) for the r = 1 polynomial p, so
// grad_d B = (I - u u^T) grad p(u) / r.  gx, gy, gz receive the components.
__device__ __forceinline__ void harmonics_grad(float x, float y, float z, float rinv,
                                               float (&B)[NLM], float (&gx)[NLM],
                                               float (&gy)[NLM], float (&gz)[NLM]) {
  harmonics(x, y, z, B);
  const float x2 = x * x, y2 = y * y, z2 = z * z;
  // gradients of the unit-sphere polynomials
  gx[0] = 0.f; gy[0] = 0.f; gz[0] = 1.f;
  gx[1] = 1.f; gy[1] = 0.f; gz[1] = 0.f;
  gx[2] = 0.f; gy[2] = 1.f; gz[2] = 0.f;
  gx[3] = 0.f; gy[3] = 0.f; gz[3] = 6.f * z;
  gx[4] = z; gy[4] = 0.f; gz[4] = x;
  gx[5] = 0.f; gy[5] = z; gz[5] = y;
  gx[6] = 2.f * x; gy[6] = -2.f * y; gz[6] = 0.f;
  gx[7] = 2.f * y; gy[7] = 2.f * x; gz[7] = 0.f;
  const float p3 = 5.f * z2 - 1.f;
  gx[8] = 0.f; gy[8] = 0.f; gz[8] = 15.f * z2 - 3.f;
  gx[9] = p3; gy[9] = 0.f; gz[9] = 10.f * x * z;
  gx[10] = 0.f; gy[10] = p3; gz[10] = 10.f * y * z;
  gx[11] = 2.f * x * z; gy[11] = -2.f * y * z; gz[11] = x2 - y2;
  gx[12] = 2.f * y * z; gy[12] = 2.f * x * z; gz[12] = 2.f * x * y;
  gx[13] = 3.f * (x2 - y2); gy[13] = -6.f * x * y; gz[13] = 0.f;
  gx[14] = 6.f * x * y; gy[14] = 3.f * (x2 - y2); gz[14] = 0.f;
  const float w4 = (7.f * z2 - 3.f) * z, dw4 = 21.f * z2 - 3.f, p4 = 7.f * z2 - 1.f;
  gx[15] = 0.f; gy[15] = 0.f; gz[15] = (140.f * z2 - 60.f) * z;
  gx[16] = w4; gy[16] = 0.f; gz[16] = dw4 * x;
  gx[17] = 0.f; gy[17] = w4; gz[17] = dw4 * y;
  gx[18] = 2.f * x * p4; gy[18] = -2.f * y * p4; gz[18] = 14.f * z * (x2 - y2);
  gx[19] = 2.f * y * p4; gy[19] = 2.f * x * p4; gz[19] = 28.f * x * y * z;
  gx[20] = 3.f * (x2 - y2) * z; gy[20] = -6.f * x * y * z; gz[20] = (x2 - 3.f * y2) * x;
  gx[21] = 6.f * x * y * z; gy[21] = 3.f * (x2 - y2) * z; gz[21] = (3.f * x2 - y2) * y;
  gx[22] = 4.f * x * (x2 - 3.f * y2); gy[22] = 4.f * y * (y2 - 3.f * x2); gz[22] = 0.f;
  gx[23] = 4.f * y * (3.f * x2 - y2); gy[23] = 4.f * x * (x2 - 3.f * y2); gz[23] = 0.f;
#pragma unroll
  for (int q = 0; q < NLM; ++q) {
    const float ud = x * gx[q] + y * gy[q] + z * gz[q];
    gx[q] = (gx[q] - ud * x) * rinv;
    gy[q] = (gy[q] - ud * y) * rinv;
    gz[q] = (gz[q] - ud * z) * rinv;
  }
}

// Harmonics on the unit vector u and, for a direction w, the directional
// derivatives D_lm = grad_d B_lm . w (B9.2).  Each B_lm is the degree-l
// homogeneous polynomial h_lm (the r = 1 forms with 1 read as r^2) on u, so
// grad_d B_lm = (grad h_lm(u) - l h_lm(u) u) / r (Euler's relation u . grad h =
// l h removes the radial part), and grad h_lm(u) . w is the derivative of h_lm
// along w, evaluated here with dx = w_x, dy = w_y, dz = w_z, d(r^2) = 2 u . w.
__device__ __forceinline__ void harmonics_dir(float x, float y, float z, float rinv, float wx, float wy, float wz,
                                              float (&B)[NLM], float (&Dd)[NLM]) {
  harmonics(x, y, z, B);
  const float ru = x * wx + y * wy + z * wz;  // u . w; d(r^2) = 2 ru
  const float x2 = x * x, y2 = y * y, z2 = z * z;
  const float dx2 = 2.f * x * wx, dy2 = 2.f * y * wy, dz2 = 2.f * z * wz, dr2 = 2.f * ru;
  float d[NLM];
  // l = 1
  d[0] = wz; d[1] = wx; d[2] = wy;
  // l = 2
  d[3] = 3.f * dz2 - dr2;
  d[4] = wx * z + x * wz;
  d[5] = wy * z + y * wz;
  d[6] = dx2 - dy2;
  d[7] = 2.f * (wx * y + x * wy);
  // l = 3: p3 = 5 z^2 - r^2
  const float p3 = 5.f * z2 - 1.f, dp3 = 5.f * dz2 - dr2;
  d[8] = (5.f * dz2 - 3.f * dr2) * z + (5.f * z2 - 3.f) * wz;
  d[9] = dp3 * x + p3 * wx;
  d[10] = dp3 * y + p3 * wy;
  const float xmy = x2 - y2, dxmy = dx2 - dy2;
  d[11] = dxmy * z + xmy * wz;
  d[12] = 2.f * ((wx * y + x * wy) * z + x * y * wz);
  const float a13 = x2 - 3.f * y2, da13 = dx2 - 3.f * dy2;
  const float a14 = 3.f * x2 - y2, da14 = 3.f * dx2 - dy2;
  d[13] = da13 * x + a13 * wx;
  d[14] = da14 * y + a14 * wy;
  // l = 4: w4 = (7 z^2 - 3 r^2) z, p4 = 7 z^2 - r^2
  const float w4 = (7.f * z2 - 3.f) * z, dw4 = (7.f * dz2 - 3.f * dr2) * z + (7.f * z2 - 3.f) * wz;
  const float p4 = 7.f * z2 - 1.f, dp4 = 7.f * dz2 - dr2;
  d[15] = 35.f * 2.f * z2 * dz2 - 30.f * (dz2 + z2 * dr2) + 3.f * 2.f * dr2;
  d[16] = dw4 * x + w4 * wx;
  d[17] = dw4 * y + w4 * wy;
  d[18] = dp4 * xmy + p4 * dxmy;
  const float xy = x * y, dxy = wx * y + x * wy;
  d[19] = 2.f * (dp4 * xy + p4 * dxy);
  d[20] = da13 * x * z + a13 * (wx * z + x * wz);
  d[21] = da14 * y * z + a14 * (wy * z + y * wz);
  d[22] = 2.f * x2 * dx2 - 6.f * (dx2 * y2 + x2 * dy2) + 2.f * y2 * dy2;
  d[23] = 4.f * (dxy * xmy + xy * dxmy);
#pragma unroll
  for (int q = 0; q < NLM; ++q) Dd[q] = (d[q] - (float)lm_l(q) * B[q] * ru) * rinv;
}


// 4-body invariant q4 = tr(Q^3) with Q = sum_j g (3 u u^T - I)/2, written in the
// l = 2 moments S_2m (m = 0..4, i.e. lm = 3..7):
//   Q_zz = S0/2, Q_xz = 3 S1/2, Q_yz = 3 S2/2, Q_xy = 3 S4/4,
//   Q_xx = -S0/4 + 3 S3/4, Q_yy = -S0/4 - 3 S3/4.
struct Sym3 { float xx, yy, zz, xy, yz, xz; };

__device__ __forceinline__ Sym3 quad_from_s2(const float* s) {
  Sym3 q;
  q.zz = 0.5f * s[0];
  q.xz = 1.5f * s[1];
  q.yz = 1.5f * s[2];
  q.xx = -0.25f * s[0] + 0.75f * s[3];
  q.yy = -0.25f * s[0] - 0.75f * s[3];
  q.xy = 0.75f * s[4];
  return q;
}

// Product P = A B of two symmetric matrices, symmetrised (A B + B A) / 2.
__device__ __forceinline__ Sym3 sym_prod(const Sym3& a, const Sym3& b) {
  Sym3 p;
  const float axx = a.xx, ayy = a.yy, azz = a.zz, axy = a.xy, ayz = a.yz, axz = a.xz;
  const float bxx = b.xx, byy = b.yy, bzz = b.zz, bxy = b.xy, byz = b.yz, bxz = b.xz;
  p.xx = axx * bxx + axy * bxy + axz * bxz;
  p.yy = axy * bxy + ayy * byy + ayz * byz;
  p.zz = axz * bxz + ayz * byz + azz * bzz;
  p.xy = 0.5f * ((axx * bxy + axy * byy + axz * byz) + (bxx * axy + bxy * ayy + bxz * ayz));
  p.yz = 0.5f * ((axy * bxz + ayy * byz + ayz * bzz) + (bxy * axz + byy * ayz + byz * azz));
  p.xz = 0.5f * ((axx * bxz + axy * byz + axz * bzz) + (bxx * axz + bxy * ayz + bxz * azz));
  return p;
}

__device__ __forceinline__ float sym_trace_prod(const Sym3& a, const Sym3& b) {
  return a.xx * b.xx + a.yy * b.yy + a.zz * b.zz +
         2.f * (a.xy * b.xy + a.yz * b.yz + a.xz * b.xz);
}

// Pull a symmetric matrix M (a gradient dq/dQ) back to the five S_2m.
__device__ __forceinline__ void s2_from_grad(const Sym3& m, float* g) {
  g[0] = 0.5f * m.zz - 0.25f * (m.xx + m.yy);
  g[1] = 3.f * m.xz;
  g[2] = 3.f * m.yz;
  g[3] = 0.75f * (m.xx - m.yy);
  g[4] = 1.5f * m.xy;
}

__device__ __forceinline__ float q4_value(const float* s2) {
  const Sym3 q = quad_from_s2(s2);
  return sym_trace_prod(sym_prod(q, q), q);
}

// dq4/dS_2m: dq4/dQ = 3 Q^2.
__device__ __forceinline__ void q4_grad(const float* s2, float* g) {
  const Sym3 q = quad_from_s2(s2);
  Sym3 m = sym_prod(q, q);
  m.xx *= 3.f; m.yy *= 3.f; m.zz *= 3.f; m.xy *= 3.f; m.yz *= 3.f; m.xz *= 3.f;
  s2_from_grad(m, g);
}

// Hessian-vector product of q4 in S_2m space along sd: d/dt [3 Q^2] = 3 (Q Qd + Qd Q).
__device__ __forceinline__ void q4_hvp(const float* s2, const float* sd, float* g) {
  const Sym3 q = quad_from_s2(s2), qd = quad_from_s2(sd);
  Sym3 m = sym_prod(q, qd);  // (Q Qd + Qd Q)/2
  m.xx *= 6.f; m.yy *= 6.f; m.zz *= 6.f; m.xy *= 6.f; m.yz *= 6.f; m.xz *= 6.f;
  s2_from_grad(m, g);
}

}  // namespace gnep
