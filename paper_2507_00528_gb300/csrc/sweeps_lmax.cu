// Angular sweeps for l_max > 4: the terms l = 5..8 of Eq. 7 (App. B, B5-B8),
// with the same four sweeps as the l_max = 4 kernels of sweeps.cu (descriptor,
// pair force, tangent, coefficient gradient; see there for the gradient route).
//
// Harmonic basis.  q_nl = sum_m C_lm S_nlm^2 depends only on the addition
// theorem sum_m C_lm B_lm(u) B_lm(v) = P_l(u.v), not on the basis chosen
// within one l.  For l <= 4 these kernels take the printed forms B1-B4 with
// their C_lm (device_math.cuh), which the 4-body term is written in; for
// l = 5..8 they take the real regular solid harmonics in Racah normalisation,
// generated by the three-term recurrences in x, y, z and r^2
//   R_00 = 1,
//   R_{l+1,l+1}^c = -sqrt((2l+1)/(2l+2)) (x R_ll^c - y R_ll^s),
//   R_{l+1,l+1}^s = -sqrt((2l+1)/(2l+2)) (y R_ll^c + x R_ll^s),
//   R_{l+1,m} = ((2l+1) z R_lm - sqrt((l+m)(l-m)) r^2 R_{l-1,m})
//               / sqrt((l+m+1)(l-m+1)),
// for which R_l0(u) R_l0(v) + 2 sum_{m>0} (R^c(u) R^c(v) + R^s(u) R^s(v)) =
// P_l(u.v): the weight C is 1 for m = 0 and 2 for m > 0.  Components of
// degree l >= 5 are stored from index l^2 - 1 on as m = 0, then (c, s) for
// m = 1..l.  The recurrence runs on the unit vector u (a homogeneous
// polynomial of degree l in its components, r^2 kept as x^2 + y^2 + z^2) with
// forward-mode dual numbers, which give its directional derivatives; B(d) =
// R(d) / |d|^l is homogeneous of degree 0, so its gradient is
// (grad R(u) - l R(u) u) / r (Euler's relation).
//
// Thread map: one warp per atom, persistent blocks of four warps.  A chunk of
// up to 32 of the atom's pairs is evaluated one pair per lane into the warp's
// shared memory; then each lane takes (n, q) components (or, in the
// c-gradient, (J, n, k) entries) and sums over the chunk's pairs in list
// order.  Every sum has a fixed order (no atomics).
#include "device_math.cuh"
#include "gnep_internal.h"
#include "shape.cuh"
#include "sweeps_lmax.cuh"

namespace gnep {

namespace {

constexpr int kHiWarps = 4;   // warps (atoms in flight) per block
constexpr int kHiChunk = 32;  // pairs per chunk (one per lane)
constexpr int kForcePairs = 10;  // pairs per round of the force sweep (three lanes each)

constexpr double csqrt(double x) {  // square root by Newton's method, for compile-time constants
  double r = x > 1.0 ? x : 1.0;
  for (int i = 0; i < 60; ++i) r = 0.5 * (r + x / r);
  return x > 0.0 ? r : 0.0;
}

// A value with its derivatives along K directions (K = 0: the value alone).
template <int K>
struct Dn {
  float v;
  float d[K > 0 ? K : 1];
};
template <int K>
__device__ __forceinline__ Dn<K> dn(float v) {
  Dn<K> r;
  r.v = v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = 0.f;
  return r;
}
template <int K>
__device__ __forceinline__ Dn<K> dn_mul(const Dn<K>& a, const Dn<K>& b) {
  Dn<K> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = fmaf(a.d[i], b.v, a.v * b.d[i]);
  return r;
}
// s a + t b
template <int K>
__device__ __forceinline__ Dn<K> dn_lin(float s, const Dn<K>& a, float t, const Dn<K>& b) {
  Dn<K> r;
  r.v = fmaf(s, a.v, t * b.v);
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = fmaf(s, a.d[i], t * b.d[i]);
  return r;
}

// The recurrence above, from l = 0 to LMAX; each component of degree l >= 5 is
// handed to emit(q, l, value) with q its index.
template <int LMAX, int K, class F>
__device__ __forceinline__ void solid_hi(const Dn<K>& x, const Dn<K>& y, const Dn<K>& z, F&& emit) {
  const Dn<K> r2 = dn_lin(1.f, dn_lin(1.f, dn_mul(x, x), 1.f, dn_mul(y, y)), 1.f, dn_mul(z, z));
  Dn<K> pc[LMAX + 2], ps[LMAX + 2], cc[LMAX + 2], cs[LMAX + 2];
#pragma unroll
  for (int m = 0; m < LMAX + 2; ++m) {
    pc[m] = dn<K>(0.f); ps[m] = dn<K>(0.f); cc[m] = dn<K>(0.f); cs[m] = dn<K>(0.f);
  }
  cc[0] = dn<K>(1.f);
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    Dn<K> nc[LMAX + 2], ns[LMAX + 2];
#pragma unroll
    for (int m = 0; m <= l; ++m) {
      const float b = (float)((2.0 * l + 1.0) / csqrt((double)((l + m + 1) * (l - m + 1))));
      const float a = (float)(csqrt((double)((l + m) * (l - m))) / csqrt((double)((l + m + 1) * (l - m + 1))));
      nc[m] = dn_lin(b, dn_mul(z, cc[m]), -a, dn_mul(r2, pc[m]));
      ns[m] = dn_lin(b, dn_mul(z, cs[m]), -a, dn_mul(r2, ps[m]));
    }
    const float f = -(float)csqrt((2.0 * l + 1.0) / (2.0 * l + 2.0));
    nc[l + 1] = dn_lin(f, dn_mul(x, cc[l]), -f, dn_mul(y, cs[l]));
    ns[l + 1] = dn_lin(f, dn_mul(y, cc[l]), f, dn_mul(x, cs[l]));
    if (l + 1 >= 5) {
      const int base = (l + 1) * (l + 1) - 1;
      emit(base, l + 1, nc[0]);
#pragma unroll
      for (int m = 1; m <= l + 1; ++m) {
        emit(base + 2 * m - 1, l + 1, nc[m]);
        emit(base + 2 * m, l + 1, ns[m]);
      }
    }
#pragma unroll
    for (int m = 0; m <= l + 1; ++m) {
      pc[m] = cc[m]; ps[m] = cs[m];
      cc[m] = nc[m]; cs[m] = ns[m];
    }
  }
}

// Weight C of component q and its degree l.
__device__ __forceinline__ int deg_of(int q) {
  if (q < NLM) return lm_l(q);
  int l = 5;
  while ((l + 1) * (l + 1) - 1 <= q) ++l;
  return l;
}
__device__ __forceinline__ float weight_of(int q) {
  if (q < NLM) return kClm[q];
  const int l = deg_of(q);
  return q == l * l - 1 ? 1.f : 2.f;
}

__device__ __forceinline__ float3 sym_apply3(const float* b, float3 r) {  // b = xx yy zz xy yz zx
  return make_float3(b[0] * r.x + b[3] * r.y + b[5] * r.z, b[3] * r.x + b[1] * r.y + b[4] * r.z,
                     b[5] * r.x + b[4] * r.y + b[2] * r.z);
}

// Per-warp shared memory: the chunk's per-pair rows and the atom's rows.
template <class C>
struct HiSm {
  static constexpr int NLP = C::NLX + 1;  // odd row length
  float B[kHiChunk][NLP];
  float D[kHiChunk][NLP];
  float g[kHiChunk][C::NQA];
  float ga[kHiChunk][C::NQA];
  float f[kHiChunk][C::KA];
  float fu[kHiChunk][C::KA];
  float A[C::NQA][C::NLX];
  float A2[C::NQA][C::NLX];
  int J[kHiChunk];
};

template <class C>
constexpr size_t hi_smem() {
  return kHiWarps * sizeof(HiSm<C>);
}
// The force sweep keeps only the atom's rows per warp.
template <class C>
struct HiForceSm {
  float A[C::NQA][C::NLX];
};
template <class C>
constexpr size_t hi_force_smem() {
  return kHiWarps * sizeof(HiForceSm<C>);
}

// ------------------------------------------------------------- sweep 1

template <class C>
__global__ void __launch_bounds__(32 * kHiWarps) k_desc_hi(int N, DevModel dm, const int* __restrict__ type,
                                                           const int* __restrict__ off, const float4* __restrict__ rij,
                                                           float* __restrict__ Sout, float* __restrict__ G) {
  GNEP_PDL_WAIT();
  constexpr int NQA = C::NQA, KA = C::KA, NLX = C::NLX, NE = NQA * NLX, NT = (NE + 31) / 32;
  extern __shared__ float4 smraw[];
  __shared__ float cA[C::NCA];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  HiSm<C>& sm = reinterpret_cast<HiSm<C>*>(smraw)[warp];
  for (int q = threadIdx.x; q < C::NCA; q += blockDim.x) cA[q] = dm.params[dm.off_cA + q];
  __syncthreads();
  for (int i = blockIdx.x * kHiWarps + warp; i < N; i += gridDim.x * kHiWarps) {
    const int I = type[i], p0 = off[i], p1 = off[i + 1];
    float acc[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) acc[t] = 0.f;
    for (int cs = p0; cs < p1; cs += kHiChunk) {
      const int p = cs + lane;
      if (p < p1) {
        const float4 r = rij[p];
        const int J = (int)r.w;
        const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z), ri = 1.f / rr;
        float f[KA];
        radial_basis<KA>(rr, dm.rca_inv, f);
        const float* c = cA + (I * C::NS + J) * NQA * KA;
#pragma unroll
        for (int n = 0; n < NQA; ++n) {
          float g = 0.f;
#pragma unroll
          for (int k = 0; k < KA; ++k) g = fmaf(c[n * KA + k], f[k], g);
          sm.g[lane][n] = g;
        }
        const float ux = r.x * ri, uy = r.y * ri, uz = r.z * ri;
        float Bl[NLM];
        harmonics(ux, uy, uz, Bl);
#pragma unroll
        for (int q = 0; q < NLM; ++q) sm.B[lane][q] = Bl[q];
        solid_hi<C::LMAX, 0>(dn<0>(ux), dn<0>(uy), dn<0>(uz),
                             [&](int q, int, const Dn<0>& h) { sm.B[lane][q] = h.v; });
      }
      __syncwarp();
      const int np = min(kHiChunk, p1 - cs);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int e = lane + 32 * t;
        if (e < NE) {
          const int n = e / NLX, q = e % NLX;
          float s = acc[t];
          for (int pp = 0; pp < np; ++pp) s = fmaf(sm.g[pp][n], sm.B[pp][q], s);  // Eq. 8
          acc[t] = s;
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int e = lane + 32 * t;
      if (e < NE) {
        sm.A[e / NLX][e % NLX] = acc[t];
        Sout[(size_t)i * NE + e] = acc[t];
      }
    }
    __syncwarp();
    float* gi = G + (size_t)i * C::NDES;
    for (int e = lane; e < NQA * C::LMAX; e += 32) {  // q_nl = sum_m C_lm S_nlm^2 (Eq. 7)
      const int n = e / C::LMAX, l = e % C::LMAX + 1, q0 = l * l - 1;
      float s = 0.f;
      for (int m = 0; m <= 2 * l; ++m) {
        const float v = sm.A[n][q0 + m];
        s = fmaf(weight_of(q0 + m), v * v, s);
      }
      gi[C::vang(n, l)] = s;
    }
    if (C::FB && lane < NQA) gi[C::v4b(lane)] = q4_value(&sm.A[lane][3]);
    __syncwarp();
  }
}

// ------------------------------------------------------------- sweep 2

// dE_i/dr_ij = sum_q [ghat'_q B_q u + ghat_q grad B_q], ghat_q = sum_n g_n Shat_nq,
// ghat'_q = sum_n g_n' Shat_nq, Shat_nq = dE_i/dS_nq = 2 C_q E'_{n l(q)} S_nq
// (+ E'_4b,n dq4/dS_n2m)  (C2.1, C2.3, C3.6).
template <class C>
__global__ void __launch_bounds__(32 * kHiWarps) k_force_hi(int N, DevModel dm, const int* __restrict__ type,
                                                            const int* __restrict__ off,
                                                            const float4* __restrict__ rij,
                                                            const float* __restrict__ S, const float* __restrict__ Ep,
                                                            float4* __restrict__ dA) {
  GNEP_PDL_WAIT();
  constexpr int NQA = C::NQA, KA = C::KA, NLX = C::NLX, NE = NQA * NLX;
  extern __shared__ float4 smraw[];
  __shared__ float cA[C::NCA];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  HiForceSm<C>& sm = reinterpret_cast<HiForceSm<C>*>(smraw)[warp];
  const int fslot = lane / 3, fdir = lane - 3 * fslot;  // pair slot and direction of this lane
  for (int q = threadIdx.x; q < C::NCA; q += blockDim.x) cA[q] = dm.params[dm.off_cA + q];
  __syncthreads();
  for (int i = blockIdx.x * kHiWarps + warp; i < N; i += gridDim.x * kHiWarps) {
    const int I = type[i], p0 = off[i], p1 = off[i + 1];
    const float* ep = Ep + (size_t)i * C::NDES;
    const float* Si = S + (size_t)i * NE;
    for (int e = lane; e < NE; e += 32) {
      const int n = e / NLX, q = e % NLX;
      sm.A[n][q] = 2.f * weight_of(q) * ep[C::vang(n, deg_of(q))] * Si[e];
    }
    __syncwarp();
    if (C::FB && lane < NQA) {
      float g4[5];
      q4_grad(Si + lane * NLX + 3, g4);
      const float e4 = ep[C::v4b(lane)];
#pragma unroll
      for (int m = 0; m < 5; ++m) sm.A[lane][3 + m] = fmaf(e4, g4[m], sm.A[lane][3 + m]);
    }
    __syncwarp();
    // Lane 3 s + e takes Cartesian direction e of the round's pair s (ten
    // pairs a round; an atom has about eight angular pairs, so a pair per
    // lane with the three directions in turn left most lanes idle).
    for (int pb = p0; pb < p1; pb += kForcePairs) {
      const int p = pb + fslot;
      const bool act = fslot < kForcePairs && p < p1;
      float P = 0.f, vd = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;
      if (act) {
        const float4 r = rij[p];
        const int J = (int)r.w;
        const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z), ri = 1.f / rr;
        ux = r.x * ri;
        uy = r.y * ri;
        uz = r.z * ri;
        float f[KA], fp[KA];
        radial_basis_d<KA>(rr, dm.rca_inv, f, fp);
        const float* c = cA + (I * C::NS + J) * NQA * KA;
        float g[NQA], gp[NQA];
#pragma unroll
        for (int n = 0; n < NQA; ++n) {
          float a1 = 0.f, a2 = 0.f;
#pragma unroll
          for (int k = 0; k < KA; ++k) {
            a1 = fmaf(c[n * KA + k], f[k], a1);
            a2 = fmaf(c[n * KA + k], fp[k], a2);
          }
          g[n] = a1;
          gp[n] = a2;
        }
        // direction e: D_q = grad B_q . e (the printed forms for l <= 4, the
        // recurrence with one dual component for l >= 5), V_e = sum_q ghat_q
        // D_q; direction 0 also forms P = sum_q ghat'_q B_q.
        const float ex = fdir == 0 ? 1.f : 0.f, ey = fdir == 1 ? 1.f : 0.f, ez = fdir == 2 ? 1.f : 0.f;
        const float ue = fdir == 0 ? ux : (fdir == 1 ? uy : uz);
        {
          float Bl[NLM], Dl[NLM];
          harmonics_dir(ux, uy, uz, ri, ex, ey, ez, Bl, Dl);
#pragma unroll
          for (int q = 0; q < NLM; ++q) {
            float gh = 0.f, ghp = 0.f;
#pragma unroll
            for (int n = 0; n < NQA; ++n) {
              gh = fmaf(g[n], sm.A[n][q], gh);
              ghp = fmaf(gp[n], sm.A[n][q], ghp);
            }
            vd = fmaf(gh, Dl[q], vd);
            if (fdir == 0) P = fmaf(ghp, Bl[q], P);
          }
        }
        Dn<1> X = dn<1>(ux), Y = dn<1>(uy), Z = dn<1>(uz);
        X.d[0] = ex; Y.d[0] = ey; Z.d[0] = ez;
        solid_hi<C::LMAX, 1>(X, Y, Z, [&](int q, int l, const Dn<1>& h) {
          float gh = 0.f, ghp = 0.f;
#pragma unroll
          for (int n = 0; n < NQA; ++n) {
            gh = fmaf(g[n], sm.A[n][q], gh);
            ghp = fmaf(gp[n], sm.A[n][q], ghp);
          }
          vd = fmaf(gh, (h.d[0] - (float)l * h.v * ue) * ri, vd);
          if (fdir == 0) P = fmaf(ghp, h.v, P);
        });
      }
      // directions 1 and 2 of the pair to its direction-0 lane
      const float v1 = __shfl_down_sync(0xffffffffu, vd, 1), v2 = __shfl_down_sync(0xffffffffu, vd, 2);
      if (act && fdir == 0) dA[p] = make_float4(P * ux + vd, P * uy + v1, P * uz + v2, 0.f);
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------- sweep 3

// Sdot_nq = sum_j [g_n'(r_ij) (u . w_ij) B_q + g_n(r_ij) D_q], D_q = grad B_q . w_ij,
// with the tangent direction w_ij = (a_j - a_i) + B_s r_ij (stored for sweep 4);
// qdot_nl = 2 sum_m C_q S_nq Sdot_nq and the 4-body tangent.
template <class C>
__global__ void __launch_bounds__(32 * kHiWarps) k_tangent_hi(int N, DevModel dm, const int* __restrict__ type,
                                                              const int* __restrict__ atom_struct,
                                                              const int* __restrict__ off, const int* __restrict__ jj,
                                                              const float4* __restrict__ rij,
                                                              const float4* __restrict__ a,
                                                              const float* __restrict__ Bs,
                                                              const float* __restrict__ Sin, float* __restrict__ Sout,
                                                              float* __restrict__ Gd, float4* __restrict__ wij) {
  GNEP_PDL_WAIT();
  constexpr int NQA = C::NQA, KA = C::KA, NLX = C::NLX, NE = NQA * NLX, NT = (NE + 31) / 32;
  extern __shared__ float4 smraw[];
  __shared__ float cA[C::NCA];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  HiSm<C>& sm = reinterpret_cast<HiSm<C>*>(smraw)[warp];
  for (int q = threadIdx.x; q < C::NCA; q += blockDim.x) cA[q] = dm.params[dm.off_cA + q];
  __syncthreads();
  for (int i = blockIdx.x * kHiWarps + warp; i < N; i += gridDim.x * kHiWarps) {
    const int I = type[i], p0 = off[i], p1 = off[i + 1];
    const float4 ai = a[i];
    float bs[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) bs[q] = Bs[6 * atom_struct[i] + q];
    float acc[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) acc[t] = 0.f;
    for (int cs = p0; cs < p1; cs += kHiChunk) {
      const int p = cs + lane;
      if (p < p1) {
        const float4 r = rij[p];
        const int J = (int)r.w;
        const float4 aj = a[jj[p]];
        const float3 br = sym_apply3(bs, make_float3(r.x, r.y, r.z));
        const float wx = aj.x - ai.x + br.x, wy = aj.y - ai.y + br.y, wz = aj.z - ai.z + br.z;
        wij[p] = make_float4(wx, wy, wz, 0.f);
        const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z), ri = 1.f / rr;
        const float ux = r.x * ri, uy = r.y * ri, uz = r.z * ri;
        const float ru = ux * wx + uy * wy + uz * wz;
        float f[KA], fp[KA];
        radial_basis_d<KA>(rr, dm.rca_inv, f, fp);
        const float* c = cA + (I * C::NS + J) * NQA * KA;
#pragma unroll
        for (int n = 0; n < NQA; ++n) {
          float a1 = 0.f, a2 = 0.f;
#pragma unroll
          for (int k = 0; k < KA; ++k) {
            a1 = fmaf(c[n * KA + k], f[k], a1);
            a2 = fmaf(c[n * KA + k], fp[k], a2);
          }
          sm.g[lane][n] = a1;
          sm.ga[lane][n] = a2 * ru;
        }
        {
          float Bl[NLM], Dl[NLM];
          harmonics_dir(ux, uy, uz, ri, wx, wy, wz, Bl, Dl);
#pragma unroll
          for (int q = 0; q < NLM; ++q) {
            sm.B[lane][q] = Bl[q];
            sm.D[lane][q] = Dl[q];
          }
        }
        Dn<1> X = dn<1>(ux), Y = dn<1>(uy), Z = dn<1>(uz);
        X.d[0] = wx; Y.d[0] = wy; Z.d[0] = wz;
        solid_hi<C::LMAX, 1>(X, Y, Z, [&](int q, int l, const Dn<1>& h) {
          sm.B[lane][q] = h.v;
          sm.D[lane][q] = (h.d[0] - (float)l * h.v * ru) * ri;
        });
      }
      __syncwarp();
      const int np = min(kHiChunk, p1 - cs);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int e = lane + 32 * t;
        if (e < NE) {
          const int n = e / NLX, q = e % NLX;
          float s = acc[t];
          for (int pp = 0; pp < np; ++pp) s = fmaf(sm.ga[pp][n], sm.B[pp][q], fmaf(sm.g[pp][n], sm.D[pp][q], s));
          acc[t] = s;
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int e = lane + 32 * t;
      if (e < NE) {
        sm.A[e / NLX][e % NLX] = acc[t];
        Sout[(size_t)i * NE + e] = acc[t];
      }
    }
    __syncwarp();
    const float* Si = Sin + (size_t)i * NE;
    float* gi = Gd + (size_t)i * C::NDES;
    for (int e = lane; e < NQA * C::LMAX; e += 32) {
      const int n = e / C::LMAX, l = e % C::LMAX + 1, q0 = l * l - 1;
      float s = 0.f;
      for (int m = 0; m <= 2 * l; ++m) s = fmaf(weight_of(q0 + m) * Si[n * NLX + q0 + m], sm.A[n][q0 + m], s);
      gi[C::vang(n, l)] = 2.f * s;
    }
    if (C::FB && lane < NQA) {
      float g4[5];
      q4_grad(Si + lane * NLX + 3, g4);
      float s = 0.f;
#pragma unroll
      for (int m = 0; m < 5; ++m) s = fmaf(g4[m], sm.A[lane][3 + m], s);
      gi[C::v4b(lane)] = s;
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------- sweep 4

// dL/dc^A_nk^{IJ} += P_n f_k + R_n fu_k per pair, with
//   P_n = sum_q Sbar_nq B_q + Sdbar_nq D_q,  R_n = sum_q Sdbar_nq B_q,
//   Sbar_nq = 2 C_q (Gbar_nl S_nq - E'_nl Sdot_nq) (+ 4-body terms),
//   Sdbar_nq = -2 C_q E'_nl S_nq (+ 4-body term),  fu_k = f_k' (u . w_ij).
// Each block writes its partial of the angular coefficients once.
template <class C>
__global__ void __launch_bounds__(32 * kHiWarps) k_cgrad_hi(int N, DevModel dm, const int* __restrict__ type,
                                                            const int* __restrict__ off,
                                                            const float4* __restrict__ rij,
                                                            const float4* __restrict__ wij,
                                                            const float* __restrict__ S, const float* __restrict__ Sd,
                                                            const float* __restrict__ Gb,
                                                            const float* __restrict__ Ep, float* __restrict__ cpart) {
  GNEP_PDL_WAIT();
  constexpr int NQA = C::NQA, KA = C::KA, NS = C::NS, NLX = C::NLX, NE = NQA * NLX;
  constexpr int NEA = NS * NQA * KA, NTA = (NEA + 31) / 32;  // (J, n, k) entries of one species I
  extern __shared__ float4 smraw[];
  __shared__ float red[kHiWarps][C::NCA];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  HiSm<C>& sm = reinterpret_cast<HiSm<C>*>(smraw)[warp];
  float acc[NS][NTA];
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int t = 0; t < NTA; ++t) acc[s][t] = 0.f;
  for (int i = blockIdx.x * kHiWarps + warp; i < N; i += gridDim.x * kHiWarps) {
    const int I = type[i], p0 = off[i], p1 = off[i + 1];
    const float* Si = S + (size_t)i * NE;
    const float* Di = Sd + (size_t)i * NE;
    const float* gb = Gb + (size_t)i * C::NDES;
    const float* ep = Ep + (size_t)i * C::NDES;
    for (int e = lane; e < NE; e += 32) {
      const int n = e / NLX, q = e % NLX, v = C::vang(n, deg_of(q));
      const float c2 = 2.f * weight_of(q);
      sm.A[n][q] = c2 * (gb[v] * Si[e] - ep[v] * Di[e]);
      sm.A2[n][q] = -c2 * ep[v] * Si[e];
    }
    __syncwarp();
    if (C::FB && lane < NQA) {
      float g4[5], h4[5];
      q4_grad(Si + lane * NLX + 3, g4);
      q4_hvp(Si + lane * NLX + 3, Di + lane * NLX + 3, h4);
      const float gb4 = gb[C::v4b(lane)], ep4 = ep[C::v4b(lane)];
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        sm.A[lane][3 + m] += gb4 * g4[m] - ep4 * h4[m];
        sm.A2[lane][3 + m] -= ep4 * g4[m];
      }
    }
    __syncwarp();
    for (int cs = p0; cs < p1; cs += kHiChunk) {
      const int p = cs + lane;
      if (p < p1) {
        const float4 r = rij[p], w = wij[p];
        const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z), ri = 1.f / rr;
        const float ux = r.x * ri, uy = r.y * ri, uz = r.z * ri;
        const float ru = ux * w.x + uy * w.y + uz * w.z;
        float f[KA], fp[KA];
        radial_basis_d<KA>(rr, dm.rca_inv, f, fp);
#pragma unroll
        for (int k = 0; k < KA; ++k) {
          sm.f[lane][k] = f[k];
          sm.fu[lane][k] = fp[k] * ru;
        }
        sm.J[lane] = (int)r.w;
        float P[NQA], R[NQA];
#pragma unroll
        for (int n = 0; n < NQA; ++n) P[n] = R[n] = 0.f;
        {
          float Bl[NLM], Dl[NLM];
          harmonics_dir(ux, uy, uz, ri, w.x, w.y, w.z, Bl, Dl);
#pragma unroll
          for (int q = 0; q < NLM; ++q)
#pragma unroll
            for (int n = 0; n < NQA; ++n) {
              P[n] = fmaf(sm.A[n][q], Bl[q], fmaf(sm.A2[n][q], Dl[q], P[n]));
              R[n] = fmaf(sm.A2[n][q], Bl[q], R[n]);
            }
        }
        Dn<1> X = dn<1>(ux), Y = dn<1>(uy), Z = dn<1>(uz);
        X.d[0] = w.x; Y.d[0] = w.y; Z.d[0] = w.z;
        solid_hi<C::LMAX, 1>(X, Y, Z, [&](int q, int l, const Dn<1>& h) {
          const float Bq = h.v, Dq = (h.d[0] - (float)l * h.v * ru) * ri;
#pragma unroll
          for (int n = 0; n < NQA; ++n) {
            P[n] = fmaf(sm.A[n][q], Bq, fmaf(sm.A2[n][q], Dq, P[n]));
            R[n] = fmaf(sm.A2[n][q], Bq, R[n]);
          }
        });
#pragma unroll
        for (int n = 0; n < NQA; ++n) {
          sm.g[lane][n] = P[n];
          sm.ga[lane][n] = R[n];
        }
      }
      __syncwarp();
      const int np = min(kHiChunk, p1 - cs);
#pragma unroll
      for (int t = 0; t < NTA; ++t) {
        const int e = lane + 32 * t;
        if (e < NEA) {
          const int J = e / (NQA * KA), n = (e / KA) % NQA, k = e % KA;
          float s = 0.f;
          for (int pp = 0; pp < np; ++pp)
            if (sm.J[pp] == J) s = fmaf(sm.g[pp][n], sm.f[pp][k], fmaf(sm.ga[pp][n], sm.fu[pp][k], s));
#pragma unroll
          for (int s2 = 0; s2 < NS; ++s2) acc[s2][t] += (s2 == I) ? s : 0.f;
        }
      }
      __syncwarp();
    }
  }
  // fold the warps in order; layout c^A[I][J][n][k]
#pragma unroll
  for (int s2 = 0; s2 < NS; ++s2)
#pragma unroll
    for (int t = 0; t < NTA; ++t) {
      const int e = lane + 32 * t;
      if (e < NEA) red[warp][s2 * NEA + e] = acc[s2][t];
    }
  __syncthreads();
  for (int q = threadIdx.x; q < C::NCA; q += blockDim.x) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < kHiWarps; ++w) v += red[w][q];
    cpart[(size_t)blockIdx.x * (C::NCR + C::NCA) + C::NCR + q] = v;
  }
}

int hi_grid(int n) {
  const int b = (n + kHiWarps - 1) / kHiWarps;
  return b < 1 ? 1 : (b > 4096 ? 4096 : b);
}

}  // namespace

// ------------------------------------------------------------- launchers

template <class C>
int hi_setup() {
  const int sm = (int)hi_smem<C>();
  GNEP_CUDA(cudaFuncSetAttribute(k_desc_hi<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  GNEP_CUDA(cudaFuncSetAttribute(k_force_hi<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hi_force_smem<C>()));
  GNEP_CUDA(cudaFuncSetAttribute(k_tangent_hi<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  GNEP_CUDA(cudaFuncSetAttribute(k_cgrad_hi<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  return GNEP_OK;
}

template <class C>
int hi_desc_angular(const gnep_model* m, const gnep_nlist* nl, cudaStream_t st, float* S, float* G) {
  const int N = nl->n_atoms;
  if (N == 0) return GNEP_OK;
  (void)launch_pdl(k_desc_hi<C>, hi_grid(N), 32 * kHiWarps, hi_smem<C>(), st, N, m->dev(), nl->type, nl->L[1].off, nl->L[1].rij,
                                                                S, G);
  GNEP_CHECK_LAUNCH("k_desc_hi");
  return GNEP_OK;
}

template <class C>
int hi_force_angular(const gnep_model* m, const gnep_nlist* nl, cudaStream_t st, const float* S, const float* Ep,
                     float4* dA) {
  const int N = nl->n_atoms;
  if (N == 0 || nl->L[1].n == 0) return GNEP_OK;
  (void)launch_pdl(k_force_hi<C>, hi_grid(N), 32 * kHiWarps, hi_force_smem<C>(), st, N, m->dev(), nl->type, nl->L[1].off,
                                                                 nl->L[1].rij, S, Ep, dA);
  GNEP_CHECK_LAUNCH("k_force_hi");
  return GNEP_OK;
}

template <class C>
int hi_tangent_angular(const gnep_model* m, const gnep_nlist* nl, cudaStream_t st, const float4* a, const float* Bs,
                       const float* S, float* Sd, float* Gd, float4* wij) {
  const int N = nl->n_atoms;
  if (N == 0) return GNEP_OK;
  (void)launch_pdl(k_tangent_hi<C>, hi_grid(N), 32 * kHiWarps, hi_smem<C>(), st, N, m->dev(), nl->type, nl->atom_struct,
                                                                   nl->L[1].off, nl->L[1].j, nl->L[1].rij, a, Bs, S,
                                                                   Sd, Gd, wij);
  GNEP_CHECK_LAUNCH("k_tangent_hi");
  return GNEP_OK;
}

template <class C>
int hi_cgrad_angular(const gnep_model* m, const gnep_nlist* nl, cudaStream_t st, int nb, const float4* wij,
                     const float* S, const float* Sd, const float* Gb, const float* Ep, float* cpart) {
  (void)launch_pdl(k_cgrad_hi<C>, nb, 32 * kHiWarps, hi_smem<C>(), st, nl->n_atoms, m->dev(), nl->type, nl->L[1].off,
                                                          nl->L[1].rij, wij, S, Sd, Gb, Ep, cpart);
  GNEP_CHECK_LAUNCH("k_cgrad_hi");
  return GNEP_OK;
}

// Shapes with l_max > 4 (species, n_max+1, basis+1 radial; same angular; 4-body; l_max).
#define GNEP_HI(NS, NQR, KR, NQA, KA, FB, LM)                                                                   \
  template int hi_setup<Sh<NS, NQR, KR, NQA, KA, FB, LM>>();                                                  \
  template int hi_desc_angular<Sh<NS, NQR, KR, NQA, KA, FB, LM>>(const gnep_model*, const gnep_nlist*,        \
                                                                 cudaStream_t, float*, float*);               \
  template int hi_force_angular<Sh<NS, NQR, KR, NQA, KA, FB, LM>>(const gnep_model*, const gnep_nlist*,       \
                                                                  cudaStream_t, const float*, const float*,   \
                                                                  float4*);                                   \
  template int hi_tangent_angular<Sh<NS, NQR, KR, NQA, KA, FB, LM>>(                                          \
      const gnep_model*, const gnep_nlist*, cudaStream_t, const float4*, const float*, const float*, float*,  \
      float*, float4*);                                                                                       \
  template int hi_cgrad_angular<Sh<NS, NQR, KR, NQA, KA, FB, LM>>(const gnep_model*, const gnep_nlist*,       \
                                                                  cudaStream_t, int, const float4*,           \
                                                                  const float*, const float*, const float*,   \
                                                                  const float*, float*);
GNEP_HI(2, 5, 9, 5, 9, false, 6)
GNEP_HI(2, 5, 9, 5, 9, true, 8)
#undef GNEP_HI

}  // namespace gnep
