// Shape-specialised sweeps of one training step over a packed batch.
//
//   sweep 1  descriptors  q_n (Eqs. 5-6), S_nlm and q_nl (Eqs. 7-8), 4-body q4_n
//   network  E_i = F(s.G_i) (D1.1) with E'_i = dE_i/dG_i (D1.5)
//   sweep 2  dE_i/dr_ij (C3.6) per pair, forces (Eq. 3), per-atom virial (Eq. 4)
//   sweep 3  tangent  Gdot_i = sum_j dG_i/dr_ij . u_ij
//   network  tangent and reverse pass, adjoints Gbar_i
//   sweep 4  per-atom contributions to dL/dc^A
//
// Gradient route.  With a_i = dL/dF_i and B_s = dL/dW_s held fixed (Eqs. 11-12),
//   sum_i a_i.F_i + sum_s B_s:W_s = - sum_i sum_j u_ij . dE_i/dr_ij,
//   u_ij = (a_j - a_i) + B_s r_ij,
// because F_i = sum_j (dE_i/dr_ij - dE_j/dr_ji) (Eq. 3) and W_s = -sum r_ij (x) dE_i/dr_ij
// (Eq. 4 summed).  Hence the force and virial parts of dL/dtheta (Eqs. 15-16 with
// the mixed derivatives of App. C3 and D1.11-D1.17) equal -d/dtheta sum_i E'_i.Gdot_i:
// one forward-mode sweep (3) and one reverse sweep (4) instead of explicit second
// derivative tensors.
#include <cstdio>
#include <mutex>
#include <string>

#include "device_math.cuh"
#include "gnep_internal.h"

namespace gnep {

template <int NS_, int NQR_, int KR_, int NQA_, int KA_, bool FB_>
struct Sh {
  static constexpr int NS = NS_, NQR = NQR_, KR = KR_, NQA = NQA_, KA = KA_;
  static constexpr bool FB = FB_;
  static constexpr int NDES = NQR + NQA * 4 + (FB ? NQA : 0);
  __host__ __device__ static constexpr int vang(int n, int l) { return NQR + n * 4 + (l - 1); }
  __host__ __device__ static constexpr int v4b(int n) { return NQR + NQA * 4 + n; }
  static constexpr int NCR = NS * NS * NQR * KR;
  static constexpr int NCA = NS * NS * NQA * KA;
};

namespace {

// Accumulate v into row J of acc[NS][K] without dynamic register indexing.
template <int NS, int K>
__device__ __forceinline__ void acc_row(float (&acc)[NS][K], int J, const float (&v)[K], float w) {
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const float ws = (s == J) ? w : 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) acc[s][k] = fmaf(ws, v[k], acc[s][k]);
  }
}

template <int NS, int K>
__device__ __forceinline__ float dot_row(const float (&c)[NS][K], int J, const float (&v)[K]) {
  float r = 0.f;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) t = fmaf(c[s][k], v[k], t);
    r = (s == J) ? t : r;
  }
  return r;
}

__device__ __forceinline__ float3 sym_apply(const float* b, float3 r) {  // b = xx yy zz xy yz zx
  return make_float3(b[0] * r.x + b[3] * r.y + b[5] * r.z, b[3] * r.x + b[1] * r.y + b[4] * r.z,
                     b[5] * r.x + b[4] * r.y + b[2] * r.z);
}

// ------------------------------------------------------------- sweep 1

template <class C>
__global__ void __launch_bounds__(128) k_desc_radial(int N, DevModel dm, const int* __restrict__ type,
                                                     const int* __restrict__ off, const float4* __restrict__ rij,
                                                     float* __restrict__ FR, float* __restrict__ G) {
  __shared__ float cR[C::NCR];
  for (int q = threadIdx.x; q < C::NCR; q += blockDim.x) cR[q] = dm.params[dm.off_cR + q];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  float acc[C::NS][C::KR];
#pragma unroll
  for (int s = 0; s < C::NS; ++s)
#pragma unroll
    for (int k = 0; k < C::KR; ++k) acc[s][k] = 0.f;
  const int p1 = off[i + 1];
  for (int p = off[i]; p < p1; ++p) {
    const float4 r = rij[p];
    const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
    float f[C::KR];
    radial_basis<C::KR>(rr, dm.rcr_inv, f);
    acc_row<C::NS, C::KR>(acc, (int)r.w, f, 1.f);
  }
  float* fr = FR + (size_t)i * C::NS * C::KR;
#pragma unroll
  for (int s = 0; s < C::NS; ++s)
#pragma unroll
    for (int k = 0; k < C::KR; ++k) fr[s * C::KR + k] = acc[s][k];
  const int I = type[i];
  // q_n = sum_J sum_k c^R_nk^{IJ} sum_{j in J} f_k(r_ij)   (Eqs. 5-6)
#pragma unroll
  for (int n = 0; n < C::NQR; ++n) {
    float q = 0.f;
#pragma unroll
    for (int s = 0; s < C::NS; ++s)
#pragma unroll
      for (int k = 0; k < C::KR; ++k) q = fmaf(cR[((I * C::NS + s) * C::NQR + n) * C::KR + k], acc[s][k], q);
    G[(size_t)i * C::NDES + n] = q;
  }
}

template <class C>
__global__ void __launch_bounds__(128) k_desc_angular(int N, DevModel dm, const int* __restrict__ type,
                                                      const int* __restrict__ off, const float4* __restrict__ rij,
                                                      float* __restrict__ Sout, float* __restrict__ G) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t / C::NQA, n = t - i * C::NQA;
  if (i >= N) return;
  const int I = type[i];
  float c[C::NS][C::KA];
#pragma unroll
  for (int s = 0; s < C::NS; ++s)
#pragma unroll
    for (int k = 0; k < C::KA; ++k) c[s][k] = dm.params[dm.off_cA + ((I * C::NS + s) * C::NQA + n) * C::KA + k];
  float S[NLM];
#pragma unroll
  for (int q = 0; q < NLM; ++q) S[q] = 0.f;
  const int p1 = off[i + 1];
  for (int p = off[i]; p < p1; ++p) {
    const float4 r = rij[p];
    const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
    const float ri = 1.f / rr;
    float f[C::KA];
    radial_basis<C::KA>(rr, dm.rca_inv, f);
    const float g = dot_row<C::NS, C::KA>(c, (int)r.w, f);  // Eq. 6
    float B[NLM];
    harmonics(r.x * ri, r.y * ri, r.z * ri, B);
#pragma unroll
    for (int q = 0; q < NLM; ++q) S[q] = fmaf(g, B[q], S[q]);  // Eq. 8
  }
  float* so = Sout + ((size_t)i * C::NQA + n) * NLM;
#pragma unroll
  for (int q = 0; q < NLM; ++q) so[q] = S[q];
  float* gi = G + (size_t)i * C::NDES;
#pragma unroll
  for (int l = 1; l <= 4; ++l) {
    float q = 0.f;  // Eq. 7
#pragma unroll
    for (int lm = l * l - 1; lm < (l + 1) * (l + 1) - 1; ++lm) q = fmaf(kClm[lm] * S[lm], S[lm], q);
    gi[C::vang(n, l)] = q;
  }
  if (C::FB) gi[C::v4b(n)] = q4_value(&S[3]);
}

// ------------------------------------------------------------- network

// Network forward per atom (D1.1-D1.5): z = W0 (s.G) + b0, x = tanh z,
// E = w1.x + b1, E' = s . (W0^T (w1 (1 - x^2))).  Weights of all species in smem.
template <class C>
__global__ void __launch_bounds__(128) k_mlp_fwd(int N, DevModel dm, const int* __restrict__ type,
                                                 const float* __restrict__ G, float* __restrict__ X,
                                                 float* __restrict__ Ep, float* __restrict__ Eatom) {
  extern __shared__ float sm[];
  const int H = dm.H;
  for (int q = threadIdx.x; q < C::NS * dm.net_size; q += blockDim.x) sm[q] = dm.params[q];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int e = type[i];
  const float* W0 = sm + e * dm.net_size;
  const float* b0 = W0 + C::NDES * H;
  const float* w1 = b0 + H;
  float g[C::NDES], ep[C::NDES];
#pragma unroll
  for (int v = 0; v < C::NDES; ++v) {
    g[v] = dm.scale[v] * G[(size_t)i * C::NDES + v];
    ep[v] = 0.f;
  }
  float E = w1[H];
  for (int mu = 0; mu < H; ++mu) {
    const float* w = W0 + mu * C::NDES;
    float z = b0[mu];
#pragma unroll
    for (int v = 0; v < C::NDES; ++v) z = fmaf(w[v], g[v], z);
    const float x = tanhf(z);
    X[(size_t)i * H + mu] = x;
    E = fmaf(w1[mu], x, E);
    const float beta = w1[mu] * (1.f - x * x);
#pragma unroll
    for (int v = 0; v < C::NDES; ++v) ep[v] = fmaf(beta, w[v], ep[v]);
  }
#pragma unroll
  for (int v = 0; v < C::NDES; ++v) Ep[(size_t)i * C::NDES + v] = ep[v] * dm.scale[v];
  Eatom[i] = E;
}

// ------------------------------------------------------------- sweep 2

// dE_i/dS_nlm = E'_nl 2 C_lm S_nlm (+ E'_4b,n dq4/dS_n2m), one thread per (atom, n).
template <class C>
__global__ void __launch_bounds__(128) k_shat(int N, const float* __restrict__ Sang, const float* __restrict__ Ep,
                                              float* __restrict__ Shat) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t / C::NQA, n = t - i * C::NQA;
  if (i >= N) return;
  const float* S = Sang + ((size_t)i * C::NQA + n) * NLM;
  const float* ep = Ep + (size_t)i * C::NDES;
  float* o = Shat + ((size_t)i * C::NQA + n) * NLM;
  float s[NLM];
#pragma unroll
  for (int q = 0; q < NLM; ++q) s[q] = S[q];
#pragma unroll
  for (int lm = 0; lm < NLM; ++lm) o[lm] = 2.f * kClm[lm] * ep[C::vang(n, lm_l(lm))] * s[lm];
  if (C::FB) {
    float g4[5];
    q4_grad(&s[3], g4);
    const float e4 = ep[C::v4b(n)];
#pragma unroll
    for (int m = 0; m < 5; ++m) o[3 + m] = fmaf(e4, g4[m], o[3 + m]);
  }
}

// Radial pairs: dE_i/dr_ij = (sum_k chat_k^J f_k'(r)) r_ij / r with the per-atom
// contraction chat_k^J = sum_n E'_n c^R_nk^{IJ}  (C1.1, C3.6).
template <class C>
__global__ void __launch_bounds__(128) k_force_radial(int N, DevModel dm, const int* __restrict__ type,
                                                      const int* __restrict__ off, const float4* __restrict__ rij,
                                                      const float* __restrict__ Ep, float4* __restrict__ dR) {
  __shared__ float cR[C::NCR];
  for (int q = threadIdx.x; q < C::NCR; q += blockDim.x) cR[q] = dm.params[dm.off_cR + q];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int I = type[i];
  float ch[C::NS][C::KR];
#pragma unroll
  for (int s = 0; s < C::NS; ++s)
#pragma unroll
    for (int k = 0; k < C::KR; ++k) ch[s][k] = 0.f;
#pragma unroll
  for (int n = 0; n < C::NQR; ++n) {
    const float e = Ep[(size_t)i * C::NDES + n];
#pragma unroll
    for (int s = 0; s < C::NS; ++s)
#pragma unroll
      for (int k = 0; k < C::KR; ++k) ch[s][k] = fmaf(e, cR[((I * C::NS + s) * C::NQR + n) * C::KR + k], ch[s][k]);
  }
  const int p1 = off[i + 1];
  for (int p = off[i]; p < p1; ++p) {
    const float4 r = rij[p];
    const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
    float f[C::KR], fp[C::KR];
    radial_basis_d<C::KR>(rr, dm.rcr_inv, f, fp);
    const float ds = dot_row<C::NS, C::KR>(ch, (int)r.w, fp) / rr;
    dR[p] = make_float4(ds * r.x, ds * r.y, ds * r.z, 0.f);
  }
}

// Angular pairs, one thread per pair: dE_i/dr_ij = sum_n [g_n' (Shat_n . B) u + g_n Shat_n . grad B]
// (C2.1, C2.3, C3.6 and the 4-body term through Shat).
template <class C>
__global__ void __launch_bounds__(128) k_force_angular(int64_t P, DevModel dm, const int* __restrict__ type,
                                                       const int* __restrict__ own, const float4* __restrict__ rij,
                                                       const float* __restrict__ Shat, float4* __restrict__ dA) {
  __shared__ float cA[C::NCA];
  for (int q = threadIdx.x; q < C::NCA; q += blockDim.x) cA[q] = dm.params[dm.off_cA + q];
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int i = own[p];
  const int I = type[i];
  const float4 r = rij[p];
  const int J = (int)r.w;
  const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
  const float ri = 1.f / rr;
  const float ux = r.x * ri, uy = r.y * ri, uz = r.z * ri;
  float f[C::KA], fp[C::KA];
  radial_basis_d<C::KA>(rr, dm.rca_inv, f, fp);
  float B[NLM], gx[NLM], gy[NLM], gz[NLM];
  harmonics_grad(ux, uy, uz, ri, B, gx, gy, gz);
  const float* cIJ = cA + (I * C::NS + J) * C::NQA * C::KA;
  float dx = 0.f, dy = 0.f, dz = 0.f;
  for (int n = 0; n < C::NQA; ++n) {
    float g = 0.f, gp = 0.f;
#pragma unroll
    for (int k = 0; k < C::KA; ++k) {
      g = fmaf(cIJ[n * C::KA + k], f[k], g);
      gp = fmaf(cIJ[n * C::KA + k], fp[k], gp);
    }
    const float* sh = Shat + ((size_t)i * C::NQA + n) * NLM;
    float pb = 0.f, vx = 0.f, vy = 0.f, vz = 0.f;
#pragma unroll
    for (int q = 0; q < NLM; ++q) {
      const float s = sh[q];
      pb = fmaf(s, B[q], pb);
      vx = fmaf(s, gx[q], vx);
      vy = fmaf(s, gy[q], vy);
      vz = fmaf(s, gz[q], vz);
    }
    const float a = gp * pb;
    dx += a * ux + g * vx;
    dy += a * uy + g * vy;
    dz += a * uz + g * vz;
  }
  dA[p] = make_float4(dx, dy, dz, 0.f);
}

}  // namespace

// F_i = sum_j (d_ij - d_{rev(ij)}) over both lists (Eq. 3); per-atom virial
// -sum_j r_ij (x) d_ij, symmetrised (Eq. 4 summed over atoms gives the total).
__global__ void __launch_bounds__(128) k_force_gather(int N, const int* __restrict__ offR, const int* __restrict__ revR,
                                                      const float4* __restrict__ rijR, const float4* __restrict__ dR,
                                                      const int* __restrict__ offA, const int* __restrict__ revA,
                                                      const float4* __restrict__ rijA, const float4* __restrict__ dA,
                                                      float* __restrict__ F, float* __restrict__ Wat) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  float fx = 0.f, fy = 0.f, fz = 0.f;
  float w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int L = 0; L < 2; ++L) {
    const int* off = L ? offA : offR;
    const int* rev = L ? revA : revR;
    const float4* rij = L ? rijA : rijR;
    const float4* d = L ? dA : dR;
    const int p1 = off[i + 1];
    for (int p = off[i]; p < p1; ++p) {
      const float4 a = d[p], b = d[rev[p]], r = rij[p];
      fx += a.x - b.x;
      fy += a.y - b.y;
      fz += a.z - b.z;
      w[0] -= r.x * a.x;
      w[1] -= r.y * a.y;
      w[2] -= r.z * a.z;
      w[3] -= 0.5f * (r.x * a.y + r.y * a.x);
      w[4] -= 0.5f * (r.y * a.z + r.z * a.y);
      w[5] -= 0.5f * (r.z * a.x + r.x * a.z);
    }
  }
  F[3 * (size_t)i] = fx;
  F[3 * (size_t)i + 1] = fy;
  F[3 * (size_t)i + 2] = fz;
#pragma unroll
  for (int q = 0; q < 6; ++q) Wat[6 * (size_t)i + q] = w[q];
}

// E_s = sum_i E_i and W_s = sum_i w_i in FP64, one block per structure.
__global__ void __launch_bounds__(128) k_struct_sum(const int* __restrict__ soff, const float* __restrict__ Eatom,
                                                    const float* __restrict__ Wat, double* __restrict__ Es,
                                                    double* __restrict__ Ws) {
  const int s = blockIdx.x;
  const int a0 = soff[s], a1 = soff[s + 1];
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int i = a0 + threadIdx.x; i < a1; i += blockDim.x) {
    acc[0] += Eatom[i];
#pragma unroll
    for (int q = 0; q < 6; ++q) acc[1 + q] += Wat[6 * (size_t)i + q];
  }
  __shared__ double sh[7][128];
#pragma unroll
  for (int q = 0; q < 7; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int q = 0; q < 7; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    Es[s] = sh[0][0];
#pragma unroll
    for (int q = 0; q < 6; ++q) Ws[6 * s + q] = sh[1 + q][0];
  }
}

namespace {

// ------------------------------------------------------------- sweep 3

// Radial tangent: qdot_n = sum_J sum_k c^R_nk^{IJ} sum_{j in J} f_k'(r_ij) (u_hat . u_ij).
template <class C>
__global__ void __launch_bounds__(128) k_tangent_radial(int N, DevModel dm, const int* __restrict__ type,
                                                        const int* __restrict__ atom_struct, const int* __restrict__ off,
                                                        const int* __restrict__ jj, const float4* __restrict__ rij,
                                                        const float4* __restrict__ a, const float* __restrict__ Bs,
                                                        float* __restrict__ FRd, float* __restrict__ Gd) {
  __shared__ float cR[C::NCR];
  for (int q = threadIdx.x; q < C::NCR; q += blockDim.x) cR[q] = dm.params[dm.off_cR + q];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float4 ai = a[i];
  float b[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) b[q] = Bs[6 * atom_struct[i] + q];
  float acc[C::NS][C::KR];
#pragma unroll
  for (int s = 0; s < C::NS; ++s)
#pragma unroll
    for (int k = 0; k < C::KR; ++k) acc[s][k] = 0.f;
  const int p1 = off[i + 1];
  for (int p = off[i]; p < p1; ++p) {
    const float4 r = rij[p];
    const float4 aj = a[jj[p]];
    const float3 br = sym_apply(b, make_float3(r.x, r.y, r.z));
    const float ux = aj.x - ai.x + br.x, uy = aj.y - ai.y + br.y, uz = aj.z - ai.z + br.z;
    const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
    const float ru = (r.x * ux + r.y * uy + r.z * uz) / rr;
    float f[C::KR], fp[C::KR];
    radial_basis_d<C::KR>(rr, dm.rcr_inv, f, fp);
    acc_row<C::NS, C::KR>(acc, (int)r.w, fp, ru);
  }
  float* fr = FRd + (size_t)i * C::NS * C::KR;
#pragma unroll
  for (int s = 0; s < C::NS; ++s)
#pragma unroll
    for (int k = 0; k < C::KR; ++k) fr[s * C::KR + k] = acc[s][k];
  const int I = type[i];
#pragma unroll
  for (int n = 0; n < C::NQR; ++n) {
    float q = 0.f;
#pragma unroll
    for (int s = 0; s < C::NS; ++s)
#pragma unroll
      for (int k = 0; k < C::KR; ++k) q = fmaf(cR[((I * C::NS + s) * C::NQR + n) * C::KR + k], acc[s][k], q);
    Gd[(size_t)i * C::NDES + n] = q;
  }
}

// Angular tangent, one thread per (atom, n):
// Sdot_nlm = sum_j [g_n' (u_hat . u) B_lm + g_n grad B_lm . u],
// qdot_nl = 2 sum_m C_lm S_nlm Sdot_nlm, qdot4_n = dq4/dS . Sdot.
template <class C>
__global__ void __launch_bounds__(128) k_tangent_angular(int N, DevModel dm, const int* __restrict__ type,
                                                         const int* __restrict__ atom_struct, const int* __restrict__ off,
                                                         const int* __restrict__ jj, const float4* __restrict__ rij,
                                                         const float4* __restrict__ a, const float* __restrict__ Bs,
                                                         const float* __restrict__ Sang, float* __restrict__ Sd,
                                                         float* __restrict__ Gd) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t / C::NQA, n = t - i * C::NQA;
  if (i >= N) return;
  const int I = type[i];
  float c[C::NS][C::KA];
#pragma unroll
  for (int s = 0; s < C::NS; ++s)
#pragma unroll
    for (int k = 0; k < C::KA; ++k) c[s][k] = dm.params[dm.off_cA + ((I * C::NS + s) * C::NQA + n) * C::KA + k];
  const float4 ai = a[i];
  float b[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) b[q] = Bs[6 * atom_struct[i] + q];
  float sd[NLM];
#pragma unroll
  for (int q = 0; q < NLM; ++q) sd[q] = 0.f;
  const int p1 = off[i + 1];
  for (int p = off[i]; p < p1; ++p) {
    const float4 r = rij[p];
    const float4 aj = a[jj[p]];
    const float3 br = sym_apply(b, make_float3(r.x, r.y, r.z));
    const float vx = aj.x - ai.x + br.x, vy = aj.y - ai.y + br.y, vz = aj.z - ai.z + br.z;
    const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
    const float ri = 1.f / rr;
    const float ux = r.x * ri, uy = r.y * ri, uz = r.z * ri;
    float f[C::KA], fp[C::KA];
    radial_basis_d<C::KA>(rr, dm.rca_inv, f, fp);
    float g = 0.f, gp = 0.f;
    {
      const int J = (int)r.w;
#pragma unroll
      for (int s = 0; s < C::NS; ++s) {
        float tg = 0.f, tp = 0.f;
#pragma unroll
        for (int k = 0; k < C::KA; ++k) {
          tg = fmaf(c[s][k], f[k], tg);
          tp = fmaf(c[s][k], fp[k], tp);
        }
        g = (s == J) ? tg : g;
        gp = (s == J) ? tp : gp;
      }
    }
    float B[NLM], gx[NLM], gy[NLM], gz[NLM];
    harmonics_grad(ux, uy, uz, ri, B, gx, gy, gz);
    const float a1 = gp * (ux * vx + uy * vy + uz * vz);
#pragma unroll
    for (int q = 0; q < NLM; ++q) sd[q] += a1 * B[q] + g * (gx[q] * vx + gy[q] * vy + gz[q] * vz);
  }
  float* so = Sd + ((size_t)i * C::NQA + n) * NLM;
#pragma unroll
  for (int q = 0; q < NLM; ++q) so[q] = sd[q];
  const float* S = Sang + ((size_t)i * C::NQA + n) * NLM;
  float s[NLM];
#pragma unroll
  for (int q = 0; q < NLM; ++q) s[q] = S[q];
  float* gi = Gd + (size_t)i * C::NDES;
#pragma unroll
  for (int l = 1; l <= 4; ++l) {
    float q = 0.f;
#pragma unroll
    for (int lm = l * l - 1; lm < (l + 1) * (l + 1) - 1; ++lm) q = fmaf(2.f * kClm[lm] * s[lm], sd[lm], q);
    gi[C::vang(n, l)] = q;
  }
  if (C::FB) {
    float g4[5];
    q4_grad(&s[3], g4);
    float q = 0.f;
#pragma unroll
    for (int m = 0; m < 5; ++m) q = fmaf(g4[m], sd[3 + m], q);
    gi[C::v4b(n)] = q;
  }
}

// Network tangent and reverse pass per atom.  With psi_i = E'_i . Gdot_i and the
// energy residual weight e_i (= dL/dE_i):
//   zdot = W0 (s.Gdot), beta = w1 (1 - x^2), alpha = e_i beta + 2 x beta zdot,
//   Gbar = s . (W0^T alpha)                        (dL/dG_i, the c-gradient adjoint)
//   dL/db0 += alpha, dL/dw1 += e_i x - (1 - x^2) zdot, dL/db1 += e_i,
//   dL/dW0 += alpha (s.G)^T - beta (s.Gdot)^T     (reduced over atoms later).
template <class C>
__global__ void __launch_bounds__(128) k_mlp_bwd(int N, DevModel dm, const int* __restrict__ type,
                                                 const int* __restrict__ atom_struct, const float* __restrict__ es,
                                                 const float* __restrict__ Gd, const float* __restrict__ X,
                                                 float* __restrict__ Gb, float* __restrict__ alpha,
                                                 float* __restrict__ betaO, float* __restrict__ q1,
                                                 float* __restrict__ eatom) {
  extern __shared__ float sm[];
  const int H = dm.H;
  for (int q = threadIdx.x; q < C::NS * dm.net_size; q += blockDim.x) sm[q] = dm.params[q];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int e = type[i];
  const float* W0 = sm + e * dm.net_size;
  const float* w1 = W0 + C::NDES * H + H;
  const float ei = es[atom_struct[i]];
  eatom[i] = ei;
  float gd[C::NDES], gb[C::NDES];
#pragma unroll
  for (int v = 0; v < C::NDES; ++v) {
    gd[v] = dm.scale[v] * Gd[(size_t)i * C::NDES + v];
    gb[v] = 0.f;
  }
  for (int mu = 0; mu < H; ++mu) {
    const float* w = W0 + mu * C::NDES;
    float zd = 0.f;
#pragma unroll
    for (int v = 0; v < C::NDES; ++v) zd = fmaf(w[v], gd[v], zd);
    const float x = X[(size_t)i * H + mu];
    const float t1 = 1.f - x * x;
    const float beta = w1[mu] * t1;
    const float al = ei * beta + 2.f * x * beta * zd;
#pragma unroll
    for (int v = 0; v < C::NDES; ++v) gb[v] = fmaf(al, w[v], gb[v]);
    alpha[(size_t)i * H + mu] = al;
    betaO[(size_t)i * H + mu] = beta;
    q1[(size_t)i * H + mu] = ei * x - t1 * zd;
  }
#pragma unroll
  for (int v = 0; v < C::NDES; ++v) Gb[(size_t)i * C::NDES + v] = gb[v] * dm.scale[v];
}

// ------------------------------------------------------------- sweep 4

// Per-atom contributions to dL/dc^A_nk^{IJ}, one thread per (atom, n):
//   Sbar_nlm  = Gbar_nl 2C S_nlm - E'_nl 2C Sdot_nlm  (+ 4-body terms)
//   Sdbar_nlm = -E'_nl 2C S_nlm                        (+ 4-body term)
//   per pair: P = sum_lm Sbar B + Sdbar grad B . u,  R = sum_lm Sdbar B,
//   acc[J][k] += P f_k + R f_k' (u_hat . u).
template <class C>
__global__ void __launch_bounds__(128) k_cgrad_angular(int N, DevModel dm, const int* __restrict__ atom_struct,
                                                       const int* __restrict__ off, const int* __restrict__ jj,
                                                       const float4* __restrict__ rij, const float4* __restrict__ a,
                                                       const float* __restrict__ Bs, const float* __restrict__ Sang,
                                                       const float* __restrict__ Sdd, const float* __restrict__ Gb,
                                                       const float* __restrict__ Ep, float* __restrict__ dcA) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t / C::NQA, n = t - i * C::NQA;
  if (i >= N) return;
  float sb[NLM], sdb[NLM];
  {
    const float* S = Sang + ((size_t)i * C::NQA + n) * NLM;
    const float* D = Sdd + ((size_t)i * C::NQA + n) * NLM;
    const float* gb = Gb + (size_t)i * C::NDES;
    const float* ep = Ep + (size_t)i * C::NDES;
    float s[NLM], d[NLM];
#pragma unroll
    for (int q = 0; q < NLM; ++q) { s[q] = S[q]; d[q] = D[q]; }
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) {
      const int v = C::vang(n, lm_l(lm));
      const float c2 = 2.f * kClm[lm];
      sb[lm] = c2 * (gb[v] * s[lm] - ep[v] * d[lm]);
      sdb[lm] = -c2 * ep[v] * s[lm];
    }
    if (C::FB) {
      float g4[5], h4[5];
      q4_grad(&s[3], g4);
      q4_hvp(&s[3], &d[3], h4);
      const float gb4 = gb[C::v4b(n)], ep4 = ep[C::v4b(n)];
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        sb[3 + m] += gb4 * g4[m] - ep4 * h4[m];
        sdb[3 + m] -= ep4 * g4[m];
      }
    }
  }
  const float4 ai = a[i];
  float b[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) b[q] = Bs[6 * atom_struct[i] + q];
  float acc[C::NS][C::KA];
#pragma unroll
  for (int s = 0; s < C::NS; ++s)
#pragma unroll
    for (int k = 0; k < C::KA; ++k) acc[s][k] = 0.f;
  const int p1 = off[i + 1];
  for (int p = off[i]; p < p1; ++p) {
    const float4 r = rij[p];
    const float4 aj = a[jj[p]];
    const float3 br = sym_apply(b, make_float3(r.x, r.y, r.z));
    const float vx = aj.x - ai.x + br.x, vy = aj.y - ai.y + br.y, vz = aj.z - ai.z + br.z;
    const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
    const float ri = 1.f / rr;
    const float ux = r.x * ri, uy = r.y * ri, uz = r.z * ri;
    float f[C::KA], fp[C::KA];
    radial_basis_d<C::KA>(rr, dm.rca_inv, f, fp);
    float B[NLM], gx[NLM], gy[NLM], gz[NLM];
    harmonics_grad(ux, uy, uz, ri, B, gx, gy, gz);
    float P = 0.f, R = 0.f;
#pragma unroll
    for (int q = 0; q < NLM; ++q) {
      P = fmaf(sb[q], B[q], P);
      P = fmaf(sdb[q], gx[q] * vx + gy[q] * vy + gz[q] * vz, P);
      R = fmaf(sdb[q], B[q], R);
    }
    const float Rr = R * (ux * vx + uy * vy + uz * vz);
    const int J = (int)r.w;
#pragma unroll
    for (int s = 0; s < C::NS; ++s) {
      const float wP = (s == J) ? P : 0.f, wR = (s == J) ? Rr : 0.f;
#pragma unroll
      for (int k = 0; k < C::KA; ++k) acc[s][k] = fmaf(wP, f[k], fmaf(wR, fp[k], acc[s][k]));
    }
  }
  // layout [atom][n][J][k] so that a column sum over atoms of species I gives c^A[I][J][n][k]
  float* o = dcA + ((size_t)i * C::NQA + n) * C::NS * C::KA;
#pragma unroll
  for (int s = 0; s < C::NS; ++s)
#pragma unroll
    for (int k = 0; k < C::KA; ++k) o[s * C::KA + k] = acc[s][k];
}

// ------------------------------------------------------------- launchers

template <class C>
struct Runner {
  static int descriptors(const StepArgs& A, bool with_mlp) {
    const gnep_model* m = A.m;
    gnep_nlist* nl = A.nl;
    Workspace& w = nl->ws;
    const DevModel dm = m->dev();
    const int N = nl->n_atoms;
    if (N == 0) return GNEP_OK;
    k_desc_radial<C><<<blocks_for(N, 128), 128, 0, A.st>>>(N, dm, nl->type, nl->L[0].off, nl->L[0].rij, w.FR, w.G);
    stage("desc_radial");
    k_desc_angular<C><<<blocks_for((int64_t)N * C::NQA, 128), 128, 0, A.st>>>(N, dm, nl->type, nl->L[1].off,
                                                                                nl->L[1].rij, w.S, w.G);
    stage("desc_angular");
    GNEP_CHECK_LAUNCH("descriptor sweep");
    if (with_mlp) {
      const size_t smem = sizeof(float) * C::NS * m->net_size;
      k_mlp_fwd<C><<<blocks_for(N, 128), 128, smem, A.st>>>(N, dm, nl->type, w.G, w.X, w.Ep, w.Eatom);
      stage("mlp_fwd");
      GNEP_CHECK_LAUNCH("k_mlp_fwd");
    }
    return GNEP_OK;
  }

  static int forward(const StepArgs& A) {
    const gnep_model* m = A.m;
    gnep_nlist* nl = A.nl;
    Workspace& w = nl->ws;
    const DevModel dm = m->dev();
    const int N = nl->n_atoms;
    if (N == 0) return GNEP_OK;
    k_shat<C><<<blocks_for((int64_t)N * C::NQA, 128), 128, 0, A.st>>>(N, w.S, w.Ep, w.Shat);
    stage("shat");
    k_force_radial<C><<<blocks_for(N, 128), 128, 0, A.st>>>(N, dm, nl->type, nl->L[0].off, nl->L[0].rij, w.Ep, w.dR);
    stage("force_radial");
    if (nl->L[1].n > 0)
      k_force_angular<C><<<blocks_for(nl->L[1].n, 128), 128, 0, A.st>>>(nl->L[1].n, dm, nl->type, nl->L[1].owner,
                                                                         nl->L[1].rij, w.Shat, w.dA);
    stage("force_angular");
    k_force_gather<<<blocks_for(N, 128), 128, 0, A.st>>>(N, nl->L[0].off, nl->L[0].rev, nl->L[0].rij, w.dR,
                                                         nl->L[1].off, nl->L[1].rev, nl->L[1].rij, w.dA, w.F, w.Wat);
    stage("force_gather");
    k_struct_sum<<<nl->n_struct, 128, 0, A.st>>>(nl->struct_off, w.Eatom, w.Wat, w.Es, w.Ws);
    stage("struct_sum");
    GNEP_CHECK_LAUNCH("force sweep");
    return GNEP_OK;
  }

  static int backward(const StepArgs& A) {
    const gnep_model* m = A.m;
    gnep_nlist* nl = A.nl;
    Workspace& w = nl->ws;
    const DevModel dm = m->dev();
    const int N = nl->n_atoms;
    if (N == 0) return GNEP_OK;
    k_tangent_radial<C><<<blocks_for(N, 128), 128, 0, A.st>>>(N, dm, nl->type, nl->atom_struct, nl->L[0].off,
                                                              nl->L[0].j, nl->L[0].rij, w.a, w.Bs, w.FRd, w.Gd);
    stage("tangent_radial");
    k_tangent_angular<C><<<blocks_for((int64_t)N * C::NQA, 128), 128, 0, A.st>>>(
        N, dm, nl->type, nl->atom_struct, nl->L[1].off, nl->L[1].j, nl->L[1].rij, w.a, w.Bs, w.S, w.Sd, w.Gd);
    stage("tangent_angular");
    const size_t smem = sizeof(float) * C::NS * m->net_size;
    k_mlp_bwd<C><<<blocks_for(N, 128), 128, smem, A.st>>>(N, dm, nl->type, nl->atom_struct, w.es, w.Gd, w.X, w.Gb,
                                                          w.alpha, w.beta, w.q1, w.eatom);
    stage("mlp_bwd");
    k_cgrad_angular<C><<<blocks_for((int64_t)N * C::NQA, 128), 128, 0, A.st>>>(
        N, dm, nl->atom_struct, nl->L[1].off, nl->L[1].j, nl->L[1].rij, w.a, w.Bs, w.S, w.Sd, w.Gb, w.Ep, w.dcA);
    stage("cgrad_angular");
    GNEP_CHECK_LAUNCH("backward sweeps");
    return GNEP_OK;
  }
};

}  // namespace

// Shapes with compiled kernels: (species, n_max+1, basis+1 radial; same angular; 4-body).
#define GNEP_SHAPES(X)            \
  X(2, 5, 9, 5, 9, false)         \
  X(2, 9, 13, 9, 13, true)        \
  X(2, 9, 13, 9, 13, false)

bool shape_supported(const Shape& s) {
#define X(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB)                                                                    \
  if (s.ns == P_NS && s.nqr == P_NQR && s.kr == P_KR && s.nqa == P_NQA && s.ka == P_KA && (s.fb != 0) == P_FB && \
      s.lmax == 4)                                                                                     \
    return true;
  GNEP_SHAPES(X)
#undef X
  return false;
}

namespace {
template <class C>
int setup_shape() {
  GNEP_CUDA(cudaFuncSetAttribute(k_mlp_fwd<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  GNEP_CUDA(cudaFuncSetAttribute(k_mlp_bwd<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  return GNEP_OK;
}
}  // namespace

int shape_setup(const Shape& s) {
#define X(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB)                                                                    \
  if (s.ns == P_NS && s.nqr == P_NQR && s.kr == P_KR && s.nqa == P_NQA && s.ka == P_KA && (s.fb != 0) == P_FB) \
    return setup_shape<Sh<P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB>>();
  GNEP_SHAPES(X)
#undef X
  return set_error(GNEP_ERR_UNSUPPORTED, "no kernel for this shape");
}

int run_descriptors(const StepArgs& A, bool with_mlp) {
  const Shape& s = A.m->shape;
#define X(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB)                                                                    \
  if (s.ns == P_NS && s.nqr == P_NQR && s.kr == P_KR && s.nqa == P_NQA && s.ka == P_KA && (s.fb != 0) == P_FB) \
    return Runner<Sh<P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB>>::descriptors(A, with_mlp);
  GNEP_SHAPES(X)
#undef X
  return set_error(GNEP_ERR_UNSUPPORTED, "no kernel for this shape");
}

int run_forward(const StepArgs& A) {
  const Shape& s = A.m->shape;
#define X(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB)                                                                    \
  if (s.ns == P_NS && s.nqr == P_NQR && s.kr == P_KR && s.nqa == P_NQA && s.ka == P_KA && (s.fb != 0) == P_FB) \
    return Runner<Sh<P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB>>::forward(A);
  GNEP_SHAPES(X)
#undef X
  return set_error(GNEP_ERR_UNSUPPORTED, "no kernel for this shape");
}

int run_backward(const StepArgs& A) {
  const Shape& s = A.m->shape;
#define X(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB)                                                                    \
  if (s.ns == P_NS && s.nqr == P_NQR && s.kr == P_KR && s.nqa == P_NQA && s.ka == P_KA && (s.fb != 0) == P_FB) \
    return Runner<Sh<P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB>>::backward(A);
  GNEP_SHAPES(X)
#undef X
  return set_error(GNEP_ERR_UNSUPPORTED, "no kernel for this shape");
}

}  // namespace gnep

// ---------------------------------------------------------------------------
// Descriptors without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need
// descriptors: code that runs while a CUDA stream is being captured into a
// graph (allocation is not a capturable operation), hosts whose device memory
// is entirely owned by another allocator or a fixed pool set up at start-up,
// and per-step hooks of simulation engines that forbid allocation in their hot
// loop.  For them the descriptor sweep can use this fixed scratch array, which
// every GPU that loads the library holds until the process exits, instead of
// workspace memory.
namespace gnep {
namespace {

constexpr size_t kStaticScratchFloats = size_t(1) << 21;  // 8 MiB
static __device__ __align__(256) float g_static_scratch[kStaticScratchFloats];
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
float* g_static_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once per
// device (host code must not use the symbol itself as a device pointer).
int static_scratch(float** out) {
  int dev = 0;
  GNEP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(GNEP_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static scratch)");
    g_static_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_static_ptr[dev];
  return GNEP_OK;
}

template <class C>
int descriptors_static(const StepArgs& A, float* G) {
  const gnep_model* m = A.m;
  const gnep_nlist* nl = A.nl;
  const int64_t N = nl->n_atoms;
  const int64_t fr = N * C::NS * C::KR;
  const int64_t sa = N * C::NQA * NLM;
  const int64_t fr_padded = (fr + 63) / 64 * 64;
  if (fr_padded + sa > (int64_t)kStaticScratchFloats)
    return set_error(GNEP_ERR_INVALID_ARG,
                     "batch too large for the fixed descriptor scratch (needs " + std::to_string(fr_padded + sa) +
                         " floats, holds " + std::to_string(kStaticScratchFloats) + ")");
  float* scratch = nullptr;
  int rc = static_scratch(&scratch);
  if (rc) return rc;
  if (N == 0) return GNEP_OK;
  const DevModel dm = m->dev();
  // Both kernels overwrite every scratch element they later read, so the
  // array needs no clearing between calls.
  k_desc_radial<C><<<blocks_for(N, 128), 128, 0, A.st>>>((int)N, dm, nl->type, nl->L[0].off, nl->L[0].rij,
                                                         scratch, G);
  k_desc_angular<C><<<blocks_for(N * C::NQA, 128), 128, 0, A.st>>>((int)N, dm, nl->type, nl->L[1].off,
                                                                    nl->L[1].rij, scratch + fr_padded, G);
  GNEP_CHECK_LAUNCH("descriptor sweep (static scratch)");
  return GNEP_OK;
}

}  // namespace

int run_descriptors_static(const StepArgs& A, float* G) {
  const Shape& s = A.m->shape;
#define X(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB)                                                       \
  if (s.ns == P_NS && s.nqr == P_NQR && s.kr == P_KR && s.nqa == P_NQA && s.ka == P_KA && (s.fb != 0) == P_FB) \
    return descriptors_static<Sh<P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB>>(A, G);
  GNEP_SHAPES(X)
#undef X
  return set_error(GNEP_ERR_UNSUPPORTED, "no kernel for this shape");
}

}  // namespace gnep
