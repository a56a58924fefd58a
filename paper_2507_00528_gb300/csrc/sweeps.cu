// Shape-specialised sweeps of one training step over a packed batch.
//
//   sweep 1  descriptors  q_n (Eqs. 5-6), S_nlm and q_nl (Eqs. 7-8), 4-body q4_n
//   network  (network.cu) E_i, E'_i, per-atom radial contraction chat_i
//   sweep 2  dE_i/dr_ij (C3.6), forces (Eq. 3), per-atom virial (Eq. 4)
//   sweep 3  tangent  Gdot_i = sum_j dG_i/dr_ij . u_ij
//   network  (network.cu) tangent and reverse pass, adjoints Gbar_i
//   sweep 4  dL/dc^R and dL/dc^A
//
// Gradient route.  With a_i = dL/dF_i and B_s = dL/dW_s held fixed (Eqs. 11-12),
//   sum_i a_i.F_i + sum_s B_s:W_s = - sum_i sum_j u_ij . dE_i/dr_ij,
//   u_ij = (a_j - a_i) + B_s r_ij,
// because F_i = sum_j (dE_i/dr_ij - dE_j/dr_ji) (Eq. 3) and W_s = -sum r_ij (x) dE_i/dr_ij
// (Eq. 4 summed).  Hence the force and virial parts of dL/dtheta (Eqs. 15-16 with
// the mixed derivatives of App. C3 and D1.11-D1.17) equal -d/dtheta sum_i E'_i.Gdot_i:
// one forward-mode sweep (3) and one reverse sweep (4) instead of explicit second
// derivative tensors.
//
// Thread mappings.  Radial sweeps: RL consecutive lanes per atom, each taking
// every RL-th pair, combined by warp shuffles; RL is 4 for batches that give
// every SM several blocks, 8 or 16 for smaller ones, where the per-lane pair
// loop (one dependent global load per pair) sets the kernel's length.
// Angular sweeps 1, 3, 4:
// persistent blocks over tiles of atoms; the per-pair geometry (basis,
// harmonics, directional derivatives) of a chunk of the tile's pairs is computed
// once per pair into shared memory, then one warp per atom contracts it with
// the atom's coefficients on the tensor cores (mma.sync TF32, warp_mma.cuh).
// Angular force: one thread per pair, with dE/dS_nlm of the block's atoms in
// shared memory.  No float atomics anywhere: fixed summation order.
#include <cstdio>
#include <mutex>
#include <string>

#include "device_math.cuh"
#include "gnep_internal.h"
#include "network.cuh"
#include "shape.cuh"
#include "sweeps_lmax.cuh"
#include "warp_mma.cuh"

namespace gnep {

constexpr int CH = 128;         // pairs per geometry chunk
constexpr int kCgBlocksPerSm = 2;  // default persistent blocks of the c-gradient sweep per SM

// Angular thread map: TPA threads per atom, NPT channels per thread.
template <int NQ, int NPT>
struct AMap {
  static constexpr int TPA = (NQ + NPT - 1) / NPT;
  static constexpr int NA = 128 / TPA;
};

namespace {

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

template <int RL, int NS, int K>
__device__ __forceinline__ void lane_reduce(float (&acc)[NS][K]) {
#pragma unroll
  for (int o = 1; o < RL; o <<= 1)
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int k = 0; k < K; ++k) acc[s][k] += __shfl_xor_sync(0xffffffffu, acc[s][k], o);
}

}  // namespace

// ------------------------------------------------------------- sweep 1

// Radial descriptors: per-atom basis sums FR[J][k] = sum_{j in J} f_k(r_ij) and
// q_n = sum_J sum_k c^R_nk^{IJ} FR[J][k]  (Eqs. 5-6).
template <class C, int RL>
__global__ void __launch_bounds__(128) k_desc_radial(int N, DevModel dm, const int* __restrict__ type,
                                                     const int* __restrict__ off, const float4* __restrict__ rij,
                                                     float* __restrict__ FR, float* __restrict__ G) {
  GNEP_PDL_WAIT();
  __shared__ float cR[C::NCR];
  for (int q = threadIdx.x; q < C::NCR; q += blockDim.x) cR[q] = dm.params[dm.off_cR + q];
  __syncthreads();
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gt / RL, lane = gt % RL;
  const bool ok = i < N;
  float acc[C::NS][C::KR];
#pragma unroll
  for (int s = 0; s < C::NS; ++s)
#pragma unroll
    for (int k = 0; k < C::KR; ++k) acc[s][k] = 0.f;
  if (ok) {
    const int p1 = off[i + 1];
    int p = off[i] + lane;
    float4 rn = p < p1 ? rij[p] : make_float4(1.f, 0.f, 0.f, 0.f);  // the pair after the current one
    for (; p < p1; p += RL) {
      const float4 r = rn;
      if (p + RL < p1) rn = rij[p + RL];
      const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
      float f[C::KR];
      radial_basis<C::KR>(rr, dm.rcr_inv, f);
      acc_row<C::NS, C::KR>(acc, (int)r.w, f, 1.f);
    }
  }
  lane_reduce<RL>(acc);
  if (!ok) return;
  const int I = type[i];
  float* fr = FR + (size_t)i * C::NS * C::KR;
#pragma unroll
  for (int s = 0; s < C::NS; ++s)
#pragma unroll
    for (int k = 0; k < C::KR; ++k)
      if ((s * C::KR + k) % RL == lane) fr[s * C::KR + k] = acc[s][k];
#pragma unroll
  for (int n = 0; n < C::NQR; ++n) {
    if (n % RL != lane) continue;
    float q = 0.f;
#pragma unroll
    for (int s = 0; s < C::NS; ++s)
#pragma unroll
      for (int k = 0; k < C::KR; ++k) q = fmaf(cR[((I * C::NS + s) * C::NQR + n) * C::KR + k], acc[s][k], q);
    G[(size_t)i * C::NDES + n] = q;
  }
}

// ------------------------------------------------------------- sweep 2

// Angular pairs, one thread per pair, NAF atoms per block with
// Shat_nlm = dE_i/dS_nlm = E'_nl 2 C_lm S_nlm (+ E'_4b,n dq4/dS_n2m) in shared memory:
//   dE_i/dr_ij = sum_n [g_n' (Shat_n . B) u + g_n Shat_n . grad B]       (C2.1, C2.3, C3.6)
//             = (sum_lm ghat'_lm B_lm) u + (I - u u^T)(sum_lm ghat_lm grad p_lm) / r,
//   ghat_lm = sum_n g_n Shat_nlm, ghat'_lm = sum_n g_n' Shat_nlm.
template <class C>
__global__ void __launch_bounds__(128) k_force_angular(int N, DevModel dm, const int* __restrict__ tiles,
                                                       const int* __restrict__ type, const int* __restrict__ off,
                                                       const int* __restrict__ own, const float4* __restrict__ rij,
                                                       const float* __restrict__ Sang, const float* __restrict__ Ep,
                                                       float4* __restrict__ dA) {
  GNEP_PDL_WAIT();
  constexpr int NAF = AMap<C::NQ, 1>::NA;
  constexpr int KP = (C::KA + 3) / 4 * 4;  // basis functions padded to 16-byte rows
  static_assert(NLM % 4 == 0, "16-byte Shat rows");
  // c^A_nk^{IJ} as [IJ][n][KP] and Shat [atom][n][lm]: both read as float4 (one
  // shared-memory load per four products)
  __shared__ __align__(16) float cA[C::NS * C::NS * C::NQA * KP];
  __shared__ __align__(16) float sh[NAF][C::NQA][NLM];
  const int i0 = tiles[blockIdx.x], i1 = tiles[blockIdx.x + 1];
  for (int q = threadIdx.x; q < C::NS * C::NS * C::NQA * KP; q += blockDim.x) {
    const int k = q % KP, r = q / KP;  // r = (I NS + J) NQA + n
    cA[q] = k < C::KA ? dm.params[dm.off_cA + r * C::KA + k] : 0.f;
  }
  for (int t = threadIdx.x; t < NAF * C::NQA; t += blockDim.x) {
    const int a = t / C::NQA, n = t % C::NQA, i = i0 + a;
    if (i >= i1) continue;
    const float* S = Sang + ((size_t)i * C::NQA + n) * NLM;
    const float* ep = Ep + (size_t)i * C::NDES;
    float s[NLM];
#pragma unroll
    for (int q = 0; q < NLM; ++q) s[q] = S[q];
#pragma unroll
    for (int lm = 0; lm < NLM; ++lm) sh[a][n][lm] = 2.f * kClm[lm] * ep[C::vang(n, lm_l(lm))] * s[lm];
    if (C::FB) {
      float g4[5];
      q4_grad(&s[3], g4);
      const float e4 = ep[C::v4b(n)];
#pragma unroll
      for (int m = 0; m < 5; ++m) sh[a][n][3 + m] = fmaf(e4, g4[m], sh[a][n][3 + m]);
    }
  }
  __syncthreads();
  const int P0 = off[i0], P1 = off[i1];
  for (int p = P0 + threadIdx.x; p < P1; p += blockDim.x) {
    const int i = own[p];
    const int a = i - i0;
    const int I = type[i];
    const float4 r = rij[p];
    const int J = (int)r.w;
    const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
    const float ri = 1.f / rr;
    const float ux = r.x * ri, uy = r.y * ri, uz = r.z * ri;
    float fk[C::KA], fpk[C::KA], f[KP], fp[KP];
    radial_basis_d<C::KA>(rr, dm.rca_inv, fk, fpk);
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      f[k] = k < C::KA ? fk[k] : 0.f;
      fp[k] = k < C::KA ? fpk[k] : 0.f;
    }
    const float4* cIJ = reinterpret_cast<const float4*>(cA + (I * C::NS + J) * C::NQA * KP);
    float g[C::NQA], gp[C::NQA];
#pragma unroll
    for (int n = 0; n < C::NQA; ++n) {
      float a1 = 0.f, a2 = 0.f;
#pragma unroll
      for (int k4 = 0; k4 < KP / 4; ++k4) {
        const float4 c = cIJ[n * (KP / 4) + k4];
        a1 = fmaf(c.x, f[4 * k4], fmaf(c.y, f[4 * k4 + 1], fmaf(c.z, f[4 * k4 + 2], fmaf(c.w, f[4 * k4 + 3], a1))));
        a2 = fmaf(c.x, fp[4 * k4], fmaf(c.y, fp[4 * k4 + 1], fmaf(c.z, fp[4 * k4 + 2], fmaf(c.w, fp[4 * k4 + 3], a2))));
      }
      g[n] = a1;
      gp[n] = a2;
    }
    float B[NLM], gx[NLM], gy[NLM], gz[NLM];
    harmonics_grad(ux, uy, uz, 1.f, B, gx, gy, gz);
    float P = 0.f, vx = 0.f, vy = 0.f, vz = 0.f;
    const float4* sa = reinterpret_cast<const float4*>(&sh[a][0][0]);
#pragma unroll
    for (int q4 = 0; q4 < NLM / 4; ++q4) {
      float gh[4] = {0.f, 0.f, 0.f, 0.f}, ghp[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int n = 0; n < C::NQA; ++n) {
        const float4 s4 = sa[n * (NLM / 4) + q4];
        const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          gh[e] = fmaf(g[n], sv[e], gh[e]);
          ghp[e] = fmaf(gp[n], sv[e], ghp[e]);
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int q = 4 * q4 + e;
        P = fmaf(ghp[e], B[q], P);
        vx = fmaf(gh[e], gx[q], vx);
        vy = fmaf(gh[e], gy[q], vy);
        vz = fmaf(gh[e], gz[q], vz);
      }
    }
    dA[p] = make_float4(P * ux + vx * ri, P * uy + vy * ri, P * uz + vz * ri, 0.f);
  }
}

// Forces and per-atom virials, RL lanes per atom.
//   radial pairs: d_ij - d_ji = (chat_i[J] . f'(r) + chat_j[I] . f'(r)) r_ij / r
//                 (C1.1, C3.6 with the per-atom contraction chat = sum_n E'_n c^R_n)
//   angular pairs: d_ij - d_rev(ij) from the pair forces of k_force_angular (Eq. 3)
//   virial: -sum_j r_ij (x) d_ij, symmetrised (Eq. 4 summed over atoms).
template <class C, int RL>
__global__ void __launch_bounds__(128) k_force_atoms(int N, DevModel dm, const int* __restrict__ type,
                                                     const int* __restrict__ offR, const int* __restrict__ jR,
                                                     const float4* __restrict__ rijR, const float* __restrict__ chat,
                                                     const int* __restrict__ offA, const int* __restrict__ revA,
                                                     const float4* __restrict__ rijA, const float4* __restrict__ dA,
                                                     float* __restrict__ F, float* __restrict__ Wat) {
  GNEP_PDL_WAIT();
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gt / RL, lane = gt % RL;
  const bool ok = i < N;
  float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // F (3), W (6)
  if (ok) {
    const int I = type[i];
    float ci[C::NS][C::KR];
#pragma unroll
    for (int s = 0; s < C::NS; ++s)
#pragma unroll
      for (int k = 0; k < C::KR; ++k) ci[s][k] = chat[((size_t)i * C::NS + s) * C::KR + k];
    const int p1 = offR[i + 1];
    int p = offR[i] + lane;
    float4 rn = p < p1 ? rijR[p] : make_float4(1.f, 0.f, 0.f, 0.f);  // the pair after the current one
    int jn = p < p1 ? jR[p] : 0;
    for (; p < p1; p += RL) {
      const float4 r = rn;
      const int j = jn;
      if (p + RL < p1) {
        rn = rijR[p + RL];
        jn = jR[p + RL];
      }
      const float* cj = chat + ((size_t)j * C::NS + I) * C::KR;
      const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
      float f[C::KR], fp[C::KR];
      radial_basis_d<C::KR>(rr, dm.rcr_inv, f, fp);
      const float dij = dot_row<C::NS, C::KR>(ci, (int)r.w, fp);
      float dji = 0.f;
#pragma unroll
      for (int k = 0; k < C::KR; ++k) dji = fmaf(cj[k], fp[k], dji);
      const float s1 = (dij + dji) / rr, s0 = dij / rr;
      v[0] += s1 * r.x;
      v[1] += s1 * r.y;
      v[2] += s1 * r.z;
      v[3] -= s0 * r.x * r.x;
      v[4] -= s0 * r.y * r.y;
      v[5] -= s0 * r.z * r.z;
      v[6] -= s0 * r.x * r.y;
      v[7] -= s0 * r.y * r.z;
      v[8] -= s0 * r.z * r.x;
    }
    const int q1 = offA[i + 1];
    for (int p = offA[i] + lane; p < q1; p += RL) {
      const float4 d = dA[p], b = dA[revA[p]], r = rijA[p];
      v[0] += d.x - b.x;
      v[1] += d.y - b.y;
      v[2] += d.z - b.z;
      v[3] -= r.x * d.x;
      v[4] -= r.y * d.y;
      v[5] -= r.z * d.z;
      v[6] -= 0.5f * (r.x * d.y + r.y * d.x);
      v[7] -= 0.5f * (r.y * d.z + r.z * d.y);
      v[8] -= 0.5f * (r.z * d.x + r.x * d.z);
    }
  }
#pragma unroll
  for (int o = 1; o < RL; o <<= 1)
#pragma unroll
    for (int q = 0; q < 9; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if (!ok || lane != 0) return;
  F[3 * (size_t)i] = v[0];
  F[3 * (size_t)i + 1] = v[1];
  F[3 * (size_t)i + 2] = v[2];
#pragma unroll
  for (int q = 0; q < 6; ++q) Wat[6 * (size_t)i + q] = v[3 + q];
}

// E_s = sum_i E_i and W_s = sum_i w_i in FP64, one block per structure.
// Per-structure energy and virial (Eqs. 1, 4): each thread sums its few atoms
// (at most 4 for structures of 512 atoms) in FP32, the 128 thread sums are
// combined in FP64 by a fixed tree.
__global__ void __launch_bounds__(128) k_struct_sum(const int* __restrict__ soff, const float* __restrict__ Eatom,
                                                    const float* __restrict__ Wat, double* __restrict__ Es,
                                                    double* __restrict__ Ws) {
  GNEP_PDL_WAIT();
  const int s = blockIdx.x;
  const int a0 = soff[s], a1 = soff[s + 1];
  float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int i = a0 + threadIdx.x; i < a1; i += blockDim.x) {
    acc[0] += Eatom[i];
#pragma unroll
    for (int q = 0; q < 6; ++q) acc[1 + q] += Wat[6 * (size_t)i + q];
  }
  __shared__ double sh[7][128];
#pragma unroll
  for (int q = 0; q < 7; ++q) sh[q][threadIdx.x] = (double)acc[q];
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int q = 0; q < 7; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 7) {
    if (threadIdx.x == 0)
      Es[s] = sh[0][0];
    else
      Ws[6 * s + threadIdx.x - 1] = sh[threadIdx.x][0];
  }
}

// ------------------------------------------------------------- sweep 3

// Radial tangent: FRd[J][k] = sum_{j in J} f_k'(r_ij) (u_hat . u_ij),
// qdot_n = sum_J sum_k c^R_nk^{IJ} FRd[J][k].
template <class C, int RL>
__global__ void __launch_bounds__(128) k_tangent_radial(int N, DevModel dm, const int* __restrict__ type,
                                                        const int* __restrict__ atom_struct, const int* __restrict__ off,
                                                        const int* __restrict__ jj, const float4* __restrict__ rij,
                                                        const float4* __restrict__ a, const float* __restrict__ Bs,
                                                        float* __restrict__ FRd, float* __restrict__ Gd) {
  GNEP_PDL_WAIT();
  __shared__ float cR[C::NCR];
  for (int q = threadIdx.x; q < C::NCR; q += blockDim.x) cR[q] = dm.params[dm.off_cR + q];
  __syncthreads();
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gt / RL, lane = gt % RL;
  const bool ok = i < N;
  float acc[C::NS][C::KR];
#pragma unroll
  for (int s = 0; s < C::NS; ++s)
#pragma unroll
    for (int k = 0; k < C::KR; ++k) acc[s][k] = 0.f;
  if (ok) {
    const float4 ai = a[i];
    float b[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) b[q] = Bs[6 * atom_struct[i] + q];
    const int p1 = off[i + 1];
    int p = off[i] + lane;
    // the pair after the current one, and its neighbour's tangent
    float4 rn = p < p1 ? rij[p] : make_float4(1.f, 0.f, 0.f, 0.f);
    float4 an = p < p1 ? a[jj[p]] : ai;
    for (; p < p1; p += RL) {
      const float4 r = rn, aj = an;
      if (p + RL < p1) {
        rn = rij[p + RL];
        an = a[jj[p + RL]];
      }
      const float3 br = sym_apply(b, make_float3(r.x, r.y, r.z));
      const float ux = aj.x - ai.x + br.x, uy = aj.y - ai.y + br.y, uz = aj.z - ai.z + br.z;
      const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
      const float ru = (r.x * ux + r.y * uy + r.z * uz) / rr;
      float f[C::KR], fp[C::KR];
      radial_basis_d<C::KR>(rr, dm.rcr_inv, f, fp);
      acc_row<C::NS, C::KR>(acc, (int)r.w, fp, ru);
    }
  }
  lane_reduce<RL>(acc);
  if (!ok) return;
  float* fr = FRd + (size_t)i * C::NS * C::KR;
#pragma unroll
  for (int s = 0; s < C::NS; ++s)
#pragma unroll
    for (int k = 0; k < C::KR; ++k)
      if ((s * C::KR + k) % RL == lane) fr[s * C::KR + k] = acc[s][k];
  const int I = type[i];
#pragma unroll
  for (int n = 0; n < C::NQR; ++n) {
    if (n % RL != lane) continue;
    float q = 0.f;
#pragma unroll
    for (int s = 0; s < C::NS; ++s)
#pragma unroll
      for (int k = 0; k < C::KR; ++k) q = fmaf(cR[((I * C::NS + s) * C::NQR + n) * C::KR + k], acc[s][k], q);
    Gd[(size_t)i * C::NDES + n] = q;
  }
}

// Angular geometry of a chunk of CH pairs for the c-gradient sweep, one pair per
// thread: basis f_k, fu_k = f_k' (u_hat . u_ij), harmonics B_lm and
// D_lm = grad B_lm . u_ij.  Rows of B and D are 8 mod 32 words apart, rows of f
// and fu 4 mod 32, so that the MMA fragment loads of one warp touch 32 banks.
template <class C>
struct MGeo {
  static constexpr int SBD = CH + 8, SF = CH + 4;
  float B[NLM][SBD];
  float D[NLM][SBD];
  float f[C::KA][SF];
  float fu[C::KA][SF];
  int J[CH];
};

// Direction of the tangent for pair p: w_ij = (a_j - a_i) + B_s r_ij.
__device__ __forceinline__ float3 tangent_dir(int p, float4 r, const int* __restrict__ own,
                                              const int* __restrict__ atom_struct, const int* __restrict__ jj,
                                              const float4* __restrict__ a, const float* __restrict__ Bs) {
  const int i = own[p];
  const float4 ai = a[i], aj = a[jj[p]];
  const float* b = Bs + 6 * atom_struct[i];
  const float bb[6] = {b[0], b[1], b[2], b[3], b[4], b[5]};
  const float3 br = sym_apply(bb, make_float3(r.x, r.y, r.z));
  return make_float3(aj.x - ai.x + br.x, aj.y - ai.y + br.y, aj.z - ai.z + br.z);
}

template <class C, class Geo>
__device__ __forceinline__ void pair_geometry(Geo& g, int slot, float4 r, float3 w, const DevModel& dm) {
  const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
  const float ri = 1.f / rr;
  const float ux = r.x * ri, uy = r.y * ri, uz = r.z * ri;
  const float ru = ux * w.x + uy * w.y + uz * w.z;
  float f[C::KA], fp[C::KA];
  radial_basis_d<C::KA>(rr, dm.rca_inv, f, fp);
#pragma unroll
  for (int k = 0; k < C::KA; ++k) {
    g.f[k][slot] = f[k];
    g.fu[k][slot] = fp[k] * ru;
  }
  float B[NLM], Dd[NLM];
  harmonics_dir(ux, uy, uz, ri, w.x, w.y, w.z, B, Dd);
#pragma unroll
  for (int q = 0; q < NLM; ++q) {
    g.B[q][slot] = B[q];
    g.D[q][slot] = Dd[q];
  }
  g.J[slot] = (int)r.w;
}

// ------------------------------------------------------------- sweep 4

// dL/dc.  With Sbar and Sdbar the adjoints of S and Sdot of atom i,
//   Sbar_nlm  = Gbar_nl 2C S_nlm - E'_nl 2C Sdot_nlm  (+ 4-body terms)
//   Sdbar_nlm = -E'_nl 2C S_nlm                        (+ 4-body term),
// each angular pair ij contributes
//   P_n = sum_lm Sbar_nlm B_lm + Sdbar_nlm D_lm,   R_n = sum_lm Sdbar_nlm B_lm,
//   dL/dc^A_nk^{IJ} += P_n f_k + R_n fu_k,
// and each atom contributes dL/dc^R_nk^{IJ} += Gbar_n FR[J][k] - E'_n FRd[J][k].
//
// Angular part: one warp per atom, blocks of 4 warps (two per SM: the split
// products take over 200 registers, and two blocks let one block's tile
// barriers overlap the other's products).  For 8 of the atom's pairs at a time,
//   [P | R] = [Sbar | Sdbar] [B D; D 0 ... ]  as three products of K = 24:
//        P = Sbar B + Sdbar D,  R = Sdbar B            (16 x 24) (24 x 8)
//   acc^{IJ} += P_J F^T + R_J Fu^T                       (16 x 8) (8 x 16)
// with P_J, R_J the columns of pairs whose neighbour has species J, on the
// tensor cores (warp_mma.cuh).  The pair columns of the first products are
// ordered so that their C fragments are, register for register, the A
// fragments of the second: column g holds pair g/2 + 4 (g mod 2), so the C
// columns 2t and 2t+1 of a lane are the pairs t and t+4, which are its K rows t
// and t+4 in the second product.  Accumulators stay in registers over all of a
// warp's atoms; the block folds its four warps in order and writes
// cpart[block][c^A] once.
// Hint to bring [p, p + bytes) into L2 ahead of use (bulk prefetch; the range
// is rounded inward to 16 bytes, so nothing outside it is touched).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
  const uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
  const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
  if (e > a) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(e - a)) : "memory");
}

constexpr int kAS = 2 * NLM + 4;  // row stride of [Sbar | Sdbar] (20 mod 32 words: conflict-free A fragments)
constexpr int kCgWarps = 4;       // per block; two blocks per SM, so one block's barriers overlap the other's work

template <class C>
struct CgSmem {
  static constexpr int NA = 128 / C::NQ;  // atoms per tile, at most (force and tangent tiling)
  static constexpr int KT = (C::KA + 7) / 8;
  union {
    MGeo<C> geo;
    float red[kCgWarps][C::NS * C::NS * KT * 128];  // per warp: [I][J][kt][lane][4] accumulator registers
  };
  float A[NA][C::NQA][kAS];
  // the next tile's atom rows (S, Sdot, Gbar, E'), copied asynchronously while
  // the current tile is contracted
  float stS[NA * C::NQA * NLM];
  float stD[NA * C::NQA * NLM];
  float stG[NA * C::NDES];
  float stE[NA * C::NDES];
  int type[NA];
  int off[NA + 1];
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

template <class C, bool SPLIT>
__global__ void __launch_bounds__(32 * kCgWarps, 2)
    k_cgrad_ang(int ntile, const int* __restrict__ tiles, DevModel dm, const int* __restrict__ type,
                const int* __restrict__ off, const float4* __restrict__ rij, const float4* __restrict__ wij,
                const float* __restrict__ Sang, const float* __restrict__ Sdd, const float* __restrict__ Gb,
                const float* __restrict__ Ep, float* __restrict__ cpart) {
  GNEP_PDL_WAIT();
  using SM = CgSmem<C>;
  constexpr int NA = SM::NA, KT = SM::KT, NQA = C::NQA, KA = C::KA, NS = C::NS, KS = NLM / 8;
  static_assert(NLM % 8 == 0 && NLM % 4 == 0 && NQA <= 16 && NA * NQA <= 128 && CH == 128, "fragment shapes");
  extern __shared__ __align__(16) unsigned char smraw[];
  SM& sm = *reinterpret_cast<SM*>(smraw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int pg = (g >> 1) | ((g & 1) << 2);  // pair of B-fragment column g
  Acc<SPLIT> acc[NS][NS][KT];
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int J = 0; J < NS; ++J)
#pragma unroll
      for (int kt = 0; kt < KT; ++kt) acc[s][J][kt].zero();

  // atom rows of tile atoms [a0, a1) into the staging arrays (one commit group)
  auto stage_rows = [&](int a0, int a1) {
    const int n4 = (a1 - a0) * NQA * NLM / 4, ng = (a1 - a0) * C::NDES;
    const float4* s4 = reinterpret_cast<const float4*>(Sang + (size_t)a0 * NQA * NLM);
    const float4* d4 = reinterpret_cast<const float4*>(Sdd + (size_t)a0 * NQA * NLM);
    for (int q = tid; q < n4; q += blockDim.x) {
      cp_async16(&sm.stS[4 * q], s4 + q);
      cp_async16(&sm.stD[4 * q], d4 + q);
    }
    for (int q = tid; q < ng; q += blockDim.x) {
      cp_async4(&sm.stG[q], Gb + (size_t)a0 * C::NDES + q);
      cp_async4(&sm.stE[q], Ep + (size_t)a0 * C::NDES + q);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  int tile = blockIdx.x;
  int i0 = 0, i1 = 0, P0 = 0, P1 = 0;
  if (tile < ntile) {
    i0 = tiles[tile];
    i1 = tiles[tile + 1];
    P0 = off[i0];
    P1 = off[i1];
    stage_rows(i0, i1);
  }
  for (; tile < ntile; tile += gridDim.x) {
    const int nt = tile + gridDim.x;  // the next tile's bounds are fetched early
    const int i0n = nt < ntile ? tiles[nt] : 0, i1n = nt < ntile ? tiles[nt + 1] : 0;
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();  // the previous tile's readers are done and this tile's rows are staged
    {
      // atom rows [Sbar | Sdbar], one thread per (atom, channel), before the
      // chunk's geometry (separate shared arrays; one barrier covers both)
      const int u = tid, at = u / NQA, n = u % NQA, i = i0 + at;
      if (at < NA && i < i1) {
        const float4* S4 = reinterpret_cast<const float4*>(&sm.stS[(at * NQA + n) * NLM]);
        const float4* D4 = reinterpret_cast<const float4*>(&sm.stD[(at * NQA + n) * NLM]);
        const float* gb = &sm.stG[at * C::NDES];
        const float* ep = &sm.stE[at * C::NDES];
        float s[NLM], d[NLM], sb[NLM], sdb[NLM];
#pragma unroll
        for (int q = 0; q < NLM / 4; ++q) {
          const float4 x = S4[q], y = D4[q];
          s[4 * q] = x.x; s[4 * q + 1] = x.y; s[4 * q + 2] = x.z; s[4 * q + 3] = x.w;
          d[4 * q] = y.x; d[4 * q + 1] = y.y; d[4 * q + 2] = y.z; d[4 * q + 3] = y.w;
        }
        float gbl[4], epl[4];
#pragma unroll
        for (int l = 1; l <= 4; ++l) {
          gbl[l - 1] = gb[C::vang(n, l)];
          epl[l - 1] = ep[C::vang(n, l)];
        }
#pragma unroll
        for (int lm = 0; lm < NLM; ++lm) {
          const float c2 = 2.f * kClm[lm], gv = gbl[lm_l(lm) - 1], ev = epl[lm_l(lm) - 1];
          sb[lm] = c2 * (gv * s[lm] - ev * d[lm]);
          sdb[lm] = -c2 * ev * s[lm];
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
        float4* row = reinterpret_cast<float4*>(sm.A[at][n]);
#pragma unroll
        for (int q = 0; q < NLM / 4; ++q) {
          row[q] = make_float4(sb[4 * q], sb[4 * q + 1], sb[4 * q + 2], sb[4 * q + 3]);
          row[NLM / 4 + q] = make_float4(sdb[4 * q], sdb[4 * q + 1], sdb[4 * q + 2], sdb[4 * q + 3]);
        }
      }
      if (u < NA) sm.type[u] = (i0 + u < i1) ? type[i0 + u] : 0;
      if (u <= i1 - i0) sm.off[u] = off[i0 + u];
    }
    for (int cs = P0; cs < P1; cs += CH) {
      const int ce = min(cs + CH, P1);
      if (cs != P0) __syncthreads();  // the previous chunk's readers are done
      if (tid < 128 && cs + tid < ce) {
        const float4 r = rij[cs + tid], w = wij[cs + tid];
        pair_geometry<C>(sm.geo, tid, r, make_float3(w.x, w.y, w.z), dm);
      }
      __syncthreads();
      if (cs == P0 && nt < ntile) {
        // while this tile is contracted: the next tile's atom rows to shared
        // memory, its pair rows into L2 (the last warp has the fewest atoms)
        stage_rows(i0n, i1n);
        if (tid == 32 * kCgWarps - 1) {
          const int p0n = off[i0n], p1n = off[i1n];
          prefetch_l2(rij + p0n, (size_t)(p1n - p0n) * sizeof(float4));
          prefetch_l2(wij + p0n, (size_t)(p1n - p0n) * sizeof(float4));
        }
      }
      for (int at = warp; at < i1 - i0; at += kCgWarps) {
        const int q0 = max(sm.off[at], cs) - cs, q1 = min(sm.off[at + 1], ce) - cs;
        if (q0 >= q1) continue;
        FragA fa[2 * KS];  // [Sbar | Sdbar], k-steps of 8 columns
        const float* Am = &sm.A[at][0][0];
#pragma unroll
        for (int ks = 0; ks < 2 * KS; ++ks) {
          const int c = 8 * ks + t;
          frag_a<SPLIT>(fa[ks], g < NQA ? Am[g * kAS + c] : 0.f, g + 8 < NQA ? Am[(g + 8) * kAS + c] : 0.f,
                        g < NQA ? Am[g * kAS + c + 4] : 0.f, g + 8 < NQA ? Am[(g + 8) * kAS + c + 4] : 0.f);
        }
        const int I = sm.type[at];
        for (int p0 = q0; p0 < q1; p0 += 8) {
          const int sc = p0 + pg;
          const bool vc = sc < q1;
          Acc<SPLIT> Pb, Pd, Rc;
          Pb.zero();
          Pd.zero();
          Rc.zero();
#pragma unroll
          for (int ks = 0; ks < KS; ++ks) {
            const int r0 = 8 * ks + t;
            FragB fb, fd;
            frag_b<SPLIT>(fb, vc ? sm.geo.B[r0][sc] : 0.f, vc ? sm.geo.B[r0 + 4][sc] : 0.f);
            frag_b<SPLIT>(fd, vc ? sm.geo.D[r0][sc] : 0.f, vc ? sm.geo.D[r0 + 4][sc] : 0.f);
            mma_acc<SPLIT>(Pb, fa[ks], fb);
            mma_acc<SPLIT>(Pd, fa[KS + ks], fd);
            mma_acc<SPLIT>(Rc, fa[KS + ks], fb);
          }
          float P[4], R[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            P[r] = Pb.get(r) + Pd.get(r);
            R[r] = Rc.get(r);
          }
          const int s0 = p0 + t, s1 = p0 + t + 4;  // K rows t and t+4 of the second products
          const bool v0 = s0 < q1, v1 = s1 < q1;
          const int J0 = v0 ? sm.geo.J[s0] : -1, J1 = v1 ? sm.geo.J[s1] : -1;
          FragB ff[KT], fu[KT];
#pragma unroll
          for (int kt = 0; kt < KT; ++kt) {
            const int k = 8 * kt + g;
            const bool kv = k < KA;
            frag_b<SPLIT>(ff[kt], (kv && v0) ? sm.geo.f[k][s0] : 0.f, (kv && v1) ? sm.geo.f[k][s1] : 0.f);
            frag_b<SPLIT>(fu[kt], (kv && v0) ? sm.geo.fu[k][s0] : 0.f, (kv && v1) ? sm.geo.fu[k][s1] : 0.f);
          }
#pragma unroll
          for (int J = 0; J < NS; ++J) {
            const bool m0 = J0 == J, m1 = J1 == J;
            FragA ap, ar;
            frag_a<SPLIT>(ap, m0 ? P[0] : 0.f, m0 ? P[2] : 0.f, m1 ? P[1] : 0.f, m1 ? P[3] : 0.f);
            frag_a<SPLIT>(ar, m0 ? R[0] : 0.f, m0 ? R[2] : 0.f, m1 ? R[1] : 0.f, m1 ? R[3] : 0.f);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
              if (s != I) continue;
#pragma unroll
              for (int kt = 0; kt < KT; ++kt) {
                mma_acc<SPLIT>(acc[s][J][kt], ap, ff[kt]);
                mma_acc<SPLIT>(acc[s][J][kt], ar, fu[kt]);
              }
            }
          }
        }
      }
    }
    i0 = i0n;
    i1 = i1n;
    if (nt < ntile) {
      P0 = off[i0];
      P1 = off[i1];
    }
  }
  // fold the warps in order
  __syncthreads();
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int J = 0; J < NS; ++J)
#pragma unroll
      for (int kt = 0; kt < KT; ++kt)
#pragma unroll
        for (int r = 0; r < 4; ++r) sm.red[warp][((s * NS + J) * KT + kt) * 128 + lane * 4 + r] = acc[s][J][kt].get(r);
  __syncthreads();
  for (int q = tid; q < C::NCA; q += blockDim.x) {
    const int k = q % KA, n = (q / KA) % NQA, sj = q / (KA * NQA);  // sj = I NS + J
    const int kt = k / 8, kk = k % 8;
    const int idx = (sj * KT + kt) * 128 + ((n % 8) * 4 + kk / 2) * 4 + (n / 8) * 2 + kk % 2;
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < kCgWarps; ++w) v += sm.red[w][idx];
    cpart[(size_t)blockIdx.x * (C::NCR + C::NCA) + C::NCR + q] = v;
  }
}

// Radial part: one block per contiguous range of atoms, lane = column (J, k),
// warp r takes the range's atoms r, r + 16, ... (two per iteration, loads
// first); the block folds its warps in order and writes cpart[block][c^R].
constexpr int kCgRadialWarps = 16;

template <class C>
__global__ void __launch_bounds__(32 * kCgRadialWarps) k_cgrad_radial(int N, const int* __restrict__ type,
                                                                    const float* __restrict__ Gb,
                                                                    const float* __restrict__ Ep,
                                                                    const float* __restrict__ FR,
                                                                    const float* __restrict__ FRd,
                                                                    float* __restrict__ cpart) {
  GNEP_PDL_WAIT();
  constexpr int NCOL = C::NS * C::KR, NW = kCgRadialWarps;
  static_assert(NCOL <= 32, "one lane per radial column");
  __shared__ float red[NW][C::NS][C::NQR][32];
  const int lane = threadIdx.x & 31, r = threadIdx.x >> 5;
  const int per = (N + gridDim.x - 1) / gridDim.x;
  const int lo = min(N, (int)blockIdx.x * per), hi = min(N, lo + per);
  float acc[C::NS][C::NQR];
#pragma unroll
  for (int s = 0; s < C::NS; ++s)
#pragma unroll
    for (int n = 0; n < C::NQR; ++n) acc[s][n] = 0.f;
  if (lane < NCOL) {
    for (int i = lo + r; i < hi; i += 2 * NW) {
      int I[2];
      float fr[2], frd[2], gb[2][C::NQR], ep[2][C::NQR];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int iu = i + u * NW;
        const bool ok = iu < hi;
        I[u] = ok ? type[iu] : -1;
        fr[u] = ok ? FR[(size_t)iu * NCOL + lane] : 0.f;
        frd[u] = ok ? FRd[(size_t)iu * NCOL + lane] : 0.f;
#pragma unroll
        for (int n = 0; n < C::NQR; ++n) {
          gb[u][n] = ok ? Gb[(size_t)iu * C::NDES + n] : 0.f;
          ep[u][n] = ok ? Ep[(size_t)iu * C::NDES + n] : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int n = 0; n < C::NQR; ++n) {
          const float v = gb[u][n] * fr[u] - ep[u][n] * frd[u];
#pragma unroll
          for (int s = 0; s < C::NS; ++s) acc[s][n] += (s == I[u]) ? v : 0.f;
        }
    }
  }
#pragma unroll
  for (int s = 0; s < C::NS; ++s)
#pragma unroll
    for (int n = 0; n < C::NQR; ++n) red[r][s][n][lane] = acc[s][n];
  __syncthreads();
  for (int q = threadIdx.x; q < C::NCR; q += blockDim.x) {
    const int k = q % C::KR, n = (q / C::KR) % C::NQR, J = (q / (C::KR * C::NQR)) % C::NS,
              I = q / (C::KR * C::NQR * C::NS);
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) v += red[w][I][n][J * C::KR + k];
    cpart[(size_t)blockIdx.x * (C::NCR + C::NCA) + q] = v;
  }
}

// ------------------------------------------------------------- warp-product sweeps 1 and 3

// Angular descriptor and tangent sweeps on warp-level tensor cores, one warp
// per atom i (species I).  For each run of 8 of its pairs (columns),
//   G   = sum_J C^{IJ} F_J          (16 x 16) (16 x 8):  g_n(r_ij) of Eq. 6
//   Ga  = sum_J C^{IJ} Fu_J          tangent: g_n'(r_ij) (u_hat . u)
//   S  += G B^T                      (16 x 8) (8 x 24):   S_nlm of Eq. 8
//   Sd += Ga B^T + G D^T             tangent: Sdot_nlm
// where C^{IJ}[n][k] = c^A_nk^{IJ} and F_J holds f_k of the pairs whose
// neighbour has species J (zero elsewhere).  As in the c-gradient sweep, the
// C fragments of the first products are the A fragments of the second (column
// g holds pair g/2 + 4 (g mod 2)).  The epilogue forms q_nl (Eq. 7) and q4_n,
// or their tangents, from the accumulator fragments with lane shuffles.
template <class C, bool TAN>
struct AGeo {
  static constexpr int CHT = 256;                   // pairs per chunk
  static constexpr int SF = CHT + 8, SB = CHT + 4;  // f, fu rows 8 mod 32 words apart; B, D rows 4 mod 32
  float f[C::KA][SF];
  float fu[TAN ? C::KA : 1][SF];
  float B[NLM][SB];
  float D[TAN ? NLM : 1][SB];
  int J[CHT];
};
constexpr int kCS = 20;            // row stride of the staged C^{IJ} blocks (conflict-free A fragments)
constexpr int kAngWarps = 8;
constexpr int kAngMaxAtoms = 128;  // atoms per tile, at most

template <class C, bool TAN>
struct AngSmem {
  AGeo<C, TAN> geo;
  float c[C::NS * C::NS][16][kCS];  // C^{IJ}[n][k], zero-padded to 16 x 16
  int off[kAngMaxAtoms + 1];
  int type[kAngMaxAtoms];
};

// Lane (g, t) of an accumulator holds S[n][q] for n = g + 8h (h = r / 2) and
// q = 8 nq + 2t + (r mod 2).  Sum over the lane's q of C_q x_q y_q per degree
// l, completed over the four lanes of the row.  With l = 1 for q < 3, 2 for
// q < 8, 3 for q < 15 and 4 above, a lane's positions fall as: nq = 0 into
// l = 1 or 2 (by t), nq = 1 into l = 3 (q = 15 into l = 4), nq = 2 into l = 4.
// cq[nq][e] = C_q of the lane's positions.  The four sums are completed by
// halving exchanges (lane distance 2, then 1: each lane sends the half of its
// partial sums that it does not keep), so that lane t ends with the sum of
// degree l = t + 1 of each row half: out[h].
__device__ __forceinline__ void lsum_rows(const float (&x)[3][4], const float (&y)[3][4], const float (&cq)[3][2],
                                          int t, float (&out)[2]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float v[3][2], p[4];
#pragma unroll
    for (int nq = 0; nq < 3; ++nq)
#pragma unroll
      for (int e = 0; e < 2; ++e) v[nq][e] = cq[nq][e] * x[nq][2 * h + e] * y[nq][2 * h + e];
    p[0] = t == 0 ? v[0][0] + v[0][1] : (t == 1 ? v[0][0] : 0.f);
    p[1] = t == 1 ? v[0][1] : (t >= 2 ? v[0][0] + v[0][1] : 0.f);
    p[2] = v[1][0] + (t == 3 ? 0.f : v[1][1]);
    p[3] = (t == 3 ? v[1][1] : 0.f) + v[2][0] + v[2][1];
    const bool hi = t & 2, odd = t & 1;
    const float k0 = (hi ? p[2] : p[0]) + __shfl_xor_sync(0xffffffffu, hi ? p[0] : p[2], 2);
    const float k1 = (hi ? p[3] : p[1]) + __shfl_xor_sync(0xffffffffu, hi ? p[1] : p[3], 2);
    out[h] = (odd ? k1 : k0) + __shfl_xor_sync(0xffffffffu, odd ? k0 : k1, 1);
  }
}

// The five l = 2 moments (q = 3..7) of row half h, gathered from the lanes t = 1..3 of the row.
__device__ __forceinline__ void gather_l2(const float (&x)[3][4], int h, int lane, float (&s)[5]) {
  const int base = lane & ~3;
  s[0] = __shfl_sync(0xffffffffu, x[0][2 * h + 1], base + 1);
  s[1] = __shfl_sync(0xffffffffu, x[0][2 * h], base + 2);
  s[2] = __shfl_sync(0xffffffffu, x[0][2 * h + 1], base + 2);
  s[3] = __shfl_sync(0xffffffffu, x[0][2 * h], base + 3);
  s[4] = __shfl_sync(0xffffffffu, x[0][2 * h + 1], base + 3);
}

template <class C, bool TAN, bool SPLIT>
__global__ void __launch_bounds__(32 * kAngWarps, (TAN || SPLIT) ? 2 : 3)
    k_ang_mma(int ntile, const int* __restrict__ tiles, DevModel dm, const int* __restrict__ type,
              const int* __restrict__ atom_struct, const int* __restrict__ off, const int* __restrict__ own,
              const int* __restrict__ jj, const float4* __restrict__ rij, const float4* __restrict__ a,
              const float* __restrict__ Bs, const float* __restrict__ Sin, float* __restrict__ Sout,
              float* __restrict__ Gout, float4* __restrict__ wij) {
  GNEP_PDL_WAIT();
  using SM = AngSmem<C, TAN>;
  using GEO = AGeo<C, TAN>;
  constexpr int CHT = GEO::CHT, NQA = C::NQA, KA = C::KA, NS = C::NS;
  static_assert(NLM == 24 && NQA <= 16 && KA <= 16, "fragment shapes");
  extern __shared__ __align__(16) unsigned char smraw[];
  SM& sm = *reinterpret_cast<SM*>(smraw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int pg = (g >> 1) | ((g & 1) << 2);  // pair of B-fragment column g
  for (int q = tid; q < NS * NS * 16 * kCS; q += blockDim.x) {
    const int ij = q / (16 * kCS), r = q % (16 * kCS), n = r / kCS, k = r % kCS;
    sm.c[ij][n][k] = (n < NQA && k < KA) ? dm.params[dm.off_cA + (ij * NQA + n) * KA + k] : 0.f;
  }
  float cq[3][2];  // C_lm at this lane's accumulator positions
#pragma unroll
  for (int nq = 0; nq < 3; ++nq)
#pragma unroll
    for (int e = 0; e < 2; ++e) cq[nq][e] = kClm[8 * nq + 2 * t + e];

  int tile = blockIdx.x;
  int i0 = 0, i1 = 0, P0 = 0, P1 = 0;
  if (tile < ntile) {
    i0 = tiles[tile];
    i1 = tiles[tile + 1];
    P0 = off[i0];
    P1 = off[i1];
  }
  for (; tile < ntile; tile += gridDim.x) {
    const int nt = tile + gridDim.x;  // the next tile's bounds are fetched early
    const int i0n = nt < ntile ? tiles[nt] : 0, i1n = nt < ntile ? tiles[nt + 1] : 0;
    __syncthreads();  // the previous tile's readers are done (and the staged C^{IJ} is complete)
    if (tid <= i1 - i0) sm.off[tid] = off[i0 + tid];
    if (tid < i1 - i0) sm.type[tid] = type[i0 + tid];
    for (int cs = P0; cs < P1 || cs == P0; cs += CHT) {  // one pass even for a tile without pairs
      const int ce = min(cs + CHT, P1);
      if (cs != P0) __syncthreads();  // the previous chunk's readers are done
      if (cs + tid < ce) {
        const int p = cs + tid;
        const float4 r = rij[p];
        if (TAN) {
          const float3 w = tangent_dir(p, r, own, atom_struct, jj, a, Bs);
          wij[p] = make_float4(w.x, w.y, w.z, 0.f);  // reused by the c-gradient sweep
          pair_geometry<C>(sm.geo, tid, r, w, dm);
        } else {
          const float rr = sqrtf(r.x * r.x + r.y * r.y + r.z * r.z);
          const float ri = 1.f / rr;
          float f[KA], B[NLM];
          radial_basis<KA>(rr, dm.rca_inv, f);
          harmonics(r.x * ri, r.y * ri, r.z * ri, B);
#pragma unroll
          for (int k = 0; k < KA; ++k) sm.geo.f[k][tid] = f[k];
#pragma unroll
          for (int q = 0; q < NLM; ++q) sm.geo.B[q][tid] = B[q];
          sm.geo.J[tid] = (int)r.w;
        }
      }
      __syncthreads();
      if (tid == 32 * kAngWarps - 1 && cs == P0 && nt < ntile) {
        // the next tile's pair inputs move into L2 while this one is contracted
        const int p0n = off[i0n], p1n = off[i1n];
        prefetch_l2(rij + p0n, (size_t)(p1n - p0n) * sizeof(float4));
        if (TAN) {
          prefetch_l2(own + p0n, (size_t)(p1n - p0n) * sizeof(int));
          prefetch_l2(jj + p0n, (size_t)(p1n - p0n) * sizeof(int));
          prefetch_l2(Sin + (size_t)i0n * NQA * NLM, (size_t)(i1n - i0n) * NQA * NLM * sizeof(float));
        }
      }
      for (int at = warp; at < i1 - i0; at += kAngWarps) {
        const int ia0 = sm.off[at], ia1 = sm.off[at + 1];
        const int q0 = max(ia0, cs) - cs, q1 = min(ia1, ce) - cs;
        const bool first = ia0 >= cs, last = ia1 <= ce;  // the atom's pairs start / end in this chunk
        // an atom without pairs is written by the chunk that holds its position in the list
        const bool mine = ia0 < ia1 ? q0 < q1 : ((ia0 >= cs && ia0 < ce) || (ia0 == P1 && ce == P1));
        if (!mine) continue;
        const int I = sm.type[at], i = i0 + at;
        FragA fc[NS][2];  // C^{IJ}, k-steps of 8 basis functions
#pragma unroll
        for (int J = 0; J < NS; ++J)
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const float* cm = &sm.c[I * NS + J][0][0];
            const int c0 = 8 * ks + t;
            frag_a<SPLIT>(fc[J][ks], cm[g * kCS + c0], cm[(g + 8) * kCS + c0], cm[g * kCS + c0 + 4],
                          cm[(g + 8) * kCS + c0 + 4]);
          }
        Acc<SPLIT> sacc[3];
#pragma unroll
        for (int nq = 0; nq < 3; ++nq) sacc[nq].zero();
        float sv[3][4];  // tangent: S at the lane's accumulator positions, loaded ahead of the products
        if (TAN) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float* srow_in = Sin + ((size_t)i * NQA + min(g + 8 * h, NQA - 1)) * NLM;
#pragma unroll
            for (int nq = 0; nq < 3; ++nq) {
              const float2 v = g + 8 * h < NQA ? *reinterpret_cast<const float2*>(srow_in + 8 * nq + 2 * t)
                                               : make_float2(0.f, 0.f);
              sv[nq][2 * h] = v.x;
              sv[nq][2 * h + 1] = v.y;
            }
          }
        }
        for (int p0 = q0; p0 < q1; p0 += 8) {
          const int sc = p0 + pg;
          const int Jc = sc < q1 ? sm.geo.J[sc] : -1;
          Acc<SPLIT> G, Ga;
          G.zero();
          Ga.zero();
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const int k0 = 8 * ks + t, k1 = k0 + 4;
            const float f0 = (Jc >= 0 && k0 < KA) ? sm.geo.f[k0][sc] : 0.f;
            const float f1 = (Jc >= 0 && k1 < KA) ? sm.geo.f[k1][sc] : 0.f;
            float u0 = 0.f, u1 = 0.f;
            if (TAN) {
              u0 = (Jc >= 0 && k0 < KA) ? sm.geo.fu[k0][sc] : 0.f;
              u1 = (Jc >= 0 && k1 < KA) ? sm.geo.fu[k1][sc] : 0.f;
            }
#pragma unroll
            for (int J = 0; J < NS; ++J) {
              const bool m = Jc == J;
              FragB bf;
              frag_b<SPLIT>(bf, m ? f0 : 0.f, m ? f1 : 0.f);
              mma_acc<SPLIT>(G, fc[J][ks], bf);
              if (TAN) {
                FragB bu;
                frag_b<SPLIT>(bu, m ? u0 : 0.f, m ? u1 : 0.f);
                mma_acc<SPLIT>(Ga, fc[J][ks], bu);
              }
            }
          }
          // second products: K rows t and t+4 are the pairs t and t+4
          const int s0 = p0 + t, s1 = p0 + t + 4;
          const bool v0 = s0 < q1, v1 = s1 < q1;
          FragA ag, aga;
          frag_a<SPLIT>(ag, G.get(0), G.get(2), G.get(1), G.get(3));
          if (TAN) frag_a<SPLIT>(aga, Ga.get(0), Ga.get(2), Ga.get(1), Ga.get(3));
#pragma unroll
          for (int nq = 0; nq < 3; ++nq) {
            const int q = 8 * nq + g;
            FragB bb;
            frag_b<SPLIT>(bb, v0 ? sm.geo.B[q][s0] : 0.f, v1 ? sm.geo.B[q][s1] : 0.f);
            if (TAN) {
              FragB bd;
              frag_b<SPLIT>(bd, v0 ? sm.geo.D[q][s0] : 0.f, v1 ? sm.geo.D[q][s1] : 0.f);
              mma_acc<SPLIT>(sacc[nq], aga, bb);
              mma_acc<SPLIT>(sacc[nq], ag, bd);
            } else {
              mma_acc<SPLIT>(sacc[nq], ag, bb);
            }
          }
        }
        float acc[3][4];
#pragma unroll
        for (int nq = 0; nq < 3; ++nq)
#pragma unroll
          for (int r = 0; r < 4; ++r) acc[nq][r] = sacc[nq].get(r);
        // S (or Sdot) of row n = g + 8h at q = 8 nq + 2t, +1
        float* srow[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) srow[h] = Sout + ((size_t)i * NQA + min(g + 8 * h, NQA - 1)) * NLM;
        if (!first) {  // earlier chunks of this tile left a partial sum
#pragma unroll
          for (int h = 0; h < 2; ++h)
            if (g + 8 * h < NQA)
#pragma unroll
              for (int nq = 0; nq < 3; ++nq) {
                const float2 v = *reinterpret_cast<const float2*>(srow[h] + 8 * nq + 2 * t);
                acc[nq][2 * h] += v.x;
                acc[nq][2 * h + 1] += v.y;
              }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
          if (g + 8 * h < NQA)
#pragma unroll
            for (int nq = 0; nq < 3; ++nq)
              *reinterpret_cast<float2*>(srow[h] + 8 * nq + 2 * t) = make_float2(acc[nq][2 * h], acc[nq][2 * h + 1]);
        if (!last) continue;  // completed in a later chunk
        float* gi = Gout + (size_t)i * C::NDES;
        if (!TAN) {
          float ql[2];
          lsum_rows(acc, acc, cq, t, ql);  // q_nl = sum_m C_lm S_nlm^2 (Eq. 7)
#pragma unroll
          for (int h = 0; h < 2; ++h)
            if (g + 8 * h < NQA) gi[C::vang(g + 8 * h, t + 1)] = ql[h];
          if (C::FB) {  // q4 of row g + 8h on lane t = h: one evaluation per lane for both halves
            float s2[2][5];
            gather_l2(acc, 0, lane, s2[0]);
            gather_l2(acc, 1, lane, s2[1]);
            const int h = t & 1, n = g + 8 * h;
            float sel[5];
#pragma unroll
            for (int m = 0; m < 5; ++m) sel[m] = h ? s2[1][m] : s2[0][m];
            const float q4 = q4_value(sel);
            if (t < 2 && n < NQA) gi[C::v4b(n)] = q4;
          }
        } else {
          float ql[2];
          lsum_rows(sv, acc, cq, t, ql);  // qdot_nl = 2 sum_m C_lm S_nlm Sdot_nlm
#pragma unroll
          for (int h = 0; h < 2; ++h)
            if (g + 8 * h < NQA) gi[C::vang(g + 8 * h, t + 1)] = 2.f * ql[h];
          if (C::FB) {  // qdot4 of row g + 8h on lane t = h: one evaluation per lane for both halves
            float s2[2][5], d2[2][5];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              gather_l2(sv, h, lane, s2[h]);
              gather_l2(acc, h, lane, d2[h]);
            }
            const int h = t & 1, n = g + 8 * h;
            float ss[5], dd[5], g4[5];
#pragma unroll
            for (int m = 0; m < 5; ++m) {
              ss[m] = h ? s2[1][m] : s2[0][m];
              dd[m] = h ? d2[1][m] : d2[0][m];
            }
            q4_grad(ss, g4);
            float q = 0.f;
#pragma unroll
            for (int m = 0; m < 5; ++m) q = fmaf(g4[m], dd[m], q);
            if (t < 2 && n < NQA) gi[C::v4b(n)] = q;
          }
        }
      }
      if (ce >= P1) break;
    }
    i0 = i0n;
    i1 = i1n;
    if (nt < ntile) {
      P0 = off[i0];
      P1 = off[i1];
    }
  }
}

template <class C, bool TAN, bool SPLIT>
int ang_grid_cap() {
  static int cap = 0;  // resident blocks on this GPU (the same value on every call)
  if (!cap) {
    int per_sm = 0, dev = 0, sms = 0;
    GNEP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ang_mma<C, TAN, SPLIT>, 32 * kAngWarps,
                                                            sizeof(AngSmem<C, TAN>)));
    GNEP_CUDA(cudaGetDevice(&dev));
    GNEP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cap = (per_sm > 0 ? per_sm : 1) * sms;
  }
  return cap;
}

// Descriptor (TAN = false: S, q_nl, q4 into Sout, Gout) or tangent (TAN = true:
// Sdot, qdot into Sout, Gout; w_ij into wij) sweep over the tiles of atile[0].
// Products carry FP32 accuracy (split TF32) in every precision mode: the
// precision modes narrow the network contractions only.
template <class C, bool TAN>
int launch_ang(const gnep_model* m, const gnep_nlist* nl, cudaStream_t st, const float4* a, const float* Bs,
               const float* Sin, float* Sout, float* Gout, float4* wij) {
  (void)m;
  const int ntile = nl->natile[0];
  if (ntile < 1) return GNEP_OK;
  const int cap = ang_grid_cap<C, TAN, true>();
  const int nb = ntile < cap ? ntile : cap;
  auto kern = k_ang_mma<C, TAN, true>;
  (void)launch_pdl(kern, nb, 32 * kAngWarps, sizeof(AngSmem<C, TAN>), st, ntile, nl->atile[0], m->dev(), nl->type, nl->atom_struct,
                                                            nl->L[1].off, nl->L[1].owner, nl->L[1].j, nl->L[1].rij,
                                                            a, Bs, Sin, Sout, Gout, wij);
  return GNEP_OK;
}

template <class C, bool TAN, bool SPLIT>
int setup_ang() {
  GNEP_CUDA(cudaFuncSetAttribute(k_ang_mma<C, TAN, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(AngSmem<C, TAN>)));
  GNEP_CUDA(cudaFuncSetAttribute(k_ang_mma<C, TAN, SPLIT>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  return ang_grid_cap<C, TAN, SPLIT>() > 0 ? GNEP_OK : GNEP_ERR_CUDA;
}

// ------------------------------------------------------------- launchers

// Launch CALL (which names RL) with RL = the radial sweeps' lanes per atom.
// The radial sweep of a phase beside its angular sweep: the radial kernel goes
// to the list's second stream, which first waits for the caller's stream (fork)
// and which the caller's stream waits for before the phase's consumer (join).
// The two kernels write disjoint columns of G, Gdot and the c-gradient
// partials.  Per-stage timing keeps them in turn.  *rs is the radial stream.
static int radial_fork(gnep_nlist* nl, cudaStream_t st, cudaStream_t* rs) {
  *rs = st;
  if (g_prof.on || !nl->side || !radial_beside(nl)) return GNEP_OK;
  GNEP_CUDA(cudaEventRecord(nl->fork_ev, st));
  GNEP_CUDA(cudaStreamWaitEvent(nl->side, nl->fork_ev, 0));
  *rs = nl->side;
  return GNEP_OK;
}
static int radial_join(gnep_nlist* nl, cudaStream_t st, cudaStream_t rs) {
  if (rs == st) return GNEP_OK;
  GNEP_CUDA(cudaEventRecord(nl->join_ev, rs));
  GNEP_CUDA(cudaStreamWaitEvent(st, nl->join_ev, 0));
  return GNEP_OK;
}

#define GNEP_RADIAL_LANES(RLV, CALL)  \
  switch (RLV) {                      \
    case 16: {                        \
      constexpr int RL = 16;          \
      CALL;                           \
    } break;                          \
    case 8: {                         \
      constexpr int RL = 8;           \
      CALL;                           \
    } break;                          \
    default: {                        \
      constexpr int RL = 4;           \
      CALL;                           \
    }                                 \
  }

namespace {

template <class C>
struct Runner {
  // Network forward/backward in the model's precision: plain FP32 tiles, or
  // tensor-core tiles with TF32 or BF16 operands.
  static int network_forward(const gnep_model* m, gnep_nlist* nl, cudaStream_t st) {
    if (C::LMAX > 4 || m->precision == GNEP_PREC_FP32) {
      switch (hidden_pad(m->shape.H)) {
        case 32: return mlp_forward<C::NDES, 32, C::NS, C::NQR, C::KR>(m, nl, st);
        case 64: return mlp_forward<C::NDES, 64, C::NS, C::NQR, C::KR>(m, nl, st);
        default: return mlp_forward<C::NDES, 128, C::NS, C::NQR, C::KR>(m, nl, st);
      }
    }
    if constexpr (C::LMAX > 4) {
      return set_error(GNEP_ERR_UNSUPPORTED, "l_max > 4 runs the FP32 network only");
    } else {
      const bool tf = m->precision == GNEP_PREC_TF32;
      switch (hidden_pad_tc(m->shape.H)) {
        case 32:
          return tf ? mlp_forward_tc<true, C::NDES, 32, C::NS, C::NQR, C::KR>(m, nl, st)
                    : mlp_forward_tc<false, C::NDES, 32, C::NS, C::NQR, C::KR>(m, nl, st);
        case 64:
          return tf ? mlp_forward_tc<true, C::NDES, 64, C::NS, C::NQR, C::KR>(m, nl, st)
                    : mlp_forward_tc<false, C::NDES, 64, C::NS, C::NQR, C::KR>(m, nl, st);
        default:
          return tf ? mlp_forward_tc<true, C::NDES, 112, C::NS, C::NQR, C::KR>(m, nl, st)
                    : mlp_forward_tc<false, C::NDES, 112, C::NS, C::NQR, C::KR>(m, nl, st);
      }
    }
  }

  static int network_backward(const gnep_model* m, gnep_nlist* nl, cudaStream_t st) {
    if (C::LMAX > 4 || m->precision == GNEP_PREC_FP32) {
      switch (hidden_pad(m->shape.H)) {
        case 32: return mlp_backward<C::NDES, 32>(m, nl, st);
        case 64: return mlp_backward<C::NDES, 64>(m, nl, st);
        default: return mlp_backward<C::NDES, 128>(m, nl, st);
      }
    }
    if constexpr (C::LMAX > 4) {
      return set_error(GNEP_ERR_UNSUPPORTED, "l_max > 4 runs the FP32 network only");
    } else {
      const bool tf = m->precision == GNEP_PREC_TF32;
      switch (hidden_pad_tc(m->shape.H)) {
        case 32:
          return tf ? mlp_backward_tc<true, C::NDES, 32>(m, nl, st) : mlp_backward_tc<false, C::NDES, 32>(m, nl, st);
        case 64:
          return tf ? mlp_backward_tc<true, C::NDES, 64>(m, nl, st) : mlp_backward_tc<false, C::NDES, 64>(m, nl, st);
        default:
          return tf ? mlp_backward_tc<true, C::NDES, 112>(m, nl, st)
                    : mlp_backward_tc<false, C::NDES, 112>(m, nl, st);
      }
    }
  }

  static int descriptors(const StepArgs& A, bool with_mlp) {
    const gnep_model* m = A.m;
    gnep_nlist* nl = A.nl;
    Workspace& w = nl->ws;
    const DevModel dm = m->dev();
    const int N = nl->n_atoms;
    if (N == 0) return GNEP_OK;
    cudaStream_t rs;
    if (int rc = radial_fork(nl, A.st, &rs)) return rc;
    GNEP_RADIAL_LANES(radial_lanes(nl), ((void)launch_on(rs == A.st, k_desc_radial<C, RL>,
                                             blocks_for((int64_t)N * RL, 128), 128, 0, rs,
                                             N, dm, nl->type, nl->L[0].off, nl->L[0].rij, w.FR, w.G)));
    stage("desc_radial");
    if constexpr (C::LMAX > 4) {
      if (int rc = hi_desc_angular<C>(m, nl, A.st, w.S, w.G)) return rc;
    } else {
      if (int rc = launch_ang<C, false>(m, nl, A.st, nullptr, nullptr, nullptr, w.S, w.G, nullptr)) return rc;
    }
    stage("desc_angular");
    if (int rc = radial_join(nl, A.st, rs)) return rc;
    GNEP_CHECK_LAUNCH("descriptor sweep");
    if (with_mlp) {
      if (int rc = network_forward(m, nl, A.st)) return rc;
      stage("mlp_fwd");
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
    if (nl->L[1].n > 0) {
      if constexpr (C::LMAX > 4) {
        if (int rc = hi_force_angular<C>(m, nl, A.st, w.S, w.Ep, w.dA)) return rc;
      } else {
        (void)launch_pdl(k_force_angular<C>, nl->natile[1], 128, 0, A.st, N, dm, nl->atile[1], nl->type, nl->L[1].off,
                                                             nl->L[1].owner, nl->L[1].rij, w.S, w.Ep, w.dA);
      }
      stage("force_angular");
    }
    GNEP_RADIAL_LANES(radial_lanes(nl), ((void)launch_pdl(k_force_atoms<C, RL>, blocks_for((int64_t)N * RL, 128), 128, 0, A.st, 
                                             N, dm, nl->type, nl->L[0].off, nl->L[0].j, nl->L[0].rij, w.chat,
                                             nl->L[1].off, nl->L[1].rev, nl->L[1].rij, w.dA, w.F, w.Wat)));
    stage("force_atoms");
    if (!A.loss_follows) {  // otherwise the loss kernel forms these sums
      (void)launch_pdl(k_struct_sum, nl->n_struct, 128, 0, A.st, nl->struct_off, w.Eatom, w.Wat, w.Es, w.Ws);
      stage("struct_sum");
    }
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
    cudaStream_t rs;
    if (int rc = radial_fork(nl, A.st, &rs)) return rc;
    GNEP_RADIAL_LANES(radial_lanes(nl),
                      ((void)launch_on(rs == A.st, k_tangent_radial<C, RL>, blocks_for((int64_t)N * RL, 128), 128, 0,
                          rs, N, dm, nl->type, nl->atom_struct, nl->L[0].off, nl->L[0].j, nl->L[0].rij, w.a, w.Bs,
                          w.FRd, w.Gd)));
    stage("tangent_radial");
    if constexpr (C::LMAX > 4) {
      if (int rc = hi_tangent_angular<C>(m, nl, A.st, w.a, w.Bs, w.S, w.Sd, w.Gd, w.wij)) return rc;
    } else {
      if (int rc = launch_ang<C, true>(m, nl, A.st, w.a, w.Bs, w.S, w.Sd, w.Gd, w.wij)) return rc;
    }
    stage("tangent_angular");
    if (int rc = radial_join(nl, A.st, rs)) return rc;
    if (int rc = network_backward(m, nl, A.st)) return rc;
    stage("mlp_bwd");
    const int nb = cgrad_blocks(nl);
    if (int rc = radial_fork(nl, A.st, &rs)) return rc;
    (void)launch_on(rs == A.st, k_cgrad_radial<C>, nb, 32 * kCgRadialWarps, 0, rs, N, nl->type, w.Gb, w.Ep, w.FR,
                    w.FRd, w.cpart);
    stage("cgrad_radial");
    if constexpr (C::LMAX > 4) {
      if (int rc = hi_cgrad_angular<C>(m, nl, A.st, nb, w.wij, w.S, w.Sd, w.Gb, w.Ep, w.cpart)) return rc;
    } else {
      auto ang = k_cgrad_ang<C, true>;  // split TF32 in every precision mode
      (void)launch_pdl(ang, nb, 32 * kCgWarps, sizeof(CgSmem<C>), A.st, nl->natile[1], nl->atile[1], dm, nl->type, nl->L[1].off,
                                                           nl->L[1].rij, w.wij, w.S, w.Sd, w.Gb, w.Ep, w.cpart);
    }
    stage("cgrad");
    if (int rc = radial_join(nl, A.st, rs)) return rc;
    GNEP_CHECK_LAUNCH("backward sweeps");
    return GNEP_OK;
  }
};

}  // namespace

// Shapes with compiled kernels: (species, n_max+1, basis+1 radial; same angular; 4-body; l_max).
#define GNEP_SHAPES(X)            \
  X(2, 5, 9, 5, 9, false, 4)      \
  X(2, 9, 13, 9, 13, true, 4)     \
  X(2, 9, 13, 9, 13, false, 4)    \
  X(2, 5, 9, 5, 9, false, 6)      \
  X(2, 5, 9, 5, 9, true, 8)

#define GNEP_MATCH(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM)                                                \
  (s.ns == P_NS && s.nqr == P_NQR && s.kr == P_KR && s.nqa == P_NQA && s.ka == P_KA && (s.fb != 0) == P_FB && \
   s.lmax == P_LM)

bool shape_supported(const Shape& s) {
#define X(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM) \
  if (GNEP_MATCH(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM)) return true;
  GNEP_SHAPES(X)
#undef X
  return false;
}

namespace {
template <class C>
int setup_shape() {
  if constexpr (C::LMAX > 4) {
    int rc = hi_setup<C>();
    if (!rc) rc = mlp_setup<C::NDES, 32, C::NS, C::NQR, C::KR>();
    if (!rc) rc = mlp_setup<C::NDES, 64, C::NS, C::NQR, C::KR>();
    if (!rc) rc = mlp_setup<C::NDES, 128, C::NS, C::NQR, C::KR>();
    return rc;
  } else {
    if (int rc = setup_ang<C, false, true>()) return rc;
    if (int rc = setup_ang<C, true, true>()) return rc;
    GNEP_CUDA(cudaFuncSetAttribute(k_cgrad_ang<C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(CgSmem<C>)));
    GNEP_CUDA(cudaFuncSetAttribute(k_cgrad_ang<C, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int rc = mlp_setup<C::NDES, 32, C::NS, C::NQR, C::KR>();
    if (!rc) rc = mlp_setup<C::NDES, 64, C::NS, C::NQR, C::KR>();
    if (!rc) rc = mlp_setup<C::NDES, 128, C::NS, C::NQR, C::KR>();
    if (!rc) rc = mlp_setup_tc<false, C::NDES, 32, C::NS, C::NQR, C::KR>();
    if (!rc) rc = mlp_setup_tc<false, C::NDES, 64, C::NS, C::NQR, C::KR>();
    if (!rc) rc = mlp_setup_tc<false, C::NDES, 112, C::NS, C::NQR, C::KR>();
    if (!rc) rc = mlp_setup_tc<true, C::NDES, 32, C::NS, C::NQR, C::KR>();
    if (!rc) rc = mlp_setup_tc<true, C::NDES, 64, C::NS, C::NQR, C::KR>();
    if (!rc) rc = mlp_setup_tc<true, C::NDES, 112, C::NS, C::NQR, C::KR>();
    return rc;
  }
}
}  // namespace

int shape_setup(const Shape& s) {
#define X(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM) \
  if (GNEP_MATCH(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM)) \
    return setup_shape<Sh<P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM>>();
  GNEP_SHAPES(X)
#undef X
  return set_error(GNEP_ERR_UNSUPPORTED, "no kernel for this shape");
}

int run_descriptors(const StepArgs& A, bool with_mlp) {
  const Shape& s = A.m->shape;
#define X(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM) \
  if (GNEP_MATCH(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM)) \
    return Runner<Sh<P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM>>::descriptors(A, with_mlp);
  GNEP_SHAPES(X)
#undef X
  return set_error(GNEP_ERR_UNSUPPORTED, "no kernel for this shape");
}

int run_forward(const StepArgs& A) {
  const Shape& s = A.m->shape;
#define X(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM) \
  if (GNEP_MATCH(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM)) \
    return Runner<Sh<P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM>>::forward(A);
  GNEP_SHAPES(X)
#undef X
  return set_error(GNEP_ERR_UNSUPPORTED, "no kernel for this shape");
}

int run_backward(const StepArgs& A) {
  const Shape& s = A.m->shape;
#define X(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM) \
  if (GNEP_MATCH(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM)) \
    return Runner<Sh<P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM>>::backward(A);
  GNEP_SHAPES(X)
#undef X
  return set_error(GNEP_ERR_UNSUPPORTED, "no kernel for this shape");
}

// SMs of this GPU (looked up once).
int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n < 1)
      n = 1;
    sms = n;
  }
  return sms;
}

// Lanes per atom of the radial sweeps: the tuned value, else 4 while that
// gives every SM at least four blocks of 128 threads, and 8 or 16 below.
int radial_lanes(const gnep_nlist* nl) {
  if (nl->tune.radial_lanes > 0) return nl->tune.radial_lanes;
  const int64_t full = 4LL * 128 * sm_count();  // threads of four blocks per SM
  const int64_t N = nl->n_atoms;
  return 4 * N >= full ? 4 : 8 * N >= full ? 8 : 16;
}

// The radial sweeps run beside the angular ones when tuned so, and by default
// while the angular descriptor sweep has fewer than eight tiles per SM.  The
// sweeps of both kinds are chains of dependent loads and products with idle
// issue slots: on a small batch neither fills the GPU and the two at once hide
// the shorter one; up to a few tiles per SM the radial warps still fill issue
// slots the angular warps leave (on the 256-structure workload, about 1,900
// tiles, the two placements time the same).
bool radial_beside(const gnep_nlist* nl) {
  if (nl->tune.beside > 0) return nl->tune.beside == 2;
  return nl->natile[0] < 8 * sm_count();
}

// Persistent blocks of the c-gradient sweep: one per tile up to the default
// (or tuned) count, at most kCgBlocksMax (the size of the partial buffer).
int cgrad_blocks(const gnep_nlist* nl) {
  const int ntiles = nl->natile[1];
  int cap = nl->tune.cg_blocks > 0 ? nl->tune.cg_blocks : kCgBlocksPerSm * sm_count();
  if (cap > kCgBlocksMax) cap = kCgBlocksMax;
  return ntiles < cap ? (ntiles > 0 ? ntiles : 1) : cap;
}

// Tile limits of the angular sweeps: [0] descriptor and tangent sweeps (one
// warp per atom, chunks of 256 pairs: 32 atoms, 256 pairs), [1] force and
// c-gradient sweeps (one thread per (atom, channel) in the force sweep, CH pairs).
void angular_tile_limits(const Shape& s, int which, int* na, int* ch) {
  const int nq = s.nqr > s.nqa ? s.nqr : s.nqa;
  if (which == 0) {
    *na = 32;
    *ch = AGeo<Sh<1, 1, 1, 1, 1, false>, false>::CHT;
  } else {
    *na = 128 / nq;
    *ch = CH;
  }
}

}  // namespace gnep

// ---------------------------------------------------------------------------
// Descriptors without any device allocation.
//
// Some callers must not allocate device memory at the point where they need
// descriptors: hosts whose device memory is reserved up front by another
// allocator or a fixed pool (a cudaMalloc there fails or fragments the pool),
// and per-step hooks of simulation engines that forbid allocation in their hot
// loop (cudaMalloc and cudaFree may synchronise the device).  For them the
// descriptor sweep can use this fixed scratch array, which every GPU that
// loads the library holds until the process exits, instead of workspace
// memory.  Calls share the array; calls that overlap on the GPU race.
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
  const int64_t sa = N * C::NQA * C::NLX;
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
  GNEP_RADIAL_LANES(radial_lanes(nl), ((void)launch_pdl(k_desc_radial<C, RL>, blocks_for(N * RL, 128), 128, 0, A.st, 
                                           (int)N, dm, nl->type, nl->L[0].off, nl->L[0].rij, scratch, G)));
  if constexpr (C::LMAX > 4) {
    if ((rc = hi_desc_angular<C>(m, nl, A.st, scratch + fr_padded, G))) return rc;
  } else {
    if ((rc = launch_ang<C, false>(m, nl, A.st, nullptr, nullptr, nullptr, scratch + fr_padded, G, nullptr))) return rc;
  }
  GNEP_CHECK_LAUNCH("descriptor sweep (static scratch)");
  return GNEP_OK;
}

}  // namespace

int run_descriptors_static(const StepArgs& A, float* G) {
  const Shape& s = A.m->shape;
#define X(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM) \
  if (GNEP_MATCH(P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM)) \
    return descriptors_static<Sh<P_NS, P_NQR, P_KR, P_NQA, P_KA, P_FB, P_LM>>(A, G);
  GNEP_SHAPES(X)
#undef X
  return set_error(GNEP_ERR_UNSUPPORTED, "no kernel for this shape");
}

}  // namespace gnep
