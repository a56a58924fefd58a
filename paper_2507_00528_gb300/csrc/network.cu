// Per-element one-hidden-layer network (D1.1-D1.10) on species-homogeneous
// tiles of 32 atoms.  The contractions are register-blocked FP32 tile GEMMs
// from shared memory; the network-parameter gradient (D1.18-D1.21 through the
// tangent/reverse pass) is accumulated in registers over the tiles a
// persistent block visits and written once per block and species.  Every sum
// runs in a fixed order (no atomics), so results are bit-reproducible.
#include <cstdio>

#include "gnep_internal.h"
#include "network.cuh"

namespace gnep {

namespace {

constexpr int TM = kTileAtoms;  // atoms per tile
constexpr int NT = 128;         // threads per block

__device__ __forceinline__ void tile_of(const Tiles& T, int t, int& e, int& a0, int& na) {
  e = 0;
  while (e + 1 < T.ns && t >= T.tbase[e + 1]) ++e;
  a0 = T.soff[e] + (t - T.tbase[e]) * TM;
  na = min(TM, T.soff[e + 1] - a0);
}

// C[m][n] (TM rows, NP cols) = sum_k A[k][m] B[k][n]; A and B k-major in shared
// memory.  Thread t owns 4x4 blocks t, t+NT, ...; f(m0, n0, acc) gets each.
template <int NP, int K, int LDA, int LDB, class F>
__device__ __forceinline__ void tile_gemm(const float* A, const float* B, F f) {
  constexpr int NB = (TM / 4) * (NP / 4);
  for (int blk = threadIdx.x; blk < NB; blk += NT) {
    const int m0 = (blk / (NP / 4)) * 4, n0 = (blk % (NP / 4)) * 4;
    float acc[4][4] = {};
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(A + k * LDA + m0);
      const float4 b = *reinterpret_cast<const float4*>(B + k * LDB + n0);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[u][w] = fmaf(av[u], bv[w], acc[u][w]);
    }
    f(m0, n0, acc);
  }
}

// Weights of species e, zero-padded: W0t [DP][HP] (for z = G W0^T) and
// W0n [HP][DP] (for E' = beta W0), b0 and w1 [HP].
template <int D, int DP, int HP>
__device__ void load_weights(const DevModel& dm, int e, float* W0t, float* W0n, float* b0, float* w1) {
  const float* P = dm.params + (size_t)e * dm.net_size;
  const int H = dm.H;
  for (int q = threadIdx.x; q < DP * HP; q += NT) {
    const int v = q / HP, mu = q % HP;
    const float w = (v < D && mu < H) ? P[mu * D + v] : 0.f;
    W0t[q] = w;
    W0n[mu * DP + v] = w;
  }
  for (int mu = threadIdx.x; mu < HP; mu += NT) {
    b0[mu] = mu < H ? P[D * H + mu] : 0.f;
    w1[mu] = mu < H ? P[D * H + H + mu] : 0.f;
  }
}

}  // namespace

template <int D, int HP, int NS, int NQR, int KR>
size_t mlp_fwd_smem() {
  constexpr int DP = (D + 3) / 4 * 4;
  return sizeof(float) * (2 * DP * HP + 2 * HP + DP * TM + 2 * HP * TM + NS * NQR * KR);
}

// Forward per tile: z = W0 (s.G) + b0, x = tanh z, E = w1.x + b1,
// E' = s . (W0^T (w1 (1 - x^2)))  (D1.1-D1.5), and the per-atom radial
// contraction chat_i[J][k] = sum_n E'_n c^R_nk^{IJ} the force sweep uses.
template <int D, int HP, int NS, int NQR, int KR>
__global__ void __launch_bounds__(NT) k_mlp_fwd_tile(Tiles T, DevModel dm, const float* __restrict__ G,
                                                     float* __restrict__ X, float* __restrict__ Ep,
                                                     float* __restrict__ Eatom, float* __restrict__ chat) {
  constexpr int DP = (D + 3) / 4 * 4;
  extern __shared__ float4 sm4[];
  float* sm = reinterpret_cast<float*>(sm4);
  float* W0t = sm;                // [DP][HP]
  float* W0n = W0t + DP * HP;     // [HP][DP]
  float* b0 = W0n + HP * DP;      // [HP]
  float* w1 = b0 + HP;            // [HP]
  float* Gt = w1 + HP;            // [DP][TM] scaled inputs, later E'
  float* Bt = Gt + DP * TM;       // [HP][TM] beta
  float* Xs = Bt + HP * TM;       // [TM][HP] x
  float* cR = Xs + TM * HP;       // [NS][NQR][KR] of this species
  __shared__ int rows[TM];
  int e, a0, na;
  tile_of(T, blockIdx.x, e, a0, na);
  load_weights<D, DP, HP>(dm, e, W0t, W0n, b0, w1);
  for (int q = threadIdx.x; q < NS * NQR * KR; q += NT) cR[q] = dm.params[dm.off_cR + e * NS * NQR * KR + q];
  if (threadIdx.x < TM) rows[threadIdx.x] = threadIdx.x < na ? T.perm[a0 + threadIdx.x] : -1;
  __syncthreads();
  for (int q = threadIdx.x; q < DP * TM; q += NT) {
    const int v = q / TM, a = q % TM, r = rows[a];
    Gt[q] = (r >= 0 && v < D) ? dm.scale[v] * G[(size_t)r * D + v] : 0.f;
  }
  __syncthreads();
  const int H = dm.H;
  tile_gemm<HP, DP, TM, HP>(Gt, W0t, [&](int m0, int n0, float (&acc)[4][4]) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int a = m0 + u, mu = n0 + w;
        const float x = mu < H ? tanhf(acc[u][w] + b0[mu]) : 0.f;
        Xs[a * HP + mu] = x;
        Bt[mu * TM + a] = w1[mu] * (1.f - x * x);
      }
  });
  __syncthreads();
  // energies (thread a, fixed order) and x to global
  if (threadIdx.x < na) {
    const int a = threadIdx.x;
    float E = 0.f;
    for (int mu = 0; mu < H; ++mu) E = fmaf(w1[mu], Xs[a * HP + mu], E);
    Eatom[rows[a]] = E + dm.params[(size_t)e * dm.net_size + D * H + 2 * H];
  }
  for (int q = threadIdx.x; q < na * H; q += NT) {
    const int a = q / H, mu = q % H;
    X[(size_t)rows[a] * H + mu] = Xs[a * HP + mu];
  }
  tile_gemm<DP, HP, TM, DP>(Bt, W0n, [&](int m0, int n0, float (&acc)[4][4]) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int a = m0 + u, v = n0 + w;
        Gt[v * TM + a] = v < D ? acc[u][w] * dm.scale[v] : 0.f;  // Gt no longer read by the GEMM above
      }
  });
  __syncthreads();
  for (int q = threadIdx.x; q < na * D; q += NT) {
    const int a = q / D, v = q % D;
    Ep[(size_t)rows[a] * D + v] = Gt[v * TM + a];
  }
  for (int q = threadIdx.x; q < na * NS * KR; q += NT) {
    const int a = q / (NS * KR), jk = q % (NS * KR), J = jk / KR, k = jk % KR;
    float s = 0.f;
#pragma unroll
    for (int n = 0; n < NQR; ++n) s = fmaf(Gt[n * TM + a], cR[(J * NQR + n) * KR + k], s);
    chat[(size_t)rows[a] * NS * KR + jk] = s;
  }
}

template <int D, int HP>
size_t mlp_bwd_smem() {
  constexpr int DP = (D + 3) / 4 * 4;
  return sizeof(float) * (2 * DP * HP + 2 * HP + 3 * TM * DP + 4 * HP * TM);
}

// Tangent and reverse pass per tile, with the energy residual weight e_i:
//   zdot = W0 (s.Gdot), beta = w1 (1 - x^2), alpha = e_i beta + 2 x beta zdot,
//   Gbar = s . (W0^T alpha),
//   dW0 += alpha (s.G)^T - beta (s.Gdot)^T, db0 += alpha,
//   dw1 += e_i x - (1 - x^2) zdot, db1 += e_i.
// Persistent blocks visit tiles blockIdx.x, +gridDim.x, ... (species in
// order) and write one partial per species visited into part[block][species]
// (zeroed beforehand).
template <int D, int HP>
__global__ void __launch_bounds__(NT) k_mlp_bwd_tile(Tiles T, int ntiles, DevModel dm,
                                                     const int* __restrict__ atom_struct,
                                                     const float* __restrict__ es, const float* __restrict__ G,
                                                     const float* __restrict__ Gd, const float* __restrict__ X,
                                                     float* __restrict__ Gb, float* __restrict__ part,
                                                     int part_stride) {
  constexpr int DP = (D + 3) / 4 * 4;
  constexpr int NBLK = (HP / 4) * (DP / 4);
  constexpr int NBW = (NBLK + NT - 1) / NT;
  extern __shared__ float4 sm4[];
  float* sm = reinterpret_cast<float*>(sm4);
  float* W0t = sm;               // [DP][HP]
  float* W0n = W0t + DP * HP;    // [HP][DP]
  float* b0 = W0n + HP * DP;
  float* w1 = b0 + HP;
  float* Gt = w1 + HP;           // [TM][DP] s.G, atom-major
  float* Gdk = Gt + TM * DP;     // [DP][TM] s.Gdot, k-major
  float* Gda = Gdk + DP * TM;    // [TM][DP] s.Gdot, atom-major
  float* Al = Gda + TM * DP;     // [HP][TM] alpha, k-major
  float* Ala = Al + HP * TM;     // [TM][HP] alpha, atom-major
  float* Bea = Ala + TM * HP;    // [TM][HP] -beta, atom-major
  float* Q1 = Bea + TM * HP;     // [TM][HP] e x - (1 - x^2) zdot
  __shared__ int rows[TM];
  __shared__ float ei[TM];
  const int H = dm.H;
  float accW[NBW][4][4];
  float sb0 = 0.f, sw1 = 0.f, sb1 = 0.f;  // column mu = threadIdx.x (and b1 on thread 0)
  int cur_e = -1;

  auto reset = [&]() {
#pragma unroll
    for (int q = 0; q < NBW; ++q)
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) accW[q][u][w] = 0.f;
    sb0 = sw1 = sb1 = 0.f;
  };
  auto flush = [&](int e) {
    float* out = part + ((size_t)blockIdx.x * T.ns + e) * part_stride;
#pragma unroll
    for (int q = 0; q < NBW; ++q) {
      const int blk = threadIdx.x + q * NT;
      if (blk >= NBLK) continue;
      const int m0 = (blk / (DP / 4)) * 4, n0 = (blk % (DP / 4)) * 4;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int mu = m0 + u, v = n0 + w;
          if (mu < H && v < D) out[mu * D + v] = accW[q][u][w];
        }
    }
    if (threadIdx.x < H) {
      out[D * H + threadIdx.x] = sb0;
      out[D * H + H + threadIdx.x] = sw1;
    }
    if (threadIdx.x == 0) out[D * H + 2 * H] = sb1;
  };
  reset();

  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int e, a0, na;
    tile_of(T, t, e, a0, na);
    __syncthreads();
    if (e != cur_e) {
      if (cur_e >= 0) flush(cur_e);
      reset();
      load_weights<D, DP, HP>(dm, e, W0t, W0n, b0, w1);
      cur_e = e;
    }
    if (threadIdx.x < TM) {
      const int r = threadIdx.x < na ? T.perm[a0 + threadIdx.x] : -1;
      rows[threadIdx.x] = r;
      ei[threadIdx.x] = r >= 0 ? es[atom_struct[r]] : 0.f;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < TM * DP; q += NT) {
      const int a = q / DP, v = q % DP, r = rows[a];
      const bool ok = r >= 0 && v < D;
      const float s = ok ? dm.scale[v] : 0.f;
      const float g = ok ? s * G[(size_t)r * D + v] : 0.f;
      const float gd = ok ? s * Gd[(size_t)r * D + v] : 0.f;
      Gt[a * DP + v] = g;
      Gda[a * DP + v] = gd;
      Gdk[v * TM + a] = gd;
    }
    __syncthreads();
    tile_gemm<HP, DP, TM, HP>(Gdk, W0t, [&](int m0, int n0, float (&acc)[4][4]) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int a = m0 + u, r = rows[a];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int mu = n0 + w;
          const float x = (r >= 0 && mu < H) ? X[(size_t)r * H + mu] : 0.f;
          const float t1 = 1.f - x * x;
          const float beta = w1[mu] * t1;
          const float zd = acc[u][w];
          const float al = ei[a] * beta + 2.f * x * beta * zd;
          Al[mu * TM + a] = al;
          Ala[a * HP + mu] = al;
          Bea[a * HP + mu] = -beta;
          Q1[a * HP + mu] = (r >= 0 && mu < H) ? ei[a] * x - t1 * zd : 0.f;
        }
      }
    });
    __syncthreads();
    if (threadIdx.x < HP) {  // column sums in atom order
      const int mu = threadIdx.x;
      for (int a = 0; a < na; ++a) {
        sb0 += Ala[a * HP + mu];
        sw1 += Q1[a * HP + mu];
      }
    }
    if (threadIdx.x == 0)
      for (int a = 0; a < na; ++a) sb1 += ei[a];
    tile_gemm<DP, HP, TM, DP>(Al, W0n, [&](int m0, int n0, float (&acc)[4][4]) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = rows[m0 + u];
        if (r < 0) continue;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int v = n0 + w;
          if (v < D) Gb[(size_t)r * D + v] = acc[u][w] * dm.scale[v];
        }
      }
    });
#pragma unroll
    for (int q = 0; q < NBW; ++q) {
      const int blk = threadIdx.x + q * NT;
      if (blk >= NBLK) continue;
      const int m0 = (blk / (DP / 4)) * 4, n0 = (blk % (DP / 4)) * 4;
      for (int a = 0; a < na; ++a) {
        const float4 al = *reinterpret_cast<const float4*>(Ala + a * HP + m0);
        const float4 be = *reinterpret_cast<const float4*>(Bea + a * HP + m0);
        const float4 g = *reinterpret_cast<const float4*>(Gt + a * DP + n0);
        const float4 gd = *reinterpret_cast<const float4*>(Gda + a * DP + n0);
        const float av[4] = {al.x, al.y, al.z, al.w}, bv[4] = {be.x, be.y, be.z, be.w};
        const float gv[4] = {g.x, g.y, g.z, g.w}, dv[4] = {gd.x, gd.y, gd.z, gd.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int w = 0; w < 4; ++w) accW[q][u][w] = fmaf(av[u], gv[w], fmaf(bv[u], dv[w], accW[q][u][w]));
      }
    }
  }
  if (cur_e >= 0) flush(cur_e);
}

// ------------------------------------------------------------- launchers

Tiles make_tiles(const gnep_nlist* nl, int ns) {
  Tiles T;
  T.perm = nl->perm;
  T.ns = ns;
  int t = 0;
  for (int e = 0; e <= ns; ++e) {
    T.soff[e] = nl->species_off[e];
    T.tbase[e] = t;
    if (e < ns) t += (nl->species_off[e + 1] - nl->species_off[e] + TM - 1) / TM;
  }
  return T;
}

template <int D, int HP, int NS, int NQR, int KR>
int mlp_setup() {
  GNEP_CUDA(cudaFuncSetAttribute(k_mlp_fwd_tile<D, HP, NS, NQR, KR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)mlp_fwd_smem<D, HP, NS, NQR, KR>()));
  GNEP_CUDA(cudaFuncSetAttribute(k_mlp_bwd_tile<D, HP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)mlp_bwd_smem<D, HP>()));
  return GNEP_OK;
}

template <int D, int HP, int NS, int NQR, int KR>
int mlp_forward(const gnep_model* m, gnep_nlist* nl, cudaStream_t st) {
  const Tiles T = make_tiles(nl, NS);
  const int ntiles = T.tbase[NS];
  if (ntiles == 0) return GNEP_OK;
  Workspace& w = nl->ws;
  k_mlp_fwd_tile<D, HP, NS, NQR, KR><<<ntiles, NT, mlp_fwd_smem<D, HP, NS, NQR, KR>(), st>>>(
      T, m->dev(), w.G, w.X, w.Ep, w.Eatom, w.chat);
  GNEP_CHECK_LAUNCH("k_mlp_fwd_tile");
  return GNEP_OK;
}

template <int D, int HP>
int mlp_backward(const gnep_model* m, gnep_nlist* nl, cudaStream_t st) {
  const int ns = m->shape.ns;
  const Tiles T = make_tiles(nl, ns);
  const int ntiles = T.tbase[ns];
  Workspace& w = nl->ws;
  const int grid = ntiles < kNetBlocks ? (ntiles > 0 ? ntiles : 1) : kNetBlocks;
  GNEP_CUDA(cudaMemsetAsync(w.net_part, 0, sizeof(float) * (size_t)kNetBlocks * ns * m->net_size, st));
  if (ntiles == 0) return GNEP_OK;
  k_mlp_bwd_tile<D, HP><<<grid, NT, mlp_bwd_smem<D, HP>(), st>>>(T, ntiles, m->dev(), nl->atom_struct, w.es, w.G,
                                                                 w.Gd, w.X, w.Gb, w.net_part, m->net_size);
  GNEP_CHECK_LAUNCH("k_mlp_bwd_tile");
  return GNEP_OK;
}

// Instantiations: descriptor length D (with the radial block NQR x KR) and the
// hidden width padded to HP.
#define GNEP_NET(D, NQR, KR)                                                                             \
  template int mlp_setup<D, 32, 2, NQR, KR>();                                                           \
  template int mlp_setup<D, 64, 2, NQR, KR>();                                                           \
  template int mlp_setup<D, 128, 2, NQR, KR>();                                                          \
  template int mlp_forward<D, 32, 2, NQR, KR>(const gnep_model*, gnep_nlist*, cudaStream_t);             \
  template int mlp_forward<D, 64, 2, NQR, KR>(const gnep_model*, gnep_nlist*, cudaStream_t);             \
  template int mlp_forward<D, 128, 2, NQR, KR>(const gnep_model*, gnep_nlist*, cudaStream_t);            \
  template int mlp_backward<D, 32>(const gnep_model*, gnep_nlist*, cudaStream_t);                        \
  template int mlp_backward<D, 64>(const gnep_model*, gnep_nlist*, cudaStream_t);                        \
  template int mlp_backward<D, 128>(const gnep_model*, gnep_nlist*, cudaStream_t);
GNEP_NET(25, 5, 9)
GNEP_NET(54, 9, 13)
GNEP_NET(45, 9, 13)
#undef GNEP_NET

}  // namespace gnep
