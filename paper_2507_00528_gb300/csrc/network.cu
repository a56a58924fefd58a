// Per-element one-hidden-layer network (D1.1-D1.10) on species-homogeneous
// tiles of 32 atoms.  The contractions are register-blocked FP32 tile GEMMs
// from shared memory; persistent blocks keep one species' weights resident and
// walk the tiles of the species-grouped atom order.  The network-parameter
// gradient (D1.18-D1.21 through the tangent/reverse pass) is accumulated in
// registers and written once per block and species.  Every sum runs in a fixed
// order (no atomics), so results are bit-reproducible.
//
// Tile GEMM layout: C[m][n] = sum_k A[k][m] B[k][n] with A, B k-major in shared
// memory; thread t owns the 4x4 block (m0, n0) with m0 = 4 (t mod 8) and
// n0 = 4 (t div 8), so the 8 threads sharing n0 read 128 contiguous bytes of A
// and write transposed results as conflict-free 16-byte stores.
#include <cstdio>

#include "gnep_internal.h"
#include "network.cuh"

namespace gnep {

namespace {

constexpr int TM = kTileAtoms;  // atoms per tile (32)
constexpr int NT = 128;         // threads per block
constexpr int MB = TM / 4;      // m-blocks per tile (8)

__device__ __forceinline__ void tile_of(const Tiles& T, int t, int& e, int& a0, int& na) {
  e = 0;
  while (e + 1 < T.ns && t >= T.tbase[e + 1]) ++e;
  a0 = T.soff[e] + (t - T.tbase[e]) * TM;
  na = min(TM, T.soff[e + 1] - a0);
}

// Blocks of a TM x NP product: thread t handles blocks t, t + NT, ...
template <int NP, int K, int LDA, int LDB, class F>
__device__ __forceinline__ void tile_gemm(const float* A, const float* B, F f) {
  constexpr int NB = MB * (NP / 4);
  for (int blk = threadIdx.x; blk < NB; blk += NT) {
    const int m0 = (blk % MB) * 4, n0 = (blk / MB) * 4;
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
  for (int q = threadIdx.x; q < DP * HP; q += NT) {  // W0n row-major, coalesced reads
    const int mu = q / DP, v = q % DP;
    W0n[q] = (v < D && mu < H) ? P[mu * D + v] : 0.f;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < DP * HP; q += NT) {  // W0t from W0n
    const int v = q / HP, mu = q % HP;
    W0t[q] = W0n[mu * DP + v];
  }
  for (int mu = threadIdx.x; mu < HP; mu += NT) {
    b0[mu] = mu < H ? P[D * H + mu] : 0.f;
    w1[mu] = mu < H ? P[D * H + H + mu] : 0.f;
  }
}

// Stage rows of a per-atom array (row stride D) into A[k][a] (k-major), zero-padded.
template <int D, int DP>
__device__ __forceinline__ void stage_kmajor(const float* __restrict__ src, const int* rows, const float* scale,
                                             float* dst) {
  for (int q = threadIdx.x; q < DP * TM; q += NT) {
    const int v = q / TM, a = q % TM, r = rows[a];
    dst[q] = (r >= 0 && v < D) ? scale[v] * src[(size_t)r * D + v] : 0.f;
  }
}

// Stage rows into R[a][DP] (atom-major), zero-padded.
template <int D, int DP>
__device__ __forceinline__ void stage_rows(const float* __restrict__ src, const int* rows, const float* scale,
                                           float* dst) {
  for (int q = threadIdx.x; q < DP * TM; q += NT) {
    const int a = q / DP, v = q % DP, r = rows[a];
    dst[q] = (r >= 0 && v < D) ? scale[v] * src[(size_t)r * D + v] : 0.f;
  }
}

}  // namespace

template <int D, int HP, int NS, int NQR, int KR>
size_t mlp_fwd_smem() {
  constexpr int DP = (D + 3) / 4 * 4;
  return sizeof(float) * (2 * DP * HP + 2 * HP + DP * TM + HP * TM + (HP / 4) * TM + NS * NQR * KR);
}

// Forward, persistent over tiles: z = W0 (s.G) + b0, x = tanh z, E = w1.x + b1,
// E' = s . (W0^T (w1 (1 - x^2)))  (D1.1-D1.5), and the per-atom radial
// contraction chat_i[J][k] = sum_n E'_n c^R_nk^{IJ} used by the force sweep.
// X is stored with row pitch HP.
template <int D, int HP, int NS, int NQR, int KR>
__global__ void __launch_bounds__(NT) k_mlp_fwd_tile(Tiles T, int ntiles, DevModel dm, const float* __restrict__ G,
                                                     float* __restrict__ X, float* __restrict__ Ep,
                                                     float* __restrict__ Eatom, float* __restrict__ chat) {
  constexpr int DP = (D + 3) / 4 * 4;
  extern __shared__ float4 sm4[];
  float* sm = reinterpret_cast<float*>(sm4);
  float* W0t = sm;                // [DP][HP]
  float* W0n = W0t + DP * HP;     // [HP][DP]
  float* b0 = W0n + HP * DP;      // [HP]
  float* w1 = b0 + HP;            // [HP]
  float* Gt = w1 + HP;            // [DP][TM] scaled inputs, then E'
  float* Bt = Gt + DP * TM;       // [HP][TM] beta
  float* Ep4 = Bt + HP * TM;      // [HP/4][TM] partial energies per hidden block
  float* cR = Ep4 + (HP / 4) * TM;  // [NS][NQR][KR] of this species
  __shared__ int rows[TM];
  const int H = dm.H;
  int cur_e = -1;
  float b1 = 0.f;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int e, a0, na;
    tile_of(T, t, e, a0, na);
    __syncthreads();
    if (e != cur_e) {
      load_weights<D, DP, HP>(dm, e, W0t, W0n, b0, w1);
      for (int q = threadIdx.x; q < NS * NQR * KR; q += NT) cR[q] = dm.params[dm.off_cR + e * NS * NQR * KR + q];
      b1 = dm.params[(size_t)e * dm.net_size + D * H + 2 * H];
      cur_e = e;
    }
    if (threadIdx.x < TM) rows[threadIdx.x] = threadIdx.x < na ? T.perm[a0 + threadIdx.x] : -1;
    __syncthreads();
    stage_kmajor<D, DP>(G, rows, dm.scale, Gt);
    __syncthreads();
    tile_gemm<HP, DP, TM, HP>(Gt, W0t, [&](int m0, int n0, float (&acc)[4][4]) {
      float4 bt[4];
      float ep[4] = {0.f, 0.f, 0.f, 0.f};
      float xv[4][4];
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int mu = n0 + w;
        float bb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float x = mu < H ? tanhf(acc[u][w] + b0[mu]) : 0.f;
          xv[u][w] = x;
          bb[u] = w1[mu] * (1.f - x * x);
          ep[u] = fmaf(w1[mu], x, ep[u]);
        }
        bt[w] = make_float4(bb[0], bb[1], bb[2], bb[3]);
      }
#pragma unroll
      for (int w = 0; w < 4; ++w) *reinterpret_cast<float4*>(Bt + (n0 + w) * TM + m0) = bt[w];
      *reinterpret_cast<float4*>(Ep4 + (n0 / 4) * TM + m0) = make_float4(ep[0], ep[1], ep[2], ep[3]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = rows[m0 + u];
        if (r >= 0) *reinterpret_cast<float4*>(X + (size_t)r * HP + n0) = make_float4(xv[u][0], xv[u][1], xv[u][2], xv[u][3]);
      }
    });
    __syncthreads();
    if (threadIdx.x < na) {  // energies, hidden blocks summed in order
      const int a = threadIdx.x;
      float E = 0.f;
      for (int b = 0; b < HP / 4; ++b) E += Ep4[b * TM + a];
      Eatom[rows[a]] = E + b1;
    }
    tile_gemm<DP, HP, TM, DP>(Bt, W0n, [&](int m0, int n0, float (&acc)[4][4]) {
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int v = n0 + w;
        const float s = v < D ? dm.scale[v] : 0.f;
        *reinterpret_cast<float4*>(Gt + v * TM + m0) =
            make_float4(acc[0][w] * s, acc[1][w] * s, acc[2][w] * s, acc[3][w] * s);
      }
    });
    __syncthreads();
    for (int q = threadIdx.x; q < na * D; q += NT) {
      const int a = q / D, v = q % D;
      Ep[(size_t)rows[a] * D + v] = Gt[v * TM + a];
    }
    for (int q = threadIdx.x; q < TM * NS * KR; q += NT) {
      const int a = q % TM, jk = q / TM, J = jk / KR, k = jk % KR;
      if (a >= na) continue;
      float s = 0.f;
#pragma unroll
      for (int n = 0; n < NQR; ++n) s = fmaf(Gt[n * TM + a], cR[(J * NQR + n) * KR + k], s);
      chat[(size_t)rows[a] * NS * KR + jk] = s;
    }
  }
}

template <int D, int HP>
size_t mlp_bwd_smem() {
  constexpr int DP = (D + 3) / 4 * 4;
  return sizeof(float) * (2 * DP * HP + 2 * HP + 3 * TM * DP + 2 * HP * TM + TM * HP);
}

// Tangent and reverse pass, persistent over tiles, with the energy residual
// weight e_i:
//   zdot = W0 (s.Gdot), beta = w1 (1 - x^2), alpha = e_i beta + 2 x beta zdot,
//   Gbar = s . (W0^T alpha),
//   dW0 += alpha (s.G)^T - beta (s.Gdot)^T, db0 += alpha,
//   dw1 += e_i x - (1 - x^2) zdot, db1 += e_i.
// Each block writes one partial per species it visited into
// part[block][species] (zeroed beforehand).
template <int D, int HP>
__global__ void __launch_bounds__(NT) k_mlp_bwd_tile(Tiles T, int ntiles, DevModel dm,
                                                     const int* __restrict__ atom_struct,
                                                     const float* __restrict__ es, const float* __restrict__ G,
                                                     const float* __restrict__ Gd, const float* __restrict__ X,
                                                     float* __restrict__ Gb, float* __restrict__ part,
                                                     int part_stride) {
  constexpr int DP = (D + 3) / 4 * 4;
  constexpr int NBW = ((HP / 4) * (DP / 4) + NT - 1) / NT;  // dW0 4x4 blocks per thread
  extern __shared__ float4 sm4[];
  float* sm = reinterpret_cast<float*>(sm4);
  float* W0t = sm;               // [DP][HP]
  float* W0n = W0t + DP * HP;    // [HP][DP]
  float* b0 = W0n + HP * DP;
  float* w1 = b0 + HP;
  float* Gr = w1 + HP;           // [TM][DP] s.G, atom-major
  float* Gdr = Gr + TM * DP;     // [TM][DP] s.Gdot, atom-major
  float* Gdk = Gdr + TM * DP;    // [DP][TM] s.Gdot, k-major
  float* Al = Gdk + DP * TM;     // [HP][TM] alpha, k-major
  float* Be = Al + HP * TM;      // [HP][TM] -beta, k-major
  float* Xs = Be + HP * TM;      // [TM][HP] x
  __shared__ int rows[TM];
  __shared__ float ei[TM];
  const int H = dm.H;
  constexpr int NCB = (MB * (HP / 4) + NT - 1) / NT;  // GEMM blocks per thread (column groups)
  float accW[NBW][4][4];
  float cb0[NCB][4], cw1[NCB][4], cb1 = 0.f;  // column sums of the thread's column groups
  int cur_e = -1;

  auto reset = [&]() {
#pragma unroll
    for (int q = 0; q < NBW; ++q)
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) accW[q][u][w] = 0.f;
#pragma unroll
    for (int c = 0; c < NCB; ++c)
#pragma unroll
      for (int w = 0; w < 4; ++w) cb0[c][w] = cw1[c][w] = 0.f;
    cb1 = 0.f;
  };
  auto flush = [&](int e) {
    float* out = part + ((size_t)blockIdx.x * T.ns + e) * part_stride;
#pragma unroll
    for (int q = 0; q < NBW; ++q) {
      const int blk = threadIdx.x + q * NT;
      if (blk >= (HP / 4) * (DP / 4)) continue;
      const int m0 = (blk / (DP / 4)) * 4, n0 = (blk % (DP / 4)) * 4;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int mu = m0 + u, v = n0 + w;
          if (mu < H && v < D) out[mu * D + v] = accW[q][u][w];
        }
    }
    // column sums live in the lanes with m-block 0 (threadIdx % MB == 0)
#pragma unroll
    for (int c = 0; c < NCB; ++c) {
      const int blk = threadIdx.x + c * NT;
      if (threadIdx.x % MB != 0 || blk >= MB * (HP / 4)) continue;
      const int n0 = (blk / MB) * 4;
#pragma unroll
      for (int w = 0; w < 4; ++w)
        if (n0 + w < H) {
          out[D * H + n0 + w] = cb0[c][w];
          out[D * H + H + n0 + w] = cw1[c][w];
        }
    }
    if (threadIdx.x == 0) out[D * H + 2 * H] = cb1;
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
    stage_rows<D, DP>(G, rows, dm.scale, Gr);
    stage_rows<D, DP>(Gd, rows, dm.scale, Gdr);
    stage_kmajor<D, DP>(Gd, rows, dm.scale, Gdk);
    for (int q = threadIdx.x; q < TM * (HP / 4); q += NT) {
      const int a = q / (HP / 4), c4 = (q % (HP / 4)) * 4, r = rows[a];
      const float4 x = r >= 0 ? *reinterpret_cast<const float4*>(X + (size_t)r * HP + c4) : make_float4(0.f, 0.f, 0.f, 0.f);
      *reinterpret_cast<float4*>(Xs + a * HP + c4) = x;
    }
    if (threadIdx.x == 0)
      for (int a = 0; a < na; ++a) cb1 += ei[a];
    __syncthreads();
    // zdot = (s.Gdot) W0^T; alpha, beta; column sums of alpha and q1 = e x - (1-x^2) zdot
    tile_gemm<HP, DP, TM, HP>(Gdk, W0t, [&](int m0, int n0, float (&acc)[4][4]) {
      float s0[4] = {0.f, 0.f, 0.f, 0.f}, s1[4] = {0.f, 0.f, 0.f, 0.f};
      float4 al[4], be[4];
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int mu = n0 + w;
        float av[4], bv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int a = m0 + u;
          const float x = Xs[a * HP + mu];
          const float t1 = 1.f - x * x;
          const float beta = w1[mu] * t1;
          const float zd = acc[u][w];
          const float ea = ei[a];
          const float alpha = ea * beta + 2.f * x * beta * zd;
          av[u] = alpha;
          bv[u] = -beta;
          s0[w] += alpha;
          s1[w] += ea * x - t1 * zd;  // zero for padded atoms (x = 0, zd = 0)
        }
        al[w] = make_float4(av[0], av[1], av[2], av[3]);
        be[w] = make_float4(bv[0], bv[1], bv[2], bv[3]);
      }
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        *reinterpret_cast<float4*>(Al + (n0 + w) * TM + m0) = al[w];
        *reinterpret_cast<float4*>(Be + (n0 + w) * TM + m0) = be[w];
      }
      // the 8 lanes sharing n0 hold the 32 atoms: sum them in a fixed order
      const int c = (MB * (n0 / 4) + m0 / 4 - (int)threadIdx.x) / NT;  // this thread's block index
#pragma unroll
      for (int w = 0; w < 4; ++w) {
#pragma unroll
        for (int o = 1; o < MB; o <<= 1) {
          s0[w] += __shfl_xor_sync(0xffffffffu, s0[w], o);
          s1[w] += __shfl_xor_sync(0xffffffffu, s1[w], o);
        }
#pragma unroll
        for (int cc = 0; cc < NCB; ++cc)
          if (cc == c) {
            cb0[cc][w] += s0[w];
            cw1[cc][w] += s1[w];
          }
      }
    });
    __syncthreads();
    // Gbar = s . (alpha W0)
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
    // dW0 += alpha^T (s.G) - beta^T (s.Gdot) over the tile's atoms (K = atoms)
#pragma unroll
    for (int q = 0; q < NBW; ++q) {
      const int blk = threadIdx.x + q * NT;
      if (blk >= (HP / 4) * (DP / 4)) continue;
      const int m0 = (blk / (DP / 4)) * 4, n0 = (blk % (DP / 4)) * 4;
      for (int a = 0; a < na; ++a) {
        float av[4], bv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          av[u] = Al[(m0 + u) * TM + a];
          bv[u] = Be[(m0 + u) * TM + a];
        }
        const float4 g = *reinterpret_cast<const float4*>(Gr + a * DP + n0);
        const float4 gd = *reinterpret_cast<const float4*>(Gdr + a * DP + n0);
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

Tiles make_tiles(const gnep_nlist* nl, int ns, int tile_atoms) {
  Tiles T;
  T.perm = nl->perm;
  T.ns = ns;
  int t = 0;
  for (int e = 0; e <= ns; ++e) {
    T.soff[e] = nl->species_off[e];
    T.tbase[e] = t;
    if (e < ns) t += (nl->species_off[e + 1] - nl->species_off[e] + tile_atoms - 1) / tile_atoms;
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
  const int grid = net_blocks(nl, ntiles < kNetBlocks ? ntiles : kNetBlocks);
  k_mlp_fwd_tile<D, HP, NS, NQR, KR><<<grid, NT, mlp_fwd_smem<D, HP, NS, NQR, KR>(), st>>>(
      T, ntiles, m->dev(), w.G, w.X, w.Ep, w.Eatom, w.chat);
  GNEP_CHECK_LAUNCH("k_mlp_fwd_tile");
  return GNEP_OK;
}

template <int D, int HP>
int mlp_backward(const gnep_model* m, gnep_nlist* nl, cudaStream_t st) {
  const int ns = m->shape.ns;
  const Tiles T = make_tiles(nl, ns);
  const int ntiles = T.tbase[ns];
  Workspace& w = nl->ws;
  const int grid = net_blocks(nl, ntiles < kNetBlocks ? (ntiles > 0 ? ntiles : 1) : kNetBlocks);
  w.net_blocks = grid;
  GNEP_CUDA(cudaMemsetAsync(w.net_part, 0, sizeof(float) * (size_t)grid * ns * m->net_size, st));
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
