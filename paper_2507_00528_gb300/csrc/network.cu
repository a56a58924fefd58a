// Per-element one-hidden-layer network (D1.1-D1.10) in FP32 on the CUDA
// cores, and its tangent/reverse pass (D1.18-D1.21 through the tangent/adjoint
// route), over species-homogeneous tiles of the species-grouped atom order:
// 128 atoms per tile, or 32 for batches too small to give every SM a tile.  Persistent blocks keep one species' weights in shared memory
// and walk the tiles.  Every sum runs in a fixed order (no atomics), so results
// are bit-reproducible.
//
// Thread map: 256 threads, G per atom (G = 2 for 128-atom tiles, 8 for 32).
// With AW = 32 / G atoms per warp, lane l of warp w takes atom AW w + (l mod AW)
// and part l / AW of the hidden units (the units padded to a multiple of G), so
// that each thread's descriptor row (and, backward, its tangent row and the
// adjoint it accumulates) lives in registers while the weight row of hidden
// unit mu is read by 16-byte loads that the AW lanes of a part share.  For each
// mu a thread forms z = W0_mu . (s.G) (interleaved partial sums), the
// element-wise terms and then the rank-one update of E' (forward) or Gbar
// (backward) with the same row.  The hidden activations are recomputed in the
// backward pass instead of being stored.  The parts are combined by exchanges
// between lanes l and l ^ AW, l ^ 2 AW, ... (a butterfly, so every part's lane
// holds the same sum).
//
// The weight gradient dW0 += alpha^T (s.G) - beta^T (s.Gdot) contracts over the
// tile's atoms: after the per-atom phase alpha and -beta are in shared memory
// and each thread accumulates 4 x 4 blocks of dW0 in registers across all
// tiles of one species, from four 16-byte loads per atom (alpha, -beta, s.G,
// s.Gdot).  db0 and dw1 are column sums of alpha and of e x - (1 - x^2) zdot
// over the tile's atoms, taken from shared memory in the same phase (hidden
// widths up to 64; above that the rows would not fit and the sums are formed
// by shuffles over the lanes of each part in the per-atom phase).
#include <cstdio>

#include "gnep_internal.h"
#include "network.cuh"

namespace gnep {

namespace {

constexpr int NT = 256;  // threads per block
constexpr int NW = NT / 32;

// Tile of TA atoms: G = NT / TA threads per atom, AW = 32 / G atoms per warp.
template <int TA>
struct TileMap {
  static_assert(TA == 32 || TA == 128, "network tiles hold 32 or 128 atoms");
  static constexpr int G = NT / TA, AW = 32 / G;
};

template <int TA>
__device__ __forceinline__ void tile_of(const Tiles& T, int t, int& e, int& a0, int& na) {
  e = 0;
  while (e + 1 < T.ns && t >= T.tbase[e + 1]) ++e;
  a0 = T.soff[e] + (t - T.tbase[e]) * TA;
  na = min(TA, T.soff[e + 1] - a0);
}

// Row widths: descriptor rows padded to 16 bytes; hidden units padded to a
// multiple of G (the parts take the same number of units; padding units have
// zero weights) and the alpha / beta rows to a multiple of 4.
template <int D>
struct RowW {
  static constexpr int DW = (D + 3) / 4 * 4;
};
template <int G>
__host__ __device__ inline int h_even(int H) { return (H + G - 1) / G * G; }
template <int G>
__host__ __device__ inline int h_row(int H) { return (h_even<G>(H) + 3) / 4 * 4; }

// Weights of species e: W [H2][DW] (row mu = W0_mu, zero beyond D and H),
// b0, w1 [H2] (zero beyond H).
template <int D, int G>
__device__ void load_weights(const DevModel& dm, int e, float* W, float* b0, float* w1) {
  constexpr int DW = RowW<D>::DW;
  const float* P = dm.params + (size_t)e * dm.net_size;
  const int H = dm.H, H2 = h_even<G>(H);
  for (int q = threadIdx.x; q < H2 * DW; q += NT) {
    const int mu = q / DW, v = q % DW;
    W[q] = (v < D && mu < H) ? P[mu * D + v] : 0.f;
  }
  for (int mu = threadIdx.x; mu < H2; mu += NT) {
    b0[mu] = mu < H ? P[D * H + mu] : 0.f;
    w1[mu] = mu < H ? P[D * H + H + mu] : 0.f;
  }
}

// Scaled rows s.src of the tile's atoms into R [TA][DW] (zero padding), for
// NA arrays at once: every thread issues all of its gathered loads before the
// first store, so that a tile waits for one global-memory latency, not one per
// element.
template <int D, int NA, int TA>
__device__ __forceinline__ void stage_rows(const float* __restrict__ s0, const float* __restrict__ s1,
                                           const int* rows, const float* sc, float* R0, float* R1) {
  constexpr int DW = RowW<D>::DW, N = TA * DW, IT = (N + NT - 1) / NT;
  float x[NA][IT];
#pragma unroll
  for (int k = 0; k < IT; ++k) {
    const int q = threadIdx.x + k * NT, a = q / DW, v = q % DW;
    const int r = q < N ? rows[a] : -1;
    const bool in = r >= 0 && v < D;
    x[0][k] = in ? __ldg(s0 + (size_t)r * D + v) : 0.f;
    if constexpr (NA > 1) x[NA - 1][k] = in ? __ldg(s1 + (size_t)r * D + v) : 0.f;
  }
#pragma unroll
  for (int k = 0; k < IT; ++k) {
    const int q = threadIdx.x + k * NT;
    if (q < N) {
      const float c = sc[q % DW];
      R0[q] = c * x[0][k];
      if constexpr (NA > 1) R1[q] = c * x[NA - 1][k];
    }
  }
}

template <int DW>
__device__ __forceinline__ void load_row(const float* R, float (&x)[DW]) {
#pragma unroll
  for (int v4 = 0; v4 < DW / 4; ++v4) {
    const float4 t = reinterpret_cast<const float4*>(R)[v4];
    x[4 * v4] = t.x; x[4 * v4 + 1] = t.y; x[4 * v4 + 2] = t.z; x[4 * v4 + 3] = t.w;
  }
}

// Dot product of a register row with a shared-memory weight row, four chains.
template <int DW>
__device__ __forceinline__ float dot_row(const float (&x)[DW], const float4* w, float init) {
  float s0 = init, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
  for (int v4 = 0; v4 < DW / 4; ++v4) {
    const float4 t = w[v4];
    s0 = fmaf(x[4 * v4], t.x, s0);
    s1 = fmaf(x[4 * v4 + 1], t.y, s1);
    s2 = fmaf(x[4 * v4 + 2], t.z, s2);
    s3 = fmaf(x[4 * v4 + 3], t.w, s3);
  }
  return (s0 + s1) + (s2 + s3);
}

// Two dot products with the same weight row, four chains each.
template <int DW>
__device__ __forceinline__ void dot_row2(const float (&x)[DW], const float (&y)[DW], const float4* w, float init,
                                         float& zx, float& zy) {
  float a0 = init, a1 = 0.f, a2 = 0.f, a3 = 0.f, b0 = 0.f, b1 = 0.f, b2 = 0.f, b3 = 0.f;
#pragma unroll
  for (int v4 = 0; v4 < DW / 4; ++v4) {
    const float4 t = w[v4];
    a0 = fmaf(x[4 * v4], t.x, a0);
    a1 = fmaf(x[4 * v4 + 1], t.y, a1);
    a2 = fmaf(x[4 * v4 + 2], t.z, a2);
    a3 = fmaf(x[4 * v4 + 3], t.w, a3);
    b0 = fmaf(y[4 * v4], t.x, b0);
    b1 = fmaf(y[4 * v4 + 1], t.y, b1);
    b2 = fmaf(y[4 * v4 + 2], t.z, b2);
    b3 = fmaf(y[4 * v4 + 3], t.w, b3);
  }
  zx = (a0 + a1) + (a2 + a3);
  zy = (b0 + b1) + (b2 + b3);
}

// acc += c * (weight row)
template <int DW>
__device__ __forceinline__ void axpy_row(float (&acc)[DW], float c, const float4* w) {
#pragma unroll
  for (int v4 = 0; v4 < DW / 4; ++v4) {
    const float4 t = w[v4];
    acc[4 * v4] = fmaf(c, t.x, acc[4 * v4]);
    acc[4 * v4 + 1] = fmaf(c, t.y, acc[4 * v4 + 1]);
    acc[4 * v4 + 2] = fmaf(c, t.z, acc[4 * v4 + 2]);
    acc[4 * v4 + 3] = fmaf(c, t.w, acc[4 * v4 + 3]);
  }
}

}  // namespace

template <int D, int NS, int NQR, int KR, int TA>
size_t mlp_fwd_smem(int H) {
  constexpr int DW = RowW<D>::DW;
  const int H2 = h_even<TileMap<TA>::G>(H);
  return sizeof(float) * ((size_t)H2 * DW + (size_t)TA * DW + 2 * H2 + DW + NS * NQR * KR);
}

// Forward, persistent over tiles: z = W0 (s.G) + b0, x = tanh z, E = w1.x + b1,
// E' = s . (W0^T (w1 (1 - x^2)))  (D1.1-D1.5), and the per-atom radial
// contraction chat_i[J][k] = sum_n E'_n c^R_nk^{IJ} used by the force sweep.
template <int D, int NS, int NQR, int KR, int TA>
__global__ void __launch_bounds__(NT, 1) k_mlp_fwd_row(Tiles T, int ntiles, DevModel dm, const float* __restrict__ G,
                                                       float* __restrict__ Ep, float* __restrict__ Eatom,
                                                       float* __restrict__ chat) {
  constexpr int DW = RowW<D>::DW, NJK = NS * KR, GP = TileMap<TA>::G, AW = TileMap<TA>::AW;
  extern __shared__ float4 sm4[];
  const int H = dm.H, H2 = h_even<GP>(H), Hh = H2 / GP;
  float* W = reinterpret_cast<float*>(sm4);  // [H2][DW]
  float* R = W + H2 * DW;                    // [TA][DW] s.G, then the scaled E'
  float* b0 = R + TA * DW;                   // [H2]
  float* w1 = b0 + H2;                       // [H2]
  float* sc = w1 + H2;                       // [DW]
  float* cR = sc + DW;                       // [NS][NQR][KR] of the tile's species
  __shared__ int rows[TA];
  const int tid = threadIdx.x, lane = tid & 31;
  const int a = AW * (tid >> 5) + (lane % AW), hpart = lane / AW;
  for (int v = tid; v < DW; v += NT) sc[v] = v < D ? dm.scale[v] : 0.f;
  int cur_e = -1;
  float b1 = 0.f;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int e, a0, na;
    tile_of<TA>(T, t, e, a0, na);
    __syncthreads();  // the previous tile's readers of R, rows and the weights are done
    if (e != cur_e) {
      load_weights<D, GP>(dm, e, W, b0, w1);
      for (int q = tid; q < NS * NQR * KR; q += NT) cR[q] = dm.params[dm.off_cR + e * NS * NQR * KR + q];
      b1 = dm.params[(size_t)e * dm.net_size + D * H + 2 * H];
      cur_e = e;
    }
    if (tid < TA) rows[tid] = tid < na ? T.perm[a0 + tid] : -1;
    __syncthreads();
    stage_rows<D, 1, TA>(G, nullptr, rows, sc, R, nullptr);
    __syncthreads();
    float g[DW], ep[DW];
    load_row<DW>(R + a * DW, g);
#pragma unroll
    for (int v = 0; v < DW; ++v) ep[v] = 0.f;
    float E = 0.f;
    for (int mu = hpart * Hh; mu < (hpart + 1) * Hh; ++mu) {
      const float4* wr = reinterpret_cast<const float4*>(W + mu * DW);
      const float x = tanhf(dot_row<DW>(g, wr, b0[mu]));
      E = fmaf(w1[mu], x, E);
      axpy_row<DW>(ep, w1[mu] * (1.f - x * x), wr);
    }
#pragma unroll
    for (int o = AW; o < 32; o <<= 1) {
#pragma unroll
      for (int v = 0; v < DW; ++v) ep[v] += __shfl_xor_sync(0xffffffffu, ep[v], o);
      E += __shfl_xor_sync(0xffffffffu, E, o);
    }
    __syncthreads();  // every row of R has been read
    if (hpart == 0 && a < na) {
      Eatom[rows[a]] = E + b1;
      float4* o = reinterpret_cast<float4*>(R + a * DW);
#pragma unroll
      for (int v4 = 0; v4 < DW / 4; ++v4)
        o[v4] = make_float4(ep[4 * v4] * sc[4 * v4], ep[4 * v4 + 1] * sc[4 * v4 + 1], ep[4 * v4 + 2] * sc[4 * v4 + 2],
                            ep[4 * v4 + 3] * sc[4 * v4 + 3]);
    }
    __syncthreads();
    // coalesced row writes: E' and chat
    for (int q = tid; q < na * D; q += NT) {
      const int r = q / D, v = q % D;
      Ep[(size_t)rows[r] * D + v] = R[r * DW + v];
    }
    for (int q = tid; q < na * NJK; q += NT) {
      const int r = q / NJK, jk = q % NJK, J = jk / KR, k = jk % KR;
      float s = 0.f;
#pragma unroll
      for (int n = 0; n < NQR; ++n) s = fmaf(R[r * DW + n], cR[(J * NQR + n) * KR + k], s);
      chat[(size_t)rows[r] * NJK + jk] = s;
    }
  }
}

template <int D, int HP, int TA>
size_t mlp_bwd_smem(int H) {
  constexpr int DW = RowW<D>::DW, GP = TileMap<TA>::G;
  const int H2 = h_even<GP>(H), HR = h_row<GP>(H);
  const size_t rows = HP <= 64 ? 3 * (size_t)TA * HR : 2 * (size_t)TA * HR + 2 * (size_t)NW * HP;
  return sizeof(float) * ((size_t)H2 * DW + 2 * (size_t)TA * DW + rows + 2 * H2 + DW + TA);
}

// Tangent and reverse pass, persistent over tiles, with e_i the energy residual
// weight of the atom's structure:
//   z = W0 (s.G) + b0, zdot = W0 (s.Gdot), x = tanh z, beta = w1 (1 - x^2),
//   alpha = e_i beta + 2 x beta zdot, Gbar = s . (W0^T alpha),
//   dW0 += alpha (s.G)^T - beta (s.Gdot)^T, db0 += alpha,
//   dw1 += e_i x - (1 - x^2) zdot, db1 += e_i.
// Each block writes one partial per species it visited into
// part[block][species] (zeroed beforehand).  HP: hidden width padded to 32, 64
// or 128 (sets the dW0 blocks a thread owns); TA: atoms per tile.
template <int D, int HP, int TA>
__global__ void __launch_bounds__(NT, 1) k_mlp_bwd_row(Tiles T, int ntiles, DevModel dm,
                                                       const int* __restrict__ atom_struct,
                                                       const float* __restrict__ es, const float* __restrict__ G,
                                                       const float* __restrict__ Gd, float* __restrict__ Gb,
                                                       float* __restrict__ part, int part_stride) {
  constexpr int DW = RowW<D>::DW, NVB = DW / 4, GP = TileMap<TA>::G, AW = TileMap<TA>::AW;
  constexpr int NBK = ((HP / 4) * NVB + NT - 1) / NT;  // dW0 4 x 4 blocks per thread
  extern __shared__ float4 sm4[];
  const int H = dm.H, H2 = h_even<GP>(H), Hh = H2 / GP, HR = h_row<GP>(H);
  float* W = reinterpret_cast<float*>(sm4);  // [H2][DW]
  float* SG = W + H2 * DW;                   // [TA][DW] s.G, then the Gbar output rows
  float* SD = SG + TA * DW;                  // [TA][DW] s.Gdot
  float* Al = SD + TA * DW;                  // [TA][HR] alpha
  float* Be = Al + TA * HR;                  // [TA][HR] -beta
  constexpr bool kRows = HP <= 64;          // column sums from shared rows (else per-warp shuffles)
  float* Q1 = Be + TA * HR;                  // [TA][HR] e_i x - (1 - x^2) zdot (kRows)
  float* wdw1 = Q1;                          // [NW][HP] per-warp sums over atoms (!kRows)
  float* wdb0 = wdw1 + NW * HP;              // [NW][HP] (!kRows)
  float* b0 = Q1 + (kRows ? TA * HR : 2 * NW * HP);  // [H2]
  float* w1 = b0 + H2;                       // [H2]
  float* sc = w1 + H2;                       // [DW]
  float* ev = sc + DW;                       // [TA] e_i of the tile's atoms
  __shared__ int rows[TA];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int a = AW * warp + (lane % AW), hpart = lane / AW;
  for (int v = tid; v < DW; v += NT) sc[v] = v < D ? dm.scale[v] : 0.f;
  for (int q = tid; q < 2 * TA * HR + (kRows ? TA * HR : 0); q += NT) Al[q] = 0.f;  // Be, Q1 follow Al
  float acc[NBK][4][4];
  float cdb0 = 0.f, cdw1 = 0.f;  // column sums of hidden unit tid (tid < H2)
  float cb1 = 0.f;
  int cur_e = -1;

  auto reset = [&]() {
#pragma unroll
    for (int k = 0; k < NBK; ++k)
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[k][u][c] = 0.f;
    cdb0 = cdw1 = 0.f;
    if constexpr (!kRows)
      for (int q = tid; q < 2 * NW * HP; q += NT) wdw1[q] = 0.f;  // wdb0 follows wdw1
    cb1 = 0.f;
  };
  auto flush = [&](int e) {  // after a barrier that follows the last tile of species e
    float* out = part + ((size_t)blockIdx.x * T.ns + e) * part_stride;
#pragma unroll
    for (int k = 0; k < NBK; ++k) {
      const int q = tid + k * NT, mb = q / NVB, vb = q % NVB;
      if (q >= (HP / 4) * NVB) continue;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int mu = 4 * mb + u, v = 4 * vb + c;
          if (mu < H && v < D) out[mu * D + v] = acc[k][u][c];
        }
    }
    if constexpr (kRows) {
      if (tid < H) {
        out[D * H + tid] = cdb0;
        out[D * H + H + tid] = cdw1;
      }
    } else {
      for (int mu = tid; mu < H; mu += NT) {
        float s0 = 0.f, s1 = 0.f;
        for (int w = 0; w < NW; ++w) {  // warps in order
          s0 += wdb0[w * HP + mu];
          s1 += wdw1[w * HP + mu];
        }
        out[D * H + mu] = s0;
        out[D * H + H + mu] = s1;
      }
    }
    if (tid == 0) out[D * H + 2 * H] = cb1;
  };
  reset();

  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int e, a0, na;
    tile_of<TA>(T, t, e, a0, na);
    __syncthreads();  // the previous tile is done with every shared array
    if (e != cur_e) {
      if (cur_e >= 0) flush(cur_e);
      __syncthreads();
      reset();
      load_weights<D, GP>(dm, e, W, b0, w1);
      cur_e = e;
    }
    if (tid < TA) {
      const int r = tid < na ? T.perm[a0 + tid] : -1;
      rows[tid] = r;
      ev[tid] = r >= 0 ? es[atom_struct[r]] : 0.f;
    }
    __syncthreads();
    stage_rows<D, 2, TA>(G, Gd, rows, sc, SG, SD);
    if (tid == 0)
      for (int r = 0; r < na; ++r) cb1 += ev[r];
    __syncthreads();
    // per atom: z, zdot, alpha, -beta, q1 and Gbar
    float gb[DW];
    {
      float g[DW], gd[DW];
      load_row<DW>(SG + a * DW, g);
      load_row<DW>(SD + a * DW, gd);
#pragma unroll
      for (int v = 0; v < DW; ++v) gb[v] = 0.f;
      const float ea = ev[a];
      for (int mu = hpart * Hh; mu < (hpart + 1) * Hh; ++mu) {
        const float4* wr = reinterpret_cast<const float4*>(W + mu * DW);
        float z, zd;
        dot_row2<DW>(g, gd, wr, b0[mu], z, zd);
        const float x = tanhf(z);
        const float t1 = 1.f - x * x;
        const float beta = w1[mu] * t1;
        const float alpha = ea * beta + 2.f * x * beta * zd;
        Al[a * HR + mu] = alpha;
        Be[a * HR + mu] = -beta;
        float q1 = ea * x - t1 * zd;  // zero for padding atoms (e = 0, zdot = 0) and the padding unit
        axpy_row<DW>(gb, alpha, wr);
        if constexpr (kRows) {
          Q1[a * HR + mu] = q1;
        } else {
          float as = alpha;  // summed over the AW atoms of this part in the warp
#pragma unroll
          for (int o = 1; o < AW; o <<= 1) {
            as += __shfl_xor_sync(0xffffffffu, as, o);
            q1 += __shfl_xor_sync(0xffffffffu, q1, o);
          }
          if (lane % AW == 0) {
            wdb0[warp * HP + mu] += as;
            wdw1[warp * HP + mu] += q1;
          }
        }
      }
    }
#pragma unroll
    for (int o = AW; o < 32; o <<= 1)
#pragma unroll
      for (int v = 0; v < DW; ++v) gb[v] += __shfl_xor_sync(0xffffffffu, gb[v], o);
    __syncthreads();  // alpha and -beta of the tile are complete
    // dW0 += alpha^T (s.G) - beta^T (s.Gdot) over the tile's atoms
#pragma unroll
    for (int k = 0; k < NBK; ++k) {
      const int q = tid + k * NT, mb = q / NVB, vb = q % NVB;
      if (q >= (HP / 4) * NVB || 4 * mb >= H2) continue;
#pragma unroll 4
      for (int r = 0; r < na; ++r) {
        const float4 al = *reinterpret_cast<const float4*>(Al + r * HR + 4 * mb);
        const float4 be = *reinterpret_cast<const float4*>(Be + r * HR + 4 * mb);
        const float4 g4 = *reinterpret_cast<const float4*>(SG + r * DW + 4 * vb);
        const float4 d4 = *reinterpret_cast<const float4*>(SD + r * DW + 4 * vb);
        const float av[4] = {al.x, al.y, al.z, al.w}, bv[4] = {be.x, be.y, be.z, be.w};
        const float gv[4] = {g4.x, g4.y, g4.z, g4.w}, dv[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[k][u][c] = fmaf(av[u], gv[c], fmaf(bv[u], dv[c], acc[k][u][c]));
      }
    }
    if (kRows && tid < H2) {  // db0, dw1: sums over the tile's atoms in order
      float s0 = 0.f, s1 = 0.f;
      for (int r = 0; r < na; ++r) {
        s0 += Al[r * HR + tid];
        s1 += Q1[r * HR + tid];
      }
      cdb0 += s0;
      cdw1 += s1;
    }
    __syncthreads();  // s.G rows are no longer read: they take the Gbar rows
    if (hpart == 0) {
      float4* o = reinterpret_cast<float4*>(SG + a * DW);
#pragma unroll
      for (int v4 = 0; v4 < DW / 4; ++v4)
        o[v4] = make_float4(gb[4 * v4] * sc[4 * v4], gb[4 * v4 + 1] * sc[4 * v4 + 1], gb[4 * v4 + 2] * sc[4 * v4 + 2],
                            gb[4 * v4 + 3] * sc[4 * v4 + 3]);
    }
    __syncthreads();
    for (int q = tid; q < na * D; q += NT) {
      const int r = q / D, v = q % D;
      Gb[(size_t)rows[r] * D + v] = SG[r * DW + v];
    }
  }
  __syncthreads();
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

namespace {
// Resident blocks of a kernel on this GPU.
template <class K>
int resident_blocks(K kern, size_t smem, int& out) {
  int per_sm = 0, dev = 0, sms = 0;
  GNEP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
  GNEP_CUDA(cudaGetDevice(&dev));
  GNEP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (per_sm < 1) return set_error(GNEP_ERR_CUDA, "FP32 network kernel does not fit on an SM");
  out = per_sm * sms;
  return GNEP_OK;
}
}  // namespace

// Atoms per network tile: the tuned value, else 128 while the batch has at
// least one such tile per two SMs, and 32 below (four times the tiles, each
// with four times the threads per atom, so that small batches spread over more
// SMs and each atom's hidden-unit loop is a quarter as long).
int net_tile_atoms(const gnep_nlist* nl, int ns) {
  if (nl->tune.net_tile > 0) return nl->tune.net_tile;
  return 2 * make_tiles(nl, ns, 128).tbase[ns] >= sm_count() ? 128 : 32;
}

template <int D, int HP, int NS, int NQR, int KR, int TA>
int mlp_setup_ta() {
  // shared memory for the largest hidden width of this padding
  GNEP_CUDA(cudaFuncSetAttribute(k_mlp_fwd_row<D, NS, NQR, KR, TA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)mlp_fwd_smem<D, NS, NQR, KR, TA>(kMaxHidden)));
  GNEP_CUDA(cudaFuncSetAttribute(k_mlp_bwd_row<D, HP, TA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)mlp_bwd_smem<D, HP, TA>(HP)));
  GNEP_CUDA(cudaFuncSetAttribute(k_mlp_bwd_row<D, HP, TA>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  return GNEP_OK;
}

template <int D, int HP, int NS, int NQR, int KR>
int mlp_setup() {
  if (int rc = mlp_setup_ta<D, HP, NS, NQR, KR, 128>()) return rc;
  return mlp_setup_ta<D, HP, NS, NQR, KR, 32>();
}

template <int D, int NS, int NQR, int KR, int TA>
int mlp_forward_ta(const gnep_model* m, gnep_nlist* nl, cudaStream_t st) {
  const Tiles T = make_tiles(nl, NS, TA);
  const int ntiles = T.tbase[NS];
  if (ntiles == 0) return GNEP_OK;
  Workspace& w = nl->ws;
  auto kern = k_mlp_fwd_row<D, NS, NQR, KR, TA>;
  const size_t smem = mlp_fwd_smem<D, NS, NQR, KR, TA>(m->shape.H);
  int cap = 0;
  if (int rc = resident_blocks(kern, smem, cap)) return rc;
  const int grid = net_blocks(nl, ntiles < cap ? ntiles : cap);
  kern<<<grid, NT, smem, st>>>(T, ntiles, m->dev(), w.G, w.Ep, w.Eatom, w.chat);
  GNEP_CHECK_LAUNCH("k_mlp_fwd_row");
  return GNEP_OK;
}

template <int D, int HP, int NS, int NQR, int KR>
int mlp_forward(const gnep_model* m, gnep_nlist* nl, cudaStream_t st) {
  return net_tile_atoms(nl, NS) == 32 ? mlp_forward_ta<D, NS, NQR, KR, 32>(m, nl, st)
                                      : mlp_forward_ta<D, NS, NQR, KR, 128>(m, nl, st);
}

template <int D, int HP, int TA>
int mlp_backward_ta(const gnep_model* m, gnep_nlist* nl, cudaStream_t st) {
  const int ns = m->shape.ns;
  const Tiles T = make_tiles(nl, ns, TA);
  const int ntiles = T.tbase[ns];
  Workspace& w = nl->ws;
  auto kern = k_mlp_bwd_row<D, HP, TA>;
  const size_t smem = mlp_bwd_smem<D, HP, TA>(m->shape.H);
  int cap = 0;
  if (int rc = resident_blocks(kern, smem, cap)) return rc;
  if (cap > kNetBlocks) cap = kNetBlocks;  // net_part holds kNetBlocks partials
  const int grid = net_blocks(nl, ntiles < cap ? (ntiles > 0 ? ntiles : 1) : cap);
  w.net_blocks = grid;
  GNEP_CUDA(cudaMemsetAsync(w.net_part, 0, sizeof(float) * (size_t)grid * ns * m->net_size, st));
  if (ntiles == 0) return GNEP_OK;
  kern<<<grid, NT, smem, st>>>(T, ntiles, m->dev(), nl->atom_struct, w.es, w.G, w.Gd, w.Gb, w.net_part,
                               m->net_size);
  GNEP_CHECK_LAUNCH("k_mlp_bwd_row");
  return GNEP_OK;
}

template <int D, int HP>
int mlp_backward(const gnep_model* m, gnep_nlist* nl, cudaStream_t st) {
  return net_tile_atoms(nl, m->shape.ns) == 32 ? mlp_backward_ta<D, HP, 32>(m, nl, st)
                                               : mlp_backward_ta<D, HP, 128>(m, nl, st);
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
GNEP_NET(35, 5, 9)
GNEP_NET(50, 5, 9)
#undef GNEP_NET

}  // namespace gnep
