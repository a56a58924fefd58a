// Per-element one-hidden-layer network (D1.1-D1.10) with FP32 accuracy, and
// its tangent/reverse pass (D1.18-D1.21 through the tangent/adjoint route),
// over species-homogeneous tiles of the species-grouped atom order, in two
// forms: 128-atom tiles on warp-level tensor cores in split TF32 (the second
// half of this file), and CUDA-core kernels (below) on 32-atom tiles for
// batches too small to give every other SM a tile, and for the backward pass
// above 64 hidden units on 128-atom tiles.  Persistent blocks keep one
// species' weights in shared memory and walk the tiles.  Every sum runs in a
// fixed order (no atomics), so results are bit-reproducible.
//
// CUDA-core thread map: 256 threads, G per atom (G = 2 for 128-atom tiles, 8
// for 32).
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
#include "warp_mma.cuh"

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
  const int H = dm.H, H2 = h_even<G>(H), N = H2 * DW;
  for (int q0 = threadIdx.x; q0 < N; q0 += 4 * NT) {  // four loads in flight per thread
    float x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int q = q0 + k * NT, mu = q / DW, v = q % DW;
      x[k] = (q < N && v < D && mu < H) ? __ldg(P + mu * D + v) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (q0 + k * NT < N) W[q0 + k * NT] = x[k];
  }
  for (int mu = threadIdx.x; mu < H2; mu += NT) {
    b0[mu] = mu < H ? P[D * H + mu] : 0.f;
    w1[mu] = mu < H ? P[D * H + H + mu] : 0.f;
  }
}

// Scaled rows s.src of the tile's atoms into R [TA][RS] (zero padding), for
// NA arrays at once: every thread issues all of its gathered loads before the
// first store, so that a tile waits for one global-memory latency, not one per
// element.
template <int D, int NA, int TA, int RS = RowW<D>::DW, int NTH = NT>
__device__ __forceinline__ void stage_rows(const float* __restrict__ s0, const float* __restrict__ s1,
                                           const int* rows, const float* sc, float* R0, float* R1) {
  constexpr int DW = RS, N = TA * DW, IT = (N + NTH - 1) / NTH;
  float x[NA][IT];
#pragma unroll
  for (int k = 0; k < IT; ++k) {
    const int q = threadIdx.x + k * NTH, a = q / DW, v = q % DW;
    const int r = q < N ? rows[a] : -1;
    const bool in = r >= 0 && v < D;
    x[0][k] = in ? __ldg(s0 + (size_t)r * D + v) : 0.f;
    if constexpr (NA > 1) x[NA - 1][k] = in ? __ldg(s1 + (size_t)r * D + v) : 0.f;
  }
#pragma unroll
  for (int k = 0; k < IT; ++k) {
    const int q = threadIdx.x + k * NTH;
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
  GNEP_PDL_WAIT();
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
  GNEP_PDL_WAIT();
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
  unsigned visited = 0;  // species whose partial this block writes

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
      visited |= 1u << e;
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
  // the partials of the species this block did not visit are zero (the
  // gradient assembly reads every block's row of every species)
  for (int e = 0; e < T.ns; ++e)
    if (!(visited & (1u << e)))
      for (int q = threadIdx.x; q < part_stride; q += blockDim.x)
        part[((size_t)blockIdx.x * T.ns + e) * part_stride + q] = 0.f;
}

// ------------------------------------------------------------- tensor-core tiles (FP32 accuracy)
//
// The same forward and backward passes on the warp-level tensor cores, with
// every product carried in split TF32 (hi*hi plus the two cross terms in two
// accumulators, warp_mma.cuh), which keeps FP32 accuracy.  128-atom tiles,
// eight warps; warp w owns the tile's atoms 16 w .. 16 w + 15 as the M = 16
// rows of its products:
//   Z  = (s.G) W0^T      M 16 atoms, N 8 hidden units, K 8 descriptors
//   Zd = (s.Gdot) W0^T   (backward; same B fragments)
//   E' = beta W0         (forward)   M 16 atoms, N 8 descriptors, K 8 units
//   Gb = alpha W0        (backward)
// The hidden units go in chunks of 16 (two N tiles).  The B columns of the
// first products are permuted (column c holds unit c/2 + 4 (c mod 2)) so that
// a lane's C fragment of Z is, register for register, its A fragment of the
// second product: the element-wise terms never leave the registers.  W0 sits
// in shared memory already split (hi and lo TF32 words).  The weight gradient
// dW0 and its column sums take the contraction over atoms as before.
template <int D>
struct MmaW {
  static constexpr int DP = (D + 7) / 8 * 8;  // descriptors padded to k-steps of 8
  static constexpr int KD = DP / 8;
  static constexpr int SW = DP + 4;  // row stride (4 mod 8 words: the A and Z-product B fragments hit 32 banks)
};

// Weights of species e split into TF32 hi / lo words: Wh, Wl [HP][SW] (zero
// beyond D and H), b0, w1 [HP] (zero beyond H).
template <int D, int HP, int NTH>
__device__ void load_weights_split(const DevModel& dm, int e, uint32_t* Wh, uint32_t* Wl, float* b0, float* w1) {
  constexpr int SW = MmaW<D>::SW;
  const float* P = dm.params + (size_t)e * dm.net_size;
  const int H = dm.H;
  constexpr int N = HP * SW;
  for (int q0 = threadIdx.x; q0 < N; q0 += 4 * NTH) {  // four loads in flight per thread
    float x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int q = q0 + k * NTH, mu = q / SW, v = q % SW;
      x[k] = (q < N && v < D && mu < H) ? __ldg(P + mu * D + v) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (q0 + k * NTH < N) split_tf32<true>(x[k], Wh[q0 + k * NTH], Wl[q0 + k * NTH]);
  }
  for (int mu = threadIdx.x; mu < HP; mu += NTH) {
    b0[mu] = mu < H ? P[D * H + mu] : 0.f;
    w1[mu] = mu < H ? P[D * H + H + mu] : 0.f;
  }
}

// B fragment of a first product: column g of hidden chunk n0 (unit n0 + pg),
// rows c and c + 4 of the descriptor k-step.
template <int SW>
__device__ __forceinline__ void frag_w_cols(FragB& b, const uint32_t* Wh, const uint32_t* Wl, int mu, int c) {
  b.h[0] = Wh[mu * SW + c];
  b.l[0] = Wl[mu * SW + c];
  b.h[1] = Wh[mu * SW + c + 4];
  b.l[1] = Wl[mu * SW + c + 4];
}
// B fragment of a second product: rows k0 and k0 + 4 (hidden units), column d.
template <int SW>
__device__ __forceinline__ void frag_w_rows(FragB& b, const uint32_t* Wh, const uint32_t* Wl, int k0, int d) {
  b.h[0] = Wh[k0 * SW + d];
  b.l[0] = Wl[k0 * SW + d];
  b.h[1] = Wh[(k0 + 4) * SW + d];
  b.l[1] = Wl[(k0 + 4) * SW + d];
}

template <int D, int HP, int NS, int NQR, int KR, int TA>
size_t mlp_fwd_mma_smem() {
  constexpr int SW = MmaW<D>::SW;
  return sizeof(float) * (2 * (size_t)HP * SW + 2 * TA * (size_t)SW + 2 * HP + SW + NS * NQR * KR);
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

// Forward on tensor cores: z = W0 (s.G) + b0, x = tanh z, E = w1.x + b1,
// E' = s . (W0^T (w1 (1 - x^2)))  (D1.1-D1.5), and chat as in k_mlp_fwd_row.
template <int D, int HP, int NS, int NQR, int KR, int TA>
__global__ void __launch_bounds__(2 * TA, 1) k_mlp_fwd_mma(Tiles T, int ntiles, DevModel dm, const float* __restrict__ G,
                                                       float* __restrict__ Ep, float* __restrict__ Eatom,
                                                       float* __restrict__ chat) {
  GNEP_PDL_WAIT();
  constexpr int NTB = 2 * TA, SW = MmaW<D>::SW, KD = MmaW<D>::KD, NJK = NS * KR;
  static_assert(HP % 16 == 0 && TA == 128, "16-unit chunks, 16 atoms per warp");
  extern __shared__ float4 sm4[];
  uint32_t* Wh = reinterpret_cast<uint32_t*>(sm4);  // [HP][SW]
  uint32_t* Wl = Wh + HP * SW;                       // [HP][SW]
  float* Rbuf = reinterpret_cast<float*>(Wl + HP * SW);  // [2][TA][SW] s.G, then the scaled E'
  float* b0 = Rbuf + 2 * TA * SW;                    // [HP]
  float* w1 = b0 + HP;                               // [HP]
  float* sc = w1 + HP;                               // [SW]
  float* cR = sc + SW;                               // [NS][NQR][KR] of the tile's species
  __shared__ int rowsb[2][TA];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3, pg = (g >> 1) | ((g & 1) << 2);
  const int H = dm.H;
  // Staging: the rows of a tile are copied into one of two buffers with
  // cp.async (thread 2a + h copies the elements h, h + 2, ... of atom a's row)
  // while the previous tile writes its outputs, then scaled in place by the
  // thread that copied them.  Columns beyond D stay zero (the buffers start
  // zeroed and the E' rows written there carry s = 0 beyond D); rows beyond a
  // tile's atoms keep earlier finite values and only feed discarded rows.
  const int sa = tid >> 1, sh = tid & 1;
  for (int q = tid; q < 2 * TA * SW; q += NTB) Rbuf[q] = 0.f;
  for (int v = tid; v < SW; v += NTB) sc[v] = v < D ? dm.scale[v] : 0.f;
  __syncthreads();
  auto issue = [&](int r, int buf) {  // row r of G into this thread's atom slot of buffer buf
    rowsb[buf][sa] = r;  // both threads of the atom write the same value
    if (r >= 0) {
      float* dst = Rbuf + (size_t)buf * TA * SW + sa * SW;
      const float* src = G + (size_t)r * D;
      for (int v = sh; v < D; v += 2) cp_async4(dst + v, src + v);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  auto tile_row = [&](int tt) {  // row index of this thread's atom in tile tt (-1 beyond it)
    if (tt >= ntiles) return -1;
    int e, a0, na;
    tile_of<TA>(T, tt, e, a0, na);
    return sa < na ? T.perm[a0 + sa] : -1;
  };
  int cur_e = -1;
  float b1 = 0.f;
  int buf = 0;
  if (blockIdx.x < ntiles) issue(tile_row(blockIdx.x), 0);
  for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x, buf ^= 1) {
    int e, a0, na;
    tile_of<TA>(T, tt, e, a0, na);
    const int rnext = tile_row(tt + gridDim.x);  // loaded now, used after the products
    __syncthreads();  // the previous tile's readers of the weights are done
    if (e != cur_e) {
      load_weights_split<D, HP, NTB>(dm, e, Wh, Wl, b0, w1);
      for (int q = tid; q < NS * NQR * KR; q += NTB) cR[q] = dm.params[dm.off_cR + e * NS * NQR * KR + q];
      b1 = dm.params[(size_t)e * dm.net_size + D * H + 2 * H];
      cur_e = e;
    }
    float* R = Rbuf + (size_t)buf * TA * SW;
    const int* rows = rowsb[buf];
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (sa < na)
      for (int v = sh; v < D; v += 2) R[sa * SW + v] *= sc[v];
    __syncthreads();
    float* Rw = R + 16 * warp * SW;  // this warp's 16 rows
    Acc<true> ep[KD];
#pragma unroll
    for (int nd = 0; nd < KD; ++nd) ep[nd].zero();
    float Eg = 0.f, Eg8 = 0.f;  // energies of atoms g and g + 8 (this lane's units)
    if (16 * warp < na) {
      for (int hc = 0; hc < HP / 16 && 16 * hc < H; ++hc) {
        Acc<true> z[2];
        z[0].zero();
        z[1].zero();
#pragma unroll
        for (int ks = 0; ks < KD; ++ks) {
          const int c = 8 * ks + t;
          FragA a;
          frag_a<true>(a, Rw[g * SW + c], Rw[(g + 8) * SW + c], Rw[g * SW + c + 4], Rw[(g + 8) * SW + c + 4]);
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) {
            FragB b;
            frag_w_cols<SW>(b, Wh, Wl, 16 * hc + 8 * nt + pg, c);
            mma_acc<true>(z[nt], a, b);
          }
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int m0 = 16 * hc + 8 * nt + t, m1 = m0 + 4;  // units of C columns 2t and 2t + 1
          const float x0 = tanhf(z[nt].get(0) + b0[m0]), x1 = tanhf(z[nt].get(1) + b0[m1]);
          const float x2 = tanhf(z[nt].get(2) + b0[m0]), x3 = tanhf(z[nt].get(3) + b0[m1]);
          Eg = fmaf(w1[m1], x1, fmaf(w1[m0], x0, Eg));
          Eg8 = fmaf(w1[m1], x3, fmaf(w1[m0], x2, Eg8));
          FragA ab;  // beta = w1 (1 - x^2) as the A fragment (rows g, g + 8; k = t, t + 4)
          frag_a<true>(ab, w1[m0] * (1.f - x0 * x0), w1[m0] * (1.f - x2 * x2), w1[m1] * (1.f - x1 * x1),
                       w1[m1] * (1.f - x3 * x3));
#pragma unroll
          for (int nd = 0; nd < KD; ++nd) {
            FragB b;
            frag_w_rows<SW>(b, Wh, Wl, m0, 8 * nd + g);
            mma_acc<true>(ep[nd], ab, b);
          }
        }
      }
    }
    Eg += __shfl_xor_sync(0xffffffffu, Eg, 1);
    Eg += __shfl_xor_sync(0xffffffffu, Eg, 2);
    Eg8 += __shfl_xor_sync(0xffffffffu, Eg8, 1);
    Eg8 += __shfl_xor_sync(0xffffffffu, Eg8, 2);
    __syncwarp();  // the warp's rows of R have been read: they take the scaled E'
#pragma unroll
    for (int nd = 0; nd < KD; ++nd) {
      const int d = 8 * nd + 2 * t;
      Rw[g * SW + d] = ep[nd].get(0) * sc[d];
      Rw[g * SW + d + 1] = ep[nd].get(1) * sc[d + 1];
      Rw[(g + 8) * SW + d] = ep[nd].get(2) * sc[d];
      Rw[(g + 8) * SW + d + 1] = ep[nd].get(3) * sc[d + 1];
    }
    if (t == 0) {
      if (16 * warp + g < na) Eatom[rows[16 * warp + g]] = Eg + b1;
      if (16 * warp + g + 8 < na) Eatom[rows[16 * warp + g + 8]] = Eg8 + b1;
    }
    __syncthreads();
    issue(rnext, buf ^ 1);  // the next tile's rows arrive while this one writes its outputs
    // coalesced row writes: E' and chat
    for (int q = tid; q < na * D; q += NTB) {
      const int r = q / D, v = q % D;
      Ep[(size_t)rows[r] * D + v] = R[r * SW + v];
    }
    for (int q = tid; q < na * NJK; q += NTB) {
      const int r = q / NJK, jk = q % NJK, J = jk / KR, k = jk % KR;
      float s = 0.f;
#pragma unroll
      for (int n = 0; n < NQR; ++n) s = fmaf(R[r * SW + n], cR[(J * NQR + n) * KR + k], s);
      chat[(size_t)rows[r] * NJK + jk] = s;
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");  // no copy outlives the block
}

template <int D, int HP>
size_t mlp_bwd_mma_smem() {
  constexpr int SW = MmaW<D>::SW, HR = HP + 8, TA = 128, NWB = TA / 16;
  return sizeof(float) * (2 * (size_t)HP * SW + 2 * (size_t)TA * SW + 2 * (size_t)TA * HR + 2 * (size_t)NWB * HP +
                          2 * HP + SW + TA);
}

// Tangent and reverse pass on tensor cores (the terms of k_mlp_bwd_row):
// per chunk of 16 hidden units, Z and Zdot by split-TF32 products, the
// element-wise alpha, -beta, q1 in the accumulator registers, Gbar += alpha W0;
// alpha and -beta go to shared rows, the column sums of alpha and q1 over the
// warp's atoms to per-warp shared sums.  Then the weight gradient
//   dW0 += alpha^T (s.G) - beta^T (s.Gdot)      M 16 units, N 8 descriptors, K 8 atoms
// by split-TF32 products too: warp w takes the 16-unit block w mod (HP/16) and
// one of 8 / (HP/16) groups of the tile's atoms, keeping its partial dW0 in
// registers over all tiles of a species; the partials are added in warp order
// when the block flushes.  Writes part[block][species] like k_mlp_bwd_row.
// 128-atom tiles, HP (hidden width padded) 32 or 64.
template <int D, int HP>
__global__ void __launch_bounds__(256, 1) k_mlp_bwd_mma(Tiles T, int ntiles, DevModel dm,
                                                       const int* __restrict__ atom_struct,
                                                       const float* __restrict__ es, const float* __restrict__ G,
                                                       const float* __restrict__ Gd, float* __restrict__ Gb,
                                                       float* __restrict__ part, int part_stride) {
  GNEP_PDL_WAIT();
  constexpr int TA = 128, NTB = 256, NWB = 8, SW = MmaW<D>::SW, KD = MmaW<D>::KD, HR = HP + 8;
  constexpr int MT = HP / 16, KG = NWB / MT, KA = TA / KG;  // dW0: unit blocks, atom groups, atoms per group
  static_assert(HP % 16 == 0 && HP <= 64 && NWB % MT == 0, "16-unit chunks, 16 atoms per warp");
  extern __shared__ float4 sm4[];
  uint32_t* Wh = reinterpret_cast<uint32_t*>(sm4);  // [HP][SW]
  uint32_t* Wl = Wh + HP * SW;                       // [HP][SW]
  float* SG = reinterpret_cast<float*>(Wl + HP * SW);  // [TA][SW] s.G, then the Gbar output rows
  float* SD = SG + TA * SW;                          // [TA][SW] s.Gdot
  float* Al = SD + TA * SW;                          // [TA][HR] alpha
  float* Be = Al + TA * HR;                          // [TA][HR] -beta
  float* wdb0 = Be + TA * HR;                        // [NWB][HP] per-warp column sums of alpha
  float* wdw1 = wdb0 + NWB * HP;                     // [NWB][HP] per-warp column sums of q1
  float* b0 = wdw1 + NWB * HP;                       // [HP]
  float* w1 = b0 + HP;                               // [HP]
  float* sc = w1 + HP;                               // [SW]
  float* ev = sc + SW;                               // [TA] e_i of the tile's atoms
  __shared__ int rows[TA];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3, pg = (g >> 1) | ((g & 1) << 2);
  const int mw = warp % MT, kw = warp / MT;  // this warp's dW0 unit block and atom group
  const int H = dm.H;
  for (int v = tid; v < SW; v += NTB) sc[v] = v < D ? dm.scale[v] : 0.f;
  for (int q = tid; q < 2 * TA * HR; q += NTB) Al[q] = 0.f;  // Be follows Al
  Acc<true> dw[KD];  // dW0[16 mw + (g, g + 8)][8 nd + 2t, + 1], partial over atom group kw
  float cb1 = 0.f;
  int cur_e = -1;
  unsigned visited = 0;  // species whose partial this block writes

  auto reset = [&]() {
#pragma unroll
    for (int nd = 0; nd < KD; ++nd) dw[nd].zero();
    for (int q = tid; q < 2 * NWB * HP; q += NTB) wdb0[q] = 0.f;  // wdw1 follows wdb0
    cb1 = 0.f;
  };
  // after a barrier that follows the last tile of species e; uses SG as scratch
  auto flush = [&](int e) {
    float* red = SG;  // [NWB][16][8 KD] the warps' partial dW0 blocks
#pragma unroll
    for (int nd = 0; nd < KD; ++nd) {
      const int d = 8 * nd + 2 * t;
      red[(warp * 16 + g) * 8 * KD + d] = dw[nd].get(0);
      red[(warp * 16 + g) * 8 * KD + d + 1] = dw[nd].get(1);
      red[(warp * 16 + g + 8) * 8 * KD + d] = dw[nd].get(2);
      red[(warp * 16 + g + 8) * 8 * KD + d + 1] = dw[nd].get(3);
    }
    __syncthreads();
    float* out = part + ((size_t)blockIdx.x * T.ns + e) * part_stride;
    for (int q = tid; q < H * D; q += NTB) {
      const int mu = q / D, v = q % D, m = mu / 16, r = mu % 16;
      float s = 0.f;
      for (int k = 0; k < KG; ++k) s += red[((k * MT + m) * 16 + r) * 8 * KD + v];  // atom groups in order
      out[q] = s;
    }
    for (int mu = tid; mu < H; mu += NTB) {
      float s0 = 0.f, s1 = 0.f;
      for (int w = 0; w < NWB; ++w) {  // warps in order
        s0 += wdb0[w * HP + mu];
        s1 += wdw1[w * HP + mu];
      }
      out[D * H + mu] = s0;
      out[D * H + H + mu] = s1;
    }
    if (tid == 0) out[D * H + 2 * H] = cb1;
  };
  reset();

  for (int tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
    int e, a0, na;
    tile_of<TA>(T, tt, e, a0, na);
    __syncthreads();  // the previous tile is done with every shared array
    if (e != cur_e) {
      if (cur_e >= 0) flush(cur_e);
      __syncthreads();
      reset();
      load_weights_split<D, HP, NTB>(dm, e, Wh, Wl, b0, w1);
      cur_e = e;
      visited |= 1u << e;
    }
    if (tid < TA) {
      const int r = tid < na ? T.perm[a0 + tid] : -1;
      rows[tid] = r;
      ev[tid] = r >= 0 ? es[atom_struct[r]] : 0.f;
    }
    __syncthreads();
    stage_rows<D, 2, TA, SW, NTB>(G, Gd, rows, sc, SG, SD);
    if (tid == 0)
      for (int r = 0; r < na; ++r) cb1 += ev[r];
    __syncthreads();
    // per warp: Z, Zdot, the element-wise terms and Gbar of its 16 atoms
    const float* Gw = SG + 16 * warp * SW;
    const float* Dw = SD + 16 * warp * SW;
    Acc<true> gb[KD];
#pragma unroll
    for (int nd = 0; nd < KD; ++nd) gb[nd].zero();
    if (16 * warp < na) {
      const float ea = ev[16 * warp + g], ea8 = ev[16 * warp + g + 8];
      float* Alw = Al + 16 * warp * HR;
      float* Bew = Be + 16 * warp * HR;
      for (int hc = 0; hc < HP / 16 && 16 * hc < H; ++hc) {
        Acc<true> z[2], zd[2];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          z[nt].zero();
          zd[nt].zero();
        }
#pragma unroll
        for (int ks = 0; ks < KD; ++ks) {
          const int c = 8 * ks + t;
          FragA a, ad;
          frag_a<true>(a, Gw[g * SW + c], Gw[(g + 8) * SW + c], Gw[g * SW + c + 4], Gw[(g + 8) * SW + c + 4]);
          frag_a<true>(ad, Dw[g * SW + c], Dw[(g + 8) * SW + c], Dw[g * SW + c + 4], Dw[(g + 8) * SW + c + 4]);
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) {
            FragB b;
            frag_w_cols<SW>(b, Wh, Wl, 16 * hc + 8 * nt + pg, c);
            mma_acc<true>(z[nt], a, b);
            mma_acc<true>(zd[nt], ad, b);
          }
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int m[2] = {16 * hc + 8 * nt + t, 16 * hc + 8 * nt + t + 4};  // units of C columns 2t, 2t + 1
          float al[4], q1[4];  // C positions: (g, m0) (g, m1) (g + 8, m0) (g + 8, m1)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int mu = m[r & 1];
            const float ee = r < 2 ? ea : ea8;
            const float x = tanhf(z[nt].get(r) + b0[mu]);
            const float t1 = 1.f - x * x;
            const float beta = w1[mu] * t1;
            const float zdr = zd[nt].get(r);
            al[r] = ee * beta + 2.f * x * beta * zdr;
            q1[r] = ee * x - t1 * zdr;  // zero for padding atoms (e = 0, zdot = 0) and padding units
            const int row = (r < 2 ? g : g + 8) * HR + mu;
            Alw[row] = al[r];
            Bew[row] = -beta;
          }
          // column sums over the warp's 16 atoms (rows g and g + 8 of the eight lanes t)
          float s[4] = {al[0] + al[2], al[1] + al[3], q1[0] + q1[2], q1[1] + q1[3]};
#pragma unroll
          for (int o = 4; o < 32; o <<= 1)
#pragma unroll
            for (int k = 0; k < 4; ++k) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
          if (g == 0) {
            wdb0[warp * HP + m[0]] += s[0];
            wdb0[warp * HP + m[1]] += s[1];
            wdw1[warp * HP + m[0]] += s[2];
            wdw1[warp * HP + m[1]] += s[3];
          }
          FragA aa;  // alpha as the A fragment (rows g, g + 8; k = t, t + 4)
          frag_a<true>(aa, al[0], al[2], al[1], al[3]);
#pragma unroll
          for (int nd = 0; nd < KD; ++nd) {
            FragB b;
            frag_w_rows<SW>(b, Wh, Wl, m[0], 8 * nd + g);
            mma_acc<true>(gb[nd], aa, b);
          }
        }
      }
    }
    __syncthreads();  // alpha and -beta of the tile are complete
    // dW0 += alpha^T (s.G) - beta^T (s.Gdot) over this warp's atom group
    if (16 * mw < H) {
      const int k1 = min(na, KA * (kw + 1));
      for (int k0 = KA * kw; k0 < k1; k0 += 8) {
        const int u = 16 * mw + g;  // A rows g, g + 8: units; columns t, t + 4: atoms
        FragA fa, fb;
        frag_a<true>(fa, Al[(k0 + t) * HR + u], Al[(k0 + t) * HR + u + 8], Al[(k0 + t + 4) * HR + u],
                     Al[(k0 + t + 4) * HR + u + 8]);
        frag_a<true>(fb, Be[(k0 + t) * HR + u], Be[(k0 + t) * HR + u + 8], Be[(k0 + t + 4) * HR + u],
                     Be[(k0 + t + 4) * HR + u + 8]);
#pragma unroll
        for (int nd = 0; nd < KD; ++nd) {
          const int d = 8 * nd + g;  // B rows t, t + 4: atoms; column g: descriptor
          FragB bg, bd;
          frag_b<true>(bg, SG[(k0 + t) * SW + d], SG[(k0 + t + 4) * SW + d]);
          frag_b<true>(bd, SD[(k0 + t) * SW + d], SD[(k0 + t + 4) * SW + d]);
          mma_acc<true>(dw[nd], fa, bg);
          mma_acc<true>(dw[nd], fb, bd);
        }
      }
    }
    __syncthreads();  // s.G rows are no longer read: they take the Gbar rows
    {
      float* Ow = SG + 16 * warp * SW;
#pragma unroll
      for (int nd = 0; nd < KD; ++nd) {
        const int d = 8 * nd + 2 * t;
        Ow[g * SW + d] = gb[nd].get(0) * sc[d];
        Ow[g * SW + d + 1] = gb[nd].get(1) * sc[d + 1];
        Ow[(g + 8) * SW + d] = gb[nd].get(2) * sc[d];
        Ow[(g + 8) * SW + d + 1] = gb[nd].get(3) * sc[d + 1];
      }
    }
    __syncthreads();
    for (int q = tid; q < na * D; q += NTB) {
      const int r = q / D, v = q % D;
      Gb[(size_t)rows[r] * D + v] = SG[r * SW + v];
    }
  }
  __syncthreads();
  if (cur_e >= 0) flush(cur_e);
  // the partials of the species this block did not visit are zero (the
  // gradient assembly reads every block's row of every species)
  for (int e = 0; e < T.ns; ++e)
    if (!(visited & (1u << e)))
      for (int q = threadIdx.x; q < part_stride; q += blockDim.x)
        part[((size_t)blockIdx.x * T.ns + e) * part_stride + q] = 0.f;
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
int resident_blocks(K kern, int threads, size_t smem, int& out) {
  int per_sm = 0, dev = 0, sms = 0;
  GNEP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
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

template <class K>
int set_smem(K kern, size_t bytes) {
  GNEP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  GNEP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  return GNEP_OK;
}

// Kernels per tile size: 32-atom tiles on the CUDA cores (eight threads per
// atom); 128-atom tiles on the tensor cores, except the backward pass above 64
// hidden units (its alpha and beta rows would not fit next to the split
// weights), which takes the CUDA-core kernel with two threads per atom.
template <int D, int HP, int NS, int NQR, int KR>
int mlp_setup() {
  // shared memory for the largest hidden width of this padding
  if (int rc = set_smem(k_mlp_fwd_row<D, NS, NQR, KR, 32>, mlp_fwd_smem<D, NS, NQR, KR, 32>(kMaxHidden))) return rc;
  if (int rc = set_smem(k_mlp_bwd_row<D, HP, 32>, mlp_bwd_smem<D, HP, 32>(HP))) return rc;
  if (int rc = set_smem(k_mlp_fwd_mma<D, HP, NS, NQR, KR, 128>, mlp_fwd_mma_smem<D, HP, NS, NQR, KR, 128>()))
    return rc;
  if constexpr (HP <= 64) {
    return set_smem(k_mlp_bwd_mma<D, HP>, mlp_bwd_mma_smem<D, HP>());
  } else {
    return set_smem(k_mlp_bwd_row<D, HP, 128>, mlp_bwd_smem<D, HP, 128>(HP));
  }
}

template <class K>
int launch_forward(K kern, int threads, size_t smem, int tile_atoms, const gnep_model* m, gnep_nlist* nl,
                   cudaStream_t st, const char* what) {
  const Tiles T = make_tiles(nl, m->shape.ns, tile_atoms);
  const int ntiles = T.tbase[m->shape.ns];
  if (ntiles == 0) return GNEP_OK;
  Workspace& w = nl->ws;
  int cap = 0;
  if (int rc = resident_blocks(kern, threads, smem, cap)) return rc;
  const int grid = net_blocks(nl, ntiles < cap ? ntiles : cap);
  (void)launch_pdl(kern, grid, threads, smem, st, T, ntiles, m->dev(), w.G, w.Ep, w.Eatom, w.chat);
  GNEP_CHECK_LAUNCH(what);
  return GNEP_OK;
}

template <int D, int HP, int NS, int NQR, int KR>
int mlp_forward(const gnep_model* m, gnep_nlist* nl, cudaStream_t st) {
  switch (net_tile_atoms(nl, NS)) {
    case 32:
      return launch_forward(k_mlp_fwd_row<D, NS, NQR, KR, 32>, NT, mlp_fwd_smem<D, NS, NQR, KR, 32>(m->shape.H), 32,
                            m, nl, st, "k_mlp_fwd_row");
    default:
      return launch_forward(k_mlp_fwd_mma<D, HP, NS, NQR, KR, 128>, 256, mlp_fwd_mma_smem<D, HP, NS, NQR, KR, 128>(),
                            128, m, nl, st, "k_mlp_fwd_mma");
  }
}

template <class K>
int launch_backward(K kern, int threads, size_t smem, int tile_atoms, const gnep_model* m, gnep_nlist* nl,
                    cudaStream_t st, const char* what) {
  const int ns = m->shape.ns;
  const Tiles T = make_tiles(nl, ns, tile_atoms);
  const int ntiles = T.tbase[ns];
  Workspace& w = nl->ws;
  int cap = 0;
  if (int rc = resident_blocks(kern, threads, smem, cap)) return rc;
  if (cap > kNetBlocks) cap = kNetBlocks;  // net_part holds kNetBlocks partials
  const int grid = net_blocks(nl, ntiles < cap ? (ntiles > 0 ? ntiles : 1) : cap);
  w.net_blocks = grid;
  if (ntiles == 0) {  // no block runs: the single partial is zero
    GNEP_CUDA(cudaMemsetAsync(w.net_part, 0, sizeof(float) * (size_t)grid * ns * m->net_size, st));
    return GNEP_OK;
  }
  (void)launch_pdl(kern, grid, threads, smem, st, T, ntiles, m->dev(), nl->atom_struct, w.es, w.G, w.Gd, w.Gb, w.net_part,
                                    m->net_size);
  GNEP_CHECK_LAUNCH(what);
  return GNEP_OK;
}

template <int D, int HP>
int mlp_backward(const gnep_model* m, gnep_nlist* nl, cudaStream_t st) {
  const int ta = net_tile_atoms(nl, m->shape.ns);
  if (ta == 32)
    return launch_backward(k_mlp_bwd_row<D, HP, 32>, NT, mlp_bwd_smem<D, HP, 32>(m->shape.H), 32, m, nl, st,
                           "k_mlp_bwd_row");
  if constexpr (HP <= 64) {
    return launch_backward(k_mlp_bwd_mma<D, HP>, 256, mlp_bwd_mma_smem<D, HP>(), 128, m, nl, st, "k_mlp_bwd_mma");
  } else {
    return launch_backward(k_mlp_bwd_row<D, HP, 128>, NT, mlp_bwd_smem<D, HP, 128>(m->shape.H), 128, m, nl, st,
                           "k_mlp_bwd_row");
  }
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
