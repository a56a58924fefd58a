// Per-element network (D1.1-D1.10, and the tangent/reverse pass of
// D1.18-D1.21) with its contractions on the fifth-generation tensor cores:
// BF16 or TF32 operands staged in shared memory, FP32 accumulation in tensor
// memory (TMEM).  Tiles hold 128 atoms of one species, so that an atom is a
// row of every MMA and thread t of the block owns TMEM lane t, i.e. atom t of
// the tile: the element-wise epilogues (tanh, beta, alpha, energies) run
// thread-per-atom straight out of TMEM.
//
// Forward, per tile:   Z  = (s.G) W0^T                     [128 x H]
//                      E' = (w1 (1 - x^2)) W0, scaled by s  [128 x D]
// Backward, per tile:  Z, Zdot = (s.G) W0^T, (s.Gdot) W0^T
//                      Gbar = s . (alpha W0)
//                      dW0 += alpha^T (s.G) - beta^T (s.Gdot)    (K = atoms)
// dW0 stays in TMEM across all tiles a block visits for one species and is
// written once, as one partial per block and species; db0 = sum of alpha comes
// out of the same accumulator through a column of ones appended to (s.G)^T.
// All operands are K-major; the operands of the atom contraction are written
// transposed by the epilogue.  Per-atom rows are staged one 8 x 16-byte core
// matrix per warp step with 4-byte stores that fill the 32 banks, and the
// atom-contraction operands take padded core matrices where that costs no
// block per SM, so that the epilogue's transposed stores do not collide.  The
// network in FP32 (network.cu) is the plain form these modes are measured
// against.
#include "gnep_internal.h"
#include "network.cuh"
#include "tc.cuh"

namespace gnep {

namespace {

constexpr int TA = 128;                      // atoms per tile = MMA rows = TMEM lanes
constexpr int NTC = 256;                     // threads per block: warps w and w + 4 share TMEM lanes 32 (w % 4) ..
constexpr uint64_t kWaitNs = 1000000000ull;  // give up on an MMA completion after 1 s
constexpr int kSmemPerSm = 233472;           // shared memory per SM (228 KB)

__device__ __forceinline__ void tile_of(const Tiles& T, int t, int& e, int& a0, int& na) {
  e = 0;
  while (e + 1 < T.ns && t >= T.tbase[e + 1]) ++e;
  a0 = T.soff[e] + (t - T.tbase[e]) * TA;
  na = min(TA, T.soff[e + 1] - a0);
}

// Bytes of an R x C operand whose K-adjacent core matrices are L bytes apart.
template <bool TF32>
constexpr int op_bytes(int R, int C, uint32_t L) {
  return (R / 8) * (int)tc::sbo<TF32>(C, L);
}
// Blocks per SM that TMEM and shared memory admit (caps the registers per thread via launch bounds).
constexpr int tc_fits(int smem, int cols) {
  const int by_smem = kSmemPerSm / (smem + 6 * 1024), by_tmem = 512 / cols;
  const int b = by_smem < by_tmem ? by_smem : by_tmem;
  return b < 1 ? 1 : (b > 3 ? 3 : b);
}
constexpr int kMaxDynSmem = 232448;  // per block (227 KB)

template <bool TF32, int D, int HPn>
struct Layout {
  static constexpr int DPn = (D + 1 + 15) / 16 * 16;  // descriptor width + the ones column, padded
  static constexpr int bO = TA * (D + 1) * 4;
  static constexpr int fwd(uint32_t L) {
    const int g = op_bytes<TF32>(TA, DPn, L), h = op_bytes<TF32>(TA, HPn, L);
    return (g > h ? g : h) + 2 * op_bytes<TF32>(HPn, DPn, L) + bO;
  }
  // L: operands contracted over v or mu; LT: the backward's operands contracted over the tile's atoms
  static constexpr int bwd(uint32_t L, uint32_t LT) {
    const int g2 = 2 * op_bytes<TF32>(TA, DPn, L), h = op_bytes<TF32>(TA, HPn, L);
    return (g2 > h ? g2 : h) + op_bytes<TF32>(DPn, TA, LT) + op_bytes<TF32>(128, TA, LT) +
           2 * op_bytes<TF32>(HPn, DPn, L);
  }
  static constexpr int fwd_cols = tc::pow2_cols(HPn + DPn);
  static constexpr int bwd_cols = tc::pow2_cols(2 * HPn + 2 * DPn);
  // padded core matrices where they cost no block per SM and fit a block
  static constexpr uint32_t lbo() {
    return (fwd(144) <= kMaxDynSmem && bwd(144, 144) <= kMaxDynSmem &&
            tc_fits(fwd(144), fwd_cols) >= tc_fits(fwd(128), fwd_cols) &&
            tc_fits(bwd(144, 144), bwd_cols) >= tc_fits(bwd(128, 128), bwd_cols))
               ? 144u
               : 128u;
  }
  // the atom-contraction operands alone, where padding all operands costs a block
  static constexpr uint32_t lbo_t() {
    return (bwd(lbo(), 144) <= kMaxDynSmem && tc_fits(bwd(lbo(), 144), bwd_cols) >= tc_fits(bwd(lbo(), 128), bwd_cols))
               ? 144u
               : 128u;
  }
};

template <bool TF32, int D, int HPn>
struct Dims {
  using Lay = Layout<TF32, D, HPn>;
  static constexpr int DPn = Lay::DPn;
  static constexpr uint32_t LBO = Lay::lbo(), LBOT = Lay::lbo_t();
  static constexpr uint32_t sG = tc::sbo<TF32>(DPn, LBO);  // rows of length DPn:  [atoms][v], [mu][v]
  static constexpr uint32_t sH = tc::sbo<TF32>(HPn, LBO);  // rows of length HPn:  [atoms][mu], [v][mu]
  static constexpr uint32_t sA = tc::sbo<TF32>(TA, LBOT);  // rows of length TA:   [mu][atoms], [v][atoms]
  static constexpr int bG = op_bytes<TF32>(TA, DPn, LBO);
  static constexpr int bH = op_bytes<TF32>(TA, HPn, LBO);
  static constexpr int bW0 = op_bytes<TF32>(HPn, DPn, LBO);
  static constexpr int bT = op_bytes<TF32>(128, TA, LBOT);  // [mu][atoms], 128 rows (the MMA's M) whatever H is
  static constexpr int bGT = op_bytes<TF32>(DPn, TA, LBOT);
  static constexpr int OW = D + 1;          // row pitch (floats) of the FP32 output tile, odd: conflict-free rows
  static constexpr int bO = Lay::bO;
  // forward: RA (s.G, then beta) | W0 [mu][v] | W0t [v][mu] | output tile (E')
  static constexpr int fRA = bG > bH ? bG : bH;
  static constexpr int fwd_smem = fRA + 2 * bW0 + bO;
  static constexpr int fwd_cols = Lay::fwd_cols;
  // backward: RA (s.G | s.Gdot, then alpha) | RG ((s.G)^T, then (s.Gdot)^T) |
  //           RT (alpha^T, then the Gbar output tile, then -beta^T) | W0 | W0t
  static constexpr int bRA = 2 * bG > bH ? 2 * bG : bH;
  static constexpr int bwd_smem = bRA + bGT + bT + 2 * bW0;
  static constexpr int bwd_cols = Lay::bwd_cols;
  static_assert(bO <= bT, "the Gbar output tile lives in the [mu][atoms] operand");
  static_assert(fwd_smem == Lay::fwd(LBO) && bwd_smem == Lay::bwd(LBO, LBOT), "layout sizes");
  static constexpr int fwd_minb = tc_fits(fwd_smem, fwd_cols);
  static constexpr int bwd_minb = tc_fits(bwd_smem, bwd_cols);
};

// W0 of species e as [mu][v] and [v][mu] operands (zero-padded), b0 and w1.
template <bool TF32, int D, int HPn>
__device__ void stage_weights(const DevModel& dm, int e, uint8_t* W0, uint8_t* W0t, float* b0s, float* w1s) {
  using Dm = Dims<TF32, D, HPn>;
  const float* P = dm.params + (size_t)e * dm.net_size;
  const int H = dm.H;
  for (int q = threadIdx.x; q < HPn * Dm::DPn; q += NTC) {
    const int mu = q / Dm::DPn, v = q % Dm::DPn;
    const float w = (mu < H && v < D) ? P[mu * D + v] : 0.f;
    tc::st_elem<TF32>(W0, tc::core_off<TF32>(mu, v, Dm::sG, Dm::LBO), w);
    tc::st_elem<TF32>(W0t, tc::core_off<TF32>(v, mu, Dm::sH, Dm::LBO), w);
  }
  for (int mu = threadIdx.x; mu < HPn; mu += NTC) {
    b0s[mu] = mu < H ? P[D * H + mu] : 0.f;
    w1s[mu] = mu < H ? P[D * H + H + mu] : 0.f;
  }
}

// Rows `rows[a]` (a < TA, -1 = padding) of one or two per-atom arrays of
// width D, zero-padded to DPn columns, staged one core matrix per warp step:
// the atoms 8 ab .. 8 ab + 7 and the EPC columns of column chunk vc.  Lane l
// takes atom 8 ab + l / 4 and the EW = 4 / ES columns of word l % 4 of that
// core row and hands them to store(a, v, x[array][e]), so that the warp's 32
// word stores into an [atoms][v] operand fill the 32 banks.  A warp takes
// consecutive blocks (all column chunks of two atom groups) and keeps NB
// blocks of loads in flight.
template <bool TF32, int D, int DPn, int NARR, class F>
__device__ __forceinline__ void stage_blocks(const float* __restrict__ s0, const float* __restrict__ s1,
                                             const int* rows, F store) {
  constexpr int EPC = tc::Elem<TF32>::EPC, EW = 4 / tc::Elem<TF32>::ES, NVC = DPn / EPC;
  constexpr int PERW = (TA / 8) * NVC / (NTC / 32), NB = 4;
  static_assert((TA / 8) * NVC % (NTC / 32) == 0 && PERW % NB == 0, "blocks per warp");
  const int lane = threadIdx.x & 31, b0 = (threadIdx.x >> 5) * PERW, ai = lane >> 2, w = lane & 3;
#pragma unroll 1
  for (int bb = 0; bb < PERW; bb += NB) {
    float x[NB][NARR][EW];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int blk = b0 + bb + u, a = 8 * (blk / NVC) + ai, v = EPC * (blk % NVC) + EW * w, r = rows[a];
#pragma unroll
      for (int e = 0; e < EW; ++e) {
        const bool in = r >= 0 && v + e < D;
        x[u][0][e] = in ? s0[(size_t)r * D + v + e] : 0.f;
        if constexpr (NARR > 1) x[u][NARR - 1][e] = in ? s1[(size_t)r * D + v + e] : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int blk = b0 + bb + u;
      store(8 * (blk / NVC) + ai, EPC * (blk % NVC) + EW * w, x[u]);
    }
  }
}

// This lane's values of stage_blocks (atom a, columns v .. v + EW - 1) into a
// [v][atoms] operand as one word store.  BF16: lanes l and l ^ 4 (atoms a and
// a ^ 1) swap one value, so that the lane of the even atom stores column v of
// both atoms and its partner column v + 1; the warp's 32 words fill the 32
// banks.  TF32: one element per word.  Called by all 32 lanes together.
template <bool TF32>
__device__ __forceinline__ void st_trans(uint8_t* base, int a, int v, const float (&t)[4 / tc::Elem<TF32>::ES],
                                         uint32_t sbo_, uint32_t lbo) {
  if constexpr (TF32) {
    tc::st_elem<true>(base, tc::core_off<true>(v, a, sbo_, lbo), t[0]);
  } else {
    const bool odd = a & 1;
    const float recv = __shfl_xor_sync(0xffffffffu, odd ? t[0] : t[1], 4);
    const float pair[2] = {odd ? recv : t[0], odd ? t[1] : recv};
    tc::st_word<false>(base, tc::core_off<false>(odd ? v + 1 : v, a & ~1, sbo_, lbo), pair);
  }
}

// The [v][atoms] operand from an [atoms][v] operand already in shared memory
// (same values, already rounded), in the blocks and lane roles of
// stage_blocks: each lane reads its word and, for BF16, swaps one half with
// lane l ^ 4 as st_trans does.  Called by all threads of the block.
template <bool TF32, int DPn>
__device__ __forceinline__ void transpose_blocks(const uint8_t* src, uint32_t sbo_src, uint32_t lbo_src, uint8_t* dst,
                                                 uint32_t sbo_dst, uint32_t lbo_dst) {
  constexpr int EPC = tc::Elem<TF32>::EPC, EW = 4 / tc::Elem<TF32>::ES, NVC = DPn / EPC;
  constexpr int PERW = (TA / 8) * NVC / (NTC / 32);
  const int lane = threadIdx.x & 31, b0 = (threadIdx.x >> 5) * PERW, ai = lane >> 2, w = lane & 3;
#pragma unroll 4
  for (int k = 0; k < PERW; ++k) {
    const int blk = b0 + k, a = 8 * (blk / NVC) + ai, v = EPC * (blk % NVC) + EW * w;
    const uint32_t word = *reinterpret_cast<const uint32_t*>(src + tc::core_off<TF32>(a, v, sbo_src, lbo_src));
    if constexpr (TF32) {
      *reinterpret_cast<uint32_t*>(dst + tc::core_off<true>(v, a, sbo_dst, lbo_dst)) = word;
    } else {
      // low half: column v, high half: column v + 1 (of atom a)
      const bool odd = a & 1;
      const uint32_t recv = __shfl_xor_sync(0xffffffffu, odd ? (word & 0xFFFFu) : (word >> 16), 4);
      const uint32_t out = odd ? (recv | (word & 0xFFFF0000u)) : ((word & 0xFFFFu) | (recv << 16));
      *reinterpret_cast<uint32_t*>(dst + tc::core_off<false>(odd ? v + 1 : v, a & ~1, sbo_dst, lbo_dst)) = out;
    }
  }
}

// tanh of the hidden layer: the hardware approximation (relative error about
// 2^-11, below the BF16 rounding of the operands it feeds) with BF16 operands,
// the full-precision function with TF32 operands.
template <bool TF32>
__device__ __forceinline__ float act_tanh(float x) {
  if constexpr (TF32) {
    return tanhf(x);
  } else {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
}

// Sums of v[0..15] over the 32 lanes of the warp by halving exchanges (16
// shuffles instead of 80): after the exchange over lane distance 16 >> s a
// lane keeps the half of its values whose index bit 3 - s matches its lane
// bit 4 - s.  The sum of v[i] ends in lanes 2i and 2i + 1.
__device__ __forceinline__ float warp_colsum16(float (&v)[16]) {
  const int ln = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int h = 8 >> s, o = 16 >> s;
    const bool up = (ln & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = up ? v[i] : v[i + h], keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Make this thread's generic-proxy shared-memory writes and TMEM reads
// ordered before an MMA that a thread issues after the barrier.
__device__ __forceinline__ void sync_for_mma() {
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
}

// Wait for the MMAs committed on `mbar` (phase `ph`); the outcome is made
// uniform across the block so that every thread leaves the tile loop together.
__device__ __forceinline__ bool wait_mma(uint64_t* mbar, uint32_t& ph, uint64_t limit_ns = kWaitNs) {
  const bool ok = tc::mbar_wait(mbar, ph, limit_ns);
  ph ^= 1u;
  tc::fence_after();
  return __syncthreads_and(ok) != 0;
}

// After a timed-out wait: give the MMAs in flight a second bounded wait before
// the tensor memory they write is released, and raise the error flag.
__device__ __forceinline__ void on_timeout(uint64_t* mbar, uint32_t ph, int* err, uint64_t limit_ns = kWaitNs) {
  tc::mbar_wait(mbar, ph ^ 1u, limit_ns);
  if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
}

// The failure path of the bounded waits, run on purpose: one block allocates
// tensor memory as the network kernels do, waits with a limit of limit_ns on
// an mbarrier that nothing arrives on, gives up, takes the second bounded
// wait, frees its tensor memory and raises TIMEOUT in the error flag.
__global__ void __launch_bounds__(NTC) k_wait_selftest(uint64_t limit_ns, int* __restrict__ err) {
  __shared__ uint64_t mbar;
  __shared__ uint32_t tbase;
  const int warp = threadIdx.x >> 5;
  if (warp == 0) tc::tmem_alloc(&tbase, 32);
  if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm = tbase;
  uint32_t ph = 0;
  const bool ok = wait_mma(&mbar, ph, limit_ns);  // no MMA was committed: this wait runs out
  if (!ok) on_timeout(&mbar, ph, err, limit_ns);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tm, 32);
}

}  // namespace

// Forward, persistent over 128-atom tiles: energies (D1.1), E' (D1.5) and the
// per-atom radial contraction chat_i[J][k] = sum_n E'_n c^R_nk^{IJ} used by
// the force sweep.  Thread t reads TMEM lane 32 (w % 4) + (t % 32) (its atom)
// and the 16-column chunks c = w / 4, w / 4 + 2, ... of each accumulator.
template <bool TF32, int D, int HPn, int NS, int NQR, int KR>
__global__ void __launch_bounds__(NTC, (Dims<TF32, D, HPn>::fwd_minb))
    k_mlp_fwd_tc(Tiles T, int ntiles, DevModel dm, const float* __restrict__ G, float* __restrict__ Ep,
                 float* __restrict__ Eatom, float* __restrict__ chat, int* __restrict__ err) {
  GNEP_PDL_WAIT();
  using Dm = Dims<TF32, D, HPn>;
  constexpr int DPn = Dm::DPn, OW = Dm::OW, NCZ = HPn / 16, NCE = DPn / 16, NJK = NS * KR;
  constexpr int EW = 4 / tc::Elem<TF32>::ES;  // operand elements per 4-byte word
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* RA = smem;
  uint8_t* W0 = RA + Dm::fRA;
  uint8_t* W0t = W0 + Dm::bW0;
  float* O = reinterpret_cast<float*>(W0t + Dm::bW0);  // [TA][OW] scaled E'
  __shared__ float b0s[HPn], w1s[HPn], sc[DPn], cR[NS * NQR * KR], Eh[2][TA];
  __shared__ int rows[TA];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, half = warp >> 2;
  const int arow = 32 * (warp & 3) + (tid & 31);
  if (warp == 0) tc::tmem_alloc(&tbase, Dm::fwd_cols);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  for (int v = tid; v < DPn; v += NTC) sc[v] = v < D ? dm.scale[v] : 0.f;
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm = tbase;
  const uint32_t lane = tm + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t cZ = 0, cE = HPn;  // TMEM columns of Z and E'
  uint32_t ph = 0;
  bool ok = true;
  int cur_e = -1;
  float b1 = 0.f;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int e, a0, na;
    tile_of(T, t, e, a0, na);
    if (e != cur_e) {
      stage_weights<TF32, D, HPn>(dm, e, W0, W0t, b0s, w1s);
      for (int q = tid; q < NS * NQR * KR; q += NTC) cR[q] = dm.params[dm.off_cR + e * NS * NQR * KR + q];
      b1 = dm.params[(size_t)e * dm.net_size + D * dm.H + 2 * dm.H];
      cur_e = e;
    }
    if (tid < TA) rows[tid] = tid < na ? T.perm[a0 + tid] : -1;
    __syncthreads();
    stage_blocks<TF32, D, DPn, 1>(G, nullptr, rows, [&](int a, int v, const auto& x) {
      float g[EW];
#pragma unroll
      for (int e = 0; e < EW; ++e) g[e] = sc[v + e] * x[0][e];
      tc::st_word<TF32>(RA, tc::core_off<TF32>(a, v, Dm::sG, Dm::LBO), g);
    });
    sync_for_mma();
    if (tid == 0) {
      tc::mma_chain<TF32>(tm + cZ, RA, Dm::sG, W0, Dm::sG, DPn, HPn, false, Dm::LBO);
      tc::commit(&mbar);
    }
    if (!(ok = wait_mma(&mbar, ph))) break;
    // x = tanh(z + b0), E = w1.x + b1, beta = w1 (1 - x^2) -> RA as [atoms][mu]
    float E = 0.f;
    for (int c = half; c < NCZ; c += 2) {
      float z[16], bt[16];
      tc::ld16(lane + cZ + 16 * c, z);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int mu = 16 * c + q;
        const float x = act_tanh<TF32>(z[q] + b0s[mu]);
        E = fmaf(w1s[mu], x, E);
        bt[q] = w1s[mu] * (1.f - x * x);
      }
#pragma unroll
      for (int q = 0; q < 16; q += tc::Elem<TF32>::EPC)
        tc::st_chunk<TF32>(RA, tc::core_off<TF32>(arow, 16 * c + q, Dm::sH, Dm::LBO), bt + q);
    }
    Eh[half][arow] = E;
    sync_for_mma();
    if (tid == 0) {
      tc::mma_chain<TF32>(tm + cE, RA, Dm::sH, W0t, Dm::sH, HPn, DPn, false, Dm::LBO);
      tc::commit(&mbar);
    }
    if (tid < TA) {
      const int r = rows[tid];
      if (r >= 0) Eatom[r] = (Eh[0][tid] + Eh[1][tid]) + b1;
    }
    if (!(ok = wait_mma(&mbar, ph))) break;
    for (int c = half; c < NCE; c += 2) {
      float v[16];
      tc::ld16(lane + cE + 16 * c, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int vv = 16 * c + q;
        if (vv < D) O[arow * OW + vv] = v[q] * sc[vv];
      }
    }
    tc::fence_before();
    __syncthreads();
    // coalesced row writes: E' and chat
    for (int q = tid; q < TA * D; q += NTC) {
      const int a = q / D, v = q % D, r = rows[a];
      if (r >= 0) Ep[(size_t)r * D + v] = O[a * OW + v];
    }
    for (int q = tid; q < TA * NJK; q += NTC) {
      const int a = q / NJK, jk = q % NJK, r = rows[a];
      if (r < 0) continue;
      const int J = jk / KR, k = jk % KR;
      float s = 0.f;
#pragma unroll
      for (int n = 0; n < NQR; ++n) s = fmaf(O[a * OW + n], cR[(J * NQR + n) * KR + k], s);
      chat[(size_t)r * NJK + jk] = s;
    }
    __syncthreads();  // rows, RA, O and the TMEM columns are rewritten by the next tile
    tc::fence_after();
  }
  if (!ok) on_timeout(&mbar, ph, err);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tm, Dm::fwd_cols);
}

// Tangent and reverse pass, persistent over 128-atom tiles, with e_i the
// energy residual weight of the atom's structure:
//   zdot = W0 (s.Gdot), beta = w1 (1 - x^2), alpha = e_i beta + 2 x beta zdot,
//   Gbar = s . (W0^T alpha),
//   dW0 += alpha (s.G)^T - beta (s.Gdot)^T, db0 += alpha,
//   dw1 += e_i x - (1 - x^2) zdot, db1 += e_i.
// One partial per block and species visited goes to part[block][species].
template <bool TF32, int D, int HPn>
__global__ void __launch_bounds__(NTC, (Dims<TF32, D, HPn>::bwd_minb))
    k_mlp_bwd_tc(Tiles T, int ntiles, DevModel dm, const int* __restrict__ atom_struct, const float* __restrict__ es,
                 const float* __restrict__ G, const float* __restrict__ Gd, float* __restrict__ Gb,
                 float* __restrict__ part, int part_stride, int* __restrict__ err) {
  GNEP_PDL_WAIT();
  using Dm = Dims<TF32, D, HPn>;
  constexpr int DPn = Dm::DPn, OW = Dm::OW, NCZ = HPn / 16, NCD = DPn / 16;
  constexpr int EW = 4 / tc::Elem<TF32>::ES;  // operand elements per 4-byte word
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* RA = smem;          // s.G | s.Gdot as [atoms][v]; then alpha as [atoms][mu]
  uint8_t* RG = RA + Dm::bRA;  // (s.G)^T with a row of ones at v = D, then (s.Gdot)^T, as [v][atoms]
  uint8_t* RT = RG + Dm::bGT;  // alpha^T, then the Gbar output tile, then -beta^T, as [mu][atoms]
  uint8_t* W0 = RT + Dm::bT;
  uint8_t* W0t = W0 + Dm::bW0;
  float* O = reinterpret_cast<float*>(RT);
  __shared__ float b0s[HPn], w1s[HPn], sc[DPn], wpart[4][HPn];
  __shared__ int rows[TA];
  __shared__ float cbp[4];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, ln = tid & 31, half = warp >> 2;
  const int arow = 32 * (warp & 3) + ln;
  const int H = dm.H;
  // rows HPn..127 of the [mu][atoms] operand must hold zeros whenever an MMA reads it
  auto zero_pad_rows = [&]() {
    for (uint32_t o = (uint32_t)(HPn / 8) * Dm::sA + 16u * tid; o < (uint32_t)Dm::bT; o += 16u * NTC)
      *reinterpret_cast<uint4*>(RT + o) = make_uint4(0u, 0u, 0u, 0u);
  };
  if (warp == 0) tc::tmem_alloc(&tbase, Dm::bwd_cols);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  for (int v = tid; v < DPn; v += NTC) sc[v] = v < D ? dm.scale[v] : 0.f;
  zero_pad_rows();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm = tbase;
  const uint32_t lane = tm + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t cZ = 0, cZd = HPn, cGb = 2 * HPn, cW = 2 * HPn + DPn;  // TMEM columns
  uint32_t ph = 0;
  bool ok = true, fresh = true;
  int cur_e = -1;
  float acc_w1 = 0.f, cb1 = 0.f;

  auto flush = [&](int e) {
    float* out = part + ((size_t)blockIdx.x * T.ns + e) * part_stride;
    const int mu = arow;
    for (int c = half; c < NCD; c += 2) {
      float v[16];
      tc::ld16(lane + cW + 16 * c, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int vv = 16 * c + q;
        if (mu < H) {
          if (vv < D)
            out[mu * D + vv] = v[q];
          else if (vv == D)
            out[D * H + mu] = v[q];  // db0 through the ones column
        }
      }
    }
    if (tid < H) out[D * H + H + tid] = acc_w1;
    if (tid == 0) out[D * H + 2 * H] = cb1;
  };

  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int e, a0, na;
    tile_of(T, t, e, a0, na);
    if (e != cur_e) {
      if (cur_e >= 0) flush(cur_e);
      stage_weights<TF32, D, HPn>(dm, e, W0, W0t, b0s, w1s);
      acc_w1 = 0.f;
      cb1 = 0.f;
      fresh = true;
      cur_e = e;
    }
    if (tid < TA) rows[tid] = tid < na ? T.perm[a0 + tid] : -1;
    __syncthreads();
    // e_i of this thread's atom: the structure index is fetched beside the
    // staging loads and the weight during the first products
    const int s_a = rows[arow] >= 0 ? atom_struct[rows[arow]] : -1;
    stage_blocks<TF32, D, DPn, 2>(G, Gd, rows, [&](int a, int v, const auto& x) {
      float g[EW], gd[EW], gt[EW];
#pragma unroll
      for (int e = 0; e < EW; ++e) {
        g[e] = sc[v + e] * x[0][e];
        gd[e] = sc[v + e] * x[1][e];
        gt[e] = v + e == D ? (rows[a] >= 0 ? 1.f : 0.f) : g[e];
      }
      const uint32_t o = tc::core_off<TF32>(a, v, Dm::sG, Dm::LBO);
      tc::st_word<TF32>(RA, o, g);
      tc::st_word<TF32>(RA + Dm::bG, o, gd);
      st_trans<TF32>(RG, a, v, gt, Dm::sA, Dm::LBOT);
    });
    const float ea = s_a >= 0 ? es[s_a] : 0.f;
    sync_for_mma();
    if (tid == 0) {
      tc::mma_chain<TF32>(tm + cZ, RA, Dm::sG, W0, Dm::sG, DPn, HPn, false, Dm::LBO);
      tc::mma_chain<TF32>(tm + cZd, RA + Dm::bG, Dm::sG, W0, Dm::sG, DPn, HPn, false, Dm::LBO);
      tc::commit(&mbar);
    }
    if (!(ok = wait_mma(&mbar, ph))) break;
    // alpha -> RA ([atoms][mu]) and RT ([mu][atoms]); column sums of e x - (1 - x^2) zdot
    if (half == 0) {  // the tile's sum of e_i, for db1
      float se = ea;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
      if (ln == 0) cbp[warp] = se;
    }
    for (int c = half; c < NCZ; c += 2) {
      float z[16], zd[16], al[16], q1[16];
      tc::ld16(lane + cZ + 16 * c, z);
      tc::ld16(lane + cZd + 16 * c, zd);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int mu = 16 * c + q;
        const float x = act_tanh<TF32>(z[q] + b0s[mu]);
        const float t1 = 1.f - x * x;
        const float beta = w1s[mu] * t1;
        al[q] = ea * beta + 2.f * x * beta * zd[q];
        q1[q] = ea * x - t1 * zd[q];  // zero for padded atoms (e = 0, zdot = 0)
        tc::st_elem<TF32>(RT, tc::core_off<TF32>(mu, arow, Dm::sA, Dm::LBOT), al[q]);
      }
      const float q1s = warp_colsum16(q1);
      if ((ln & 1) == 0) wpart[warp & 3][16 * c + (ln >> 1)] = q1s;
#pragma unroll
      for (int q = 0; q < 16; q += tc::Elem<TF32>::EPC)
        tc::st_chunk<TF32>(RA, tc::core_off<TF32>(arow, 16 * c + q, Dm::sH, Dm::LBO), al + q);
    }
    sync_for_mma();
    if (tid < HPn) acc_w1 += ((wpart[0][tid] + wpart[1][tid]) + wpart[2][tid]) + wpart[3][tid];
    if (tid == 0) cb1 += ((cbp[0] + cbp[1]) + cbp[2]) + cbp[3];
    if (tid == 0) {
      tc::mma_chain<TF32>(tm + cGb, RA, Dm::sH, W0t, Dm::sH, HPn, DPn, false, Dm::LBO);
      tc::mma_chain<TF32>(tm + cW, RT, Dm::sA, RG, Dm::sA, TA, DPn, !fresh, Dm::LBOT);
      tc::commit(&mbar);
    }
    if (!(ok = wait_mma(&mbar, ph))) break;
    // Gbar -> output tile in RT -> coalesced rows of Gb
    for (int c = half; c < NCD; c += 2) {
      float v[16];
      tc::ld16(lane + cGb + 16 * c, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int vv = 16 * c + q;
        if (vv < D) O[arow * OW + vv] = v[q] * sc[vv];
      }
    }
    __syncthreads();
    for (int q = tid; q < TA * D; q += NTC) {
      const int a = q / D, v = q % D, r = rows[a];
      if (r >= 0) Gb[(size_t)r * D + v] = O[a * OW + v];
    }
    __syncthreads();
    // -beta -> RT ([mu][atoms]); (s.Gdot)^T -> RG
    for (int c = half; c < NCZ; c += 2) {
      float z[16];
      tc::ld16(lane + cZ + 16 * c, z);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int mu = 16 * c + q;
        const float x = act_tanh<TF32>(z[q] + b0s[mu]);
        tc::st_elem<TF32>(RT, tc::core_off<TF32>(mu, arow, Dm::sA, Dm::LBOT), -w1s[mu] * (1.f - x * x));
      }
    }
    zero_pad_rows();
    if constexpr (Dm::bH <= Dm::bG) {
      // s.Gdot is still in RA behind the alpha operand
      transpose_blocks<TF32, DPn>(RA + Dm::bG, Dm::sG, Dm::LBO, RG, Dm::sA, Dm::LBOT);
    } else {
      stage_blocks<TF32, D, DPn, 1>(Gd, nullptr, rows, [&](int a, int v, const auto& x) {
        float gt[EW];
#pragma unroll
        for (int e = 0; e < EW; ++e) gt[e] = sc[v + e] * x[0][e];
        st_trans<TF32>(RG, a, v, gt, Dm::sA, Dm::LBOT);
      });
    }
    sync_for_mma();
    if (tid == 0) {
      tc::mma_chain<TF32>(tm + cW, RT, Dm::sA, RG, Dm::sA, TA, DPn, true, Dm::LBOT);
      tc::commit(&mbar);
    }
    if (!(ok = wait_mma(&mbar, ph))) break;
    fresh = false;
  }
  if (ok && cur_e >= 0) flush(cur_e);
  if (!ok) on_timeout(&mbar, ph, err);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tm, Dm::bwd_cols);
}

// ------------------------------------------------------------- launchers

namespace {

// Dynamic shared memory for a kernel that allocates `cols` TMEM columns: at
// least `need`, and large enough that no more CTAs share an SM than its 512
// TMEM columns admit, so that an allocation never waits on another CTA.
int tc_smem(int need, int cols, int static_bytes) {
  const int cap = 512 / cols;
  const int floor_req = kSmemPerSm / (cap + 1) - 1024 - static_bytes + 16;
  return need > floor_req ? need : floor_req;
}

// Blocks per SM from the kernel's registers, shared memory and TMEM columns.
template <class K>
int tc_launch_shape(K kern, int need, int cols, int ntiles, int& smem, int& grid) {
  cudaFuncAttributes fa;
  GNEP_CUDA(cudaFuncGetAttributes(&fa, kern));
  smem = tc_smem(need, cols, (int)fa.sharedSizeBytes);
  int dev = 0, nsm = 0;
  GNEP_CUDA(cudaGetDevice(&dev));
  GNEP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
  const int by_regs = 65536 / (regs_warp * (NTC / 32));
  const int by_smem = kSmemPerSm / (smem + (int)fa.sharedSizeBytes + 1024);
  int occ = 512 / cols;
  if (by_regs < occ) occ = by_regs;
  if (by_smem < occ) occ = by_smem;
  if (occ < 1) return set_error(GNEP_ERR_CUDA, "tensor-core network kernel does not fit on an SM");
  grid = ntiles < nsm * occ ? ntiles : nsm * occ;
  return GNEP_OK;
}

template <class K>
int tc_set_smem(K kern, int need, int cols) {
  cudaFuncAttributes fa;
  GNEP_CUDA(cudaFuncGetAttributes(&fa, kern));
  GNEP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc_smem(need, cols, (int)fa.sharedSizeBytes)));
  GNEP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  return GNEP_OK;
}

}  // namespace

int wait_selftest(const gnep_model* m, uint64_t limit_ns, cudaStream_t st) {
  k_wait_selftest<<<1, NTC, 0, st>>>(limit_ns, m->err);
  GNEP_CHECK_LAUNCH("k_wait_selftest");
  return GNEP_OK;
}

template <bool TF32, int D, int HPn, int NS, int NQR, int KR>
int mlp_setup_tc() {
  using Dm = Dims<TF32, D, HPn>;
  int rc = tc_set_smem(k_mlp_fwd_tc<TF32, D, HPn, NS, NQR, KR>, Dm::fwd_smem, Dm::fwd_cols);
  if (!rc) rc = tc_set_smem(k_mlp_bwd_tc<TF32, D, HPn>, Dm::bwd_smem, Dm::bwd_cols);
  return rc;
}

template <bool TF32, int D, int HPn, int NS, int NQR, int KR>
int mlp_forward_tc(const gnep_model* m, gnep_nlist* nl, cudaStream_t st) {
  using Dm = Dims<TF32, D, HPn>;
  const Tiles T = make_tiles(nl, NS, TA);
  const int ntiles = T.tbase[NS];
  if (ntiles == 0) return GNEP_OK;
  Workspace& w = nl->ws;
  auto kern = k_mlp_fwd_tc<TF32, D, HPn, NS, NQR, KR>;
  int smem = 0, grid = 0;
  if (int rc = tc_launch_shape(kern, Dm::fwd_smem, Dm::fwd_cols, ntiles, smem, grid)) return rc;
  grid = net_blocks(nl, grid);
  (void)launch_pdl(kern, grid, NTC, smem, st, T, ntiles, m->dev(), w.G, w.Ep, w.Eatom, w.chat, m->err);
  GNEP_CHECK_LAUNCH("k_mlp_fwd_tc");
  return GNEP_OK;
}

template <bool TF32, int D, int HPn>
int mlp_backward_tc(const gnep_model* m, gnep_nlist* nl, cudaStream_t st) {
  using Dm = Dims<TF32, D, HPn>;
  const int ns = m->shape.ns;
  const Tiles T = make_tiles(nl, ns, TA);
  const int ntiles = T.tbase[ns];
  Workspace& w = nl->ws;
  auto kern = k_mlp_bwd_tc<TF32, D, HPn>;
  int smem = 0, grid = 1;
  if (ntiles > 0)
    if (int rc = tc_launch_shape(kern, Dm::bwd_smem, Dm::bwd_cols, ntiles, smem, grid)) return rc;
  if (grid > kNetBlocks) grid = kNetBlocks;  // net_part holds kNetBlocks partials
  grid = net_blocks(nl, grid);
  w.net_blocks = grid;
  GNEP_CUDA(cudaMemsetAsync(w.net_part, 0, sizeof(float) * (size_t)grid * ns * m->net_size, st));
  if (ntiles == 0) return GNEP_OK;
  (void)launch_pdl(kern, grid, NTC, smem, st, T, ntiles, m->dev(), nl->atom_struct, w.es, w.G, w.Gd, w.Gb, w.net_part,
                                m->net_size, m->err);
  GNEP_CHECK_LAUNCH("k_mlp_bwd_tc");
  return GNEP_OK;
}

#define GNEP_NET_TC1(TF, D, HPN, NQR, KR)                                                               \
  template int mlp_setup_tc<TF, D, HPN, 2, NQR, KR>();                                                 \
  template int mlp_forward_tc<TF, D, HPN, 2, NQR, KR>(const gnep_model*, gnep_nlist*, cudaStream_t);   \
  template int mlp_backward_tc<TF, D, HPN>(const gnep_model*, gnep_nlist*, cudaStream_t);
#define GNEP_NET_TC(D, NQR, KR)            \
  GNEP_NET_TC1(false, D, 32, NQR, KR)      \
  GNEP_NET_TC1(false, D, 64, NQR, KR)      \
  GNEP_NET_TC1(false, D, 112, NQR, KR)     \
  GNEP_NET_TC1(true, D, 32, NQR, KR)       \
  GNEP_NET_TC1(true, D, 64, NQR, KR)       \
  GNEP_NET_TC1(true, D, 112, NQR, KR)
GNEP_NET_TC(25, 5, 9)
GNEP_NET_TC(54, 9, 13)
GNEP_NET_TC(45, 9, 13)
#undef GNEP_NET_TC
#undef GNEP_NET_TC1

}  // namespace gnep
