// Loss (Eqs. 9-12), residual weights, parameter-gradient reductions
// (Eqs. 13-16, D1.18-D1.21), Adam with the Eq. 17 schedule, descriptor scale
// and the species-grouped atom order.  Every cross-atom sum runs in a fixed
// order, so a step is bit-reproducible: FP32 leaves, FP64 above them (the
// per-structure sums combine a warp's lanes as exact FP32 pairs first).
#include <cmath>

#include "gnep_internal.h"
#include "network.cuh"

namespace gnep {


namespace {

// Block sums of K values per thread, in a fixed order (xor butterflies within
// warps, then warps in order); the sums are valid in threads 0..K-1 (thread k
// holds sum k).  sh holds 32 K doubles.
template <int K>
__device__ __forceinline__ double block_sums(double (&v)[K], double* sh) {
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[warp * K + k] = v[k];
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < K)
    for (int w = 0; w < nw; ++w) r += sh[w * K + threadIdx.x];
  return r;
}

// Sums carried as FP32 pairs hi + lo without rounding error in the additions
// (Knuth's TwoSum for the sum of the high parts and again to renormalise), so
// that a warp's cross-atom sums keep about 44 significant bits on the FP32
// pipes; FP64 is used only above the warps.
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  const float s = a.hi + b.hi, bs = s - a.hi;
  const float e = (a.hi - (s - bs)) + (b.hi - bs);  // s + e = a.hi + b.hi exactly
  const float t = e + (a.lo + b.lo);
  const float h = s + t, bh = h - s;
  return {h, (s - (h - bh)) + (t - bh)};  // h + lo = s + t exactly
}
// The sum over the warp's 32 lanes (xor butterflies; every lane gets a sum).
__device__ __forceinline__ F2 f2_warp_sum(F2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const F2 w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = f2_add(v, w);
  }
  return v;
}

struct LossArgs {
  int N, S;
  double le, lf, lv, l2;
  int form;
  int64_t n_params;
  double inv_S, inv_3N, inv_6S, inv_np;  // reciprocal normalisers (0 for empty sets), formed on the host
};

// Loss terms and the scalar weights of the residuals, by one block:
// coef[0..3] = {L, L_e, L_f, L_v}; coef[4] = cf, coef[5] = ce, coef[6] = cv with
//   a_i = cf (F_i - F_i^tar),  e_s = ce (E_s/N_s - E_s^tar)/N_s,
//   B_s = cv (W_s/N_s - V_s^tar)/N_s  (off-diagonals halved).
__device__ void loss_final_block(const LossArgs& a, int nred, const double* __restrict__ red,
                                 const float* __restrict__ params, double* __restrict__ coef, int* __restrict__ err) {
  __shared__ double sh[32 * 4];
  __shared__ double tot[4];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nred; b += blockDim.x) {
    v[0] += red[3 * b];
    v[1] += red[3 * b + 1];
    v[2] += red[3 * b + 2];
  }
  if (a.l2 != 0.0)
    for (int64_t q = threadIdx.x; q < a.n_params; q += blockDim.x) v[3] += (double)params[q] * params[q];
  const double r = block_sums<4>(v, sh);
  if (threadIdx.x < 4) tot[threadIdx.x] = r;
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double se = tot[0], sf = tot[1], sv = tot[2], l2 = tot[3];
  const double Le = se * a.inv_S;   // Eq. 10
  const double Lf = sf * a.inv_3N;  // Eq. 11
  const double Lv = sv * a.inv_6S;  // Eq. 12
  const double reg = a.l2 * l2 * a.inv_np;
  double L, ke = 1, kf = 1, kv = 1;
  if (a.form == GNEP_LOSS_RMSE) {
    L = a.le * sqrt(Le) + a.lf * sqrt(Lf) + a.lv * sqrt(Lv) + reg;
    ke = Le > 0 ? 0.5 / sqrt(Le) : 0.0;
    kf = Lf > 0 ? 0.5 / sqrt(Lf) : 0.0;
    kv = Lv > 0 ? 0.5 / sqrt(Lv) : 0.0;
  } else {
    L = a.le * Le + a.lf * Lf + a.lv * Lv + reg;  // Eq. 9
  }
  coef[0] = L;
  coef[1] = Le;
  coef[2] = Lf;
  coef[3] = Lv;
  coef[4] = 2.0 * a.lf * kf * a.inv_3N;  // Eq. 15
  coef[5] = 2.0 * a.le * ke * a.inv_S;   // Eq. 14
  coef[6] = 2.0 * a.lv * kv * a.inv_6S;  // Eq. 16
  if (!isfinite(L)) atomicOr(err, kErrNonFinite);
}

__global__ void __launch_bounds__(256) k_loss_final(LossArgs a, int nred, const double* __restrict__ red,
                                                    const float* __restrict__ params, double* __restrict__ coef,
                                                    int* __restrict__ err) {
  GNEP_PDL_WAIT();
  loss_final_block(a, nred, red, params, coef, err);
}

// Per structure s (one block of 128 threads): the sums E_s and W_s (Eqs. 1, 4)
// and the structure's squared residuals of Eqs. 10-12 (energy, virial, and the
// force term over its atoms), and the residuals divided by N_s for the weights
// of the loss gradient: rn[7 s] = (E_s/N_s - E_s^tar)/N_s, rn[7 s + 1 + c] =
// (W_sc/N_s - V_sc^tar)/N_s.  Each thread sums its few atoms in FP32, the
// warps combine their lanes as FP32 pairs (F2) and the four warp sums are
// added in FP64 in order.  The last block to finish (counted in *done, which
// it resets) forms the loss terms from all blocks' residuals in structure
// order.  In the MSE form the residual weights cf, ce, cv are constants
// (Eqs. 14-16 without the RMSE chain factor), so each block also writes the
// residual weights a_i, e_s and B_s of its structure (what k_residuals forms
// otherwise, with the same arithmetic).
__global__ void __launch_bounds__(128) k_struct_loss(const int* __restrict__ soff, const float* __restrict__ Eatom,
                                                     const float* __restrict__ Wat, const float* __restrict__ F,
                                                     const double* __restrict__ le, const float* __restrict__ lf,
                                                     const double* __restrict__ lv, double* __restrict__ Es,
                                                     double* __restrict__ Ws, double* __restrict__ red,
                                                     double* __restrict__ rn, LossArgs la,
                                                     const float* __restrict__ params, double* __restrict__ coef,
                                                     int* __restrict__ err, int* __restrict__ done,
                                                     float4* __restrict__ aw, float* __restrict__ es,
                                                     float* __restrict__ Bs) {
  GNEP_PDL_WAIT();
  const int s = blockIdx.x;
  const int a0 = soff[s], a1 = soff[s + 1];
  const bool fused = la.form != GNEP_LOSS_RMSE;
  const float cf = (float)(2.0 * la.lf * la.inv_3N);  // coef[4] of the MSE form
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int i = a0 + threadIdx.x; i < a1; i += blockDim.x) {
    acc[0] += Eatom[i];
#pragma unroll
    for (int q = 0; q < 6; ++q) acc[1 + q] += Wat[6 * (size_t)i + q];
    float d[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      d[c] = F[3 * (size_t)i + c] - lf[3 * (size_t)i + c];
      acc[7] = fmaf(d[c], d[c], acc[7]);
    }
    if (fused) aw[i] = make_float4(cf * d[0], cf * d[1], cf * d[2], 0.f);
  }
  __shared__ float2 wsum[4][8];
  __shared__ double tot[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const F2 v = f2_warp_sum(F2{acc[q], 0.f});
    if (lane == 0) wsum[warp][q] = make_float2(v.hi, v.lo);
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 4; ++w) t += (double)wsum[w][threadIdx.x].x + (double)wsum[w][threadIdx.x].y;
    tot[threadIdx.x] = t;
  }
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) {
    const double inv = 1.0 / (double)(a1 - a0);
    const double E = tot[0];
    Es[s] = E;
    const double de = E * inv - le[s];
    rn[7 * s] = de * inv;
    double sv = 0.0;
    for (int c = 0; c < 6; ++c) {
      const double w = tot[1 + c];
      Ws[6 * s + c] = w;
      const double dv = w * inv - lv[6 * s + c];
      rn[7 * s + 1 + c] = dv * inv;
      sv += dv * dv;
    }
    red[3 * s] = de * de;
    red[3 * s + 1] = tot[7];
    red[3 * s + 2] = sv;
    if (fused) {  // coef[5], coef[6] of the MSE form times the residuals over N_s
      es[s] = (float)(2.0 * la.le * la.inv_S * rn[7 * s]);
      for (int c = 0; c < 6; ++c) {
        const double g = 2.0 * la.lv * la.inv_6S * rn[7 * s + 1 + c];
        Bs[6 * s + c] = (float)(c < 3 ? g : 0.5 * g);
      }
    }
    __threadfence();
    last = atomicAdd(done, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  loss_final_block(la, (int)gridDim.x, red, params, coef, err);
  if (threadIdx.x == 0) *done = 0;
}

// Residual weights of the loss gradient: a_i for atoms i < N, then e_s and
// B_s (off-diagonals halved) for structures s = i - N (Eqs. 14-16), from the
// structures' residuals divided by N_s (rn) that the loss kernel left.
__global__ void k_residuals(int N, int S, const float* __restrict__ F, const float* __restrict__ lf,
                            const double* __restrict__ rn, const double* __restrict__ coef, float4* __restrict__ a,
                            float* __restrict__ es, float* __restrict__ Bs) {
  GNEP_PDL_WAIT();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    const float cf = (float)coef[4];
    a[i] = make_float4(cf * (F[3 * i] - lf[3 * i]), cf * (F[3 * i + 1] - lf[3 * i + 1]),
                       cf * (F[3 * i + 2] - lf[3 * i + 2]), 0.f);
    return;
  }
  const int s = i - N;
  if (s >= S) return;
  es[s] = (float)(coef[5] * rn[7 * s]);
  for (int c = 0; c < 6; ++c) {
    const double g = coef[6] * rn[7 * s + 1 + c];
    Bs[6 * s + c] = (float)(c < 3 ? g : 0.5 * g);
  }
}

// ---------------------------------------------------------- gradient sums

// grad[q] = sum over block partials + 2 lambda_l2 theta_q / N_par; network
// parameters come from the network backward pass (net_part), the coefficients
// from the c-gradient sweeps (cpart).  A block takes 32
// consecutive parameters (coalesced rows) and 32 subsets of the partial rows:
// each thread sums its rows in FP32 (at most a few dozen leaves, eight loads
// in flight), the 32 subset sums of a parameter are combined in FP64 in a
// fixed order.
constexpr int kGfCols = 32, kGfRows = 32;

// The block's part of the gradient: returns grad[q] (also written) on the
// threads of row 0 for their column q < n_params, and 0 elsewhere.  `params`
// is read for the L2 term only.
__device__ __forceinline__ double grad_block(const DevModel& dm, int ns, int nb_net, int nb_cg,
                                             const float* __restrict__ net_part, const float* __restrict__ cpart,
                                             double l2coef, const float* params, double* __restrict__ grad) {
  __shared__ double sh[kGfRows][kGfCols];
  const int tx = threadIdx.x % kGfCols, ty = threadIdx.x / kGfCols;
  const int64_t q = (int64_t)blockIdx.x * kGfCols + tx;
  const int64_t nnet = (int64_t)ns * dm.net_size;
  float leaf = 0.f;
  if (q < dm.n_params) {
    const float* src;
    int64_t stride;
    int nb;
    if (q < nnet) {  // net_part[b][e][l] = row b, column q
      src = net_part + q;
      stride = nnet;
      nb = nb_net;
    } else {
      stride = dm.n_params - nnet;
      src = cpart + (q - dm.off_cR);
      nb = nb_cg;
    }
#pragma unroll 8
    for (int b = ty; b < nb; b += kGfRows) leaf += src[(size_t)b * stride];
  }
  sh[ty][tx] = (double)leaf;
  __syncthreads();
  double t = 0.0;
  if (ty == 0 && q < dm.n_params) {
#pragma unroll
    for (int k = 0; k < kGfRows; ++k) t += sh[k][tx];
    t += l2coef * (double)params[q];
    grad[q] = t;
  }
  return t;
}

__global__ void __launch_bounds__(kGfCols* kGfRows) k_grad_final(DevModel dm, int ns, int nb_net, int nb_cg,
                                                                 const float* __restrict__ net_part,
                                                                 const float* __restrict__ cpart, double l2coef,
                                                                 double* __restrict__ grad) {
  GNEP_PDL_WAIT();
  (void)grad_block(dm, ns, nb_net, nb_cg, net_part, cpart, l2coef, dm.params, grad);
}

// ---------------------------------------------------------- Adam, Eq. 17

struct AdamArgs {
  float lr, b1, b2, eps, wd;
  float lb1, lb2;  // log(beta1), log(beta2), formed on the host in double
  int scheduled;
  float lr_start, lr_stop;
  long long nw, nt;
};

// Eq. 17: linear warm-up from lr_stop to lr_start over nw steps, then a cosine
// decay back to lr_stop at step nt.
__device__ float lr_eq17(const AdamArgs& a, long long s) {
  if (s < a.nw) return a.lr_stop + (float)s / (float)a.nw * (a.lr_start - a.lr_stop);
  if (s > a.nt) s = a.nt;
  const long long span = a.nt - a.nw;
  const float frac = span > 0 ? (float)(s - a.nw) / (float)span : 1.f;
  return a.lr_stop + (a.lr_start - a.lr_stop) * 0.5f * (1.f + cospif(frac));
}

// Adam (Kingma-Ba bias correction, optional decoupled weight decay) with the
// step size of Eq. 17 when scheduled, in FP32 (moments are FP32).  The bias
// corrections 1 - beta^t are formed as -expm1(t log beta), accurate also when
// beta^t is close to 1.  adam_rates gives the step size and the two inverse
// corrections of update s + 1; adam_entry updates one parameter.
struct AdamRates {
  float lr, ic1, ic2;
};
__device__ __forceinline__ AdamRates adam_rates(const AdamArgs& a, long long s) {
  const float tf = (float)(s + 1);
  AdamRates r;
  r.lr = a.scheduled ? lr_eq17(a, s) : a.lr;
  r.ic1 = -1.f / expm1f(tf * a.lb1);
  r.ic2 = -1.f / expm1f(tf * a.lb2);
  return r;
}
__device__ __forceinline__ void adam_entry(int64_t q, float gq, float* p, float* __restrict__ m,
                                           float* __restrict__ v, const AdamArgs& a, const AdamRates& r) {
  const float mq = fmaf(a.b1, m[q], (1.f - a.b1) * gq);
  const float vq = fmaf(a.b2, v[q], (1.f - a.b2) * gq * gq);
  m[q] = mq;
  v[q] = vq;
  const float upd = (mq * r.ic1) / (sqrtf(vq * r.ic2) + a.eps) + a.wd * p[q];
  p[q] = p[q] - r.lr * upd;
}
// The last block to finish advances the update count (every block read it
// before its own arrival).
__device__ __forceinline__ void adam_count(long long* step, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(err + 1, 1) == (int)gridDim.x - 1) {
      *step += 1;
      err[1] = 0;
    }
  }
}

__global__ void k_adam(int64_t n, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const double* __restrict__ g, long long* __restrict__ step, int* __restrict__ err,
                       AdamArgs a) {
  GNEP_PDL_WAIT();
  if (*err & kErrNonFinite) return;  // the step is skipped (uniform over the grid)
  const AdamRates r = adam_rates(a, *step);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    adam_entry(q, (float)g[q], p, m, v, a, r);
  adam_count(step, err);
}

// The end of a captured training step in one kernel: the gradient of
// k_grad_final, the loss terms copied to loss_out (may be NULL), and then,
// unless the loss was not finite, the Adam update of k_adam on the same
// entries with the same arithmetic.
__global__ void __launch_bounds__(kGfCols* kGfRows) k_grad_adam(DevModel dm, int ns, int nb_net, int nb_cg,
                                                                const float* __restrict__ net_part,
                                                                const float* __restrict__ cpart, double l2coef,
                                                                double* __restrict__ grad, float* p, float* __restrict__ m,
                                                                float* __restrict__ v, long long* __restrict__ step,
                                                                int* __restrict__ err, AdamArgs a,
                                                                const double* __restrict__ coef,
                                                                double* __restrict__ loss_out) {
  GNEP_PDL_WAIT();
  const double gq = grad_block(dm, ns, nb_net, nb_cg, net_part, cpart, l2coef, p, grad);
  if (loss_out && blockIdx.x == 0 && threadIdx.x < 4) loss_out[threadIdx.x] = coef[threadIdx.x];
  if (*err & kErrNonFinite) return;  // the update is skipped (uniform over the grid)
  const AdamRates r = adam_rates(a, *step);
  const int64_t q = (int64_t)blockIdx.x * kGfCols + threadIdx.x;
  if (threadIdx.x < kGfCols && q < dm.n_params) adam_entry(q, (float)gq, p, m, v, a, r);
  adam_count(step, err);
}

// ---------------------------------------------------------- scale, perm

__global__ void __launch_bounds__(256) k_scale(int N, int ndes, const float* __restrict__ G, float* __restrict__ scale) {
  __shared__ float smin[256], smax[256];
  const int v = blockIdx.x;
  float lo = INFINITY, hi = -INFINITY;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float g = G[(size_t)i * ndes + v];
    lo = fminf(lo, g);
    hi = fmaxf(hi, g);
  }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      smin[threadIdx.x] = fminf(smin[threadIdx.x], smin[threadIdx.x + o]);
      smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float span = smax[0] - smin[0];
    scale[v] = span > 0.f ? 1.f / span : 1.f;
  }
}

// Stable grouping of atoms by species: perm = atoms of species 0 in order,
// then 1, ...  Three steps over blocks of 1024 atoms: per-block species counts;
// block offsets (one small block, exclusive scan in block order); scatter with
// ranks inside the block from warp ballots.
constexpr int kPermBlock = 1024;

__global__ void __launch_bounds__(kPermBlock) k_species_count(int N, int ns, const int* __restrict__ type,
                                                              int* __restrict__ bcount) {
  __shared__ int c[8];
  if (threadIdx.x < 8) c[threadIdx.x] = 0;
  __syncthreads();
  const int i = blockIdx.x * kPermBlock + threadIdx.x;
  const int t = i < N ? type[i] : -1;
  for (int e = 0; e < ns; ++e) {
    const unsigned b = __ballot_sync(0xffffffffu, t == e);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(&c[e], __popc(b));  // integer: order-free
  }
  __syncthreads();
  if (threadIdx.x < ns) bcount[(size_t)blockIdx.x * ns + threadIdx.x] = c[threadIdx.x];
}

// bcount[b][e] -> exclusive offsets boff[b][e] of the grouped order; soff[e] = species starts.
__global__ void __launch_bounds__(256) k_species_offsets(int nb, int ns, const int* __restrict__ bcount,
                                                         int* __restrict__ boff, int* __restrict__ soff) {
  if (threadIdx.x != 0) return;
  int base = 0;
  for (int e = 0; e < ns; ++e) {
    soff[e] = base;
    for (int b = 0; b < nb; ++b) {
      boff[(size_t)b * ns + e] = base;
      base += bcount[(size_t)b * ns + e];
    }
  }
  soff[ns] = base;
}

__global__ void __launch_bounds__(kPermBlock) k_species_scatter(int N, int ns, const int* __restrict__ type,
                                                                const int* __restrict__ boff, int* __restrict__ perm) {
  __shared__ int wc[8][kPermBlock / 32];
  const int i = blockIdx.x * kPermBlock + threadIdx.x;
  const int t = i < N ? type[i] : -1;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  unsigned mine = 0;
  for (int e = 0; e < ns; ++e) {
    const unsigned b = __ballot_sync(0xffffffffu, t == e);
    if (lane == 0) wc[e][w] = __popc(b);
    if (t == e) mine = b;
  }
  __syncthreads();
  if (t < 0) return;
  int r = __popc(mine & lt);
  for (int k = 0; k < w; ++k) r += wc[t][k];
  perm[boff[(size_t)blockIdx.x * ns + t] + r] = i;
}

}  // namespace

// Loss partials per structure: three squared residuals and seven residuals divided by N_s.
int64_t loss_partial_doubles(int n_struct) { return 10LL * (n_struct > 0 ? n_struct : 1); }

int run_species_perm(gnep_nlist* nl, cudaStream_t st) {
  int* soff_dev = nullptr;
  GNEP_CUDA(cudaMallocAsync(&soff_dev, sizeof(int) * 9, st));
  const int N = nl->n_atoms, ns = nl->shape.ns, nb = (N + kPermBlock - 1) / kPermBlock;
  int* tmp = nullptr;
  GNEP_CUDA(cudaMallocAsync(&tmp, sizeof(int) * 2 * (size_t)(nb > 0 ? nb : 1) * ns, st));
  if (nb > 0) {
    k_species_count<<<nb, kPermBlock, 0, st>>>(N, ns, nl->type, tmp);
    k_species_offsets<<<1, 32, 0, st>>>(nb, ns, tmp, tmp + (size_t)nb * ns, soff_dev);
    k_species_scatter<<<nb, kPermBlock, 0, st>>>(N, ns, nl->type, tmp + (size_t)nb * ns, nl->perm);
  } else {
    GNEP_CUDA(cudaMemsetAsync(soff_dev, 0, sizeof(int) * 9, st));
  }
  GNEP_CHECK_LAUNCH("species grouping");
  GNEP_CUDA(cudaFreeAsync(tmp, st));
  GNEP_CUDA(cudaMemcpyAsync(nl->species_off, soff_dev, sizeof(int) * (nl->shape.ns + 1), cudaMemcpyDeviceToHost, st));
  GNEP_CUDA(cudaFreeAsync(soff_dev, st));
  GNEP_CUDA(cudaStreamSynchronize(st));
  return GNEP_OK;
}

int run_loss_impl(const gnep_model* m, gnep_nlist* nl, const double* le, const float* lf, const double* lv,
                  const gnep_labels* y, cudaStream_t st) {
  Workspace& w = nl->ws;
  const int N = nl->n_atoms, S = nl->n_struct;
  LossArgs a;
  a.N = N; a.S = S; a.le = y->lambda_e; a.lf = y->lambda_f; a.lv = y->lambda_v; a.l2 = y->lambda_l2;
  a.form = y->loss_form; a.n_params = m->n_params;
  a.inv_S = S > 0 ? 1.0 / S : 0.0;
  a.inv_3N = N > 0 ? 1.0 / (3.0 * N) : 0.0;
  a.inv_6S = S > 0 ? 1.0 / (6.0 * S) : 0.0;
  a.inv_np = 1.0 / (double)m->n_params;
  if (S > 0) {  // per-structure residuals; the last block forms the loss terms
    (void)launch_pdl(k_struct_loss, S, 128, 0, st, nl->struct_off, w.Eatom, w.Wat, w.F, le, lf, lv, w.Es, w.Ws, w.red,
                                     w.red + 3 * (size_t)S, a, m->params, w.coef, m->err, m->err + 2, w.a, w.es,
                                     w.Bs);
  } else {
    (void)launch_pdl(k_loss_final, 1, 256, 0, st, a, 0, w.red, m->params, w.coef, m->err);
  }
  stage("struct_loss");
  if (N + S > 0 && (S == 0 || a.form == GNEP_LOSS_RMSE)) {  // the loss kernel wrote them in the MSE form
    (void)launch_pdl(k_residuals, blocks_for(N + S, 256), 256, 0, st, N, S, w.F, lf, w.red + 3 * (size_t)S, w.coef, w.a, w.es,
                                                         w.Bs);
    stage("residuals");
  }
  GNEP_CHECK_LAUNCH("loss");
  return GNEP_OK;
}

int run_grad_reduce_impl(const gnep_model* m, gnep_nlist* nl, double lambda_l2, cudaStream_t st) {
  const DevModel dm = m->dev();
  const int ns = m->shape.ns;
  const int nb_net = nl->ws.net_blocks;
  const int nb_cg = nl->n_atoms > 0 ? cgrad_blocks(nl) : 0;
  const double l2coef = 2.0 * lambda_l2 / (double)m->n_params;
  (void)launch_pdl(k_grad_final, blocks_for(m->n_params, kGfCols), kGfCols * kGfRows, 0, st, dm, ns, nb_net, nb_cg, nl->ws.net_part,
                                                                              nl->ws.cpart, l2coef, m->grad);
  stage("grad_final");
  GNEP_CHECK_LAUNCH("gradient reduction");
  return GNEP_OK;
}

static int adam_args(double lr, double b1, double b2, double eps, double wd, bool scheduled, double lr_start,
                     double lr_stop, int64_t nw, int64_t nt, AdamArgs* a) {
  if (!(b1 > 0.0 && b1 < 1.0 && b2 > 0.0 && b2 < 1.0 && eps > 0.0))
    return set_error(GNEP_ERR_INVALID_ARG, "Adam needs 0 < beta1, beta2 < 1 and eps > 0");
  a->lr = (float)lr; a->b1 = (float)b1; a->b2 = (float)b2; a->eps = (float)eps; a->wd = (float)wd;
  a->lb1 = (float)std::log(b1); a->lb2 = (float)std::log(b2);
  a->scheduled = scheduled ? 1 : 0;
  a->lr_start = (float)lr_start; a->lr_stop = (float)lr_stop; a->nw = nw; a->nt = nt;
  return GNEP_OK;
}

int run_adam(gnep_model* m, const double*, double lr, double b1, double b2, double eps, double wd, bool scheduled,
             double lr_start, double lr_stop, int64_t nw, int64_t nt, cudaStream_t st) {
  AdamArgs a;
  if (int rc = adam_args(lr, b1, b2, eps, wd, scheduled, lr_start, lr_stop, nw, nt, &a)) return rc;
  const int nb = blocks_for(m->n_params, 256);
  (void)launch_pdl(k_adam, nb < 1 ? 1 : nb, 256, 0, st, m->n_params, m->params, m->adam_m, m->adam_v, m->grad, m->step, m->err, a);
  stage("adam");
  GNEP_CHECK_LAUNCH("adam");
  return GNEP_OK;
}

int run_grad_adam(gnep_model* m, gnep_nlist* nl, double lambda_l2, double* loss_out, double b1, double b2,
                  double eps, double wd, double lr_start, double lr_stop, int64_t nw, int64_t nt, cudaStream_t st) {
  AdamArgs a;
  if (int rc = adam_args(0.0, b1, b2, eps, wd, true, lr_start, lr_stop, nw, nt, &a)) return rc;
  const DevModel dm = m->dev();
  const int nb_cg = nl->n_atoms > 0 ? cgrad_blocks(nl) : 0;
  const double l2coef = 2.0 * lambda_l2 / (double)m->n_params;
  (void)launch_pdl(k_grad_adam, blocks_for(m->n_params, kGfCols), kGfCols * kGfRows, 0, st, dm, m->shape.ns,
                   nl->ws.net_blocks, nb_cg, nl->ws.net_part, nl->ws.cpart, l2coef, m->grad, m->params, m->adam_m, m->adam_v,
                   m->step, m->err, a, nl->ws.coef, loss_out);
  stage("grad_adam");
  GNEP_CHECK_LAUNCH("gradient and adam");
  return GNEP_OK;
}

namespace {
__global__ void k_to_float(int64_t n, const double* __restrict__ g, float* __restrict__ o) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) o[q] = (float)g[q];
}
}  // namespace

int grad_to_float(const gnep_model* m, float* dst, cudaStream_t st) {
  k_to_float<<<blocks_for(m->n_params, 256), 256, 0, st>>>(m->n_params, m->grad, dst);
  GNEP_CHECK_LAUNCH("k_to_float");
  return GNEP_OK;
}

int run_scale(gnep_model* m, gnep_nlist* nl, cudaStream_t st) {
  if (nl->n_atoms == 0) return set_error(GNEP_ERR_INVALID_ARG, "empty batch");
  k_scale<<<m->shape.ndes, 256, 0, st>>>(nl->n_atoms, m->shape.ndes, nl->ws.G, m->scale);
  GNEP_CHECK_LAUNCH("k_scale");
  return GNEP_OK;
}

}  // namespace gnep
