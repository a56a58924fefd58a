// Loss (Eqs. 9-12), residual weights, parameter-gradient reductions
// (Eqs. 13-16, D1.18-D1.21), Adam with the Eq. 17 schedule, descriptor scale
// and the species-grouped atom order.  Every cross-atom sum is FP64 in a fixed
// order, so a step is bit-reproducible.
#include "gnep_internal.h"
#include "network.cuh"

namespace gnep {

constexpr int kRedBlocks = 512;  // partial sums per loss term

namespace {

__device__ __forceinline__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// Partial sums of the squared residuals of Eqs. 10-12 (fixed grid, fixed order).
__global__ void __launch_bounds__(256) k_loss_partials(int N, int S, const int* __restrict__ soff,
                                                       const double* __restrict__ Es, const double* __restrict__ Ws,
                                                       const float* __restrict__ F, const double* __restrict__ le,
                                                       const float* __restrict__ lf, const double* __restrict__ lv,
                                                       double* __restrict__ red) {
  __shared__ double sh[256];
  double se = 0, sf = 0, sv = 0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < 3LL * N; q += (int64_t)gridDim.x * blockDim.x) {
    const double d = (double)F[q] - (double)lf[q];
    sf += d * d;
  }
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
    const double ns = soff[s + 1] - soff[s];
    const double de = Es[s] / ns - le[s];
    se += de * de;
    for (int c = 0; c < 6; ++c) {
      const double dv = Ws[6 * s + c] / ns - lv[6 * s + c];
      sv += dv * dv;
    }
  }
  se = block_sum(se, sh);
  sf = block_sum(sf, sh);
  sv = block_sum(sv, sh);
  if (threadIdx.x == 0) {
    red[3 * blockIdx.x] = se;
    red[3 * blockIdx.x + 1] = sf;
    red[3 * blockIdx.x + 2] = sv;
  }
}

struct LossArgs {
  int N, S;
  double le, lf, lv, l2;
  int form;
  int64_t n_params;
};

// Loss terms and the scalar weights of the residuals:
// coef[0..3] = {L, L_e, L_f, L_v}; coef[4] = cf, coef[5] = ce, coef[6] = cv with
//   a_i = cf (F_i - F_i^tar),  e_s = ce (E_s/N_s - E_s^tar)/N_s,
//   B_s = cv (W_s/N_s - V_s^tar)/N_s  (off-diagonals halved).
__global__ void __launch_bounds__(256) k_loss_final(LossArgs a, int nred, const double* __restrict__ red,
                                                    const float* __restrict__ params, double* __restrict__ coef,
                                                    int* __restrict__ err) {
  __shared__ double sh[256];
  double se = 0, sf = 0, sv = 0, l2 = 0;
  for (int b = threadIdx.x; b < nred; b += blockDim.x) {
    se += red[3 * b];
    sf += red[3 * b + 1];
    sv += red[3 * b + 2];
  }
  for (int64_t q = threadIdx.x; q < a.n_params; q += blockDim.x) l2 += (double)params[q] * params[q];
  se = block_sum(se, sh);
  sf = block_sum(sf, sh);
  sv = block_sum(sv, sh);
  l2 = block_sum(l2, sh);
  if (threadIdx.x != 0) return;
  const double Le = a.S > 0 ? se / a.S : 0.0;           // Eq. 10
  const double Lf = a.N > 0 ? sf / (3.0 * a.N) : 0.0;   // Eq. 11
  const double Lv = a.S > 0 ? sv / (6.0 * a.S) : 0.0;   // Eq. 12
  const double reg = a.l2 * l2 / (double)a.n_params;
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
  coef[4] = a.N > 0 ? a.lf * kf * 2.0 / (3.0 * a.N) : 0.0;  // Eq. 15
  coef[5] = a.S > 0 ? a.le * ke * 2.0 / a.S : 0.0;          // Eq. 14
  coef[6] = a.S > 0 ? a.lv * kv * 2.0 / (6.0 * a.S) : 0.0;  // Eq. 16
  if (!isfinite(L)) atomicOr(err, kErrNonFinite);
}

__global__ void k_residual_atoms(int N, const float* __restrict__ F, const float* __restrict__ lf,
                                 const double* __restrict__ coef, float4* __restrict__ a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float cf = (float)coef[4];
  a[i] = make_float4(cf * (F[3 * i] - lf[3 * i]), cf * (F[3 * i + 1] - lf[3 * i + 1]),
                     cf * (F[3 * i + 2] - lf[3 * i + 2]), 0.f);
}

__global__ void k_residual_struct(int S, const int* __restrict__ soff, const double* __restrict__ Es,
                                  const double* __restrict__ Ws, const double* __restrict__ le,
                                  const double* __restrict__ lv, const double* __restrict__ coef,
                                  float* __restrict__ es, float* __restrict__ Bs) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const double ns = soff[s + 1] - soff[s];
  es[s] = (float)(coef[5] * (Es[s] / ns - le[s]) / ns);
  for (int c = 0; c < 6; ++c) {
    const double g = coef[6] * (Ws[6 * s + c] / ns - lv[6 * s + c]) / ns;
    Bs[6 * s + c] = (float)(c < 3 ? g : 0.5 * g);
  }
}

// ---------------------------------------------------------- gradient sums

// grad[q] = sum over block partials (FP64, one warp per parameter, fixed order)
//           + 2 lambda_l2 theta_q / N_par.
// Network parameters come from the network backward pass (net_part), the
// coefficients from the c-gradient sweep (cpart).
__global__ void __launch_bounds__(256) k_grad_final(DevModel dm, int ns, int nb_net, int nb_cg,
                                                    const float* __restrict__ net_part,
                                                    const float* __restrict__ cpart, double l2coef,
                                                    double* __restrict__ grad) {
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= dm.n_params) return;
  double s = 0.0;
  if (q < (int64_t)ns * dm.net_size) {
    const int e = (int)(q / dm.net_size), l = (int)(q % dm.net_size);
    for (int b = lane; b < nb_net; b += 32) s += (double)net_part[((size_t)b * ns + e) * dm.net_size + l];
  } else {
    const int64_t nc = dm.n_params - (int64_t)ns * dm.net_size;
    const int64_t c = q - dm.off_cR;
    for (int b = lane; b < nb_cg; b += 32) s += (double)cpart[(size_t)b * nc + c];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) grad[q] = s + l2coef * (double)dm.params[q];
}

// ---------------------------------------------------------- Adam, Eq. 17

struct AdamArgs {
  double lr, b1, b2, eps, wd;
  int scheduled;
  double lr_start, lr_stop;
  long long nw, nt;
};

__device__ double lr_eq17(const AdamArgs& a, long long s) {
  if (s < a.nw) return a.lr_stop + (double)s / (double)a.nw * (a.lr_start - a.lr_stop);
  if (s > a.nt) s = a.nt;
  const double span = (double)(a.nt - a.nw);
  const double frac = span > 0 ? (double)(s - a.nw) / span : 1.0;
  return a.lr_stop + (a.lr_start - a.lr_stop) * 0.5 * (1.0 + cospi(frac));
}

__global__ void k_adam(int64_t n, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const double* __restrict__ g, const long long* __restrict__ step,
                       const int* __restrict__ err, AdamArgs a) {
  if (*err & kErrNonFinite) return;  // the step is skipped
  const long long t = *step + 1;
  const double lr = a.scheduled ? lr_eq17(a, *step) : a.lr;
  const double c1 = 1.0 - pow(a.b1, (double)t), c2 = 1.0 - pow(a.b2, (double)t);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const double gq = g[q];
    const double mq = a.b1 * m[q] + (1.0 - a.b1) * gq;
    const double vq = a.b2 * v[q] + (1.0 - a.b2) * gq * gq;
    m[q] = (float)mq;
    v[q] = (float)vq;
    const double upd = (mq / c1) / (sqrt(vq / c2) + a.eps) + a.wd * p[q];
    p[q] = (float)(p[q] - lr * upd);
  }
}

__global__ void k_step_inc(long long* step, const int* err) {
  if (!(*err & kErrNonFinite)) *step += 1;
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

// Stable grouping of atoms by species: perm = atoms of species 0 in order, then 1, ...
__global__ void __launch_bounds__(1024) k_species_perm(int N, int ns, const int* __restrict__ type,
                                                       int* __restrict__ perm, int* __restrict__ soff) {
  __shared__ int sh[1024];
  int base = 0;
  for (int e = 0; e < ns; ++e) {
    if (threadIdx.x == 0) soff[e] = base;
    for (int c = 0; c < N; c += 1024) {
      const int i = c + threadIdx.x;
      const int f = (i < N && type[i] == e) ? 1 : 0;
      sh[threadIdx.x] = f;
      __syncthreads();
      for (int o = 1; o < 1024; o <<= 1) {
        const int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
      }
      if (f) perm[base + sh[threadIdx.x] - 1] = i;
      const int tot = sh[1023];
      __syncthreads();
      base += tot;
    }
  }
  if (threadIdx.x == 0) soff[ns] = base;
}

}  // namespace

int64_t loss_partial_doubles() { return 3LL * kRedBlocks; }

int run_species_perm(gnep_nlist* nl, cudaStream_t st) {
  int* soff_dev = nullptr;
  GNEP_CUDA(cudaMallocAsync(&soff_dev, sizeof(int) * 9, st));
  k_species_perm<<<1, 1024, 0, st>>>(nl->n_atoms, nl->shape.ns, nl->type, nl->perm, soff_dev);
  GNEP_CHECK_LAUNCH("k_species_perm");
  GNEP_CUDA(cudaMemcpyAsync(nl->species_off, soff_dev, sizeof(int) * (nl->shape.ns + 1), cudaMemcpyDeviceToHost, st));
  GNEP_CUDA(cudaFreeAsync(soff_dev, st));
  GNEP_CUDA(cudaStreamSynchronize(st));
  return GNEP_OK;
}

int run_loss_impl(const gnep_model* m, gnep_nlist* nl, const double* le, const float* lf, const double* lv,
                  const gnep_labels* y, cudaStream_t st) {
  Workspace& w = nl->ws;
  const int N = nl->n_atoms, S = nl->n_struct;
  k_loss_partials<<<kRedBlocks, 256, 0, st>>>(N, S, nl->struct_off, w.Es, w.Ws, w.F, le, lf, lv, w.red);
  stage("loss_partials");
  LossArgs a;
  a.N = N; a.S = S; a.le = y->lambda_e; a.lf = y->lambda_f; a.lv = y->lambda_v; a.l2 = y->lambda_l2;
  a.form = y->loss_form; a.n_params = m->n_params;
  k_loss_final<<<1, 256, 0, st>>>(a, kRedBlocks, w.red, m->params, w.coef, m->err);
  stage("loss_final");
  if (N > 0) k_residual_atoms<<<blocks_for(N, 256), 256, 0, st>>>(N, w.F, lf, w.coef, w.a);
  stage("residual_atoms");
  k_residual_struct<<<blocks_for(S, 128), 128, 0, st>>>(S, nl->struct_off, w.Es, w.Ws, le, lv, w.coef, w.es, w.Bs);
  stage("residual_struct");
  GNEP_CHECK_LAUNCH("loss");
  return GNEP_OK;
}

int run_grad_reduce_impl(const gnep_model* m, gnep_nlist* nl, double lambda_l2, cudaStream_t st) {
  const DevModel dm = m->dev();
  const int ns = m->shape.ns;
  const int nb_net = nl->ws.net_blocks;
  const int nb_cg = nl->n_atoms > 0 ? cgrad_blocks(nl) : 0;
  k_grad_final<<<blocks_for(m->n_params * 32, 256), 256, 0, st>>>(dm, ns, nb_net, nb_cg, nl->ws.net_part,
                                                                  nl->ws.cpart, 2.0 * lambda_l2 / (double)m->n_params,
                                                                  m->grad);
  stage("grad_final");
  GNEP_CHECK_LAUNCH("gradient reduction");
  return GNEP_OK;
}

int run_adam(gnep_model* m, const double*, double lr, double b1, double b2, double eps, double wd, bool scheduled,
             double lr_start, double lr_stop, int64_t nw, int64_t nt, cudaStream_t st) {
  AdamArgs a;
  a.lr = lr; a.b1 = b1; a.b2 = b2; a.eps = eps; a.wd = wd;
  a.scheduled = scheduled ? 1 : 0;
  a.lr_start = lr_start; a.lr_stop = lr_stop; a.nw = nw; a.nt = nt;
  const int nb = blocks_for(m->n_params, 256);
  k_adam<<<nb < 1 ? 1 : nb, 256, 0, st>>>(m->n_params, m->params, m->adam_m, m->adam_v, m->grad, m->step, m->err, a);
  stage("adam");
  k_step_inc<<<1, 1, 0, st>>>(m->step, m->err);
  stage("step_inc");
  GNEP_CHECK_LAUNCH("adam");
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
