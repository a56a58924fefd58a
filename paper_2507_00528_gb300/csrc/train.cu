// Loss (Eqs. 9-12), residual weights, parameter-gradient reductions
// (Eqs. 13-16, D1.18-D1.21), Adam with the Eq. 17 schedule, descriptor scale
// and the species-grouped atom order.  Every cross-atom sum is FP64 in a fixed
// order, so a step is bit-reproducible.
#include "gnep_internal.h"

namespace gnep {

constexpr int kRedBlocks = 512;  // partial sums per loss term
constexpr int kChunk = 256;      // atoms per gradient partial

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

struct Operand {
  const float* p;
  int ld, col0;
  const float* colscale;  // optional per-column factor
};

struct ChunkMap {
  const int* perm;
  int soff[9];     // species offsets in perm
  int nchunk[8];   // chunks per species
  int cmax;        // max chunks over species
  int local_size;  // partial row length per species (= n_params / ns)
  int ns;
};

__device__ __forceinline__ bool chunk_range(const ChunkMap& cm, int e, int c, int& b, int& en) {
  if (c >= cm.nchunk[e]) return false;
  b = cm.soff[e] + c * kChunk;
  en = min(b + kChunk, cm.soff[e + 1]);
  return b < en;
}

// out[a][b] += sum_i X1(i,a) Y1(i,b) + sgn X2(i,a) Y2(i,b) over one chunk of one
// species; 32 x 32 output tile per block, 256 threads x 4 outputs.
__global__ void __launch_bounds__(256) k_outer_reduce(ChunkMap cm, Operand x1, Operand y1, Operand x2,
                                                      Operand y2, float sgn, int A, int B, int out_off,
                                                      float* __restrict__ part) {
  const int tilesB = (B + 31) / 32;
  const int ta = blockIdx.x / tilesB, tb = blockIdx.x % tilesB;
  const int c = blockIdx.y, e = blockIdx.z;
  int i0, i1;
  if (!chunk_range(cm, e, c, i0, i1)) return;
  __shared__ float sx1[32][33], sy1[32][33], sx2[32][33], sy2[32][33];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 2 x 2 outputs each
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int base = i0; base < i1; base += 32) {
    for (int q = threadIdx.x; q < 32 * 32; q += 256) {
      const int r = q >> 5, col = q & 31;
      const int ii = base + r;
      float vx1 = 0.f, vy1 = 0.f, vx2 = 0.f, vy2 = 0.f;
      if (ii < i1) {
        const int at = cm.perm[ii];
        const int a = ta * 32 + col, b = tb * 32 + col;
        if (a < A) {
          vx1 = x1.p[(size_t)at * x1.ld + x1.col0 + a];
          if (x2.p) vx2 = x2.p[(size_t)at * x2.ld + x2.col0 + a];
        }
        if (b < B) {
          vy1 = y1.p[(size_t)at * y1.ld + y1.col0 + b];
          if (y1.colscale) vy1 *= y1.colscale[y1.col0 + b];
          if (y2.p) {
            vy2 = y2.p[(size_t)at * y2.ld + y2.col0 + b];
            if (y2.colscale) vy2 *= y2.colscale[y2.col0 + b];
          }
        }
      }
      sx1[r][col] = vx1;
      sy1[r][col] = vy1;
      sx2[r][col] = vx2;
      sy2[r][col] = sgn * vy2;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int w = 0; w < 2; ++w) {
          acc[u][w] = fmaf(sx1[r][ty * 2 + u], sy1[r][tx * 2 + w], acc[u][w]);
          acc[u][w] = fmaf(sx2[r][ty * 2 + u], sy2[r][tx * 2 + w], acc[u][w]);
        }
    }
    __syncthreads();
  }
  float* out = part + ((size_t)c * cm.ns + e) * cm.local_size + out_off;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const int a = ta * 32 + ty * 2 + u, b = tb * 32 + tx * 2 + w;
      if (a < A && b < B) out[a * B + b] = acc[u][w];
    }
}

// out[q] = sum_i Z(i, q) over one chunk of one species.
__global__ void __launch_bounds__(256) k_col_reduce(ChunkMap cm, Operand z, int Q, int out_off,
                                                    float* __restrict__ part) {
  const int c = blockIdx.y, e = blockIdx.z;
  int i0, i1;
  if (!chunk_range(cm, e, c, i0, i1)) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Q) return;
  float s = 0.f;
  for (int ii = i0; ii < i1; ++ii) s += z.p[(size_t)cm.perm[ii] * z.ld + z.col0 + q];
  part[((size_t)c * cm.ns + e) * cm.local_size + out_off + q] = s;
}

// grad[q] = sum over chunks (FP64) + 2 lambda_l2 theta_q / N_par.
__global__ void k_grad_final(DevModel dm, int cmax, int ns, int local_size, const float* __restrict__ part,
                             double l2coef, double* __restrict__ grad) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= dm.n_params) return;
  int e, l;
  if (q < (int64_t)ns * dm.net_size) {
    e = (int)(q / dm.net_size);
    l = (int)(q % dm.net_size);
  } else if (q < dm.off_cA) {
    const int r = (int)(q - dm.off_cR), blk = ns * dm.nqr * dm.kr;
    e = r / blk;
    const int rem = r % blk, J = rem / (dm.nqr * dm.kr), n = (rem / dm.kr) % dm.nqr, k = rem % dm.kr;
    l = dm.net_size + n * ns * dm.kr + J * dm.kr + k;
  } else {
    const int r = (int)(q - dm.off_cA), blk = ns * dm.nqa * dm.ka;
    e = r / blk;
    const int rem = r % blk, J = rem / (dm.nqa * dm.ka), n = (rem / dm.ka) % dm.nqa, k = rem % dm.ka;
    l = dm.net_size + dm.nqr * ns * dm.kr + n * ns * dm.ka + J * dm.ka + k;
  }
  double s = 0.0;
  for (int c = 0; c < cmax; ++c) s += (double)part[((size_t)c * ns + e) * local_size + l];
  grad[q] = s + l2coef * (double)dm.params[q];
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

ChunkMap make_chunk_map(const gnep_model* m, const gnep_nlist* nl) {
  ChunkMap cm;
  cm.perm = nl->perm;
  cm.ns = m->shape.ns;
  cm.cmax = 0;
  for (int e = 0; e <= cm.ns; ++e) cm.soff[e] = nl->species_off[e];
  for (int e = 0; e < cm.ns; ++e) {
    const int ne = nl->species_off[e + 1] - nl->species_off[e];
    cm.nchunk[e] = (ne + kChunk - 1) / kChunk;
    if (cm.nchunk[e] > cm.cmax) cm.cmax = cm.nchunk[e];
  }
  cm.local_size = (int)(m->n_params / cm.ns);
  return cm;
}

}  // namespace

int64_t grad_partial_floats(const gnep_model* m, int n_atoms) {
  const int cmax = (n_atoms + kChunk - 1) / kChunk + 1;
  return (int64_t)cmax * m->n_params;
}
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
  Workspace& w = nl->ws;
  const Shape& sh = m->shape;
  const ChunkMap cm = make_chunk_map(m, nl);
  const DevModel dm = m->dev();
  const int H = sh.H, D = sh.ndes, ns = sh.ns;
  const size_t part_bytes = sizeof(float) * (size_t)(cm.cmax > 0 ? cm.cmax : 1) * ns * cm.local_size;
  GNEP_CUDA(cudaMemsetAsync(w.part, 0, part_bytes, st));
  stage("memset_partials");
  if (cm.cmax > 0) {
    // dL/dW0 = sum_i alpha (s.G)^T - beta (s.Gdot)^T
    {
      Operand x1{w.alpha, H, 0, nullptr}, y1{w.G, D, 0, m->scale}, x2{w.beta, H, 0, nullptr},
          y2{w.Gd, D, 0, m->scale};
      dim3 grid(((H + 31) / 32) * ((D + 31) / 32), cm.cmax, ns);
      k_outer_reduce<<<grid, 256, 0, st>>>(cm, x1, y1, x2, y2, -1.f, H, D, 0, w.part);
      stage("reduce_W0");
    }
    // dL/dc^R = sum_i Gbar_n FR_Jk - E'_n FRdot_Jk
    {
      Operand x1{w.Gb, D, 0, nullptr}, y1{w.FR, ns * sh.kr, 0, nullptr}, x2{w.Ep, D, 0, nullptr},
          y2{w.FRd, ns * sh.kr, 0, nullptr};
      const int B = ns * sh.kr;
      dim3 grid(((sh.nqr + 31) / 32) * ((B + 31) / 32), cm.cmax, ns);
      k_outer_reduce<<<grid, 256, 0, st>>>(cm, x1, y1, x2, y2, -1.f, sh.nqr, B, m->net_size, w.part);
      stage("reduce_cR");
    }
    // b0, w1, b1, c^A column sums
    {
      dim3 g1((H + 255) / 256, cm.cmax, ns);
      k_col_reduce<<<g1, 256, 0, st>>>(cm, Operand{w.alpha, H, 0, nullptr}, H, D * H, w.part);
      stage("reduce_b0");
      k_col_reduce<<<g1, 256, 0, st>>>(cm, Operand{w.q1, H, 0, nullptr}, H, D * H + H, w.part);
      stage("reduce_w1");
      dim3 g2(1, cm.cmax, ns);
      k_col_reduce<<<g2, 256, 0, st>>>(cm, Operand{w.eatom, 1, 0, nullptr}, 1, D * H + 2 * H, w.part);
      stage("reduce_b1");
      const int QA = sh.nqa * ns * sh.ka;
      dim3 g3((QA + 255) / 256, cm.cmax, ns);
      k_col_reduce<<<g3, 256, 0, st>>>(cm, Operand{w.dcA, QA, 0, nullptr}, QA,
                                       m->net_size + sh.nqr * ns * sh.kr, w.part);
      stage("reduce_cA");
    }
  }
  k_grad_final<<<blocks_for(m->n_params, 256), 256, 0, st>>>(dm, cm.cmax, ns, cm.local_size, w.part,
                                                             2.0 * lambda_l2 / (double)m->n_params, m->grad);
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
