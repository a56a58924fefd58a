// C ABI of libgnep: models, neighbour lists, one training step, Adam, graphs,
// checkpoints and error reporting.  See include/gnep.h for the contract.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gnep_internal.h"
#include "network.cuh"

using namespace gnep;

namespace gnep {

Profiler g_prof;
static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? GNEP_ERR_OOM : GNEP_ERR_CUDA;
}

}  // namespace gnep

namespace {

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy to a caller buffer (host or device); host destinations are complete on return.
int copy_out(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (!dst || bytes == 0) return GNEP_OK;
  GNEP_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
  if (!is_device_ptr(dst)) GNEP_CUDA(cudaStreamSynchronize(st));
  return GNEP_OK;
}

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

namespace gnep {

void free_workspace(gnep_nlist* nl) {
  if (nl->ws_mem) cudaFree(nl->ws_mem);
  nl->ws_mem = nullptr;
  nl->ws = Workspace();
  nl->ws_pairs[0] = nl->ws_pairs[1] = -1;
}

int alloc_workspace(gnep_model* m, gnep_nlist* nl) {
  if (nl->ws_mem && nl->ws_pairs[0] >= nl->L[0].n && nl->ws_pairs[1] >= nl->L[1].n) return GNEP_OK;
  free_workspace(nl);
  const Shape& s = m->shape;
  const size_t N = nl->n_atoms > 0 ? nl->n_atoms : 1, S = nl->n_struct;
  // pair-sized buffers get headroom so that rebuilds with a few more pairs (MD) do not reallocate
  const size_t PR = nl->L[0].n + nl->L[0].n / 8 + 64, PA = nl->L[1].n + nl->L[1].n / 8 + 64;
  const size_t D = s.ndes, A24 = (size_t)s.nqa * ((s.lmax + 1) * (s.lmax + 1) - 1), FRn = (size_t)s.ns * s.kr;
  struct Item { void** p; size_t bytes; };
  Workspace& w = nl->ws;
  w.red_len = loss_partial_doubles(nl->n_struct);
  const size_t NC = (size_t)(m->n_params - (int64_t)s.ns * m->net_size);
  std::vector<Item> items = {
      {(void**)&w.G, 4 * N * D},        {(void**)&w.Ep, 4 * N * D},
      {(void**)&w.Eatom, 4 * N},        {(void**)&w.S, 4 * N * A24},      {(void**)&w.FR, 4 * N * FRn},
      {(void**)&w.chat, 4 * N * FRn},   {(void**)&w.dA, 16 * PA},         {(void**)&w.F, 12 * N},
      {(void**)&w.Wat, 24 * N},         {(void**)&w.Es, 8 * S},           {(void**)&w.Ws, 48 * S},
      {(void**)&w.a, 16 * N},           {(void**)&w.es, 4 * S},           {(void**)&w.Bs, 24 * S},
      {(void**)&w.Gd, 4 * N * D},       {(void**)&w.Sd, 4 * N * A24},     {(void**)&w.FRd, 4 * N * FRn},
      {(void**)&w.Gb, 4 * N * D},       {(void**)&w.wij, 16 * PA},
      {(void**)&w.net_part, 4 * (size_t)kNetBlocks * s.ns * m->net_size},
      {(void**)&w.cpart, 4 * (size_t)kCgBlocksMax * NC},
      {(void**)&w.red, 8 * (size_t)w.red_len},
      {(void**)&w.lab_e, 8 * S},        {(void**)&w.lab_f, 12 * N},       {(void**)&w.lab_v, 48 * S},
      {(void**)&w.coef, 8 * 8},         {(void**)&w.gradf, 4 * (size_t)m->n_params}};
  (void)PR;
  size_t total = 0;
  for (auto& it : items) total += align256(it.bytes);
  char* base = nullptr;
  GNEP_CUDA(cudaMalloc(&base, total));
  GNEP_CUDA(cudaMemset(base, 0, total));
  size_t off = 0;
  for (auto& it : items) {
    *it.p = base + off;
    off += align256(it.bytes);
  }
  nl->ws_mem = base;
  nl->ws_pairs[0] = (int64_t)PR;
  nl->ws_pairs[1] = (int64_t)PA;
  return GNEP_OK;
}

}  // namespace gnep

// ======================================================================= API

extern "C" {

const char* gnep_last_error(void) { return gnep::g_last_error.c_str(); }
int gnep_abi_version(void) { return GNEP_ABI_VERSION; }

int gnep_create(gnep_model** out, int n_species, const int* species_z, double rc_radial, double rc_angular,
                int n_max_radial, int n_max_angular, int basis_radial, int basis_angular, int l_max,
                int four_body, int hidden, uint64_t seed, int precision) {
  (void)species_z;
  if (!out) return set_error(GNEP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_species < 1 || n_species > 8 || !(rc_radial > 0) || !(rc_angular > 0) || rc_angular > rc_radial ||
      n_max_radial < 0 || n_max_angular < 0 || basis_radial < 0 || basis_angular < 0 || l_max < 1 ||
      l_max > 8 || hidden < 1 || hidden > kMaxHidden || precision < 0 || precision > 2)
    return set_error(GNEP_ERR_INVALID_ARG, "hyper-parameter out of range");
  Shape s;
  s.ns = n_species; s.nqr = n_max_radial + 1; s.kr = basis_radial + 1; s.nqa = n_max_angular + 1;
  s.ka = basis_angular + 1; s.lmax = l_max; s.fb = four_body ? 1 : 0; s.H = hidden;
  s.ndes = s.nqr + s.nqa * s.lmax + (s.fb ? s.nqa : 0);
  if (!shape_supported(s))
    return set_error(GNEP_ERR_UNSUPPORTED,
                     "no compiled kernel for this shape (built: 2 species; l_max 4 with n_max/basis 4/8 without "
                     "4-body or 8/12 with or without 4-body; n_max/basis 4/8 with l_max 6 without 4-body or "
                     "l_max 8 with 4-body)");
  if (precision != GNEP_PREC_FP32 && hidden > kMaxHiddenTc)
    return set_error(GNEP_ERR_UNSUPPORTED, "TF32/BF16 network tiles hold at most 112 hidden neurons");
  if (precision != GNEP_PREC_FP32 && l_max > 4)
    return set_error(GNEP_ERR_UNSUPPORTED, "l_max > 4 runs the FP32 network only");
  gnep_model* m = new gnep_model();
  m->shape = s;
  m->rcr = rc_radial;
  m->rca = rc_angular;
  m->precision = precision;
  m->net_size = s.ndes * s.H + 2 * s.H + 1;
  m->off_cR = s.ns * m->net_size;
  m->off_cA = m->off_cR + s.ns * s.ns * s.nqr * s.kr;
  m->n_params = (int64_t)m->off_cA + (int64_t)s.ns * s.ns * s.nqa * s.ka;
  cudaGetDevice(&m->device);
  {  // keep stream-ordered scratch (neighbour builds) in the pool between builds
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, m->device) == cudaSuccess) {
      uint64_t keep = 8ull << 30;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
  }
  int rc = shape_setup(s);
  if (rc) { delete m; return rc; }
  const size_t n = (size_t)m->n_params;
  auto fail = [&](cudaError_t e, const char* w) {
    gnep_destroy(m);
    return cuda_error(e, w);
  };
  cudaError_t e;
  if ((e = cudaMalloc(&m->params, 4 * n)) != cudaSuccess) return fail(e, "cudaMalloc params");
  if ((e = cudaMalloc(&m->scale, 4 * (size_t)s.ndes)) != cudaSuccess) return fail(e, "cudaMalloc scale");
  if ((e = cudaMalloc(&m->adam_m, 4 * n)) != cudaSuccess) return fail(e, "cudaMalloc adam");
  if ((e = cudaMalloc(&m->adam_v, 4 * n)) != cudaSuccess) return fail(e, "cudaMalloc adam");
  if ((e = cudaMalloc(&m->grad, 8 * n)) != cudaSuccess) return fail(e, "cudaMalloc grad");
  if ((e = cudaMalloc(&m->step, sizeof(long long))) != cudaSuccess) return fail(e, "cudaMalloc step");
  if ((e = cudaMalloc(&m->err, 3 * sizeof(int))) != cudaSuccess) return fail(e, "cudaMalloc err");
  std::vector<float> h(n);
  uint64_t st = seed;
  for (size_t q = 0; q < n; ++q) h[q] = (float)((double)(splitmix64(st) >> 11) * 0x1.0p-53 - 0.5);
  std::vector<float> one(s.ndes, 1.f);
  cudaMemcpy(m->params, h.data(), 4 * n, cudaMemcpyHostToDevice);
  cudaMemcpy(m->scale, one.data(), 4 * (size_t)s.ndes, cudaMemcpyHostToDevice);
  cudaMemset(m->adam_m, 0, 4 * n);
  cudaMemset(m->adam_v, 0, 4 * n);
  cudaMemset(m->grad, 0, 8 * n);
  cudaMemset(m->step, 0, sizeof(long long));
  if ((e = cudaMemset(m->err, 0, 3 * sizeof(int))) != cudaSuccess) return fail(e, "init");
  *out = m;
  return GNEP_OK;
}

int gnep_destroy(gnep_model* m) {
  if (!m) return GNEP_OK;
  cudaFree(m->params); cudaFree(m->scale); cudaFree(m->adam_m); cudaFree(m->adam_v);
  cudaFree(m->grad); cudaFree(m->step); cudaFree(m->err);
  delete m;
  return GNEP_OK;
}

int gnep_set_precision(gnep_model* m, int precision) {
  if (!m || precision < 0 || precision > 2) return set_error(GNEP_ERR_INVALID_ARG, "bad precision");
  if (precision != GNEP_PREC_FP32 && m->shape.H > kMaxHiddenTc)
    return set_error(GNEP_ERR_UNSUPPORTED, "TF32/BF16 network tiles hold at most 112 hidden neurons");
  if (precision != GNEP_PREC_FP32 && m->shape.lmax > 4)
    return set_error(GNEP_ERR_UNSUPPORTED, "l_max > 4 runs the FP32 network only");
  m->precision = precision;
  return GNEP_OK;
}

int gnep_num_params(const gnep_model* m, int64_t* n) {
  if (!m || !n) return set_error(GNEP_ERR_INVALID_ARG, "NULL argument");
  *n = m->n_params;
  return GNEP_OK;
}

int gnep_num_descriptors(const gnep_model* m, int32_t* n) {
  if (!m || !n) return set_error(GNEP_ERR_INVALID_ARG, "NULL argument");
  *n = m->shape.ndes;
  return GNEP_OK;
}

int gnep_get_params(gnep_model* m, float* dst, int64_t n, void* stream) {
  if (!m || !dst || n != m->n_params) return set_error(GNEP_ERR_INVALID_ARG, "bad parameter buffer");
  return copy_out(dst, m->params, 4 * (size_t)n, (cudaStream_t)stream);
}

int gnep_set_params(gnep_model* m, const float* src, int64_t n, void* stream) {
  if (!m || !src || n != m->n_params) return set_error(GNEP_ERR_INVALID_ARG, "bad parameter buffer");
  GNEP_CUDA(cudaMemcpyAsync(m->params, src, 4 * (size_t)n, cudaMemcpyDefault, (cudaStream_t)stream));
  if (!is_device_ptr(src)) GNEP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return GNEP_OK;
}

int gnep_set_descriptor_scale(gnep_model* m, const float* scale, int32_t n, void* stream) {
  if (!m || !scale || n != m->shape.ndes) return set_error(GNEP_ERR_INVALID_ARG, "bad scale buffer");
  GNEP_CUDA(cudaMemcpyAsync(m->scale, scale, 4 * (size_t)n, cudaMemcpyDefault, (cudaStream_t)stream));
  if (!is_device_ptr(scale)) GNEP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return GNEP_OK;
}

int gnep_get_descriptor_scale(gnep_model* m, float* scale, int32_t n, void* stream) {
  if (!m || !scale || n != m->shape.ndes) return set_error(GNEP_ERR_INVALID_ARG, "bad scale buffer");
  return copy_out(scale, m->scale, 4 * (size_t)n, (cudaStream_t)stream);
}

static int check_nlist(const gnep_model* m, const gnep_nlist* nl) {
  if (!m || !nl) return set_error(GNEP_ERR_INVALID_ARG, "NULL model or neighbour list");
  if (!(nl->shape == m->shape) || nl->rcr != m->rcr || nl->rca != m->rca)
    return set_error(GNEP_ERR_INVALID_ARG, "neighbour list was built for a model of another shape or cut-off");
  return GNEP_OK;
}

// Orders the work that follows on `st` after the device work of the last
// build of `nl` (a rebuild returns before that work has finished).
static int after_build(const gnep_nlist* nl, cudaStream_t st) {
  if (nl && nl->ready_ev) GNEP_CUDA(cudaStreamWaitEvent(st, nl->ready_ev, 0));
  return GNEP_OK;
}

// check_nlist, then after_build on `st`.
static int use_nlist(const gnep_model* m, const gnep_nlist* nl, cudaStream_t st) {
  const int rc = check_nlist(m, nl);
  return rc ? rc : after_build(nl, st);
}

int gnep_compute_descriptor_scale(gnep_model* m, const gnep_nlist* nl_, void* stream) {
  int rc = use_nlist(m, nl_, (cudaStream_t)stream);
  if (rc) return rc;
  gnep_nlist* nl = const_cast<gnep_nlist*>(nl_);
  cudaStream_t st = (cudaStream_t)stream;
  StepArgs A{m, nl, st};
  if ((rc = run_descriptors(A, false))) return rc;
  if ((rc = run_scale(m, nl, st))) return rc;
  GNEP_CUDA(cudaStreamSynchronize(st));
  return GNEP_OK;
}

// --------------------------------------------------------------- batches

// True when the host can read p directly (pageable or pinned host memory).
static bool host_readable(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeUnregistered || a.type == cudaMemoryTypeHost;
}

static int load_batch(gnep_model* m, const gnep_batch* b, gnep_nlist* nl, cudaStream_t st) {
  const int S = b->n_struct, N = b->n_atoms;
  std::vector<int> off_copy, typ_copy;
  const int *off = b->struct_off, *typ = b->type;
  const bool host = host_readable(b->struct_off) && (N == 0 || host_readable(b->type));
  if (!host) {  // device arrays: bring them over for the checks
    off_copy.resize(S + 1);
    typ_copy.resize(N > 0 ? N : 1);
    GNEP_CUDA(cudaMemcpyAsync(off_copy.data(), b->struct_off, sizeof(int) * (S + 1), cudaMemcpyDefault, st));
    if (N > 0) GNEP_CUDA(cudaMemcpyAsync(typ_copy.data(), b->type, sizeof(int) * N, cudaMemcpyDefault, st));
    GNEP_CUDA(cudaStreamSynchronize(st));
    off = off_copy.data();
    typ = typ_copy.data();
  }
  if (off[0] != 0 || off[S] != N) return set_error(GNEP_ERR_INVALID_ARG, "struct_off must start at 0 and end at n_atoms");
  for (int s = 0; s < S; ++s)
    if (off[s + 1] <= off[s])
      return set_error(GNEP_ERR_INVALID_ARG, "struct_off must be strictly increasing (every structure holds an atom)");
  for (int i = 0; i < N; ++i)
    if (typ[i] < 0 || typ[i] >= m->shape.ns) return set_error(GNEP_ERR_INVALID_ARG, "species index out of range");
  // the species grouping only changes with the species (a rebuild usually keeps them)
  nl->types_changed = !(nl->host_types.size() == (size_t)N && std::equal(typ, typ + N, nl->host_types.begin()));
  if (nl->types_changed) nl->host_types.assign(typ, typ + N);
  GNEP_CUDA(cudaMemcpyAsync(nl->struct_off, b->struct_off, sizeof(int) * (S + 1), cudaMemcpyDefault, st));
  if (N > 0) {
    GNEP_CUDA(cudaMemcpyAsync(nl->type, b->type, sizeof(int) * N, cudaMemcpyDefault, st));
    GNEP_CUDA(cudaMemcpyAsync(nl->pos, b->pos, sizeof(double) * 3 * (size_t)N, cudaMemcpyDefault, st));
  }
  GNEP_CUDA(cudaMemcpyAsync(nl->cell, b->cell, sizeof(double) * 9 * (size_t)S, cudaMemcpyDefault, st));
  return GNEP_OK;
}

// Greedy tiles of consecutive atoms with at most na atoms and ch angular pairs,
// cut on the host from the angular offsets of the last list build and uploaded
// from pinned staging (the upload overlaps the rest of the build).
static int build_angular_tiles(gnep_model* m, gnep_nlist* nl, cudaStream_t st) {
  const int N = nl->n_atoms;
  const long long* off = nl->host_aoff;
  if (!off || nl->host_aoff_n != (int64_t)N + 1)
    return set_error(GNEP_ERR_CUDA, "angular offsets missing (internal error)");
  if (!nl->tile_host || nl->tile_host_cap < 2 * ((int64_t)N + 1)) {
    if (nl->tile_host) {
      GNEP_CUDA(cudaEventSynchronize(nl->tile_ev));
      cudaFreeHost(nl->tile_host);
      nl->tile_host = nullptr;
    }
    GNEP_CUDA(cudaMallocHost(&nl->tile_host, sizeof(int) * 2 * ((size_t)N + 1)));
    nl->tile_host_cap = 2 * ((int64_t)N + 1);
  }
  if (!nl->tile_ev) GNEP_CUDA(cudaEventCreateWithFlags(&nl->tile_ev, cudaEventDisableTiming));
  GNEP_CUDA(cudaEventSynchronize(nl->tile_ev));  // the previous upload has left the staging
  for (int which = 0; which < 2; ++which) {
    int na = 0, ch = 0;
    angular_tile_limits(m->shape, which, &na, &ch);
    if (nl->tune.na[which] > 0 && nl->tune.na[which] < na) na = nl->tune.na[which];
    if (nl->tune.ch[which] > 0) ch = nl->tune.ch[which];
    int* t = nl->tile_host + which * ((size_t)N + 1);
    int nt = 0, i = 0;
    while (i < N) {
      t[nt++] = i;
      int j = i + 1;
      while (j < N && j - i < na && off[j + 1] - off[i] <= ch) ++j;
      i = j;
    }
    t[nt++] = N;
    if (!nl->atile[which] || nl->atile_cap[which] < (int64_t)nt) {  // at most N + 1 bounds
      cudaFree(nl->atile[which]);
      nl->atile[which] = nullptr;
      GNEP_CUDA(cudaMalloc(&nl->atile[which], sizeof(int) * (size_t)(N + 1)));
      nl->atile_cap[which] = N + 1;
    }
    GNEP_CUDA(cudaMemcpyAsync(nl->atile[which], t, sizeof(int) * nt, cudaMemcpyHostToDevice, st));
    nl->natile[which] = nt - 1;
  }
  GNEP_CUDA(cudaEventRecord(nl->tile_ev, st));
  return GNEP_OK;
}

// The lists, species grouping, angular tiles and workspace of `nl` for the
// batch already on the device.  The build synchronises with the host once the
// pair counts are known; with `wait` it also waits for the end of its device
// work and reports the lists' consistency flag, otherwise it returns after
// queueing that work (its end is nl->ready_ev, which every consumer of the
// list waits on, and the flag is reported by the next synchronising build or
// by gnep_sync_status).
static int finish_build(gnep_model* m, gnep_nlist* nl, cudaStream_t st, bool wait) {
  int rc;
  ++nl->gen;
  if (nl->n_atoms > 0) {
    if ((rc = build_lists(m, nl, st))) return rc;
    if (nl->types_changed && (rc = run_species_perm(nl, st))) return rc;
    nl->types_changed = false;
    if ((rc = build_angular_tiles(m, nl, st))) return rc;
  } else {
    for (int e = 0; e <= m->shape.ns; ++e) nl->species_off[e] = 0;
    for (int L = 0; L < 2; ++L) {
      if (!nl->L[L].off) GNEP_CUDA(cudaMalloc(&nl->L[L].off, sizeof(int)));
      GNEP_CUDA(cudaMemsetAsync(nl->L[L].off, 0, sizeof(int), st));
      nl->L[L].n = 0;
    }
  }
  if ((rc = alloc_workspace(m, nl))) return rc;
  if (!nl->ready_ev) GNEP_CUDA(cudaEventCreateWithFlags(&nl->ready_ev, cudaEventDisableTiming));
  if (!nl->side) {  // created here, outside any stream capture
    GNEP_CUDA(cudaStreamCreateWithFlags(&nl->side, cudaStreamNonBlocking));
    GNEP_CUDA(cudaEventCreateWithFlags(&nl->fork_ev, cudaEventDisableTiming));
    GNEP_CUDA(cudaEventCreateWithFlags(&nl->join_ev, cudaEventDisableTiming));
  }
  GNEP_CUDA(cudaEventRecord(nl->ready_ev, st));
  if (!wait) return GNEP_OK;
  int herr = 0;
  GNEP_CUDA(cudaMemcpyAsync(&herr, m->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GNEP_CUDA(cudaStreamSynchronize(st));
  if (herr & kErrRevMissing) {
    GNEP_CUDA(cudaMemset(m->err, 0, sizeof(int)));
    return set_error(GNEP_ERR_INVALID_ARG, "neighbour lists are not symmetric (internal error)");
  }
  return GNEP_OK;
}

int gnep_nlist_destroy(gnep_nlist* nl) {
  if (!nl) return GNEP_OK;
  cudaFree(nl->struct_off); cudaFree(nl->type); cudaFree(nl->pos); cudaFree(nl->cell);
  cudaFree(nl->atom_struct); cudaFree(nl->perm);
  cudaFree(nl->atile[0]); cudaFree(nl->atile[1]);
  if (nl->ready_ev) {
    cudaEventSynchronize(nl->ready_ev);
    cudaEventDestroy(nl->ready_ev);
  }
  if (nl->tile_ev) {
    cudaEventSynchronize(nl->tile_ev);
    cudaEventDestroy(nl->tile_ev);
  }
  if (nl->side) {
    cudaStreamSynchronize(nl->side);
    cudaStreamDestroy(nl->side);
    cudaEventDestroy(nl->fork_ev);
    cudaEventDestroy(nl->join_ev);
  }
  if (nl->tile_host) cudaFreeHost(nl->tile_host);
  if (nl->host_aoff) cudaFreeHost(nl->host_aoff);
  for (int L = 0; L < 2; ++L) {
    PairList& P = nl->L[L];
    cudaFree(P.off); cudaFree(P.j); cudaFree(P.owner); cudaFree(P.rev); cudaFree(P.rij); cudaFree(P.shift);
  }
  free_workspace(nl);
  delete nl;
  return GNEP_OK;
}

int gnep_build_neighbors(gnep_model* m, const gnep_batch* b, gnep_nlist** out, void* stream) {
  if (!m || !b || !out) return set_error(GNEP_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (b->n_struct < 1 || b->n_atoms < 0 || !b->struct_off || !b->cell || (b->n_atoms > 0 && (!b->pos || !b->type)))
    return set_error(GNEP_ERR_INVALID_ARG, "empty or incomplete batch");
  cudaStream_t st = (cudaStream_t)stream;
  gnep_nlist* nl = new gnep_nlist();
  nl->shape = m->shape;
  nl->rcr = m->rcr;
  nl->rca = m->rca;
  nl->n_struct = b->n_struct;
  nl->n_atoms = b->n_atoms;
  cudaGetDevice(&nl->device);
  const size_t N = b->n_atoms > 0 ? b->n_atoms : 1, S = b->n_struct;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&nl->struct_off, sizeof(int) * (S + 1));
  if (e == cudaSuccess) e = cudaMalloc(&nl->type, sizeof(int) * N);
  if (e == cudaSuccess) e = cudaMalloc(&nl->pos, sizeof(double) * 3 * N);
  if (e == cudaSuccess) e = cudaMalloc(&nl->cell, sizeof(double) * 9 * S);
  if (e == cudaSuccess) e = cudaMalloc(&nl->atom_struct, sizeof(int) * N);
  if (e == cudaSuccess) e = cudaMalloc(&nl->perm, sizeof(int) * N);
  if (e != cudaSuccess) {
    gnep_nlist_destroy(nl);
    return cuda_error(e, "cudaMalloc batch");
  }
  int rc = load_batch(m, b, nl, st);
  if (!rc) rc = finish_build(m, nl, st, true);
  if (rc) {
    gnep_nlist_destroy(nl);
    return rc;
  }
  *out = nl;
  return GNEP_OK;
}

int gnep_rebuild_neighbors(gnep_model* m, const gnep_batch* b, gnep_nlist* nl, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int rc = use_nlist(m, nl, st);
  if (rc) return rc;
  if (!b || b->n_struct != nl->n_struct || b->n_atoms != nl->n_atoms)
    return set_error(GNEP_ERR_INVALID_ARG, "rebuild needs the same structure and atom counts");
  if ((rc = load_batch(m, b, nl, st))) return rc;
  return finish_build(m, nl, st, false);
}

int gnep_nlist_info(const gnep_nlist* nl, int64_t* nr, int64_t* na) {
  if (!nl) return set_error(GNEP_ERR_INVALID_ARG, "NULL neighbour list");
  if (nr) *nr = nl->L[0].n;
  if (na) *na = nl->L[1].n;
  return GNEP_OK;
}

namespace {
__global__ void k_export_shift(int64_t n, const char4* __restrict__ s, int* __restrict__ o) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const char4 v = s[p];
  o[3 * p] = v.x; o[3 * p + 1] = v.y; o[3 * p + 2] = v.z;
}
}  // namespace

int gnep_nlist_export(const gnep_nlist* nl, int which, int32_t* off, int32_t* j, int32_t* shift, void* stream) {
  if (!nl || which < 0 || which > 1) return set_error(GNEP_ERR_INVALID_ARG, "bad list");
  cudaStream_t st = (cudaStream_t)stream;
  const PairList& P = nl->L[which];
  int rc = after_build(nl, st);
  if (rc) return rc;
  if ((rc = copy_out(off, P.off, sizeof(int) * ((size_t)nl->n_atoms + 1), st))) return rc;
  if (P.n == 0) return GNEP_OK;
  if ((rc = copy_out(j, P.j, sizeof(int) * (size_t)P.n, st))) return rc;
  if (shift) {
    int* tmp = nullptr;
    GNEP_CUDA(cudaMallocAsync(&tmp, sizeof(int) * 3 * (size_t)P.n, st));
    k_export_shift<<<blocks_for(P.n, 256), 256, 0, st>>>(P.n, P.shift, tmp);
    rc = copy_out(shift, tmp, sizeof(int) * 3 * (size_t)P.n, st);
    cudaFreeAsync(tmp, st);
    if (rc) return rc;
  }
  return GNEP_OK;
}

// ------------------------------------------------------------ evaluation

int gnep_descriptors(gnep_model* m, const gnep_nlist* nl_, float* G, void* stream) {
  int rc = use_nlist(m, nl_, (cudaStream_t)stream);
  if (rc) return rc;
  gnep_nlist* nl = const_cast<gnep_nlist*>(nl_);
  cudaStream_t st = (cudaStream_t)stream;
  StepArgs A{m, nl, st};
  if ((rc = run_descriptors(A, false))) return rc;
  return copy_out(G, nl->ws.G, sizeof(float) * (size_t)nl->n_atoms * m->shape.ndes, st);
}

int gnep_descriptors_noalloc(gnep_model* m, const gnep_nlist* nl_, float* G, void* stream) {
  int rc = use_nlist(m, nl_, (cudaStream_t)stream);
  if (rc) return rc;
  if (!G || !is_device_ptr(G))
    return set_error(GNEP_ERR_INVALID_ARG, "gnep_descriptors_noalloc writes G in place: G must be device memory");
  StepArgs A{m, const_cast<gnep_nlist*>(nl_), (cudaStream_t)stream};
  return run_descriptors_static(A, G);
}

int gnep_forward(gnep_model* m, const gnep_nlist* nl_, float* E_atom, double* E_struct, float* F,
                 double* W_struct, void* stream) {
  int rc = use_nlist(m, nl_, (cudaStream_t)stream);
  if (rc) return rc;
  gnep_nlist* nl = const_cast<gnep_nlist*>(nl_);
  cudaStream_t st = (cudaStream_t)stream;
  StepArgs A{m, nl, st};
  if ((rc = run_descriptors(A, true))) return rc;
  if ((rc = run_forward(A))) return rc;
  const size_t N = nl->n_atoms, S = nl->n_struct;
  if ((rc = copy_out(E_atom, nl->ws.Eatom, 4 * N, st))) return rc;
  if ((rc = copy_out(E_struct, nl->ws.Es, 8 * S, st))) return rc;
  if ((rc = copy_out(F, nl->ws.F, 12 * N, st))) return rc;
  return copy_out(W_struct, nl->ws.Ws, 48 * S, st);
}

int gnep_md_verlet(gnep_model* m, gnep_nlist* nl, double* pos, double* vel, const double* inv_mass, float* F,
                   double dt, double* E_struct, void* stream) {
  int rc = use_nlist(m, nl, (cudaStream_t)stream);
  if (rc) return rc;
  if (nl->n_atoms > 0 && (!is_device_ptr(pos) || !is_device_ptr(vel) || !is_device_ptr(inv_mass) || !is_device_ptr(F)))
    return set_error(GNEP_ERR_INVALID_ARG, "md: pos, vel, inv_mass and F must be device arrays");
  if (!(dt > 0.0)) return set_error(GNEP_ERR_INVALID_ARG, "md: dt must be positive");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t N = nl->n_atoms;
  if ((rc = md_kick_drift(nl, pos, vel, inv_mass, F, dt, st))) return rc;
  if (N > 0) GNEP_CUDA(cudaMemcpyAsync(nl->pos, pos, 24 * N, cudaMemcpyDeviceToDevice, st));
  if ((rc = finish_build(m, nl, st, true))) return rc;  // lists for the new positions
  StepArgs A{m, nl, st};
  if ((rc = run_descriptors(A, true))) return rc;
  if ((rc = run_forward(A))) return rc;
  if (N > 0) GNEP_CUDA(cudaMemcpyAsync(F, nl->ws.F, 12 * N, cudaMemcpyDeviceToDevice, st));
  if ((rc = md_kick(nl, vel, inv_mass, F, dt, st))) return rc;
  return copy_out(E_struct, nl->ws.Es, 8 * (size_t)nl->n_struct, st);
}

// Labels staged on the device, then descriptors, network, forces and the loss (Eqs. 1-12).
static int forward_loss(gnep_model* m, gnep_nlist* nl, const gnep_labels* y, cudaStream_t st) {
  if (!y || (nl->n_struct > 0 && (!y->energy || !y->virial)) || (nl->n_atoms > 0 && !y->force))
    return set_error(GNEP_ERR_INVALID_ARG, "incomplete labels");
  if (y->loss_form != GNEP_LOSS_MSE && y->loss_form != GNEP_LOSS_RMSE)
    return set_error(GNEP_ERR_INVALID_ARG, "unknown loss form");
  Workspace& w = nl->ws;
  const size_t N = nl->n_atoms, S = nl->n_struct;
  const double* le = y->energy;
  const float* lf = y->force;
  const double* lv = y->virial;
  if (!is_device_ptr(le)) { GNEP_CUDA(cudaMemcpyAsync(w.lab_e, le, 8 * S, cudaMemcpyDefault, st)); le = w.lab_e; }
  if (N > 0 && !is_device_ptr(lf)) { GNEP_CUDA(cudaMemcpyAsync(w.lab_f, lf, 12 * N, cudaMemcpyDefault, st)); lf = w.lab_f; }
  if (!is_device_ptr(lv)) { GNEP_CUDA(cudaMemcpyAsync(w.lab_v, lv, 48 * S, cudaMemcpyDefault, st)); lv = w.lab_v; }
  if (N == 0) lf = w.lab_f;
  StepArgs A{m, nl, st};
  A.loss_follows = true;
  int rc;
  if ((rc = run_descriptors(A, true))) return rc;
  if ((rc = run_forward(A))) return rc;
  return run_loss_impl(m, nl, le, lf, lv, y, st);
}

static int loss_grad_core(gnep_model* m, gnep_nlist* nl, const gnep_labels* y, cudaStream_t st) {
  int rc;
  if ((rc = forward_loss(m, nl, y, st))) return rc;
  StepArgs A{m, nl, st};
  if ((rc = run_backward(A))) return rc;
  return run_grad_reduce_impl(m, nl, y->lambda_l2, st);
}

int gnep_loss(gnep_model* m, const gnep_nlist* nl_, const gnep_labels* y, double* loss_terms, void* stream) {
  int rc = use_nlist(m, nl_, (cudaStream_t)stream);
  if (rc) return rc;
  gnep_nlist* nl = const_cast<gnep_nlist*>(nl_);
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = forward_loss(m, nl, y, st))) return rc;
  return copy_out(loss_terms, nl->ws.coef, 4 * sizeof(double), st);
}

int gnep_get_grad(gnep_model* m, double* dst, int64_t n, void* stream) {
  if (!m || !dst || n != m->n_params) return set_error(GNEP_ERR_INVALID_ARG, "gradient buffer");
  return copy_out(dst, m->grad, 8 * (size_t)n, (cudaStream_t)stream);
}

int gnep_set_grad(gnep_model* m, const double* src, int64_t n, void* stream) {
  if (!m || !src || n != m->n_params) return set_error(GNEP_ERR_INVALID_ARG, "gradient buffer");
  GNEP_CUDA(cudaMemcpyAsync(m->grad, src, 8 * (size_t)n, cudaMemcpyDefault, (cudaStream_t)stream));
  if (!is_device_ptr(src)) GNEP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return GNEP_OK;
}

int gnep_loss_grad(gnep_model* m, const gnep_nlist* nl_, const gnep_labels* y, double* loss_terms, float* grad,
                   void* stream) {
  int rc = use_nlist(m, nl_, (cudaStream_t)stream);
  if (rc) return rc;
  gnep_nlist* nl = const_cast<gnep_nlist*>(nl_);
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = loss_grad_core(m, nl, y, st))) return rc;
  if (grad) {
    if (is_device_ptr(grad)) {
      if ((rc = grad_to_float(m, grad, st))) return rc;
    } else {
      if ((rc = grad_to_float(m, nl->ws.gradf, st))) return rc;
      if ((rc = copy_out(grad, nl->ws.gradf, 4 * (size_t)m->n_params, st))) return rc;
    }
  }
  return copy_out(loss_terms, nl->ws.coef, 4 * sizeof(double), st);
}

int gnep_adam_step(gnep_model* m, double lr, double beta1, double beta2, double eps, double weight_decay,
                   void* stream) {
  if (!m) return set_error(GNEP_ERR_INVALID_ARG, "NULL model");
  return run_adam(m, nullptr, lr, beta1, beta2, eps, weight_decay, false, 0, 0, 0, 0, (cudaStream_t)stream);
}

int gnep_adam_step_scheduled(gnep_model* m, double lr_start, double lr_stop, int64_t n_warmup, int64_t n_total,
                             double beta1, double beta2, double eps, double weight_decay, void* stream) {
  if (!m || n_warmup < 0 || n_total < n_warmup) return set_error(GNEP_ERR_INVALID_ARG, "bad schedule");
  return run_adam(m, nullptr, 0.0, beta1, beta2, eps, weight_decay, true, lr_start, lr_stop, n_warmup, n_total,
                  (cudaStream_t)stream);
}

int gnep_get_step(gnep_model* m, int64_t* t, void* stream) {
  if (!m || !t) return set_error(GNEP_ERR_INVALID_ARG, "NULL argument");
  long long v = 0;
  GNEP_CUDA(cudaMemcpyAsync(&v, m->step, sizeof(long long), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  GNEP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  *t = v;
  return GNEP_OK;
}

double gnep_lr_schedule(double lr_start, double lr_stop, int64_t s, int64_t n_warmup, int64_t n_total) {
  if (s < n_warmup) return lr_stop + (double)s / (double)n_warmup * (lr_start - lr_stop);
  if (s > n_total) s = n_total;
  const double span = (double)(n_total - n_warmup);
  const double frac = span > 0 ? (double)(s - n_warmup) / span : 1.0;
  return lr_stop + (lr_start - lr_stop) * 0.5 * (1.0 + std::cos(M_PI * frac));
}

// ----------------------------------------------------------------- graphs

struct gnep_graph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  std::vector<const gnep_nlist*> nl;  // the batch of each captured step
  std::vector<uint64_t> gen;          // generation of each list at capture
};

// Captures the training steps b = 0 .. n-1 (forward, loss, backward, then the
// gradient with the scheduled Adam update in one kernel) on batches
// (nls[b], ys[b]) into one graph.
static int graph_create(gnep_model* m, const gnep_nlist* const* nls, const gnep_labels* ys, int n, double* loss_out,
                        double lr_start, double lr_stop, int64_t n_warmup, int64_t n_total, double beta1,
                        double beta2, double eps, double weight_decay, void* stream, gnep_graph** out) {
  if (!out || !nls || !ys || n < 1 || !stream)
    return set_error(GNEP_ERR_INVALID_ARG, "graph capture needs lists, labels, n >= 1 and a non-default stream");
  if (loss_out && !is_device_ptr(loss_out))
    return set_error(GNEP_ERR_INVALID_ARG, "graph capture needs a device loss buffer");
  for (int b = 0; b < n; ++b) {
    if (int rc = check_nlist(m, nls[b])) return rc;
    const gnep_labels& y = ys[b];
    if (!is_device_ptr(y.energy) || !is_device_ptr(y.force) || !is_device_ptr(y.virial))
      return set_error(GNEP_ERR_INVALID_ARG, "graph capture needs device labels");
    if (nls[b]->ready_ev) GNEP_CUDA(cudaEventSynchronize(nls[b]->ready_ev));  // a capture cannot wait on it
  }
  cudaStream_t st = (cudaStream_t)stream;
  GNEP_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  int rc = GNEP_OK;
  for (int b = 0; b < n && !rc; ++b) {
    gnep_nlist* nl = const_cast<gnep_nlist*>(nls[b]);
    rc = forward_loss(m, nl, &ys[b], st);
    StepArgs A{m, nl, st};
    if (!rc) rc = run_backward(A);
    if (!rc)
      rc = run_grad_adam(m, nl, ys[b].lambda_l2, loss_out ? loss_out + 4 * (size_t)b : nullptr, beta1, beta2, eps,
                         weight_decay, lr_start, lr_stop, n_warmup, n_total, st);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
  gnep_graph* gr = new gnep_graph();
  gr->g = g;
  for (int b = 0; b < n; ++b) {
    gr->nl.push_back(nls[b]);
    gr->gen.push_back(nls[b]->gen);
  }
  e = cudaGraphInstantiate(&gr->ge, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    delete gr;
    return cuda_error(e, "cudaGraphInstantiate");
  }
  *out = gr;
  return GNEP_OK;
}

int gnep_graph_create(gnep_model* m, const gnep_nlist* nl, const gnep_labels* y, double* loss_out,
                      double lr_start, double lr_stop, int64_t n_warmup, int64_t n_total, double beta1,
                      double beta2, double eps, double weight_decay, void* stream, gnep_graph** out) {
  if (!y) return set_error(GNEP_ERR_INVALID_ARG, "graph capture needs labels");
  return graph_create(m, &nl, y, 1, loss_out, lr_start, lr_stop, n_warmup, n_total, beta1, beta2, eps,
                      weight_decay, stream, out);
}

int gnep_graph_create_steps(gnep_model* m, const gnep_nlist* const* nls, const gnep_labels* ys, int32_t n_steps,
                            double* loss_out, double lr_start, double lr_stop, int64_t n_warmup, int64_t n_total,
                            double beta1, double beta2, double eps, double weight_decay, void* stream,
                            gnep_graph** out) {
  return graph_create(m, nls, ys, n_steps, loss_out, lr_start, lr_stop, n_warmup, n_total, beta1, beta2, eps,
                      weight_decay, stream, out);
}

int gnep_graph_launch(gnep_graph* g, void* stream) {
  if (!g) return set_error(GNEP_ERR_INVALID_ARG, "NULL graph");
  for (size_t b = 0; b < g->nl.size(); ++b)
    if (g->nl[b]->gen != g->gen[b])
      return set_error(GNEP_ERR_INVALID_ARG, "a neighbour list was rebuilt or retuned after this graph was captured");
  const gnep_nlist* last = nullptr;
  for (const gnep_nlist* nl : g->nl)
    if (nl != last) {  // consecutive repeats need one wait
      if (int rc = after_build(nl, (cudaStream_t)stream)) return rc;
      last = nl;
    }
  GNEP_CUDA(cudaGraphLaunch(g->ge, (cudaStream_t)stream));
  return GNEP_OK;
}

int gnep_graph_kernel_count(const gnep_graph* g, int32_t* n) {
  if (!g || !n) return set_error(GNEP_ERR_INVALID_ARG, "NULL argument");
  size_t nn = 0;
  GNEP_CUDA(cudaGraphGetNodes(g->g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) GNEP_CUDA(cudaGraphGetNodes(g->g, nodes.data(), &nn));
  int32_t k = 0;
  for (size_t i = 0; i < nn; ++i) {
    cudaGraphNodeType t;
    GNEP_CUDA(cudaGraphNodeGetType(nodes[i], &t));
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  *n = k;
  return GNEP_OK;
}

// ---------------------------------------------------------------- autotuner

namespace {

constexpr int kTuneKnobs = 9;  // na[0], ch[0], na[1], ch[1], cg_blocks, net_blocks, radial_lanes, net_tile, beside

int* knob(gnep_nlist* nl, int k) {
  switch (k) {
    case 0: return &nl->tune.na[0];
    case 1: return &nl->tune.ch[0];
    case 2: return &nl->tune.na[1];
    case 3: return &nl->tune.ch[1];
    case 4: return &nl->tune.cg_blocks;
    case 5: return &nl->tune.net_blocks;
    case 6: return &nl->tune.radial_lanes;
    case 7: return &nl->tune.net_tile;
    default: return &nl->tune.beside;
  }
}

// Effective value of each knob (the tuned value, or the built-in default).
void effective_tuning(const gnep_model* m, const gnep_nlist* nl, int32_t* v) {
  for (int w = 0; w < 2; ++w) {
    int na = 0, ch = 0;
    angular_tile_limits(m->shape, w, &na, &ch);
    v[2 * w] = (nl->tune.na[w] > 0 && nl->tune.na[w] < na) ? nl->tune.na[w] : na;
    v[2 * w + 1] = nl->tune.ch[w] > 0 ? nl->tune.ch[w] : ch;
  }
  v[4] = cgrad_blocks(nl);
  v[5] = nl->tune.net_blocks;  // 0: one block per tile up to the resident capacity
  v[6] = radial_lanes(nl);
  // the tensor-core network modes always take 128-atom tiles
  v[7] = (m->shape.lmax > 4 || m->precision == GNEP_PREC_FP32) ? net_tile_atoms(nl, m->shape.ns) : 128;
  v[8] = radial_beside(nl) ? 2 : 1;
}

// Median over `reps` of one loss + gradient evaluation (no update), in ms.
int time_step(gnep_model* m, gnep_nlist* nl, const gnep_labels* y, int reps, cudaStream_t st, float* ms) {
  cudaEvent_t a, b;
  GNEP_CUDA(cudaEventCreate(&a));
  GNEP_CUDA(cudaEventCreate(&b));
  std::vector<float> t;
  int rc = loss_grad_core(m, nl, y, st);  // warm-up
  for (int r = 0; r < reps && !rc; ++r) {
    cudaEventRecord(a, st);
    rc = loss_grad_core(m, nl, y, st);
    cudaEventRecord(b, st);
    if (!rc && cudaEventSynchronize(b) == cudaSuccess) {
      float x = 0.f;
      cudaEventElapsedTime(&x, a, b);
      t.push_back(x);
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  if (t.empty()) return set_error(GNEP_ERR_CUDA, "autotune timing failed");
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return GNEP_OK;
}

}  // namespace

int gnep_tuning_get(const gnep_model* m, const gnep_nlist* nl, int32_t* values) {
  if (check_nlist(m, nl) || !values) return set_error(GNEP_ERR_INVALID_ARG, "NULL argument or foreign list");
  effective_tuning(m, nl, values);
  return GNEP_OK;
}

int gnep_tuning_set(gnep_model* m, gnep_nlist* nl, const int32_t* values, void* stream) {
  int rc = use_nlist(m, nl, (cudaStream_t)stream);
  if (rc) return rc;
  if (!values) return set_error(GNEP_ERR_INVALID_ARG, "NULL values");
  for (int k = 0; k < kTuneKnobs; ++k)
    if (values[k] < 0 || values[k] > (k == 4 ? kCgBlocksMax : k == 5 ? kNetBlocks : 1 << 20))
      return set_error(GNEP_ERR_INVALID_ARG, "tuning value out of range");
  if (values[6] != 0 && values[6] != 4 && values[6] != 8 && values[6] != 16)
    return set_error(GNEP_ERR_INVALID_ARG, "radial lanes per atom must be 4, 8 or 16 (or 0)");
  if (values[7] != 0 && values[7] != 32 && values[7] != 128)
    return set_error(GNEP_ERR_INVALID_ARG, "atoms per network tile must be 32 or 128 (or 0)");
  if (values[8] > 2)
    return set_error(GNEP_ERR_INVALID_ARG, "radial sweep placement must be 1 (in turn) or 2 (beside) (or 0)");
  for (int k = 0; k < kTuneKnobs; ++k) *knob(nl, k) = values[k];
  ++nl->gen;
  if (nl->n_atoms == 0) return GNEP_OK;
  return build_angular_tiles(m, nl, (cudaStream_t)stream);
}

int gnep_autotune(gnep_model* m, gnep_nlist* nl, const gnep_labels* y, int reps, void* stream) {
  int rc = use_nlist(m, nl, (cudaStream_t)stream);
  if (rc) return rc;
  if (!y) return set_error(GNEP_ERR_INVALID_ARG, "NULL labels");
  if (nl->n_atoms == 0) return GNEP_OK;
  if (reps < 1) reps = 3;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t cur[kTuneKnobs];
  effective_tuning(m, nl, cur);
  // candidate values per knob; the compiled atom maxima bound the atom caps
  const int na0 = cur[0], na1 = cur[2];
  const std::vector<std::vector<int>> cand = {
      {na0, na0 / 2, na0 / 4},  {64, 128, 256, 384, 512},
      {na1, na1 / 2, na1 / 4},  {32, 48, 64, 96, 128, 192},
      {152, 304, 456, 608},     {0, 152, 304},
      {4, 8, 16},               {32, 128},
      {1, 2}};
  for (int k = 0; k < kTuneKnobs; ++k) *knob(nl, k) = cur[k];
  ++nl->gen;
  if ((rc = build_angular_tiles(m, nl, st))) return rc;
  float best = 0.f;
  if ((rc = time_step(m, nl, y, reps, st, &best))) return rc;
  for (int k = 0; k < kTuneKnobs; ++k) {  // coordinate descent, one pass
    const int keep = *knob(nl, k);
    int pick = keep;
    for (int v : cand[k]) {
      if ((v < 1 && k != 5) || v == keep) continue;
      *knob(nl, k) = v;
      if (k < 4 && (rc = build_angular_tiles(m, nl, st))) return rc;
      float t = 0.f;
      if ((rc = time_step(m, nl, y, reps, st, &t))) return rc;
      if (t < 0.99f * best) {
        best = t;
        pick = v;
      }
    }
    *knob(nl, k) = pick;
    if (k < 4 && (rc = build_angular_tiles(m, nl, st))) return rc;
  }
  return GNEP_OK;
}

int gnep_graph_destroy(gnep_graph* g) {
  if (!g) return GNEP_OK;
  if (g->ge) cudaGraphExecDestroy(g->ge);
  if (g->g) cudaGraphDestroy(g->g);
  delete g;
  return GNEP_OK;
}

// ------------------------------------------------------------ checkpoints

namespace {
uint32_t crc32_update(uint32_t crc, const void* data, size_t n) {
  static uint32_t table[256];
  static bool init = false;
  if (!init) {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int k = 0; k < 8; ++k) c = (c & 1) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
      table[i] = c;
    }
    init = true;
  }
  const unsigned char* p = (const unsigned char*)data;
  crc = ~crc;
  for (size_t i = 0; i < n; ++i) crc = table[(crc ^ p[i]) & 0xFF] ^ (crc >> 8);
  return ~crc;
}

struct CkptHeader {
  char magic[8];
  uint32_t version;
  int32_t shape[9];
  double rcr, rca;
  int64_t n_params;
  int64_t step;
};
}  // namespace

int gnep_save(gnep_model* m, const char* path) {
  if (!m || !path) return set_error(GNEP_ERR_INVALID_ARG, "NULL argument");
  const size_t n = (size_t)m->n_params, d = (size_t)m->shape.ndes;
  std::vector<float> p(n), mm(n), vv(n), sc(d);
  CkptHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, "GNEPCKPT", 8);
  h.version = 1;
  const Shape& s = m->shape;
  const int32_t sh[9] = {s.ns, s.nqr, s.kr, s.nqa, s.ka, s.lmax, s.fb, s.H, s.ndes};
  memcpy(h.shape, sh, sizeof(sh));
  h.rcr = m->rcr;
  h.rca = m->rca;
  h.n_params = m->n_params;
  long long stp = 0;
  GNEP_CUDA(cudaDeviceSynchronize());
  GNEP_CUDA(cudaMemcpy(p.data(), m->params, 4 * n, cudaMemcpyDeviceToHost));
  GNEP_CUDA(cudaMemcpy(mm.data(), m->adam_m, 4 * n, cudaMemcpyDeviceToHost));
  GNEP_CUDA(cudaMemcpy(vv.data(), m->adam_v, 4 * n, cudaMemcpyDeviceToHost));
  GNEP_CUDA(cudaMemcpy(sc.data(), m->scale, 4 * d, cudaMemcpyDeviceToHost));
  GNEP_CUDA(cudaMemcpy(&stp, m->step, sizeof(long long), cudaMemcpyDeviceToHost));
  h.step = stp;
  uint32_t crc = 0;
  crc = crc32_update(crc, &h, sizeof(h));
  crc = crc32_update(crc, p.data(), 4 * n);
  crc = crc32_update(crc, sc.data(), 4 * d);
  crc = crc32_update(crc, mm.data(), 4 * n);
  crc = crc32_update(crc, vv.data(), 4 * n);
  FILE* f = fopen(path, "wb");
  if (!f) return set_error(GNEP_ERR_INVALID_ARG, std::string("cannot open ") + path);
  bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(p.data(), 4, n, f) == n && fwrite(sc.data(), 4, d, f) == d &&
            fwrite(mm.data(), 4, n, f) == n && fwrite(vv.data(), 4, n, f) == n && fwrite(&crc, 4, 1, f) == 1;
  ok = (fclose(f) == 0) && ok;
  if (!ok) return set_error(GNEP_ERR_INVALID_ARG, std::string("write failed: ") + path);
  return GNEP_OK;
}

int gnep_load(gnep_model* m, const char* path) {
  if (!m || !path) return set_error(GNEP_ERR_INVALID_ARG, "NULL argument");
  FILE* f = fopen(path, "rb");
  if (!f) return set_error(GNEP_ERR_INVALID_ARG, std::string("cannot open ") + path);
  CkptHeader h;
  const size_t n = (size_t)m->n_params, d = (size_t)m->shape.ndes;
  std::vector<float> p(n), mm(n), vv(n), sc(d);
  uint32_t crc_file = 0;
  bool ok = fread(&h, sizeof(h), 1, f) == 1;
  const Shape& s = m->shape;
  const int32_t sh[9] = {s.ns, s.nqr, s.kr, s.nqa, s.ka, s.lmax, s.fb, s.H, s.ndes};
  if (ok) ok = memcmp(h.magic, "GNEPCKPT", 8) == 0 && h.version == 1 && memcmp(h.shape, sh, sizeof(sh)) == 0 &&
               h.n_params == m->n_params && h.rcr == m->rcr && h.rca == m->rca;
  if (ok) ok = fread(p.data(), 4, n, f) == n && fread(sc.data(), 4, d, f) == d && fread(mm.data(), 4, n, f) == n &&
               fread(vv.data(), 4, n, f) == n && fread(&crc_file, 4, 1, f) == 1;
  char extra;
  if (ok) ok = fread(&extra, 1, 1, f) == 0;
  fclose(f);
  if (ok) {
    uint32_t crc = 0;
    crc = crc32_update(crc, &h, sizeof(h));
    crc = crc32_update(crc, p.data(), 4 * n);
    crc = crc32_update(crc, sc.data(), 4 * d);
    crc = crc32_update(crc, mm.data(), 4 * n);
    crc = crc32_update(crc, vv.data(), 4 * n);
    ok = crc == crc_file;
  }
  if (!ok) return set_error(GNEP_ERR_CHECKPOINT_CORRUPT, std::string("checkpoint failed validation: ") + path);
  long long stp = h.step;
  GNEP_CUDA(cudaDeviceSynchronize());
  GNEP_CUDA(cudaMemcpy(m->params, p.data(), 4 * n, cudaMemcpyHostToDevice));
  GNEP_CUDA(cudaMemcpy(m->adam_m, mm.data(), 4 * n, cudaMemcpyHostToDevice));
  GNEP_CUDA(cudaMemcpy(m->adam_v, vv.data(), 4 * n, cudaMemcpyHostToDevice));
  GNEP_CUDA(cudaMemcpy(m->scale, sc.data(), 4 * d, cudaMemcpyHostToDevice));
  GNEP_CUDA(cudaMemcpy(m->step, &stp, sizeof(long long), cudaMemcpyHostToDevice));
  return GNEP_OK;
}

// -------------------------------------------------------------- profiling

static const char* g_stage_names[64];
static int g_stage_count = 0;

int gnep_profile_step(gnep_model* m, const gnep_nlist* nl_, const gnep_labels* y, float* stage_ms,
                      int32_t cap, int32_t* n_stages, void* stream) {
  int rc = use_nlist(m, nl_, (cudaStream_t)stream);
  if (rc) return rc;
  if (!stage_ms || !n_stages || cap < 1) return set_error(GNEP_ERR_INVALID_ARG, "bad output arrays");
  gnep_nlist* nl = const_cast<gnep_nlist*>(nl_);
  cudaStream_t st = (cudaStream_t)stream;
  for (int q = 0; q < 64; ++q) GNEP_CUDA(cudaEventCreate(&g_prof.ev[q]));
  g_prof.st = st;
  g_prof.n = 0;
  GNEP_CUDA(cudaEventRecord(g_prof.ev[0], st));
  g_prof.on = true;
  rc = loss_grad_core(m, nl, y, st);
  if (!rc) rc = run_adam(m, nullptr, 1e-4, 0.9, 0.999, 1e-8, 0.0, false, 0, 0, 0, 0, st);
  g_prof.on = false;
  cudaError_t e = cudaStreamSynchronize(st);
  if (!rc && e != cudaSuccess) rc = cuda_error(e, "profile step");
  if (!rc) {
    const int n = g_prof.n < cap ? g_prof.n : cap;
    for (int q = 0; q < n; ++q) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, g_prof.ev[q], g_prof.ev[q + 1]);
      stage_ms[q] = ms;
      g_stage_names[q] = g_prof.names[q];
    }
    g_stage_count = n;
    *n_stages = n;
  }
  for (int q = 0; q < 64; ++q) cudaEventDestroy(g_prof.ev[q]);
  return rc;
}

const char* gnep_profile_stage_name(int32_t i) {
  return (i >= 0 && i < g_stage_count) ? g_stage_names[i] : "";
}

// ------------------------------------------------------- data parallelism

int gnep_shard_loss_weights(double lambda_e, double lambda_f, double lambda_v, double lambda_l2, int32_t loss_form,
                            int64_t local_struct, int64_t local_atoms, int64_t total_struct, int64_t total_atoms,
                            const double* mse_total, int32_t rank, double* out) {
  if (!out || local_struct < 0 || local_atoms < 0 || total_struct < local_struct || total_atoms < local_atoms)
    return set_error(GNEP_ERR_INVALID_ARG, "shard weights: bad counts or NULL output");
  if (loss_form != GNEP_LOSS_MSE && loss_form != GNEP_LOSS_RMSE)
    return set_error(GNEP_ERR_INVALID_ARG, "shard weights: unknown loss form");
  if (loss_form == GNEP_LOSS_RMSE && !mse_total)
    return set_error(GNEP_ERR_INVALID_ARG, "shard weights: the RMSE form needs the whole-batch MSE terms");
  // Eqs. 10-12 normalise by the whole batch: a shard's share of each term is
  // its fraction of the structures (energy, virial) or atoms (forces)
  const double ws = total_struct > 0 ? (double)local_struct / (double)total_struct : 0.0;
  const double wa = total_atoms > 0 ? (double)local_atoms / (double)total_atoms : 0.0;
  double w[3] = {lambda_e * ws, lambda_f * wa, lambda_v * ws};
  if (loss_form == GNEP_LOSS_RMSE)  // d sqrt(L_x) = dL_x / (2 sqrt(L_x)), 0 where L_x = 0
    for (int x = 0; x < 3; ++x) w[x] *= mse_total[x] > 0.0 ? 0.5 / std::sqrt(mse_total[x]) : 0.0;
  out[0] = w[0];
  out[1] = w[1];
  out[2] = w[2];
  out[3] = rank == 0 ? lambda_l2 : 0.0;  // the L2 term is carried once
  return GNEP_OK;
}

int gnep_shard_mse_partials(const double* local_mse, int64_t local_struct, int64_t local_atoms, double* out) {
  if (!local_mse || !out || local_struct < 0 || local_atoms < 0)
    return set_error(GNEP_ERR_INVALID_ARG, "mse partials: bad counts or NULL pointer");
  out[0] = local_mse[0] * (double)local_struct;      // sum of squared energy residuals
  out[1] = local_mse[1] * 3.0 * (double)local_atoms;  // ... force components
  out[2] = local_mse[2] * 6.0 * (double)local_struct; // ... virial components
  out[3] = (double)local_struct;
  out[4] = (double)local_atoms;
  return GNEP_OK;
}

int gnep_shard_mse_total(const double* sums, double* out) {
  if (!sums || !out) return set_error(GNEP_ERR_INVALID_ARG, "mse total: NULL pointer");
  const double S = sums[3], N = sums[4];
  out[0] = S > 0 ? sums[0] / S : 0.0;
  out[1] = N > 0 ? sums[1] / (3.0 * N) : 0.0;
  out[2] = S > 0 ? sums[2] / (6.0 * S) : 0.0;
  return GNEP_OK;
}

// ----------------------------------------------------------------- status

int gnep_selftest_wait_timeout(gnep_model* m, int64_t limit_ns, void* stream) {
  if (!m || limit_ns < 1000 || limit_ns > 2000000000LL)
    return set_error(GNEP_ERR_INVALID_ARG, "selftest: limit_ns must lie in [1e3, 2e9]");
  cudaSetDevice(m->device);
  return wait_selftest(m, (uint64_t)limit_ns, (cudaStream_t)stream);
}

int gnep_sync_status(gnep_model* m, void* stream) {
  if (!m) return set_error(GNEP_ERR_INVALID_ARG, "NULL model");
  cudaStream_t st = (cudaStream_t)stream;
  GNEP_CUDA(cudaStreamSynchronize(st));
  GNEP_CUDA(cudaGetLastError());
  int flag = 0;
  GNEP_CUDA(cudaMemcpy(&flag, m->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) GNEP_CUDA(cudaMemset(m->err, 0, sizeof(int)));
  if (flag & kErrNonFinite) return set_error(GNEP_ERR_NONFINITE, "loss was not finite; the update was skipped");
  if (flag & kErrTimeout) return set_error(GNEP_ERR_TIMEOUT, "a device-side wait gave up");
  if (flag & kErrRevMissing) return set_error(GNEP_ERR_INVALID_ARG, "neighbour lists are not symmetric (internal error)");
  if (flag) return set_error(GNEP_ERR_INVALID_ARG, "device reported an invalid input");
  return GNEP_OK;
}

}  // extern "C"
