// Internal structures of libgnep (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/gnep.h"

namespace gnep {

// Compile-time maxima of the library.
constexpr int kMaxHidden = 128;
constexpr int kMaxDes = 64;
constexpr int kLmax = 4;

// Runtime shape of a model.
struct Shape {
  int ns, nqr, kr, nqa, ka, lmax, fb, H, ndes;
  bool operator==(const Shape& o) const {
    return ns == o.ns && nqr == o.nqr && kr == o.kr && nqa == o.nqa && ka == o.ka &&
           lmax == o.lmax && fb == o.fb && H == o.H;
  }
};

// Everything a kernel needs to know about the model, passed by value.
struct DevModel {
  int ns, nqr, kr, nqa, ka, H, ndes;
  int net_size;      // ndes*H + 2H + 1
  int off_cR, off_cA;
  long long n_params;
  float rcr_inv, rca_inv;
  const float* params;
  const float* scale;
};

// One list of Eq. 2 in CSR form.
struct PairList {
  int64_t n = 0, cap = 0;
  int* off = nullptr;      // [N+1]
  int* j = nullptr;        // [n] neighbour (global atom index)
  int* owner = nullptr;    // [n] central atom i
  int* rev = nullptr;      // [n] index of (j, i, -shift) (angular list only)
  float4* rij = nullptr;   // [n] r_ij (x, y, z), w = species of j (as float)
  char4* shift = nullptr;  // [n] image (na, nb, nc, 0)
};

// Per-step device workspace of one batch (sized at build, reused every step).
struct Workspace {
  float *G = nullptr, *Ep = nullptr, *Eatom = nullptr;
  float *S = nullptr, *FR = nullptr, *chat = nullptr;
  float4* dA = nullptr;
  float *F = nullptr, *Wat = nullptr;
  double *Es = nullptr, *Ws = nullptr;
  float4* a = nullptr;                 // force residual coefficients a_i
  float *es = nullptr, *Bs = nullptr;  // energy and virial residual coefficients
  float *Gd = nullptr, *Sd = nullptr, *FRd = nullptr, *Gb = nullptr;
  float4* wij = nullptr;               // per angular pair: tangent direction (a_j - a_i) + B_s r_ij
  float* net_part = nullptr;           // network-gradient partials [blocks][species][net_size]
  float* cpart = nullptr;              // coefficient-gradient partials [blocks][c^R + c^A]
  int net_blocks = 0;                  // blocks that wrote net_part in the last backward pass
  double* red = nullptr;               // loss partials
  int64_t red_len = 0;
  double* lab_e = nullptr;             // staged labels
  float* lab_f = nullptr;
  double* lab_v = nullptr;
  double* coef = nullptr;              // [8] loss scalars for the residual kernels
  float* gradf = nullptr;              // FP32 copy of the gradient for host output
};

}  // namespace gnep

struct gnep_nlist {
  gnep::Shape shape;
  int device = 0;
  int n_struct = 0, n_atoms = 0;
  double rcr = 0, rca = 0;
  int* struct_off = nullptr;   // device [S+1]
  int* type = nullptr;         // device [N]
  double* pos = nullptr;       // device [N*3]
  double* cell = nullptr;      // device [S*9]
  int* atom_struct = nullptr;  // device [N]
  int* perm = nullptr;         // device [N] atoms grouped by species
  int species_off[9] = {0};    // host [ns+1]
  gnep::PairList L[2];         // radial, angular
  // Atom tiles for the angular sweeps: consecutive atoms, at most NA atoms and
  // CH angular pairs per tile (a single atom above CH pairs gets its own tile).
  // [0] wide tiles (descriptor sweep), [1] narrow tiles (force, tangent, c-gradient).
  int* atile[2] = {nullptr, nullptr};
  int natile[2] = {0, 0};
  int64_t atile_cap[2] = {0, 0};  // allocated tile-bound slots
  // Launch shapes chosen by gnep_autotune (0 = built-in default): atoms and
  // pairs per tile of each tile set, persistent blocks of the c-gradient sweep
  // and of the network kernels, lanes per atom of the radial sweeps (4, 8, 16),
  // atoms per FP32 network tile (32, 128) and where the radial sweeps run
  // (1: in turn with the angular ones, 2: beside them on the second stream).
  struct Tuning {
    int na[2] = {0, 0}, ch[2] = {0, 0}, cg_blocks = 0, net_blocks = 0, radial_lanes = 0, net_tile = 0, beside = 0;
  } tune;
  uint64_t gen = 0;  // bumped whenever lists or tiles change (captured graphs check it)
  std::vector<int> host_types;  // species of the last build (host copy)
  bool types_changed = true;
  long long* host_aoff = nullptr;    // pinned: angular list offsets of the last build (for the tiles)
  int64_t host_aoff_cap = 0, host_aoff_n = 0;
  int* tile_host = nullptr;          // pinned staging of the tile bounds (both tile sets)
  int64_t tile_host_cap = 0;
  cudaEvent_t tile_ev = nullptr;     // the last upload from tile_host
  cudaEvent_t ready_ev = nullptr;    // the end of the last build's device work (consumers wait on it)
  // A second stream for the radial sweeps of small batches, with the events
  // that fork it from the caller's stream and join it back.
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  gnep::Workspace ws;
  void* ws_mem = nullptr;      // one allocation carved into the workspace
  int64_t ws_pairs[2] = {-1, -1};  // pair counts the workspace was sized for
};

struct gnep_model {
  gnep::Shape shape;
  int device = 0;
  double rcr = 0, rca = 0;
  int precision = GNEP_PREC_FP32;
  int64_t n_params = 0;
  int net_size = 0, off_cR = 0, off_cA = 0;
  float* params = nullptr;  // device [n_params]
  float* scale = nullptr;   // device [ndes]
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  double* grad = nullptr;   // device [n_params]
  long long* step = nullptr;  // device update count
  int* err = nullptr;       // device error flag, then block counters of the Adam (err[1]) and loss (err[2]) kernels
  gnep::DevModel dev() const {
    gnep::DevModel d;
    d.ns = shape.ns; d.nqr = shape.nqr; d.kr = shape.kr; d.nqa = shape.nqa; d.ka = shape.ka;
    d.H = shape.H; d.ndes = shape.ndes; d.net_size = net_size; d.off_cR = off_cR;
    d.off_cA = off_cA; d.n_params = n_params;
    d.rcr_inv = (float)(1.0 / rcr); d.rca_inv = (float)(1.0 / rca);
    d.params = params; d.scale = scale;
    return d;
  }
};

namespace gnep {

// Device error flag bits.
enum : int { kErrNonFinite = 1, kErrUnwrapped = 2, kErrRevMissing = 4, kErrTimeout = 8 };

// Error reporting helpers (api.cu).
int set_error(int code, const std::string& msg);
int cuda_error(cudaError_t e, const char* what);
#define GNEP_CUDA(call)                                        \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return gnep::cuda_error(e_, #call); \
  } while (0)
// Programmatic dependent launch.  The kernels of a step are launched with
// launch_pdl, so a kernel's blocks may be scheduled (and reach their first
// instruction) while the previous kernel's last blocks still run; every such
// kernel executes GNEP_PDL_WAIT before its first access to device memory,
// which returns once the previous kernel has completed and its writes are
// visible.  Outside a dependent launch the wait returns at once.
#define GNEP_PDL_WAIT() asm volatile("griddepcontrol.wait;" ::: "memory")

// launch_on launches as a dependent of the stream's previous kernel when `pdl`
// is set, else as an ordinary launch.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_on(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  return launch_on(true, kern, grid, block, smem, st, std::forward<Args>(args)...);
}

#define GNEP_CHECK_LAUNCH(what)                                \
  do {                                                         \
    cudaError_t e_ = cudaGetLastError();                       \
    if (e_ != cudaSuccess) return gnep::cuda_error(e_, what);  \
  } while (0)

// neighbors.cu
int build_lists(gnep_model* m, gnep_nlist* nl, cudaStream_t st);

// Shape-specialised step (sweeps.cu).
struct StepArgs {
  const gnep_model* m;
  gnep_nlist* nl;
  cudaStream_t st;
  bool loss_follows = false;  // the loss kernel forms the per-structure sums (fused)
};
bool shape_supported(const Shape& s);
int run_descriptors(const StepArgs& a, bool with_mlp);
int run_forward(const StepArgs& a);
int run_backward(const StepArgs& a);

int shape_setup(const Shape& s);
int run_descriptors_static(const StepArgs& a, float* G);
int md_kick_drift(const gnep_nlist* nl, double* pos, double* vel, const double* inv_mass, const float* F, double dt,
                  cudaStream_t st);
int md_kick(const gnep_nlist* nl, double* vel, const double* inv_mass, const float* F, double dt, cudaStream_t st);
int cgrad_blocks(const gnep_nlist* nl);
int sm_count();                                   // SMs of this GPU
int radial_lanes(const gnep_nlist* nl);           // lanes per atom of the radial sweeps
bool radial_beside(const gnep_nlist* nl);         // radial sweeps on the list's second stream
int net_tile_atoms(const gnep_nlist* nl, int ns); // atoms per FP32 network tile
// Persistent blocks of a network kernel: `fit` (resident capacity, capped at the
// tile count) or the tuned count, whichever is smaller.
inline int net_blocks(const gnep_nlist* nl, int fit) {
  const int t = nl->tune.net_blocks;
  return (t > 0 && t < fit) ? t : fit;
}
void angular_tile_limits(const Shape& s, int which, int* na, int* ch);
constexpr int kCgBlocksMax = 608;

// train.cu
int64_t loss_partial_doubles(int n_struct);
int run_loss_impl(const gnep_model* m, gnep_nlist* nl, const double* le, const float* lf, const double* lv,
                  const gnep_labels* y, cudaStream_t st);
int run_grad_reduce_impl(const gnep_model* m, gnep_nlist* nl, double lambda_l2, cudaStream_t st);
int grad_to_float(const gnep_model* m, float* dst, cudaStream_t st);
int run_adam(gnep_model* m, const double* lr_dev, double lr, double b1, double b2, double eps,
             double wd, bool scheduled, double lr_start, double lr_stop, int64_t nw, int64_t nt,
             cudaStream_t st);
// The gradient, the loss terms to loss_out (device, may be NULL) and the
// scheduled Adam update of a training step in one launch.
int run_grad_adam(gnep_model* m, gnep_nlist* nl, double lambda_l2, double* loss_out, double b1, double b2,
                  double eps, double wd, double lr_start, double lr_stop, int64_t nw, int64_t nt, cudaStream_t st);
int run_scale(gnep_model* m, gnep_nlist* nl, cudaStream_t st);
int run_species_perm(gnep_nlist* nl, cudaStream_t st);

// Workspace sizing (api.cu).
int alloc_workspace(gnep_model* m, gnep_nlist* nl);
void free_workspace(gnep_nlist* nl);

// Stage profiler: when on, an event is recorded after every kernel launch of
// a step (api.cu: gnep_profile_step).  Not thread-safe; off by default.
struct Profiler {
  bool on = false;
  cudaStream_t st = nullptr;
  int n = 0;
  cudaEvent_t ev[64];
  const char* names[64];
};
extern Profiler g_prof;
inline void stage(const char* name) {
  if (!g_prof.on || g_prof.n >= 63) return;
  cudaEventRecord(g_prof.ev[g_prof.n + 1], g_prof.st);
  g_prof.names[g_prof.n] = name;
  g_prof.n++;
}

// Small launch helpers.
inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace gnep
