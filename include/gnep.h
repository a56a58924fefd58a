/*
 * gnep.h -- C ABI of libgnep, gradient-optimised NEP training on one sm_103a GPU.
 *
 * The library evaluates, for a packed batch of periodic structures, the NEP
 * descriptor (radial Chebyshev terms, Eqs. 5-6 with App. A; angular terms from
 * real solid harmonics with l <= 4, Eqs. 7-8 with App. B; an optional 4-body
 * term), a one-hidden-layer tanh network per element (D1.1), energies, forces
 * and virials (Eqs. 1, 3, 4), the weighted energy/force/virial loss (Eqs. 9-12)
 * and its exact gradient with respect to every network weight and descriptor
 * coefficient c_nk^IJ (Eqs. 13-16, D1.18-D1.21), then an Adam update with the
 * warm-up + cosine learning rate of Eq. 17.  Every step runs in the library's
 * own CUDA kernels; there is no CPU fallback.
 *
 * Conventions for every entry point:
 *  - Return value: GNEP_OK (0) on success, a negative gnep_status otherwise;
 *    gnep_last_error() then gives a message (thread-local, valid until the next
 *    call on the same thread).
 *  - Pointers to arrays may be host or device memory; the library tells them
 *    apart (cudaPointerGetAttributes).  Host inputs are copied to library-owned
 *    device memory on `stream`; host outputs are written by a copy on `stream`
 *    that has completed when the call returns.  Device outputs are written
 *    asynchronously on `stream`.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    ordered on it; the library never synchronises the device except where a
 *    host output or a size is needed (documented per call).
 *  - The library owns models, neighbour lists and their workspaces; the caller
 *    owns every batch, label and output buffer.
 *  - Errors detected inside kernels (non-finite loss) set a device flag that
 *    gnep_sync_status() reports; a step whose loss is not finite leaves the
 *    parameters unchanged.
 *  - Positions are Cartesian (A) and must lie inside their cell (fractional
 *    coordinates in [0, 1)).  Cells are row vectors a, b, c.
 */
#ifndef GNEP_H
#define GNEP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GNEP_ABI_VERSION 5

typedef enum {
  GNEP_OK = 0,
  GNEP_ERR_INVALID_ARG = -1,       /* bad argument or inconsistent sizes */
  GNEP_ERR_OOM = -2,               /* device or host allocation failed */
  GNEP_ERR_CUDA = -3,              /* a CUDA runtime call failed */
  GNEP_ERR_NEIGHBOR_OVERFLOW = -4, /* more pairs than 32-bit indices hold */
  GNEP_ERR_NONFINITE = -5,         /* loss or gradient not finite; step skipped */
  GNEP_ERR_TIMEOUT = -6,           /* a bounded device-side wait gave up */
  GNEP_ERR_CHECKPOINT_CORRUPT = -7,/* checkpoint failed validation */
  GNEP_ERR_UNSUPPORTED = -8        /* hyper-parameters without a compiled kernel */
} gnep_status;

/* Arithmetic of the network contractions (D1.1-D1.10) only.  FP32: CUDA-core
 * FP32.  TF32 / BF16: tcgen05 tensor-core products with TF32 / BF16 operands
 * and FP32 accumulation.  In every mode the per-pair geometry is FP32, the
 * descriptor, force, tangent and coefficient-gradient contractions are
 * FP32-accurate (split-TF32 tensor-core products), and the cross-atom sums of
 * energies, virials, loss and gradient are FP64 above FP32 leaves. */
enum { GNEP_PREC_FP32 = 0, GNEP_PREC_TF32 = 1, GNEP_PREC_BF16 = 2 };
/* GNEP_LOSS_MSE: Eq. 9 with Eqs. 10-12.  GNEP_LOSS_RMSE: the same weighted sum
 * of the square roots of Eqs. 10-12. */
enum { GNEP_LOSS_MSE = 0, GNEP_LOSS_RMSE = 1 };
/* Neighbour list selector for gnep_nlist_export. */
enum { GNEP_LIST_RADIAL = 0, GNEP_LIST_ANGULAR = 1 };

typedef struct gnep_model gnep_model; /* opaque */
typedef struct gnep_nlist gnep_nlist; /* opaque: one batch's geometry, lists, workspace */

/* A packed batch of n_struct periodic structures, n_atoms atoms in total. */
typedef struct {
  int32_t n_struct;
  int32_t n_atoms;
  const int32_t *struct_off; /* [n_struct+1] strictly increasing atom offsets, [0] = 0 */
  const double *pos;         /* [n_atoms*3] positions (A), wrapped into the cell */
  const int32_t *type;       /* [n_atoms] species index, 0..n_species-1 */
  const double *cell;        /* [n_struct*9] cell rows a, b, c (A) */
} gnep_batch;

/* Labels and loss weights (Eqs. 9-12). */
typedef struct {
  const double *energy; /* [n_struct] per-atom energy E_s/N_s (eV/atom) */
  const float *force;   /* [n_atoms*3] forces (eV/A) */
  const double *virial; /* [n_struct*6] per-atom virial W_s/N_s, xx yy zz xy yz zx */
  double lambda_e, lambda_f, lambda_v; /* Eq. 9 weights */
  double lambda_l2;     /* L2 term lambda_l2 * sum(theta^2) / N_par */
  int32_t loss_form;    /* GNEP_LOSS_MSE or GNEP_LOSS_RMSE */
} gnep_labels;

/* ---------------------------------------------------------------- model */

/* Create a model (Sec. II.B-C; Eq. 6 basis, Eq. 8 harmonics, D1.1 network).
 * n_species        species count (the library compiles kernels for 2)
 * species_z        [n_species] atomic numbers, informative (may be NULL)
 * rc_radial/angular cut-offs r_c^R, r_c^A (A), 0 < rc_angular <= rc_radial
 * n_max_*          descriptors per family are n_max + 1 (n = 0..n_max)
 * basis_*          basis functions per family are basis + 1 (k = 0..N_bas, Eq. 6)
 * l_max            angular degree, up to 8 (App. B: B1-B8).  Compiled shapes
 *                  (n_max/basis both families, 4-body, l_max): 4/8 without
 *                  4-body, l_max 4; 8/12 with and without 4-body, l_max 4; 4/8 no 4-body, l_max 6;
 *                  4/8 with 4-body, l_max 8.  l_max > 4 runs the FP32 network only
 * four_body        0/1: add one tr(Q_n^3) descriptor per angular channel n
 * hidden           hidden neurons N_neu (<= 128)
 * seed             parameters are drawn U(-0.5, 0.5) from this seed
 * precision        GNEP_PREC_* for the network contractions
 * Errors: INVALID_ARG, UNSUPPORTED (no kernel for this shape), CUDA, OOM. */
int gnep_create(gnep_model **out, int n_species, const int *species_z,
                double rc_radial, double rc_angular, int n_max_radial,
                int n_max_angular, int basis_radial, int basis_angular,
                int l_max, int four_body, int hidden, uint64_t seed,
                int precision);
int gnep_destroy(gnep_model *m);
int gnep_set_precision(gnep_model *m, int precision);

/* Parameter count and descriptor length N_des = N_q^R + N_q^A l_max (+ N_q^A). */
int gnep_num_params(const gnep_model *m, int64_t *n);
int gnep_num_descriptors(const gnep_model *m, int32_t *n);

/* Parameter vector (FP32, n = gnep_num_params) in this layout:
 *   for each species e: W0[hidden][N_des] (D1.2), b0[hidden], w1[hidden], b1
 *   then c^R[I][J][n][k] (Eq. 6, radial) then c^A[I][J][n][k] (angular).
 * get: synchronises `stream` when dst is host memory. */
int gnep_get_params(gnep_model *m, float *dst, int64_t n, void *stream);
int gnep_set_params(gnep_model *m, const float *src, int64_t n, void *stream);

/* Fixed per-component input scale s (the network sees s_v G_v; not trained).
 * compute: s_v = 1 / (max_v - min_v) over the batch's atoms with the model's
 * current coefficients (1 where max = min); synchronises `stream`. */
int gnep_set_descriptor_scale(gnep_model *m, const float *scale, int32_t n, void *stream);
int gnep_get_descriptor_scale(gnep_model *m, float *scale, int32_t n, void *stream);
int gnep_compute_descriptor_scale(gnep_model *m, const gnep_nlist *nl, void *stream);

/* ------------------------------------------------------------ neighbours */

/* Build the radial and angular neighbour sets of Eq. 2 (|r_j + n.H - r_i| < r_c,
 * every periodic image n, j != i or n != 0) for a batch, in canonical order
 * (j ascending, then image shift lexicographic), with FP64 distance tests that
 * round exactly like a plain FP64 evaluation without fused multiply-add.  The
 * nlist keeps a device copy of the batch and the per-step workspace; structures
 * are fixed while it lives.  Synchronises `stream` (the pair count sizes the
 * lists).  Errors: INVALID_ARG (sizes, types, wrapping), NEIGHBOR_OVERFLOW,
 * OOM, CUDA. */
int gnep_build_neighbors(gnep_model *m, const gnep_batch *b, gnep_nlist **out,
                         void *stream);
/* Rebuild `nl` in place for a batch of the same n_struct and n_atoms (new
 * positions, cells or species); grows the lists only if the pair count grows.
 * Synchronises with the host once, when the pair counts are known (input
 * errors such as unwrapped positions are returned then), and returns with the
 * rest of the build (compaction, reverse entries, tile upload) queued on
 * `stream`: every call that reads `nl` afterwards, on any stream, is ordered
 * after that work by an event the list keeps.  The batch's host arrays may be
 * reused once this returns.  The lists' internal consistency check of that
 * queued work is reported by gnep_sync_status() (or by the next
 * gnep_build_neighbors / gnep_md_verlet).  The caller keeps the usual duty of
 * not rebuilding a list that queued work on another stream still reads. */
int gnep_rebuild_neighbors(gnep_model *m, const gnep_batch *b, gnep_nlist *nl,
                           void *stream);
int gnep_nlist_destroy(gnep_nlist *nl);
int gnep_nlist_info(const gnep_nlist *nl, int64_t *n_pairs_radial,
                    int64_t *n_pairs_angular);
/* Copy one list out: off [n_atoms+1], j [pairs] (global atom index),
 * shift [pairs*3] image (na, nb, nc).  Synchronises when any pointer is host. */
int gnep_nlist_export(const gnep_nlist *nl, int which, int32_t *off, int32_t *j,
                      int32_t *shift, void *stream);

/* ---------------------------------------------------------- evaluation */

/* Unscaled descriptors G [n_atoms][N_des] (Eqs. 5-8 and the 4-body term),
 * radial n first, then angular (n, l) n-major, then 4-body n. */
int gnep_descriptors(gnep_model *m, const gnep_nlist *nl, float *G, void *stream);

/* The same descriptors as gnep_descriptors, computed without allocating any
 * device memory.  The paper has no counterpart.  It serves callers that must
 * not allocate at the point where they need descriptors: hosts whose device
 * memory is reserved up front by another allocator or a fixed pool (a
 * cudaMalloc there fails or fragments that pool), and per-step hooks of
 * simulation engines that forbid allocation in their hot loop (cudaMalloc and
 * cudaFree may synchronise the device and stall the loop).  The call works in
 * a fixed 8 MiB scratch array built into the library (every GPU that loads
 * the library holds it until the process exits) instead of the nlist's
 * workspace.  A batch fits when
 *   roundup64(n_atoms * n_species * (basis_radial + 1))
 *     + n_atoms * 24 * (n_max_angular + 1)  <=  2^21 floats
 * (roundup64: the next multiple of 64); larger batches return INVALID_ARG.
 * G [n_atoms][N_des] must be device memory; it is written asynchronously on
 * `stream` after the nlist's last build.  The first call on each device looks
 * up the scratch address (cudaGetSymbolAddress).  All calls share one scratch
 * array per device and it keeps the last call's contents: calls whose kernels
 * may overlap on the GPU (different streams without ordering, several
 * threads) race and must not be issued; calls ordered on one stream are safe.
 * The scratch needs no clearing: every element a call reads was written
 * earlier by the same call. */
int gnep_descriptors_noalloc(gnep_model *m, const gnep_nlist *nl, float *G,
                             void *stream);

/* Energies, forces and virials (Eqs. 1, 3, 4).  Any output may be NULL.
 * E_atom [n_atoms] site energies; E_struct [n_struct] totals; F [n_atoms*3];
 * W_struct [n_struct*6] total virial, symmetrised, xx yy zz xy yz zx. */
int gnep_forward(gnep_model *m, const gnep_nlist *nl, float *E_atom,
                 double *E_struct, float *F, double *W_struct, void *stream);

/* One velocity-Verlet step of molecular dynamics (NVE) with the model's
 * forces (forward-only inference, Eqs. 1 and 3; NEXT use of a trained model
 * for EOS / RDF-style sampling).  Units A, fs, amu, eV.
 * pos [n_atoms*3] FP64 and vel [n_atoms*3] FP64 (A/fs): device arrays of this
 *   list's batch, updated in place; positions are wrapped back into their
 *   cell after the drift and the neighbour list is rebuilt from them.
 * inv_mass [n_atoms] FP64 device, 1/amu.
 * F [n_atoms*3] FP32 device: forces at pos on entry (from gnep_forward) and at
 *   the new positions on return.
 * E_struct [n_struct] FP64 (optional, host or device): potential energies at
 *   the new positions.
 * The cells stay fixed.  Graphs captured on this list are invalidated (the
 * lists are rebuilt).  Errors: INVALID_ARG (host arrays, dt <= 0), and those
 * of gnep_rebuild_neighbors and gnep_forward. */
int gnep_md_verlet(gnep_model *m, gnep_nlist *nl, double *pos, double *vel,
                   const double *inv_mass, float *F, double dt,
                   double *E_struct, void *stream);

/* Loss and exact parameter gradient of one training step (Eqs. 9-16,
 * D1.18-D1.21).  loss_terms [4] = {L, L_e, L_f, L_v} (L_x are Eqs. 10-12, L the
 * weighted total); grad [n_params] (may be NULL: the gradient stays in the
 * model for gnep_adam_step).  Both may be NULL.  Labels may be host or device
 * memory (host labels are staged on `stream`). */
int gnep_loss_grad(gnep_model *m, const gnep_nlist *nl, const gnep_labels *y,
                   double *loss_terms, float *grad, void *stream);

/* Autotuner.  Launch shapes are per batch: atoms and pairs per tile of the
 * descriptor and tangent sweeps' tiles and of the angular force and
 * c-gradient sweeps' tiles, the number of persistent blocks of the c-gradient
 * sweep and of the network kernels, the lanes per atom of the radial sweeps,
 * the atoms per tile of the FP32 network, and whether the radial sweeps run
 * beside the angular ones.  gnep_autotune times the
 * loss + gradient evaluation of this batch (median of `reps` runs, no
 * parameter update) over candidate values of each in turn and keeps the
 * fastest in the neighbour list.  It synchronizes `stream` and must not run
 * during stream capture; graphs captured earlier on this list are invalidated
 * (gnep_graph_launch then returns INVALID_ARG).  values [9] =
 *   [0] atoms per descriptor tile   [1] pairs per descriptor tile
 *   [2] atoms per force tile        [3] pairs per force tile
 *   [4] c-gradient blocks (at most 608)
 *   [5] network blocks (at most 456; 0 = one per tile up to the resident capacity)
 *   [6] radial lanes per atom: 4, 8 or 16 (default: 4 while four 128-thread
 *       blocks per SM are filled, more for smaller batches)
 *   [7] atoms per FP32 network tile: 32 or 128 (default: 128 while the batch
 *       has a tile per two SMs, else 32; the tensor-core modes always take 128).
 *   [8] radial sweeps: 1 = in turn with the angular sweeps on `stream`,
 *       2 = beside them on a second stream owned by the list, forked from and
 *       joined back to `stream` by events within each call (default: 2 while
 *       the angular descriptor sweep has fewer than eight tiles per SM, else
 *       1).  The results are the same bit for bit.
 * gnep_tuning_get gives the effective values; gnep_tuning_set takes the same
 * layout (0 = default) and rebuilds the tiles.  Results agree with the
 * untuned ones to FP32 summation order.
 * Errors: INVALID_ARG (a value out of range), CUDA, and those of
 * gnep_loss_grad. */
int gnep_autotune(gnep_model *m, gnep_nlist *nl, const gnep_labels *y,
                  int reps, void *stream);
int gnep_tuning_get(const gnep_model *m, const gnep_nlist *nl,
                    int32_t *values);
int gnep_tuning_set(gnep_model *m, gnep_nlist *nl, const int32_t *values,
                    void *stream);

/* Loss only (Eqs. 9-12): the forward pass and loss_terms [4] as in
 * gnep_loss_grad, without the backward pass.  Used where the loss must be
 * known before the gradient is formed, e.g. the whole-batch RMSE of a batch
 * split over ranks.  Errors: as gnep_loss_grad. */
int gnep_loss(gnep_model *m, const gnep_nlist *nl, const gnep_labels *y,
              double *loss_terms, void *stream);

/* The model's FP64 gradient dL/dtheta (the one gnep_adam_step applies):
 * copy it out to dst, or replace it by src ([n] doubles, host or device,
 * n = gnep_num_params).  Lets a caller sum gradients over data-parallel ranks
 * between gnep_loss_grad and gnep_adam_step.  set_grad with a host source
 * returns after the copy.  Errors: INVALID_ARG (NULL or n mismatch), CUDA. */
int gnep_get_grad(gnep_model *m, double *dst, int64_t n, void *stream);
int gnep_set_grad(gnep_model *m, const double *src, int64_t n, void *stream);

/* Adam update (Kingma & Ba, bias-corrected; AdamW decay if weight_decay > 0)
 * with the model's last gradient, in FP32 (parameters and moments are FP32).
 * The update count t lives in device memory and advances by one per call.  lr
 * is used as given.  If the last loss was not finite the update is skipped
 * and t does not advance.  Errors: INVALID_ARG unless 0 < beta1, beta2 < 1
 * and eps > 0. */
int gnep_adam_step(gnep_model *m, double lr, double beta1, double beta2,
                   double eps, double weight_decay, void *stream);
/* Same, with the learning rate of Eq. 17 evaluated on the device from the
 * update count (s = t before the update), so the call can be replayed inside a
 * captured CUDA graph. */
int gnep_adam_step_scheduled(gnep_model *m, double lr_start, double lr_stop,
                             int64_t n_warmup, int64_t n_total, double beta1,
                             double beta2, double eps, double weight_decay,
                             void *stream);
int gnep_get_step(gnep_model *m, int64_t *t, void *stream);

/* Eq. 17: linear warm-up from lr_stop to lr_start over n_warmup steps, then a
 * cosine decay to lr_stop at n_total.  Host-side scalar. */
double gnep_lr_schedule(double lr_start, double lr_stop, int64_t s,
                        int64_t n_warmup, int64_t n_total);

/* One training step captured once as a CUDA graph and replayed: loss_grad then
 * adam_step_scheduled, with the same results bit for bit (the gradient stays
 * in the model for gnep_get_grad; the gradient reduction, the copy of the loss
 * terms and the update run as one kernel).  loss_out is a device pointer [4]
 * (may be NULL) written each replay.  The nlist, labels (device pointers) and
 * loss_out must outlive the graph. */
typedef struct gnep_graph gnep_graph;
int gnep_graph_create(gnep_model *m, const gnep_nlist *nl, const gnep_labels *y,
                      double *loss_out, double lr_start, double lr_stop,
                      int64_t n_warmup, int64_t n_total, double beta1,
                      double beta2, double eps, double weight_decay,
                      void *stream, gnep_graph **out);
/* n_steps training steps captured as one CUDA graph: step b trains on the
 * batch (nls[b], ys[b]) as gnep_graph_create's step does, in order, so that
 * one launch replays, for instance, a whole epoch of one-structure batches
 * with the same results bit for bit as the n_steps single-step graphs (or the
 * eager call pairs) launched in turn.  A list may appear more than once.
 * loss_out: device [4 n_steps] (may be NULL), step b's loss terms at 4 b.
 * Lists, labels and loss_out must outlive the graph; launching after any of
 * the lists was rebuilt or retuned returns INVALID_ARG.
 * Errors: INVALID_ARG (NULL, n_steps < 1, host labels or loss buffer, the
 * default stream, a list of another model), UNSUPPORTED, OOM, CUDA. */
int gnep_graph_create_steps(gnep_model *m, const gnep_nlist *const *nls,
                            const gnep_labels *ys, int32_t n_steps,
                            double *loss_out, double lr_start, double lr_stop,
                            int64_t n_warmup, int64_t n_total, double beta1,
                            double beta2, double eps, double weight_decay,
                            void *stream, gnep_graph **out);
int gnep_graph_launch(gnep_graph *g, void *stream);
int gnep_graph_destroy(gnep_graph *g);
/* Kernels one replay launches (the graph's kernel nodes), to *n.
 * Errors: INVALID_ARG (NULL), CUDA. */
int gnep_graph_kernel_count(const gnep_graph *g, int32_t *n);

/* ------------------------------------------------------------ profiling */

/* Run one training step eagerly (loss_grad, then an Adam update with lr 1e-4)
 * with a CUDA event recorded after every launch on `stream`, and return the
 * duration of each launch in stage_ms [cap]; n_stages receives the count.
 * The step changes the parameters like any step.  Synchronises `stream`.
 * Not for concurrent use from several threads. */
int gnep_profile_step(gnep_model *m, const gnep_nlist *nl, const gnep_labels *y,
                      float *stage_ms, int32_t cap, int32_t *n_stages, void *stream);
/* Name of stage i of the last gnep_profile_step ("" when out of range). */
const char *gnep_profile_stage_name(int32_t i);

/* ------------------------------------------------------- state, errors */

/* Checkpoint: header (shape, parameter count, update count), FP32 parameters,
 * descriptor scale, Adam moments, CRC32.  load validates the header against the
 * model and the CRC; a mismatch returns CHECKPOINT_CORRUPT and leaves the model
 * unchanged.  Both synchronise the device. */
int gnep_save(gnep_model *m, const char *path);
int gnep_load(gnep_model *m, const char *path);

/* ---------------------------------------------------- data parallelism */

/* Loss weights of one data-parallel shard (Eqs. 9-12 over a batch split by
 * structure across ranks).  Eqs. 10-12 normalise by the whole batch (N_str
 * structures, N atoms), so a shard of S_r structures and N_r atoms that calls
 * gnep_loss_grad with the MSE form and these weights gets exactly its share
 * of the whole-batch gradient; summing the shards' gradients over ranks gives
 * the whole-batch gradient.  out [4] = {lambda_e S_r/N_str, lambda_f N_r/N,
 * lambda_v S_r/N_str, lambda_l2 on rank 0 else 0}; for GNEP_LOSS_RMSE each of
 * the first three is further multiplied by 1 / (2 sqrt(L_x)) (0 where L_x =
 * 0), with mse_total [3] = the whole-batch MSE terms L_e, L_f, L_v (from
 * gnep_shard_mse_total; may be NULL for the MSE form).  Host-side scalars.
 * Errors: INVALID_ARG. */
int gnep_shard_loss_weights(double lambda_e, double lambda_f, double lambda_v,
                            double lambda_l2, int32_t loss_form,
                            int64_t local_struct, int64_t local_atoms,
                            int64_t total_struct, int64_t total_atoms,
                            const double *mse_total, int32_t rank, double *out);
/* A shard's MSE terms (loss_terms[1..3] of gnep_loss) as sums that add over
 * ranks: out [5] = {L_e S_r, L_f 3 N_r, L_v 6 S_r, S_r, N_r}.  After a sum over
 * ranks, gnep_shard_mse_total turns them into the whole-batch L_e, L_f, L_v
 * (out [3]; 0 for an empty term).  Host-side.  Errors: INVALID_ARG. */
int gnep_shard_mse_partials(const double *local_mse, int64_t local_struct,
                            int64_t local_atoms, double *out);
int gnep_shard_mse_total(const double *sums, double *out);

/* Synchronise `stream`, read and clear the model's device error flag:
 * NONFINITE (a loss was not finite; that Adam update was skipped), TIMEOUT (a
 * device-side wait gave up), INVALID_ARG (a rebuild's lists failed their
 * consistency check, or another input check on the device failed). */
int gnep_sync_status(gnep_model *m, void *stream);
const char *gnep_last_error(void);
int gnep_abi_version(void);

/* Failure-path self-test of the bounded device waits (library failure
 * detection; the paper has no counterpart).  Launches one block of the
 * tensor-core kernels' wait protocol on `stream`: it allocates tensor memory,
 * waits on an mbarrier that nothing arrives on with a limit of limit_ns
 * (1e3 .. 2e9), gives up, waits once more with the same limit, frees its
 * tensor memory, raises TIMEOUT in the model's device flag and returns; the
 * next gnep_sync_status returns GNEP_ERR_TIMEOUT and clears the flag.  No
 * fault, no hang: the context stays usable.  Errors: INVALID_ARG, CUDA. */
int gnep_selftest_wait_timeout(gnep_model *m, int64_t limit_ns, void *stream);

#ifdef __cplusplus
}
#endif
#endif
