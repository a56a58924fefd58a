/*
 * FP64 CPU oracle for gradient-optimised NEP training -- declarations.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow reference that
 * the CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never does.  It
 * shares no code, header or table with the CUDA library.
 *
 * Every array is host memory, row-major, FP64 unless stated.  Positions must be
 * wrapped into their cell (fractional coordinates in [0, 1)).
 */
#ifndef GNEP_ORACLE_H
#define GNEP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int n_species;
  int nq_r, nq_a;     /* radial / angular descriptor channels (n_max + 1) */
  int k_r, k_a;       /* radial / angular basis functions (basis_size + 1) */
  int l_max;          /* 1..4 */
  int four_body;      /* 0 or 1 */
  int hidden;         /* hidden neurons N_neu */
  double rc_r, rc_a;  /* cut-offs (A) */
} orc_cfg;

typedef struct {
  int n_struct;
  const int *struct_off;  /* [n_struct+1] */
  const double *pos;      /* [N*3] */
  const int *type;        /* [N] */
  const double *cell;     /* [n_struct*9], rows a, b, c */
} orc_batch;

typedef struct {
  const double *energy;   /* [n_struct]   per-atom energy label (eV/atom) */
  const double *force;    /* [N*3]        force label (eV/A) */
  const double *virial;   /* [n_struct*6] per-atom virial label xx yy zz xy yz zx */
  double lambda_e, lambda_f, lambda_v, lambda_l2;
  int loss_form;          /* 0: MSE (Eqs. 9-12), 1: sum of weighted RMSEs */
} orc_labels;

int orc_num_des(const orc_cfg *c);
long orc_num_params(const orc_cfg *c);
const double *orc_clm(void);

void orc_chebyshev(int K, double xi, double *T, double *dT);
void orc_cutoff(double rc, double r, double *fc, double *fcp);
void orc_radial_basis(int K, double rc, double r, double *f, double *fp);
void orc_blm(const double *d, double *B, double *dB);
/* B_lm and grad B_lm for l = 1..l_max (l_max <= 8; B5-B8 from the printed
 * forms); B [nlm], dB [nlm][3], nlm = (l_max + 1)^2 - 1. */
void orc_blm_lmax(const double *d, int l_max, double *B, double *dB);
/* 4 pi / ((2l + 1) int B_lm^2 dOmega) by quadrature, for component lm. */
double orc_clm_quadrature(int lm);

long orc_neighbors(const orc_batch *b, double rc, long cap, long *off,
                   int *nbr_j, int *nbr_shift);
int orc_descriptors(const orc_cfg *c, const double *params, const orc_batch *b,
                    double *G);
int orc_ann(const orc_cfg *c, const double *params, const double *scale, int e,
            const double *G, double *E, double *Ep, double *Epp);
int orc_forward(const orc_cfg *c, const double *params, const double *scale,
                const orc_batch *b, double *E_atom, double *E_struct,
                double *F, double *W_struct);
int orc_loss(const orc_cfg *c, const double *params, const double *scale,
             const orc_batch *b, const orc_labels *y, double *terms);
int orc_loss_grad(const orc_cfg *c, const double *params, const double *scale,
                  const orc_batch *b, const orc_labels *y, double *terms,
                  double *grad);
void orc_adam(long n, double *theta, double *m, double *v, const double *g,
              long t, double lr, double beta1, double beta2, double eps,
              double weight_decay);
double orc_lr(double lr_start, double lr_stop, long s, long n_warmup,
              long n_total);

#ifdef __cplusplus
}
#endif
#endif
