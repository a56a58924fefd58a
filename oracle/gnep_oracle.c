/*
 * FP64 CPU oracle for gradient-optimised NEP training.
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct reference the
 * CUDA path is checked against.  Only tests, the smoke check and the
 * benchmark's CPU-baseline leg may call it.  It shares no code with the CUDA
 * library.  Compile with -ffp-contract=off: the neighbour test must round
 * exactly like the GPU's FP64 test (no fused multiply-add).
 *
 * What it follows, in the paper's order and notation:
 *   Eq. 2              neighbour sets, brute force over periodic images
 *   A1.1-A1.5, A2.1-2  Chebyshev basis, derivative recursion, cosine cut-off
 *   Eqs. 5-6           radial descriptors q_n
 *   B1-B4, B9.1-B9.2   real solid harmonics b_lm, B_lm = b_lm / r^l, gradients
 *   Eqs. 7-8           angular descriptors q_nl, S_nlm
 *   D1.1-D1.6          network energy, dE/dG, d2E/dG2
 *   C1.1, C2.1-C2.3,   dE_i/dr_ij (partial force)
 *   C3.6
 *   Eqs. 1, 3, 4       energy, forces, per-atom virial
 *   Eqs. 9-12          loss
 *   C1.3-C1.5, C2.5-C2.10, Alg. 1, C3.5-C3.20, D1.7-D1.17
 *                      explicit first and mixed second derivatives
 *   Eqs. 13-16, D1.18-D1.21  gradient assembly
 *   Eq. 17, Adam       learning-rate schedule and update
 *
 * Readings where the paper is silent or garbled (each one also applied by the
 * CUDA path, which is written separately):
 *   - K = basis_size + 1 functions (k = 0..N_bas inclusive, Eq. 6) and
 *     n_max + 1 channels per descriptor family.
 *   - Separate coefficient sets c^R (cut-off r_c^R) and c^A (r_c^A), ordered
 *     in the species pair (I, J).
 *   - C1.1's leading 1/2 is the one inside f_k, and the bond direction is
 *     r_ij/|r_ij|: dq_n/dr_ij = sum_k c_nk f_k'(r) r_ij/r.
 *   - C_lm: addition-theorem normalisation, sum_m C_lm B_lm(u) B_lm(v) =
 *     P_l(u.v) (Legendre).
 *   - 4-body term (the paper defers its definition elsewhere): for each angular
 *     channel n, q4_n = tr(Q_n^3) with Q_n = sum_j g_n(r_ij) (3 u u^T - I)/2,
 *     u = r_ij/r_ij, the cubic rotation invariant of the l = 2 moments.
 *   - Descriptor scale: the network sees s_v G_v with a fixed per-component
 *     scale s (not trained).
 *   - Eq. 4 governs the virial; components are symmetrised xx yy zz xy yz zx
 *     with xy = (W_xy + W_yx)/2; the label is the per-atom virial W_s / N_s.
 *   - D1.14 is read with the parameter W0_{mu v'} and the derivative direction
 *     G_v: d2E/(dW0_{mu v'} dG_v) = w1_mu (-2 x_mu (1 - x_mu^2) W0_{mu v} G_v'
 *     + delta_{v v'} (1 - x_mu^2)), as the paper's device listing computes it.
 *   - The virial analogue of D1.11-D1.17 (omitted in the paper) is Eq. 4
 *     differentiated: dV_i/dp = sum_j r_ij (x) d/dp(dE_j/dr_ji).
 *   - Loss form 1 (RMSE): L = sum_x lambda_x sqrt(L_x) + L2 term; its gradient
 *     divides each MSE gradient by 2 sqrt(L_x) (zero when L_x = 0).
 *   - L2 term: lambda_l2 * sum(theta^2) / N_par.
 */
#include "gnep_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define NLM 80 /* (l, m) components for l = 1..8, the stride of every per-(l, m) array */
#define LMAX 8

static int lm_first(int l) { return l * l - 1; } /* l=1 -> 0, 2 -> 3, 3 -> 8, 4 -> 15, ... */
static int nlm_of(int l_max) { return (l_max + 1) * (l_max + 1) - 1; }

/* C_lm of Eq. 7 (the paper only calls them constants): the addition-theorem
 * normalisation sum_m C_lm B_lm(u) B_lm(v) = P_l(u.v).  For l = 1..4 the
 * values derived from the standard real-harmonic norms, in the order of
 * App. B; for l = 5..8 (B5-B8) each value is 4 pi / ((2l + 1) int B_lm^2 dOmega)
 * by the quadrature of clm_quadrature() below, filled in on first use. */
static double C_LM[NLM] = {
    1.0, 1.0, 1.0,
    0.25, 3.0, 3.0, 0.75, 0.75,
    0.25, 0.375, 0.375, 3.75, 3.75, 0.625, 0.625,
    1.0 / 64.0, 0.625, 0.625, 0.3125, 0.3125, 4.375, 4.375, 35.0 / 64.0,
    35.0 / 64.0};
static int C_LM_ready = 0;
static void clm_init(void);

const double *orc_clm(void) {
  clm_init();
  return C_LM;
}

/* ------------------------------------------------------------------ layout */

int orc_num_des(const orc_cfg *c) {
  return c->nq_r + c->nq_a * c->l_max + (c->four_body ? c->nq_a : 0);
}

static long net_size(const orc_cfg *c) {
  long d = orc_num_des(c);
  return d * c->hidden + 2L * c->hidden + 1;
}

long orc_num_params(const orc_cfg *c) {
  long S = c->n_species;
  return S * net_size(c) + S * S * ((long)c->nq_r * c->k_r + (long)c->nq_a * c->k_a);
}

static long off_W0(const orc_cfg *c, int e) { return e * net_size(c); }
static long off_b0(const orc_cfg *c, int e) { return off_W0(c, e) + (long)orc_num_des(c) * c->hidden; }
static long off_w1(const orc_cfg *c, int e) { return off_b0(c, e) + c->hidden; }
static long off_b1(const orc_cfg *c, int e) { return off_w1(c, e) + c->hidden; }
static long off_cR(const orc_cfg *c, int I, int J, int n, int k) {
  long base = c->n_species * net_size(c);
  return base + (((long)I * c->n_species + J) * c->nq_r + n) * c->k_r + k;
}
static long off_cA(const orc_cfg *c, int I, int J, int n, int k) {
  long base = c->n_species * net_size(c) +
              (long)c->n_species * c->n_species * c->nq_r * c->k_r;
  return base + (((long)I * c->n_species + J) * c->nq_a + n) * c->k_a + k;
}
static int v_rad(const orc_cfg *c, int n) { (void)c; return n; }
static int v_ang(const orc_cfg *c, int n, int l) { return c->nq_r + n * c->l_max + (l - 1); }
static int v_4b(const orc_cfg *c, int n) { return c->nq_r + c->nq_a * c->l_max + n; }

/* --------------------------------------------------- App. A: radial basis */

/* A1.1 (T_k) and A1.3-A1.5 (dT_k/dxi). */
void orc_chebyshev(int K, double xi, double *T, double *dT) {
  for (int k = 0; k < K; ++k) {
    if (k == 0) {
      T[k] = 1.0;
      dT[k] = 0.0;
    } else if (k == 1) {
      T[k] = xi;
      dT[k] = 1.0;
    } else {
      T[k] = 2.0 * xi * T[k - 1] - T[k - 2];
      dT[k] = 2.0 * T[k - 1] + 2.0 * xi * dT[k - 1] - dT[k - 2];
    }
  }
}

/* A2.1 and A2.2. */
void orc_cutoff(double rc, double r, double *fc, double *fcp) {
  if (r <= rc) {
    *fc = 0.5 * (1.0 + cos(M_PI * r / rc));
    *fcp = -M_PI / (2.0 * rc) * sin(M_PI * r / rc);
  } else {
    *fc = 0.0;
    *fcp = 0.0;
  }
}

/* Eq. 6 basis f_k = (T_k(xi) + 1)/2 f_c(r) with xi from A1.2, and df_k/dr. */
void orc_radial_basis(int K, double rc, double r, double *f, double *fp) {
  double T[64], dT[64], fc, fcp;
  double xi = 2.0 * (r / rc - 1.0) * (r / rc - 1.0) - 1.0;
  double dxi = 4.0 * (r / rc - 1.0) / rc;
  orc_chebyshev(K, xi, T, dT);
  orc_cutoff(rc, r, &fc, &fcp);
  for (int k = 0; k < K; ++k) {
    f[k] = 0.5 * (T[k] + 1.0) * fc;
    fp[k] = 0.5 * dT[k] * dxi * fc + 0.5 * (T[k] + 1.0) * fcp;
  }
}

/* ------------------------------------------- App. B: real solid harmonics */

/* B1.1-B4.9 as printed, their Cartesian gradients, then B9.1 and B9.2:
 * B = b / r^l and grad B = grad b / r^l - l b d / r^(l+2).  dB is [24][3]. */
void orc_blm(const double *d, double *B, double *dB) {
  const double x = d[0], y = d[1], z = d[2];
  const double r2 = x * x + y * y + z * z;
  const double r = sqrt(r2);
  double b[24], g[24][3];
  /* l = 1 */
  b[0] = z;                      g[0][0] = 0;     g[0][1] = 0;     g[0][2] = 1;
  b[1] = x;                      g[1][0] = 1;     g[1][1] = 0;     g[1][2] = 0;
  b[2] = y;                      g[2][0] = 0;     g[2][1] = 1;     g[2][2] = 0;
  /* l = 2 */
  b[3] = 3 * z * z - r2;         g[3][0] = -2 * x; g[3][1] = -2 * y; g[3][2] = 4 * z;
  b[4] = x * z;                  g[4][0] = z;      g[4][1] = 0;      g[4][2] = x;
  b[5] = y * z;                  g[5][0] = 0;      g[5][1] = z;      g[5][2] = y;
  b[6] = x * x - y * y;          g[6][0] = 2 * x;  g[6][1] = -2 * y; g[6][2] = 0;
  b[7] = 2 * x * y;              g[7][0] = 2 * y;  g[7][1] = 2 * x;  g[7][2] = 0;
  /* l = 3 */
  {
    double u = 5 * z * z - r2;
    b[8] = 5 * z * z * z - 3 * z * r2;
    g[8][0] = -6 * x * z; g[8][1] = -6 * y * z; g[8][2] = 9 * z * z - 3 * r2;
    b[9] = u * x;
    g[9][0] = u - 2 * x * x; g[9][1] = -2 * x * y; g[9][2] = 8 * x * z;
    b[10] = u * y;
    g[10][0] = -2 * x * y; g[10][1] = u - 2 * y * y; g[10][2] = 8 * y * z;
    b[11] = (x * x - y * y) * z;
    g[11][0] = 2 * x * z; g[11][1] = -2 * y * z; g[11][2] = x * x - y * y;
    b[12] = 2 * x * y * z;
    g[12][0] = 2 * y * z; g[12][1] = 2 * x * z; g[12][2] = 2 * x * y;
    b[13] = (x * x - 3 * y * y) * x;
    g[13][0] = 3 * x * x - 3 * y * y; g[13][1] = -6 * x * y; g[13][2] = 0;
    b[14] = (3 * x * x - y * y) * y;
    g[14][0] = 6 * x * y; g[14][1] = 3 * x * x - 3 * y * y; g[14][2] = 0;
  }
  /* l = 4 */
  {
    double w = 7 * z * z * z - 3 * z * r2;
    double wz = 15 * z * z - 3 * r2; /* dw/dz; dw/dx = -6xz, dw/dy = -6yz */
    double p = 7 * z * z - r2;       /* dp = (-2x, -2y, 12z) */
    double q = x * x - y * y;        /* dq = (2x, -2y, 0) */
    b[15] = 35 * z * z * z * z - 30 * z * z * r2 + 3 * r2 * r2;
    g[15][0] = -60 * x * z * z + 12 * x * r2;
    g[15][1] = -60 * y * z * z + 12 * y * r2;
    g[15][2] = 80 * z * z * z - 48 * z * r2;
    b[16] = w * x;
    g[16][0] = w - 6 * x * x * z; g[16][1] = -6 * x * y * z; g[16][2] = x * wz;
    b[17] = w * y;
    g[17][0] = -6 * x * y * z; g[17][1] = w - 6 * y * y * z; g[17][2] = y * wz;
    b[18] = p * q;
    g[18][0] = -2 * x * q + 2 * x * p; g[18][1] = -2 * y * q - 2 * y * p; g[18][2] = 12 * z * q;
    b[19] = p * 2 * x * y;
    g[19][0] = -4 * x * x * y + 2 * p * y; g[19][1] = -4 * x * y * y + 2 * p * x;
    g[19][2] = 24 * x * y * z;
    b[20] = (x * x * x - 3 * x * y * y) * z;
    g[20][0] = (3 * x * x - 3 * y * y) * z; g[20][1] = -6 * x * y * z;
    g[20][2] = x * x * x - 3 * x * y * y;
    b[21] = (3 * x * x * y - y * y * y) * z;
    g[21][0] = 6 * x * y * z; g[21][1] = (3 * x * x - 3 * y * y) * z;
    g[21][2] = 3 * x * x * y - y * y * y;
    b[22] = x * x * x * x - 6 * x * x * y * y + y * y * y * y;
    g[22][0] = 4 * x * x * x - 12 * x * y * y; g[22][1] = -12 * x * x * y + 4 * y * y * y;
    g[22][2] = 0;
    b[23] = 4 * x * x * x * y - 4 * x * y * y * y;
    g[23][0] = 12 * x * x * y - 4 * y * y * y; g[23][1] = 4 * x * x * x - 12 * x * y * y;
    g[23][2] = 0;
  }
  for (int lm = 0; lm < 24; ++lm) {
    int l = lm < 3 ? 1 : lm < 8 ? 2 : lm < 15 ? 3 : 4;
    double rl = pow(r, l);
    B[lm] = b[lm] / rl;
    for (int c = 0; c < 3; ++c)
      dB[lm * 3 + c] = g[lm][c] / rl - l * b[lm] * d[c] / (rl * r2);
  }
}

/* B5.1-B8.17 as printed.  Every printed form is a product of a polynomial in
 * z and r^2, sum_k zc[k] z^(zdeg - 2k) r^(2k), and a polynomial in x and y,
 * sum_j xyc[j] x^xp[j] y^yp[j]; the table holds the two factors as printed. */
typedef struct {
  int zdeg;
  double zc[5];
  int nxy;
  double xyc[5];
  int xp[5], yp[5];
} printed_form;

#define XY1 1, {1}, {0}, {0}
#define XY_X 1, {1}, {1}, {0}
#define XY_Y 1, {1}, {0}, {1}
#define XY_C2 2, {1, -1}, {2, 0}, {0, 2}               /* x^2 - y^2 */
#define XY_S2 1, {2}, {1}, {1}                          /* 2xy */
#define XY_C3 2, {1, -3}, {3, 1}, {0, 2}               /* x^3 - 3xy^2 */
#define XY_S3 2, {3, -1}, {2, 0}, {1, 3}               /* 3x^2y - y^3 */
#define XY_C4 3, {1, -6, 1}, {4, 2, 0}, {0, 2, 4}      /* x^4 - 6x^2y^2 + y^4 */
#define XY_S4 2, {4, -4}, {3, 1}, {1, 3}               /* 4x^3y - 4xy^3 */
#define XY_C5 3, {1, -10, 5}, {5, 3, 1}, {0, 2, 4}     /* x^5 - 10x^3y^2 + 5xy^4 */
#define XY_S5 3, {5, -10, 1}, {4, 2, 0}, {1, 3, 5}     /* 5x^4y - 10x^2y^3 + y^5 */
#define XY_C6 4, {1, -15, 15, -1}, {6, 4, 2, 0}, {0, 2, 4, 6}
#define XY_S6 3, {6, -20, 6}, {5, 3, 1}, {1, 3, 5}
#define XY_C7 4, {1, -21, 35, -7}, {7, 5, 3, 1}, {0, 2, 4, 6}
#define XY_S7 4, {7, -35, 21, -1}, {6, 4, 2, 0}, {1, 3, 5, 7}
#define XY_C8 5, {1, -28, 70, -28, 1}, {8, 6, 4, 2, 0}, {0, 2, 4, 6, 8}
#define XY_S8 4, {8, -56, 56, -8}, {7, 5, 3, 1}, {1, 3, 5, 7}

static const printed_form FORMS_5_8[56] = {
    /* l = 5: B5.1-B5.11 */
    {5, {63, -70, 15}, XY1},    {4, {21, -14, 1}, XY_X},  {4, {21, -14, 1}, XY_Y},
    {3, {3, -1}, XY_C2},        {3, {3, -1}, XY_S2},      {2, {9, -1}, XY_C3},
    {2, {9, -1}, XY_S3},        {1, {1}, XY_C4},          {1, {1}, XY_S4},
    {0, {1}, XY_C5},            {0, {1}, XY_S5},
    /* l = 6: B6.1-B6.13 */
    {6, {231, -315, 105, -5}, XY1}, {5, {33, -30, 5}, XY_X}, {5, {33, -30, 5}, XY_Y},
    {4, {33, -18, 1}, XY_C2},   {4, {33, -18, 1}, XY_S2}, {3, {11, -3}, XY_C3},
    {3, {11, -3}, XY_S3},       {2, {11, -1}, XY_C4},     {2, {11, -1}, XY_S4},
    {1, {1}, XY_C5},            {1, {1}, XY_S5},          {0, {1}, XY_C6},
    {0, {1}, XY_S6},
    /* l = 7: B7.1-B7.15 */
    {7, {429, -693, 315, -35}, XY1}, {6, {429, -495, 135, -5}, XY_X},
    {6, {429, -495, 135, -5}, XY_Y}, {5, {143, -110, 15}, XY_C2}, {5, {143, -110, 15}, XY_S2},
    {4, {143, -66, 3}, XY_C3},  {4, {143, -66, 3}, XY_S3}, {3, {13, -3}, XY_C4},
    {3, {13, -3}, XY_S4},       {2, {13, -1}, XY_C5},     {2, {13, -1}, XY_S5},
    {1, {1}, XY_C6},            {1, {1}, XY_S6},          {0, {1}, XY_C7},
    {0, {1}, XY_S7},
    /* l = 8: B8.1-B8.17 */
    {8, {6435, -12012, 6930, -1260, 35}, XY1}, {7, {715, -1001, 385, -35}, XY_X},
    {7, {715, -1001, 385, -35}, XY_Y}, {6, {143, -143, 33, -1}, XY_C2},
    {6, {143, -143, 33, -1}, XY_S2}, {5, {39, -26, 3}, XY_C3}, {5, {39, -26, 3}, XY_S3},
    {4, {65, -26, 1}, XY_C4},   {4, {65, -26, 1}, XY_S4}, {3, {5, -1}, XY_C5},
    {3, {5, -1}, XY_S5},        {2, {15, -1}, XY_C6},     {2, {15, -1}, XY_S6},
    {1, {1}, XY_C7},            {1, {1}, XY_S7},          {0, {1}, XY_C8},
    {0, {1}, XY_S8}};

static double ipow(double a, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r *= a;
  return r;
}

/* b = Z(z, r^2) XY(x, y) of one printed form and its Cartesian gradient,
 * each monomial differentiated by hand (d r^2 / d x_c = 2 x_c). */
static void printed_eval(const printed_form *f, const double *d, double *b, double *g) {
  const double x = d[0], y = d[1], z = d[2], R = x * x + y * y + z * z;
  double Z = 0, Zr = 0, Zz = 0; /* Z, dZ/d(r^2), partial dZ/dz at fixed r^2 */
  for (int k = 0; 2 * k <= f->zdeg; ++k) {
    const int a = f->zdeg - 2 * k;
    Z += f->zc[k] * ipow(z, a) * ipow(R, k);
    if (k > 0) Zr += f->zc[k] * ipow(z, a) * k * ipow(R, k - 1);
    if (a > 0) Zz += f->zc[k] * a * ipow(z, a - 1) * ipow(R, k);
  }
  double P = 0, Px = 0, Py = 0;
  for (int j = 0; j < f->nxy; ++j) {
    const int p = f->xp[j], q = f->yp[j];
    P += f->xyc[j] * ipow(x, p) * ipow(y, q);
    if (p > 0) Px += f->xyc[j] * p * ipow(x, p - 1) * ipow(y, q);
    if (q > 0) Py += f->xyc[j] * q * ipow(x, p) * ipow(y, q - 1);
  }
  *b = Z * P;
  g[0] = 2 * x * Zr * P + Z * Px;
  g[1] = 2 * y * Zr * P + Z * Py;
  g[2] = (Zz + 2 * z * Zr) * P;
}

/* B_lm and grad B_lm (B9.1, B9.2) for l = 1..l_max (at most 8): B1-B4 by
 * orc_blm, B5-B8 from the printed forms.  B is [nlm], dB [nlm][3] with
 * nlm = (l_max + 1)^2 - 1. */
void orc_blm_lmax(const double *d, int l_max, double *B, double *dB) {
  orc_blm(d, B, dB);
  if (l_max <= 4) return;
  const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const double r = sqrt(r2);
  for (int lm = 24; lm < nlm_of(l_max); ++lm) {
    int l = 5;
    while (lm >= lm_first(l + 1)) ++l;
    double b, g[3];
    printed_eval(&FORMS_5_8[lm - 24], d, &b, g);
    const double rl = pow(r, l);
    B[lm] = b / rl;
    for (int c = 0; c < 3; ++c) dB[lm * 3 + c] = g[c] / rl - l * b * d[c] / (rl * r2);
  }
}

/* Gauss-Legendre nodes and weights on [-1, 1] (n points, exact for
 * polynomials of degree 2n - 1): Newton's method on P_n from the three-term
 * recurrence, started at the Chebyshev-like guess cos(pi (i + 3/4) / (n + 1/2)). */
static void gauss_legendre(int n, double *xs, double *ws) {
  for (int i = 0; i < n; ++i) {
    double t = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      const double dt = p1 / dp;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    xs[i] = t;
    ws[i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

/* 4 pi / ((2l + 1) int B_lm^2 dOmega) over the unit sphere: 12 Gauss-Legendre
 * nodes in z = cos(theta) (exact to degree 23) times 36 equal steps in phi
 * (exact for trigonometric polynomials below degree 36); B_lm^2 has degree
 * 2l <= 16 in both. */
static double clm_quadrature(int lm, int l) {
  double xs[12], ws[12], acc = 0.0;
  gauss_legendre(12, xs, ws);
  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < 36; ++j) {
      const double ph = 2.0 * M_PI * j / 36.0, st = sqrt(1.0 - xs[i] * xs[i]);
      const double u[3] = {st * cos(ph), st * sin(ph), xs[i]};
      double B[NLM], dB[NLM * 3];
      orc_blm_lmax(u, l, B, dB);
      acc += ws[i] * (2.0 * M_PI / 36.0) * B[lm] * B[lm];
    }
  return 4.0 * M_PI / ((2.0 * l + 1.0) * acc);
}

double orc_clm_quadrature(int lm) {
  int l = 1;
  while (lm >= lm_first(l + 1)) ++l;
  return clm_quadrature(lm, l);
}

static void clm_init(void) {
  if (C_LM_ready) return;
  for (int l = 5; l <= LMAX; ++l)
    for (int m = 0; m <= 2 * l; ++m) C_LM[lm_first(l) + m] = clm_quadrature(lm_first(l) + m, l);
  C_LM_ready = 1;
}

/* A(u) = (3 u u^T - I)/2 and dA_ab/dd_c for the 4-body reading. */
static void quad_tensor(const double *d, double r, double A[9], double dA[27]) {
  double u[3] = {d[0] / r, d[1] / r, d[2] / r};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      A[a * 3 + b] = 1.5 * u[a] * u[b] - (a == b ? 0.5 : 0.0);
      for (int c = 0; c < 3; ++c) {
        double dua = ((a == c ? 1.0 : 0.0) - u[a] * u[c]) / r;
        double dub = ((b == c ? 1.0 : 0.0) - u[b] * u[c]) / r;
        dA[(a * 3 + b) * 3 + c] = 1.5 * (dua * u[b] + u[a] * dub);
      }
    }
}

static void mat3_mul(const double *X, const double *Y, double *Z) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += X[a * 3 + k] * Y[k * 3 + b];
      Z[a * 3 + b] = s;
    }
}

static double mat3_trace_prod(const double *X, const double *Y) { /* tr(X Y) */
  double s = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) s += X[a * 3 + b] * Y[b * 3 + a];
  return s;
}

/* ------------------------------------------------- Eq. 2: neighbour sets */

typedef struct {
  int j;        /* structure-local neighbour index */
  int sh[3];    /* image shift (na, nb, nc) */
  double d[3];  /* r_ij = r_j + n.H - r_i */
  double r;
} opair;

typedef struct {
  int n;
  int *off;     /* [n+1] */
  opair *p;
  int *rev;     /* index of the pair (j, i, -n) */
  int np;
} olist;

/* Images needed: |n_a| <= floor(rc / w_a) + 1, w_a = V / |b x c| the cell
 * width normal to the (b, c) face. */
static void image_range(const double *H, double rc, int k[3]) {
  const double *a = H, *b = H + 3, *c = H + 6;
  double bc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
  double ca[3] = {c[1] * a[2] - c[2] * a[1], c[2] * a[0] - c[0] * a[2], c[0] * a[1] - c[1] * a[0]};
  double ab[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  double vol = fabs(a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2]);
  double w[3] = {vol / sqrt(bc[0] * bc[0] + bc[1] * bc[1] + bc[2] * bc[2]),
                 vol / sqrt(ca[0] * ca[0] + ca[1] * ca[1] + ca[2] * ca[2]),
                 vol / sqrt(ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2])};
  for (int x = 0; x < 3; ++x) k[x] = (int)floor(rc / w[x]) + 1;
}

/* The pair vector and its squared length, in a fixed operation order. */
static double pair_vec(const double *H, const double *pi, const double *pj,
                       int na, int nb, int nc, double d[3]) {
  for (int x = 0; x < 3; ++x) {
    double s = ((double)na * H[x] + (double)nb * H[3 + x]) + (double)nc * H[6 + x];
    d[x] = (pj[x] + s) - pi[x];
  }
  return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
}

/* Brute force over every atom and image of one structure, in the canonical
 * order (j ascending, then shifts lexicographic). */
static int build_list(const double *H, int n, const double *pos, double rc,
                      olist *L) {
  int k[3];
  image_range(H, rc, k);
  double rc2 = rc * rc;
  L->n = n;
  L->off = (int *)malloc(sizeof(int) * (n + 1));
  int cap = 64 * n + 16, np = 0;
  L->p = (opair *)malloc(sizeof(opair) * cap);
  for (int i = 0; i < n; ++i) {
    L->off[i] = np;
    for (int j = 0; j < n; ++j)
      for (int na = -k[0]; na <= k[0]; ++na)
        for (int nb = -k[1]; nb <= k[1]; ++nb)
          for (int nc = -k[2]; nc <= k[2]; ++nc) {
            if (j == i && na == 0 && nb == 0 && nc == 0) continue;
            double d[3];
            double d2 = pair_vec(H, pos + 3 * i, pos + 3 * j, na, nb, nc, d);
            if (!(d2 < rc2)) continue;
            if (np == cap) {
              cap *= 2;
              L->p = (opair *)realloc(L->p, sizeof(opair) * cap);
            }
            opair *p = &L->p[np++];
            p->j = j;
            p->sh[0] = na; p->sh[1] = nb; p->sh[2] = nc;
            p->d[0] = d[0]; p->d[1] = d[1]; p->d[2] = d[2];
            p->r = sqrt(d2);
          }
  }
  L->off[n] = np;
  L->np = np;
  L->rev = (int *)malloc(sizeof(int) * (np > 0 ? np : 1));
  for (int i = 0; i < n; ++i)
    for (int q = L->off[i]; q < L->off[i + 1]; ++q) {
      const opair *p = &L->p[q];
      L->rev[q] = -1;
      for (int t = L->off[p->j]; t < L->off[p->j + 1]; ++t) {
        const opair *o = &L->p[t];
        if (o->j == i && o->sh[0] == -p->sh[0] && o->sh[1] == -p->sh[1] &&
            o->sh[2] == -p->sh[2]) {
          L->rev[q] = t;
          break;
        }
      }
    }
  return np;
}

static void free_list(olist *L) {
  free(L->off);
  free(L->p);
  free(L->rev);
}

long orc_neighbors(const orc_batch *b, double rc, long cap, long *off,
                   int *nbr_j, int *nbr_shift) {
  long total = 0;
  for (int s = 0; s < b->n_struct; ++s) {
    int a0 = b->struct_off[s], n = b->struct_off[s + 1] - a0;
    olist L;
    build_list(b->cell + 9 * s, n, b->pos + 3 * a0, rc, &L);
    if (off) {
      for (int i = 0; i < n; ++i) off[a0 + i] = total + L.off[i];
      off[a0 + n] = total + L.np;
    }
    for (int q = 0; q < L.np; ++q) {
      if (total + q < cap) {
        nbr_j[total + q] = a0 + L.p[q].j;
        for (int x = 0; x < 3; ++x) nbr_shift[3 * (total + q) + x] = L.p[q].sh[x];
      }
    }
    total += L.np;
    free_list(&L);
  }
  return total;
}

/* ------------------------------------------- per-atom descriptor state */

typedef struct {
  int type;
  double E;
  double *G;    /* [n_des]            Eqs. 5, 7 and the 4-body reading */
  double *S;    /* [nq_a][24]         Eq. 8 */
  double *Q;    /* [nq_a][9]          4-body tensor */
  double *FR;   /* [n_species][k_r]   sum_{j of type J} f_k(r_ij)           (C1.3) */
  double *SA;   /* [n_species][k_a][24] sum_{j of type J} f_k B_lm          (C2.8) */
  double *QA;   /* [n_species][k_a][9]  sum_{j of type J} f_k A(u_ij) */
  double *x;    /* [hidden]           D1.3 */
  double *Ep;   /* [n_des]            D1.5 (w.r.t. the unscaled G) */
  double *Epp;  /* [n_des][n_des]     D1.6 (w.r.t. the unscaled G) */
  double *Gs;   /* [n_des]            scaled network input s * G */
} oatom;

typedef struct {
  int n;
  oatom *a;
  double *mem;
} oatoms;

static void alloc_atoms(const orc_cfg *c, int n, oatoms *A) {
  int d = orc_num_des(c), S = c->n_species;
  long per = d + c->nq_a * NLM + c->nq_a * 9 + S * c->k_r + S * c->k_a * NLM +
             S * c->k_a * 9 + c->hidden + d + (long)d * d + d;
  A->n = n;
  A->a = (oatom *)calloc(n > 0 ? n : 1, sizeof(oatom));
  A->mem = (double *)calloc(per * (n > 0 ? n : 1), sizeof(double));
  for (int i = 0; i < n; ++i) {
    double *m = A->mem + per * i;
    oatom *t = &A->a[i];
    t->G = m; m += d;
    t->S = m; m += c->nq_a * NLM;
    t->Q = m; m += c->nq_a * 9;
    t->FR = m; m += S * c->k_r;
    t->SA = m; m += S * c->k_a * NLM;
    t->QA = m; m += S * c->k_a * 9;
    t->x = m; m += c->hidden;
    t->Ep = m; m += d;
    t->Epp = m; m += (long)d * d;
    t->Gs = m;
  }
}

static void free_atoms(oatoms *A) {
  free(A->a);
  free(A->mem);
}

/* Eqs. 5-8 (and the 4-body reading) for atom i of a structure. */
static void atom_descriptors(const orc_cfg *c, const double *P, const int *type,
                             int i, const olist *LR, const olist *LA, oatom *t) {
  clm_init();
  int I = type[i];
  double f[64], fp[64];
  t->type = I;
  for (int q = LR->off[i]; q < LR->off[i + 1]; ++q) {
    const opair *p = &LR->p[q];
    int J = type[p->j];
    orc_radial_basis(c->k_r, c->rc_r, p->r, f, fp);
    for (int n = 0; n < c->nq_r; ++n) {
      double g = 0; /* Eq. 6 */
      for (int k = 0; k < c->k_r; ++k) g += P[off_cR(c, I, J, n, k)] * f[k];
      t->G[v_rad(c, n)] += g; /* Eq. 5 */
    }
    for (int k = 0; k < c->k_r; ++k) t->FR[J * c->k_r + k] += f[k];
  }
  for (int q = LA->off[i]; q < LA->off[i + 1]; ++q) {
    const opair *p = &LA->p[q];
    int J = type[p->j];
    double B[NLM], dB[NLM * 3], A[9], dA[27];
    orc_radial_basis(c->k_a, c->rc_a, p->r, f, fp);
    orc_blm_lmax(p->d, c->l_max, B, dB);
    quad_tensor(p->d, p->r, A, dA);
    for (int n = 0; n < c->nq_a; ++n) {
      double g = 0; /* Eq. 6 with c^A */
      for (int k = 0; k < c->k_a; ++k) g += P[off_cA(c, I, J, n, k)] * f[k];
      for (int lm = 0; lm < nlm_of(c->l_max); ++lm) t->S[n * NLM + lm] += g * B[lm]; /* Eq. 8 */
      for (int ab = 0; ab < 9; ++ab) t->Q[n * 9 + ab] += g * A[ab];
    }
    for (int k = 0; k < c->k_a; ++k) {
      for (int lm = 0; lm < nlm_of(c->l_max); ++lm)
        t->SA[(J * c->k_a + k) * NLM + lm] += f[k] * B[lm];
      for (int ab = 0; ab < 9; ++ab) t->QA[(J * c->k_a + k) * 9 + ab] += f[k] * A[ab];
    }
  }
  for (int n = 0; n < c->nq_a; ++n) {
    for (int l = 1; l <= c->l_max; ++l) {
      double q = 0; /* Eq. 7 */
      for (int m = 0; m <= 2 * l; ++m) {
        double s = t->S[n * NLM + lm_first(l) + m];
        q += C_LM[lm_first(l) + m] * s * s;
      }
      t->G[v_ang(c, n, l)] = q;
    }
    if (c->four_body) {
      double Q2[9], Q3[9];
      mat3_mul(t->Q + 9 * n, t->Q + 9 * n, Q2);
      mat3_mul(Q2, t->Q + 9 * n, Q3);
      t->G[v_4b(c, n)] = Q3[0] + Q3[4] + Q3[8];
    }
  }
}

/* D1.1-D1.6 for element e; derivatives are taken w.r.t. the unscaled G. */
static void ann_eval(const orc_cfg *c, const double *P, const double *scale,
                     int e, const double *G, double *Gs, double *x, double *E,
                     double *Ep, double *Epp) {
  int d = orc_num_des(c), H = c->hidden;
  const double *W0 = P + off_W0(c, e), *b0 = P + off_b0(c, e),
               *w1 = P + off_w1(c, e), *b1 = P + off_b1(c, e);
  for (int v = 0; v < d; ++v) Gs[v] = scale[v] * G[v];
  double En = 0;
  for (int v = 0; v < d; ++v) Ep[v] = 0;
  if (Epp)
    for (long q = 0; q < (long)d * d; ++q) Epp[q] = 0;
  for (int mu = 0; mu < H; ++mu) {
    double z = b0[mu]; /* D1.2 */
    for (int v = 0; v < d; ++v) z += W0[mu * d + v] * Gs[v];
    double xm = tanh(z); /* D1.3 */
    x[mu] = xm;
    En += w1[mu] * xm; /* D1.1 */
    for (int v = 0; v < d; ++v) /* D1.4-D1.5 */
      Ep[v] += w1[mu] * (1.0 - xm * xm) * W0[mu * d + v] * scale[v];
    if (Epp) /* D1.6 */
      for (int v = 0; v < d; ++v)
        for (int vp = 0; vp < d; ++vp)
          Epp[v * d + vp] += w1[mu] * W0[mu * d + v] * W0[mu * d + vp] *
                             (-2.0 * xm * (1.0 - xm * xm)) * scale[v] * scale[vp];
  }
  *E = En + b1[0];
}

int orc_ann(const orc_cfg *c, const double *params, const double *scale, int e,
            const double *G, double *E, double *Ep, double *Epp) {
  int d = orc_num_des(c);
  double *Gs = (double *)malloc(sizeof(double) * d);
  double *x = (double *)malloc(sizeof(double) * c->hidden);
  ann_eval(c, params, scale, e, G, Gs, x, E, Ep, Epp);
  free(Gs);
  free(x);
  return 0;
}

/* dG_v/dr_ij for one pair of list L (0 radial, 1 angular), owner atom t.
 * C1.1 (radial); C2.1 with C2.3 (angular); 4-body: 3 tr(Q^2 dQ/dr_ij).
 * Also returns the per-pair pieces the mixed derivatives need. */
typedef struct {
  double f[64], fp[64];
  double u[3];
  double B[NLM], dB[NLM * 3];
  double A[9], dA[27];
  double dS[16 * NLM * 3]; /* dS_nlm/dr_ij */
  double dQ[16 * 27];      /* dQ_n/dr_ij, [n][ab][c] */
} pairwork;

static void pair_dG(const orc_cfg *c, const double *P, const oatom *t, int L,
                    const opair *p, int J, double *dG, pairwork *w) {
  clm_init();
  int d = orc_num_des(c), I = t->type;
  for (int q = 0; q < 3 * d; ++q) dG[q] = 0;
  for (int x = 0; x < 3; ++x) w->u[x] = p->d[x] / p->r;
  if (L == 0) {
    orc_radial_basis(c->k_r, c->rc_r, p->r, w->f, w->fp);
    for (int n = 0; n < c->nq_r; ++n) {
      double gp = 0;
      for (int k = 0; k < c->k_r; ++k) gp += P[off_cR(c, I, J, n, k)] * w->fp[k];
      for (int x = 0; x < 3; ++x) dG[v_rad(c, n) * 3 + x] = gp * w->u[x];
    }
    return;
  }
  orc_radial_basis(c->k_a, c->rc_a, p->r, w->f, w->fp);
  orc_blm_lmax(p->d, c->l_max, w->B, w->dB);
  quad_tensor(p->d, p->r, w->A, w->dA);
  for (int n = 0; n < c->nq_a; ++n) {
    double g = 0, gp = 0;
    for (int k = 0; k < c->k_a; ++k) {
      g += P[off_cA(c, I, J, n, k)] * w->f[k];
      gp += P[off_cA(c, I, J, n, k)] * w->fp[k];
    }
    for (int lm = 0; lm < nlm_of(c->l_max); ++lm)
      for (int x = 0; x < 3; ++x) /* C2.3 */
        w->dS[(n * NLM + lm) * 3 + x] = g * w->dB[lm * 3 + x] + gp * w->u[x] * w->B[lm];
    for (int l = 1; l <= c->l_max; ++l)
      for (int x = 0; x < 3; ++x) {
        double s = 0; /* C2.1 */
        for (int m = 0; m <= 2 * l; ++m) {
          int lm = lm_first(l) + m;
          s += C_LM[lm] * t->S[n * NLM + lm] * w->dS[(n * NLM + lm) * 3 + x];
        }
        dG[v_ang(c, n, l) * 3 + x] = 2.0 * s;
      }
    for (int ab = 0; ab < 9; ++ab)
      for (int x = 0; x < 3; ++x)
        w->dQ[(n * 9 + ab) * 3 + x] = gp * w->u[x] * w->A[ab] + g * w->dA[ab * 3 + x];
    if (c->four_body) {
      double Q2[9];
      mat3_mul(t->Q + 9 * n, t->Q + 9 * n, Q2);
      for (int x = 0; x < 3; ++x) {
        double s = 0;
        for (int a = 0; a < 3; ++a)
          for (int bb = 0; bb < 3; ++bb)
            s += Q2[a * 3 + bb] * w->dQ[(n * 9 + bb * 3 + a) * 3 + x];
        dG[v_4b(c, n) * 3 + x] = 3.0 * s;
      }
    }
  }
}

/* ------------------------------------------------------ structure state */

typedef struct {
  olist L[2];    /* 0 radial, 1 angular */
  oatoms at;
  double *dpair[2]; /* dE_i/dr_ij per pair, [np][3]  (C3.6) */
} ostruct;

static void struct_forward(const orc_cfg *c, const double *P, const double *scale,
                           const orc_batch *b, int s, ostruct *st, int want_epp) {
  int a0 = b->struct_off[s], n = b->struct_off[s + 1] - a0;
  const double *H = b->cell + 9 * s, *pos = b->pos + 3 * a0;
  const int *type = b->type + a0;
  int d = orc_num_des(c);
  build_list(H, n, pos, c->rc_r, &st->L[0]);
  build_list(H, n, pos, c->rc_a, &st->L[1]);
  alloc_atoms(c, n, &st->at);
  for (int i = 0; i < n; ++i) {
    oatom *t = &st->at.a[i];
    atom_descriptors(c, P, type, i, &st->L[0], &st->L[1], t);
    ann_eval(c, P, scale, t->type, t->G, t->Gs, t->x, &t->E, t->Ep,
             want_epp ? t->Epp : NULL);
  }
  double *dG = (double *)malloc(sizeof(double) * 3 * d);
  pairwork *w = (pairwork *)malloc(sizeof(pairwork));
  for (int L = 0; L < 2; ++L) {
    olist *li = &st->L[L];
    st->dpair[L] = (double *)calloc(3 * (li->np > 0 ? li->np : 1), sizeof(double));
    for (int i = 0; i < n; ++i)
      for (int q = li->off[i]; q < li->off[i + 1]; ++q) {
        pair_dG(c, P, &st->at.a[i], L, &li->p[q], type[li->p[q].j], dG, w);
        for (int x = 0; x < 3; ++x) {
          double s2 = 0; /* C3.6 */
          for (int v = 0; v < d; ++v) s2 += st->at.a[i].Ep[v] * dG[v * 3 + x];
          st->dpair[L][3 * q + x] = s2;
        }
      }
  }
  free(dG);
  free(w);
}

static void struct_free(ostruct *st) {
  for (int L = 0; L < 2; ++L) {
    free_list(&st->L[L]);
    free(st->dpair[L]);
  }
  free_atoms(&st->at);
}

/* Eqs. 1, 3 and 4: energies, forces, total (symmetrised) virial. */
static void struct_outputs(const ostruct *st, double *E_atom, double *Es,
                           double *F, double *Wsym) {
  int n = st->at.n;
  double W[9] = {0};
  *Es = 0;
  for (int i = 0; i < n; ++i) {
    if (E_atom) E_atom[i] = st->at.a[i].E;
    *Es += st->at.a[i].E;
    double Fi[3] = {0, 0, 0};
    for (int L = 0; L < 2; ++L) {
      const olist *li = &st->L[L];
      for (int q = li->off[i]; q < li->off[i + 1]; ++q) {
        int r = li->rev[q];
        for (int x = 0; x < 3; ++x) /* Eq. 3 */
          Fi[x] += st->dpair[L][3 * q + x] - st->dpair[L][3 * r + x];
        for (int a = 0; a < 3; ++a) /* Eq. 4 */
          for (int bb = 0; bb < 3; ++bb)
            W[a * 3 + bb] += li->p[q].d[a] * st->dpair[L][3 * r + bb];
      }
    }
    for (int x = 0; x < 3; ++x) F[3 * i + x] = Fi[x];
  }
  Wsym[0] = W[0];
  Wsym[1] = W[4];
  Wsym[2] = W[8];
  Wsym[3] = 0.5 * (W[1] + W[3]);
  Wsym[4] = 0.5 * (W[5] + W[7]);
  Wsym[5] = 0.5 * (W[6] + W[2]);
}

int orc_descriptors(const orc_cfg *c, const double *params, const orc_batch *b,
                    double *G) {
  int d = orc_num_des(c);
  for (int s = 0; s < b->n_struct; ++s) {
    int a0 = b->struct_off[s], n = b->struct_off[s + 1] - a0;
    olist LR, LA;
    oatoms at;
    build_list(b->cell + 9 * s, n, b->pos + 3 * a0, c->rc_r, &LR);
    build_list(b->cell + 9 * s, n, b->pos + 3 * a0, c->rc_a, &LA);
    alloc_atoms(c, n, &at);
    for (int i = 0; i < n; ++i) {
      atom_descriptors(c, params, b->type + a0, i, &LR, &LA, &at.a[i]);
      memcpy(G + (long)(a0 + i) * d, at.a[i].G, sizeof(double) * d);
    }
    free_atoms(&at);
    free_list(&LR);
    free_list(&LA);
  }
  return 0;
}

int orc_forward(const orc_cfg *c, const double *params, const double *scale,
                const orc_batch *b, double *E_atom, double *E_struct, double *F,
                double *W_struct) {
  for (int s = 0; s < b->n_struct; ++s) {
    int a0 = b->struct_off[s];
    ostruct st;
    struct_forward(c, params, scale, b, s, &st, 0);
    struct_outputs(&st, E_atom ? E_atom + a0 : NULL, &E_struct[s], F + 3 * a0,
                   W_struct + 6 * s);
    struct_free(&st);
  }
  return 0;
}

/* ------------------------------------------------------------ Eqs. 9-12 */

static void loss_terms(const orc_cfg *c, const double *params, const orc_batch *b,
                       const orc_labels *y, const double *Es, const double *F,
                       const double *W, double *terms) {
  int S = b->n_struct, N = b->struct_off[S];
  double Le = 0, Lf = 0, Lv = 0;
  for (int s = 0; s < S; ++s) {
    double ns = b->struct_off[s + 1] - b->struct_off[s];
    double de = Es[s] / ns - y->energy[s];
    Le += de * de;
    for (int q = 0; q < 6; ++q) {
      double dv = W[6 * s + q] / ns - y->virial[6 * s + q];
      Lv += dv * dv;
    }
  }
  for (long q = 0; q < 3L * N; ++q) {
    double df = F[q] - y->force[q];
    Lf += df * df;
  }
  Le /= S;                 /* Eq. 10 */
  Lf /= 3.0 * N;           /* Eq. 11 */
  Lv /= 6.0 * S;           /* Eq. 12 */
  long np = orc_num_params(c);
  double l2 = 0;
  for (long q = 0; q < np; ++q) l2 += params[q] * params[q];
  l2 = y->lambda_l2 * l2 / np;
  double L;
  if (y->loss_form == 1)
    L = y->lambda_e * sqrt(Le) + y->lambda_f * sqrt(Lf) + y->lambda_v * sqrt(Lv) + l2;
  else
    L = y->lambda_e * Le + y->lambda_f * Lf + y->lambda_v * Lv + l2; /* Eq. 9 */
  terms[0] = L;
  terms[1] = Le;
  terms[2] = Lf;
  terms[3] = Lv;
}

int orc_loss(const orc_cfg *c, const double *params, const double *scale,
             const orc_batch *b, const orc_labels *y, double *terms) {
  int S = b->n_struct, N = b->struct_off[S];
  double *Es = (double *)malloc(sizeof(double) * S);
  double *W = (double *)malloc(sizeof(double) * 6 * S);
  double *F = (double *)malloc(sizeof(double) * 3 * (N > 0 ? N : 1));
  orc_forward(c, params, scale, b, NULL, Es, F, W);
  loss_terms(c, params, b, y, Es, F, W, terms);
  free(Es);
  free(W);
  free(F);
  return 0;
}

/* ------------------------------------------- explicit parameter gradients */

/* dE_i/dtheta: D1.7-D1.10 for the network, C3.5 (with C1.3, C2.5, C2.8) for c. */
static void energy_jacobian(const orc_cfg *c, const double *P, const oatom *t,
                            double *gE /* [N_par], accumulated */) {
  clm_init();
  int d = orc_num_des(c), H = c->hidden, e = t->type, I = t->type;
  const double *w1 = P + off_w1(c, e);
  for (int mu = 0; mu < H; ++mu) {
    double xm = t->x[mu];
    for (int v = 0; v < d; ++v) /* D1.9 */
      gE[off_W0(c, e) + mu * d + v] += w1[mu] * (1.0 - xm * xm) * t->Gs[v];
    gE[off_b0(c, e) + mu] += w1[mu] * (1.0 - xm * xm); /* D1.10 */
    gE[off_w1(c, e) + mu] += xm;                        /* D1.7 */
  }
  gE[off_b1(c, e)] += 1.0; /* D1.8 */
  for (int Jp = 0; Jp < c->n_species; ++Jp) {
    for (int n = 0; n < c->nq_r; ++n)
      for (int k = 0; k < c->k_r; ++k)
        gE[off_cR(c, I, Jp, n, k)] += t->Ep[v_rad(c, n)] * t->FR[Jp * c->k_r + k];
    for (int n = 0; n < c->nq_a; ++n)
      for (int k = 0; k < c->k_a; ++k) {
        double s = 0;
        const double *SA = t->SA + (Jp * c->k_a + k) * NLM;
        for (int l = 1; l <= c->l_max; ++l) {
          double dq = 0; /* C2.5 with C2.8 */
          for (int m = 0; m <= 2 * l; ++m) {
            int lm = lm_first(l) + m;
            dq += 2.0 * C_LM[lm] * t->S[n * NLM + lm] * SA[lm];
          }
          s += t->Ep[v_ang(c, n, l)] * dq;
        }
        if (c->four_body) {
          double Q2[9];
          mat3_mul(t->Q + 9 * n, t->Q + 9 * n, Q2);
          s += t->Ep[v_4b(c, n)] * 3.0 * mat3_trace_prod(Q2, t->QA + (Jp * c->k_a + k) * 9);
        }
        gE[off_cA(c, I, Jp, n, k)] += s;
      }
  }
}

/* J[theta][x] = d/dtheta (dE_a/dr_ab) for one pair owned by atom t (list L).
 * Network parameters: D1.11-D1.17.  Coefficients: C3.7-C3.8 expanded as
 * C3.9 / C3.16 (radial pairs) and C3.12 / C3.14 (angular pairs), with the
 * mixed terms C1.4, C2.6, C2.9 and the species mapping of Alg. 1.
 * Every entry of the owner's element network and of c^{type(t), *} is
 * written; all other entries are zero by construction and left untouched. */
static void pair_jacobian(const orc_cfg *c, const double *P, const double *scale,
                          const oatom *t, int L, const opair *p, int typej,
                          double *J, double *dG, double *h, pairwork *w) {
  clm_init();
  int d = orc_num_des(c), H = c->hidden, e = t->type, I = t->type;
  pair_dG(c, P, t, L, p, typej, dG, w);
  const double *W0 = P + off_W0(c, e), *w1 = P + off_w1(c, e);

  for (int mu = 0; mu < H; ++mu) {
    double xm = t->x[mu];
    double t1 = 1.0 - xm * xm, t2 = -2.0 * xm * t1;
    for (int vp = 0; vp < d; ++vp) /* W0_{mu v'}: D1.14 contracted as D1.13 */
      for (int x = 0; x < 3; ++x) {
        double acc = 0;
        for (int v = 0; v < d; ++v) {
          double ep = w1[mu] * (t2 * W0[mu * d + v] * t->Gs[vp] + (v == vp ? t1 : 0.0));
          acc += scale[v] * ep * dG[v * 3 + x];
        }
        J[(off_W0(c, e) + mu * d + vp) * 3 + x] = acc;
      }
    for (int x = 0; x < 3; ++x) {
      double ab0 = 0, aw1 = 0;
      for (int v = 0; v < d; ++v) {
        ab0 += scale[v] * (t2 * w1[mu] * W0[mu * d + v]) * dG[v * 3 + x]; /* D1.16-D1.17 */
        aw1 += scale[v] * (t1 * W0[mu * d + v]) * dG[v * 3 + x];          /* D1.12-D1.13 */
      }
      J[(off_b0(c, e) + mu) * 3 + x] = ab0;
      J[(off_w1(c, e) + mu) * 3 + x] = aw1;
    }
  }
  for (int x = 0; x < 3; ++x) J[off_b1(c, e) * 3 + x] = 0.0; /* D1.15 */

  /* h_v' = sum_v E''_{v' v} dG_v/dr_ij  (C3.8) */
  for (int vp = 0; vp < d; ++vp)
    for (int x = 0; x < 3; ++x) {
      double s = 0;
      for (int v = 0; v < d; ++v) s += t->Epp[vp * d + v] * dG[v * 3 + x];
      h[vp * 3 + x] = s;
    }

  for (int Jp = 0; Jp < c->n_species; ++Jp) {
    /* radial coefficients c^R_{nk}^{I J'} */
    for (int n = 0; n < c->nq_r; ++n)
      for (int k = 0; k < c->k_r; ++k)
        for (int x = 0; x < 3; ++x) {
          double val = t->FR[Jp * c->k_r + k] * h[v_rad(c, n) * 3 + x];
          if (L == 0 && typej == Jp) /* C1.4 */
            val += t->Ep[v_rad(c, n)] * w->fp[k] * w->u[x];
          J[off_cR(c, I, Jp, n, k) * 3 + x] = val;
        }
    /* angular coefficients c^A_{nk}^{I J'} */
    for (int n = 0; n < c->nq_a; ++n) {
      double Q2[9], dQ4dc_base[9];
      const double *Qn = t->Q + 9 * n;
      mat3_mul(Qn, Qn, Q2);
      (void)dQ4dc_base;
      for (int k = 0; k < c->k_a; ++k) {
        const double *SA = t->SA + (Jp * c->k_a + k) * NLM;
        const double *QA = t->QA + (Jp * c->k_a + k) * 9;
        double dGdc[LMAX + 1]; /* dq_nl/dc for l = 1..l_max, C2.5 with C2.8 */
        for (int l = 1; l <= c->l_max; ++l) {
          double s = 0;
          for (int m = 0; m <= 2 * l; ++m) {
            int lm = lm_first(l) + m;
            s += 2.0 * C_LM[lm] * t->S[n * NLM + lm] * SA[lm];
          }
          dGdc[l] = s;
        }
        double dG4dc = 0, QQA[9], QAQ[9];
        if (c->four_body) {
          dG4dc = 3.0 * mat3_trace_prod(Q2, QA);
          mat3_mul(QA, Qn, QAQ);
          mat3_mul(Qn, QA, QQA);
        }
        for (int x = 0; x < 3; ++x) {
          double val = 0;
          for (int l = 1; l <= c->l_max; ++l) val += dGdc[l] * h[v_ang(c, n, l) * 3 + x];
          if (c->four_body) val += dG4dc * h[v_4b(c, n) * 3 + x];
          if (L == 1) {
            for (int l = 1; l <= c->l_max; ++l) {
              double mixed = 0; /* C2.6 with C2.8, C2.9 and Alg. 1 */
              for (int m = 0; m <= 2 * l; ++m) {
                int lm = lm_first(l) + m;
                double term = SA[lm] * w->dS[(n * NLM + lm) * 3 + x];
                if (typej == Jp)
                  term += t->S[n * NLM + lm] *
                          (w->f[k] * w->dB[lm * 3 + x] + w->fp[k] * w->u[x] * w->B[lm]);
                mixed += 2.0 * C_LM[lm] * term;
              }
              val += t->Ep[v_ang(c, n, l)] * mixed;
            }
            if (c->four_body) {
              double dQx[9], mixed4 = 0;
              for (int ab = 0; ab < 9; ++ab) dQx[ab] = w->dQ[(n * 9 + ab) * 3 + x];
              mixed4 += 3.0 * (mat3_trace_prod(QAQ, dQx) + mat3_trace_prod(QQA, dQx));
              if (typej == Jp) {
                double dM[9];
                for (int ab = 0; ab < 9; ++ab)
                  dM[ab] = w->fp[k] * w->u[x] * w->A[ab] + w->f[k] * w->dA[ab * 3 + x];
                mixed4 += 3.0 * mat3_trace_prod(Q2, dM);
              }
              val += t->Ep[v_4b(c, n)] * mixed4;
            }
          }
          J[off_cA(c, I, Jp, n, k) * 3 + x] = val;
        }
      }
    }
  }
}

/* The parameter ranges a pair Jacobian of an atom of species e can touch:
 * its element network, c^R_{e,*} and c^A_{e,*}. */
static void owner_ranges(const orc_cfg *c, int e, long r[3][2]) {
  r[0][0] = off_W0(c, e);
  r[0][1] = off_b1(c, e) + 1;
  r[1][0] = off_cR(c, e, 0, 0, 0);
  r[1][1] = r[1][0] + (long)c->n_species * c->nq_r * c->k_r;
  r[2][0] = off_cA(c, e, 0, 0, 0);
  r[2][1] = r[2][0] + (long)c->n_species * c->nq_a * c->k_a;
}

int orc_loss_grad(const orc_cfg *c, const double *params, const double *scale,
                  const orc_batch *b, const orc_labels *y, double *terms,
                  double *grad) {
  int S = b->n_struct, N = b->struct_off[S], d = orc_num_des(c);
  long np = orc_num_params(c);
  double *Es = (double *)malloc(sizeof(double) * S);
  double *W = (double *)malloc(sizeof(double) * 6 * S);
  double *F = (double *)malloc(sizeof(double) * 3 * (N > 0 ? N : 1));
  orc_forward(c, params, scale, b, NULL, Es, F, W);
  loss_terms(c, params, b, y, Es, F, W, terms);

  double ke = 1.0, kf = 1.0, kv = 1.0; /* RMSE chain factors */
  if (y->loss_form == 1) {
    ke = terms[1] > 0 ? 0.5 / sqrt(terms[1]) : 0.0;
    kf = terms[2] > 0 ? 0.5 / sqrt(terms[2]) : 0.0;
    kv = terms[3] > 0 ? 0.5 / sqrt(terms[3]) : 0.0;
  }
  for (long q = 0; q < np; ++q) grad[q] = 2.0 * y->lambda_l2 * params[q] / np;

  double *gE = (double *)malloc(sizeof(double) * np);
  double *gW = (double *)malloc(sizeof(double) * 9 * np);
  double *gF = (double *)malloc(sizeof(double) * 3 * np);
  double *J1 = (double *)malloc(sizeof(double) * 3 * np);
  double *J2 = (double *)malloc(sizeof(double) * 3 * np);
  double *dG = (double *)malloc(sizeof(double) * 3 * d);
  double *h = (double *)malloc(sizeof(double) * 3 * d);
  pairwork *w = (pairwork *)malloc(sizeof(pairwork));

  for (int s = 0; s < S; ++s) {
    int a0 = b->struct_off[s], n = b->struct_off[s + 1] - a0;
    const int *type = b->type + a0;
    ostruct st;
    struct_forward(c, params, scale, b, s, &st, 1);
    memset(gE, 0, sizeof(double) * np);
    memset(gW, 0, sizeof(double) * 9 * np);
    for (int i = 0; i < n; ++i) {
      energy_jacobian(c, params, &st.at.a[i], gE);
      memset(gF, 0, sizeof(double) * 3 * np);
      for (int L = 0; L < 2; ++L) {
        const olist *li = &st.L[L];
        for (int q = li->off[i]; q < li->off[i + 1]; ++q) {
          const opair *p = &li->p[q];
          int r = li->rev[q];
          long r1[3][2], r2[3][2];
          /* d/dtheta (dE_i/dr_ij) and d/dtheta (dE_j/dr_ji) */
          pair_jacobian(c, params, scale, &st.at.a[i], L, p, type[p->j], J1, dG, h, w);
          pair_jacobian(c, params, scale, &st.at.a[p->j], L, &li->p[r], type[i], J2,
                        dG, h, w);
          owner_ranges(c, type[i], r1);
          owner_ranges(c, type[p->j], r2);
          for (int g = 0; g < 3; ++g) /* Eq. 3 / C3.11, C3.13, C3.15, C3.17 */
            for (long t = r1[g][0]; t < r1[g][1]; ++t)
              for (int x = 0; x < 3; ++x) gF[t * 3 + x] += J1[t * 3 + x];
          for (int g = 0; g < 3; ++g)
            for (long t = r2[g][0]; t < r2[g][1]; ++t)
              for (int x = 0; x < 3; ++x) {
                gF[t * 3 + x] -= J2[t * 3 + x];
                for (int a = 0; a < 3; ++a) /* Eq. 4 / C3.18-C3.20 */
                  gW[t * 9 + a * 3 + x] += p->d[a] * J2[t * 3 + x];
              }
        }
      }
      /* Eq. 15 / D1.20 */
      const double cf = y->lambda_f * kf * 2.0 / (3.0 * N);
      for (int x = 0; x < 3; ++x) {
        double res = F[3 * (a0 + i) + x] - y->force[3 * (a0 + i) + x];
        for (long t = 0; t < np; ++t) grad[t] += cf * res * gF[t * 3 + x];
      }
    }
    double ns = n;
    /* Eq. 14 / D1.19 */
    double ce = y->lambda_e * ke * 2.0 / S * (Es[s] / ns - y->energy[s]) / ns;
    for (long t = 0; t < np; ++t) grad[t] += ce * gE[t];
    /* Eq. 16 / D1.21 on the symmetrised components */
    for (int q = 0; q < 6; ++q) {
      static const int ia[6] = {0, 1, 2, 0, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 0};
      double cv = y->lambda_v * kv * 2.0 / (6.0 * S) * (W[6 * s + q] / ns - y->virial[6 * s + q]) / ns;
      for (long t = 0; t < np; ++t) {
        double dw = 0.5 * (gW[t * 9 + ia[q] * 3 + ib[q]] + gW[t * 9 + ib[q] * 3 + ia[q]]);
        grad[t] += cv * dw;
      }
    }
    struct_free(&st);
  }
  free(gE); free(gW); free(gF); free(J1); free(J2); free(dG); free(h); free(w);
  free(Es); free(W); free(F);
  return 0;
}

/* ------------------------------------------------------- Adam, Eq. 17 */

/* Adam (Kingma & Ba) with bias correction; optional decoupled weight decay
 * (AdamW).  t is the 1-based update count. */
void orc_adam(long n, double *theta, double *m, double *v, const double *g,
              long t, double lr, double beta1, double beta2, double eps,
              double weight_decay) {
  double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
  for (long q = 0; q < n; ++q) {
    m[q] = beta1 * m[q] + (1.0 - beta1) * g[q];
    v[q] = beta2 * v[q] + (1.0 - beta2) * g[q] * g[q];
    double mh = m[q] / c1, vh = v[q] / c2;
    theta[q] -= lr * (mh / (sqrt(vh) + eps) + weight_decay * theta[q]);
  }
}

/* Eq. 17: linear warm-up from lr_stop to lr_start, then cosine decay. */
double orc_lr(double lr_start, double lr_stop, long s, long n_warmup, long n_total) {
  if (s < n_warmup)
    return lr_stop + (double)s / (double)n_warmup * (lr_start - lr_stop);
  if (s > n_total) s = n_total;
  double span = (double)(n_total - n_warmup);
  double frac = span > 0 ? (double)(s - n_warmup) / span : 1.0;
  return lr_stop + (lr_start - lr_stop) * 0.5 * (1.0 + cos(M_PI * frac));
}
