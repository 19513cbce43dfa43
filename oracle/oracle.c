/*
 * oracle.c -- FP64 CPU oracle of the finite-thickness slice projection operator
 * of GaussianPile (arXiv 2603.20611).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py.  The product library never touches it.
 *
 * The forward pass follows the paper's own route for every (Gaussian, slice):
 *   world covariance            Sigma = R S S^T R^T                (Sec. S1)
 *   camera transform            mu_c = R_c mu + t, Sigma_c = R_c Sigma R_c^T
 *   axial re-parameterisation   Sigma_e^-1 = Sigma_c^-1 + e3 e3^T / sigma_z^2,
 *                               mu_e = Sigma_e Sigma_c^-1 mu_c      (Eq. 6)
 *   opacity modulation          opacity_r = exp(-1/2 (mu_c^T Sigma_c^-1 mu_c
 *                                            - mu_e^T Sigma_e^-1 mu_e)) (Eq. 7)
 *   screen-space projection     Sigma_2d = Sigma_e[0:2,0:2], mu_2d = mu_e[0:2] (Eq. 8)
 *   normalised intensity        a~ = alpha opacity_r / sqrt(det Sigma_2d)   (Eq. 9)
 *   additive rasterisation      I(p) = sum_i a~_i exp(-1/2 d^T Sigma_2d^-1 d) (Eq. 10)
 * with explicit 3x3 inverses, and no culling at all (brute force).
 *
 * The backward pass is reverse-mode differentiation of exactly those steps,
 * in reverse order (Sec. S2 lists the same chain; its printed formulas are not
 * transcribed -- each step below is the plain derivative of the forward step
 * above it, with every matrix treated as a general 3x3 / 2x2 matrix).
 *
 * Pins (tests/test_oracle_pins.py): closed forms for isotropic and axis-aligned
 * Gaussians, the sigma_z -> infinity and sigma_z -> 0 limits of Fig. 1(b)(c),
 * quadrature of the convolution integral Eq. 5, mass, linearity,
 * equivariances, and central finite differences of every gradient.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------- helpers */

/* Rotation matrix of the unit quaternion q/|q|, q = (w, x, y, z). */
static void quat_to_rot(const double* q, double R[3][3], double qn[4]) {
  double nrm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double w = q[0] / nrm, x = q[1] / nrm, y = q[2] / nrm, z = q[3] / nrm;
  qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z;
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}

/* dR[i][j]/d(w,x,y,z) of the formula above (unit quaternion components). */
static void rot_partials(const double qn[4], double P[4][3][3]) {
  double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
  memset(P, 0, sizeof(double) * 36);
  /* d/dw */
  P[0][0][1] = -2 * z; P[0][0][2] = 2 * y; P[0][1][0] = 2 * z;
  P[0][1][2] = -2 * x; P[0][2][0] = -2 * y; P[0][2][1] = 2 * x;
  /* d/dx */
  P[1][0][1] = 2 * y; P[1][0][2] = 2 * z; P[1][1][0] = 2 * y; P[1][1][1] = -4 * x;
  P[1][1][2] = -2 * w; P[1][2][0] = 2 * z; P[1][2][1] = 2 * w; P[1][2][2] = -4 * x;
  /* d/dy */
  P[2][0][0] = -4 * y; P[2][0][1] = 2 * x; P[2][0][2] = 2 * w; P[2][1][0] = 2 * x;
  P[2][1][2] = 2 * z; P[2][2][0] = -2 * w; P[2][2][1] = 2 * z; P[2][2][2] = -4 * y;
  /* d/dz */
  P[3][0][0] = -4 * z; P[3][0][1] = -2 * w; P[3][0][2] = 2 * x; P[3][1][0] = 2 * w;
  P[3][1][1] = -4 * z; P[3][1][2] = 2 * y; P[3][2][0] = 2 * x; P[3][2][1] = 2 * y;
}

/* Inverse of a 3x3 matrix by the adjugate: A^-1 = adj(A) / det(A). */
static double inv3(const double A[3][3], double B[3][3]) {
  double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
  double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
  double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
  double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
  double id = 1.0 / det;
  B[0][0] = c00 * id;
  B[1][0] = c01 * id;
  B[2][0] = c02 * id;
  B[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * id;
  B[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * id;
  B[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * id;
  B[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * id;
  B[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * id;
  B[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * id;
  return det;
}

static void matmul3(const double A[3][3], const double B[3][3], double C[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A[i][k] * B[k][j];
      C[i][j] = s;
    }
}

static void transpose3(const double A[3][3], double B[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) B[i][j] = A[j][i];
}

static void matvec3(const double A[3][3], const double v[3], double r[3]) {
  for (int i = 0; i < 3; ++i) r[i] = A[i][0] * v[0] + A[i][1] * v[1] + A[i][2] * v[2];
}

/* Camera axis permutation R_c: camera coordinate j is world coordinate perm[j]. */
static int axis_perm(int axis, int perm[3]) {
  if (axis == 2) { perm[0] = 0; perm[1] = 1; perm[2] = 2; return 0; }
  if (axis == 1) { perm[0] = 0; perm[1] = 2; perm[2] = 1; return 0; }
  if (axis == 0) { perm[0] = 1; perm[1] = 2; perm[2] = 0; return 0; }
  return -1;
}

static void perm_matrix(const int perm[3], double Rc[3][3]) {
  memset(Rc, 0, sizeof(double) * 9);
  for (int j = 0; j < 3; ++j) Rc[j][perm[j]] = 1.0;
}

/* View matrix [R_c | t] of a general slice orientation (Sec. S1): R_c must be
 * finite and orthonormal to within 1e-3 (the focal plane is then a true plane
 * with unit pixel spacing), t finite.  Returns -1 otherwise. */
static int view_matrix(const orc_view* v, double Rc[3][3], double tc[3]) {
  if (!v) return -1;
  for (int k = 0; k < 9; ++k)
    if (!isfinite(v->R[k])) return -1;
  for (int k = 0; k < 3; ++k)
    if (!isfinite(v->t[k])) return -1;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Rc[r][c] = v->R[3 * r + c];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double d = Rc[r][0] * Rc[c][0] + Rc[r][1] * Rc[c][1] + Rc[r][2] * Rc[c][2];
      if (fabs(d - (r == c ? 1.0 : 0.0)) > 1e-3) return -1;
    }
  for (int k = 0; k < 3; ++k) tc[k] = v->t[k];
  return 0;
}

/* The view of an axis-aligned slice: R_c the permutation of axis, t = 0. */
static int axis_view(int axis, double Rc[3][3], double tc[3]) {
  int perm[3];
  if (axis_perm(axis, perm)) return -1;
  perm_matrix(perm, Rc);
  tc[0] = tc[1] = tc[2] = 0.0;
  return 0;
}

/* World covariance of Gaussian i: Sigma = M M^T with M = R S, S = diag(mod s). */
typedef struct {
  double R[3][3], M[3][3], Sig[3][3], qn[4], qnorm, Sd[3];
} world_cov;

static void world_covariance(const orc_set* g, int64_t i, world_cov* w) {
  const double* q = g->quat + 4 * i;
  quat_to_rot(q, w->R, w->qn);
  w->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int j = 0; j < 3; ++j) w->Sd[j] = g->scale_mod * g->scale[3 * i + j];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) w->M[r][c] = w->R[r][c] * w->Sd[c];
  double Mt[3][3];
  transpose3(w->M, Mt);
  matmul3(w->M, Mt, w->Sig);
}

/* Everything the paper computes for one (Gaussian, slice), Eq. 6-9. */
typedef struct {
  double Sc[3][3];  /* Sigma_c */
  double Kc[3][3];  /* Sigma_c^-1 */
  double Ke[3][3];  /* Sigma_e^-1 */
  double Se[3][3];  /* Sigma_e */
  double muc[3];    /* mu_c */
  double b[3];      /* Sigma_c^-1 mu_c */
  double mue[3];    /* mu_e */
  double op;        /* opacity_r */
  double S2[2][2];  /* Sigma_2d */
  double det2;      /* det Sigma_2d */
  double C[2][2];   /* Sigma_2d^-1 */
  double at;        /* a~ */
} slice_proj;

static void project(const orc_set* g, int64_t i, const world_cov* w, const double Rc[3][3],
                    const double tc[3], double zs, double sigma_z, slice_proj* p) {
  /* camera transform (Sec. S1): mu_c = R_c mu + t, with the view's t shifted by
   * -z_s e3 so that the plane of slice s is z_c = 0 */
  matvec3(Rc, g->mu + 3 * i, p->muc);
  for (int k = 0; k < 3; ++k) p->muc[k] += tc[k];
  p->muc[2] -= zs;
  double Rct[3][3], tmp[3][3];
  transpose3(Rc, Rct);
  matmul3(Rc, w->Sig, tmp);
  matmul3(tmp, Rct, p->Sc);
  /* Eq. 6 */
  inv3(p->Sc, p->Kc);
  memcpy(p->Ke, p->Kc, sizeof(p->Ke));
  p->Ke[2][2] += 1.0 / (sigma_z * sigma_z);
  inv3(p->Ke, p->Se);
  matvec3(p->Kc, p->muc, p->b);
  matvec3(p->Se, p->b, p->mue);
  /* Eq. 7 */
  double Kemue[3];
  matvec3(p->Ke, p->mue, Kemue);
  double qc = p->muc[0] * p->b[0] + p->muc[1] * p->b[1] + p->muc[2] * p->b[2];
  double qe = p->mue[0] * Kemue[0] + p->mue[1] * Kemue[1] + p->mue[2] * Kemue[2];
  p->op = exp(-0.5 * (qc - qe));
  /* Eq. 8 */
  p->S2[0][0] = p->Se[0][0];
  p->S2[0][1] = p->Se[1][0];
  p->S2[1][0] = p->Se[1][0];
  p->S2[1][1] = p->Se[1][1];
  p->det2 = p->S2[0][0] * p->S2[1][1] - p->S2[0][1] * p->S2[1][0];
  p->C[0][0] = p->S2[1][1] / p->det2;
  p->C[0][1] = -p->S2[0][1] / p->det2;
  p->C[1][0] = -p->S2[1][0] / p->det2;
  p->C[1][1] = p->S2[0][0] / p->det2;
  /* Eq. 9 */
  p->at = g->alpha[i] * p->op / sqrt(p->det2);
}

/* Eq. 10 term of one Gaussian at camera point (x, y). */
static double pixel_term(const slice_proj* p, double x, double y) {
  double dx = x - p->mue[0], dy = y - p->mue[1];
  double m = dx * (p->C[0][0] * dx + p->C[0][1] * dy) + dy * (p->C[1][0] * dx + p->C[1][1] * dy);
  return p->at * exp(-0.5 * m);
}

static int check_set(const orc_set* g) {
  if (!g || g->n < 0) return -1;
  if (g->n > 0 && (!g->mu || !g->scale || !g->quat || !g->alpha)) return -1;
  return 0;
}

/* ---------------------------------------------------------------- forward */

static int render_rc(const orc_set* g, int S, const double* z, int H, int W, double sigma_z,
                     const double Rc[3][3], const double tc[3], double* out) {
  if (check_set(g) || S < 0 || H < 0 || W < 0 || !(sigma_z > 0)) return -1;
  int64_t n = g->n;
  slice_proj* P = (slice_proj*)malloc(sizeof(slice_proj) * (size_t)(n > 0 ? n : 1));
  world_cov* Wc = (world_cov*)malloc(sizeof(world_cov) * (size_t)(n > 0 ? n : 1));
  if (!P || !Wc) { free(P); free(Wc); return -2; }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) world_covariance(g, i, &Wc[i]);
  for (int s = 0; s < S; ++s) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) project(g, i, &Wc[i], Rc, tc, z[s], sigma_z, &P[i]);
#pragma omp parallel for schedule(dynamic, 1)
    for (int iy = 0; iy < H; ++iy)
      for (int ix = 0; ix < W; ++ix) {
        double acc = 0;
        for (int64_t i = 0; i < n; ++i) acc += pixel_term(&P[i], ix + 0.5, iy + 0.5);
        out[((int64_t)s * H + iy) * W + ix] = acc;
      }
  }
  free(P);
  free(Wc);
  return 0;
}

static int render_points_rc(const orc_set* g, int S, const double* z, double sigma_z,
                            const double Rc[3][3], const double tc[3], int64_t npts,
                            const int* pt_slice, const double* pt_x, const double* pt_y,
                            double* out) {
  if (check_set(g) || S < 0 || npts < 0 || !(sigma_z > 0)) return -1;
  for (int64_t k = 0; k < npts; ++k)
    if (pt_slice[k] < 0 || pt_slice[k] >= S) return -1;
  int64_t n = g->n;
  slice_proj* P = (slice_proj*)malloc(sizeof(slice_proj) * (size_t)(n > 0 ? n : 1));
  world_cov* Wc = (world_cov*)malloc(sizeof(world_cov) * (size_t)(n > 0 ? n : 1));
  if (!P || !Wc) { free(P); free(Wc); return -2; }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) world_covariance(g, i, &Wc[i]);
  for (int s = 0; s < S; ++s) {
    int used = 0;
    for (int64_t k = 0; k < npts; ++k) used |= (pt_slice[k] == s);
    if (!used) continue;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) project(g, i, &Wc[i], Rc, tc, z[s], sigma_z, &P[i]);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < npts; ++k) {
      if (pt_slice[k] != s) continue;
      double acc = 0;
      for (int64_t i = 0; i < n; ++i) acc += pixel_term(&P[i], pt_x[k], pt_y[k]);
      out[k] = acc;
    }
  }
  free(P);
  free(Wc);
  return 0;
}

/* --------------------------------------------------------------- backward */

/* Reverse-mode step from the world covariance Sigma = M M^T, M = R diag(Sd),
 * R = R(q/|q|), to (scale, quat), given the general-matrix gradient gSig. */
static void back_to_scale_quat(const orc_set* g, int64_t i, const world_cov* w,
                               const double gSig[3][3], double* gs, double* gq) {
  /* Sigma = M M^T -> gM = (gSig + gSig^T) M */
  double gS[3][3], gM[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) gS[r][c] = gSig[r][c] + gSig[c][r];
  matmul3(gS, w->M, gM);
  /* M = R D -> gR = gM D, gD_jj = sum_r R_rj gM_rj */
  double gR[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) gR[r][c] = gM[r][c] * w->Sd[c];
  for (int j = 0; j < 3; ++j) {
    double gd = 0;
    for (int r = 0; r < 3; ++r) gd += w->R[r][j] * gM[r][j];
    gs[j] += g->scale_mod * gd;
  }
  /* R = R(qn) */
  double P[4][3][3];
  rot_partials(w->qn, P);
  double gqn[4];
  for (int k = 0; k < 4; ++k) {
    double s = 0;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) s += P[k][r][c] * gR[r][c];
    gqn[k] = s;
  }
  /* qn = q / |q| -> gq = (gqn - qn (qn . gqn)) / |q| */
  double dot = gqn[0] * w->qn[0] + gqn[1] * w->qn[1] + gqn[2] * w->qn[2] + gqn[3] * w->qn[3];
  for (int k = 0; k < 4; ++k) gq[k] += (gqn[k] - w->qn[k] * dot) / w->qnorm;
}

/* Reverse-mode of project() for one (Gaussian, slice), given the gradients of
 * the rasterised quantities: g_at = dL/da~, g_mu2 = dL/dmu_2d and the
 * general-matrix gradient gC = dL/dSigma_2d^-1.  Accumulates dL/dmu, dL/dalpha
 * and the world-covariance gradient gSig. */
static void back_project(const orc_set* g, int64_t i, const double Rc[3][3],
                         const slice_proj* p, double g_at, const double g_mu2[2],
                         const double gC[2][2], double* gmu, double* galpha,
                         double gSig[3][3]) {
  double sq = sqrt(p->det2);
  double alpha = g->alpha[i];
  /* Eq. 9: a~ = alpha op det2^-1/2 */
  *galpha += g_at * p->op / sq;
  double g_op = g_at * alpha / sq;
  double g_det2 = g_at * alpha * p->op * (-0.5) / (p->det2 * sq);
  /* C = Sigma_2d^-1: gS2 = -C^T gC C^T ; det2 = det Sigma_2d: gS2 += g_det2 det2 Sigma_2d^-T */
  double gS2[2][2];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) {
      double s = 0;
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 2; ++l) s += p->C[k][r] * gC[k][l] * p->C[c][l];
      gS2[r][c] = -s + g_det2 * p->det2 * p->C[c][r];
    }
  /* Eq. 8: Sigma_2d = Sigma_e[0:2,0:2] (entry [0][1] is read from Sigma_e[1][0]) */
  double gSe[3][3];
  memset(gSe, 0, sizeof(gSe));
  gSe[0][0] = gS2[0][0];
  gSe[1][0] = gS2[0][1] + gS2[1][0];
  gSe[1][1] = gS2[1][1];
  double gmue[3] = {g_mu2[0], g_mu2[1], 0.0};
  /* Eq. 7: op = exp(-1/2 (qc - qe)), qc = mu_c^T b, qe = mu_e^T Ke mu_e */
  double g_q = g_op * (-0.5) * p->op;
  double gmuc[3] = {0, 0, 0}, gb[3] = {0, 0, 0}, gKe[3][3], gKc[3][3];
  memset(gKe, 0, sizeof(gKe));
  memset(gKc, 0, sizeof(gKc));
  /* qc = mu_c . b */
  for (int r = 0; r < 3; ++r) {
    gmuc[r] += g_q * p->b[r];
    gb[r] += g_q * p->muc[r];
  }
  /* qe = mu_e^T Ke mu_e, entering with a minus sign */
  for (int r = 0; r < 3; ++r) {
    double s = 0;
    for (int c = 0; c < 3; ++c) s += (p->Ke[r][c] + p->Ke[c][r]) * p->mue[c];
    gmue[r] += -g_q * s;
    for (int c = 0; c < 3; ++c) gKe[r][c] += -g_q * p->mue[r] * p->mue[c];
  }
  /* Eq. 6: mu_e = Se b */
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      gSe[r][c] += gmue[r] * p->b[c];
      gb[c] += p->Se[r][c] * gmue[r];
    }
  /* b = Kc mu_c */
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      gKc[r][c] += gb[r] * p->muc[c];
      gmuc[c] += p->Kc[r][c] * gb[r];
    }
  /* Se = Ke^-1: gKe += -Se^T gSe Se^T */
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) s += p->Se[k][r] * gSe[k][l] * p->Se[c][l];
      gKe[r][c] += -s;
    }
  /* Ke = Kc + e3 e3^T / sigma_z^2 */
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) gKc[r][c] += gKe[r][c];
  /* Kc = Sc^-1: gSc = -Kc^T gKc Kc^T */
  double gSc[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) s += p->Kc[k][r] * gKc[k][l] * p->Kc[c][l];
      gSc[r][c] = -s;
    }
  /* camera transform: mu_c = Rc mu + t, Sc = Rc Sigma Rc^T */
  for (int c = 0; c < 3; ++c) {
    double s = 0;
    for (int r = 0; r < 3; ++r) s += Rc[r][c] * gmuc[r];
    gmu[c] += s;
  }
  double Rct[3][3], tmp[3][3], gW[3][3];
  transpose3(Rc, Rct);
  matmul3(Rct, gSc, tmp);
  matmul3(tmp, Rc, gW);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) gSig[r][c] += gW[r][c];
}

static int render_backward_rc(const orc_set* g, int S, const double* z, int H, int W,
                              double sigma_z, const double Rc[3][3], const double tc[3],
                              const double* dL_dI, double* d_mu, double* d_scale,
                              double* d_quat, double* d_alpha) {
  if (check_set(g) || S < 0 || H < 0 || W < 0 || !(sigma_z > 0)) return -1;
  int64_t n = g->n;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n; ++i) {
    world_cov w;
    world_covariance(g, i, &w);
    double gmu[3] = {0, 0, 0}, galpha = 0, gs[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0};
    double gSig[3][3];
    memset(gSig, 0, sizeof(gSig));
    for (int s = 0; s < S; ++s) {
      slice_proj p;
      project(g, i, &w, Rc, tc, z[s], sigma_z, &p);
      /* Eq. 10 per pixel: I += a~ E, E = exp(-1/2 d^T C d), d = p - mu_2d */
      double g_at = 0, g_mu2[2] = {0, 0}, gC[2][2] = {{0, 0}, {0, 0}};
      const double* G = dL_dI + (int64_t)s * H * W;
      for (int iy = 0; iy < H; ++iy)
        for (int ix = 0; ix < W; ++ix) {
          double gp = G[(int64_t)iy * W + ix];
          if (gp == 0.0) continue;
          double dx = ix + 0.5 - p.mue[0], dy = iy + 0.5 - p.mue[1];
          double m = dx * (p.C[0][0] * dx + p.C[0][1] * dy) + dy * (p.C[1][0] * dx + p.C[1][1] * dy);
          double E = exp(-0.5 * m);
          double ge = gp * p.at * E; /* dL/d(exponent) */
          g_at += gp * E;
          /* d(-1/2 d^T C d)/dmu_2d = +1/2 (C + C^T) d */
          g_mu2[0] += ge * 0.5 * ((p.C[0][0] + p.C[0][0]) * dx + (p.C[0][1] + p.C[1][0]) * dy);
          g_mu2[1] += ge * 0.5 * ((p.C[1][0] + p.C[0][1]) * dx + (p.C[1][1] + p.C[1][1]) * dy);
          /* d(-1/2 d^T C d)/dC = -1/2 d d^T */
          gC[0][0] += -0.5 * ge * dx * dx;
          gC[0][1] += -0.5 * ge * dx * dy;
          gC[1][0] += -0.5 * ge * dy * dx;
          gC[1][1] += -0.5 * ge * dy * dy;
        }
      back_project(g, i, Rc, &p, g_at, g_mu2, gC, gmu, &galpha, gSig);
    }
    back_to_scale_quat(g, i, &w, gSig, gs, gq);
    for (int k = 0; k < 3; ++k) {
      d_mu[3 * i + k] = gmu[k];
      d_scale[3 * i + k] = gs[k];
    }
    for (int k = 0; k < 4; ++k) d_quat[4 * i + k] = gq[k];
    d_alpha[i] = galpha;
  }
  return 0;
}

/* -------------------------------------------------------------- voxelizer */

typedef struct {
  double K[3][3]; /* Sigma^-1 */
} vox_proj;

static double voxel_term(const orc_set* g, int64_t i, const vox_proj* v, double x, double y,
                         double zz) {
  const double* mu = g->mu + 3 * i;
  double d[3] = {x - mu[0], y - mu[1], zz - mu[2]};
  double m = 0;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) m += d[r] * v->K[r][c] * d[c];
  return g->alpha[i] * exp(-0.5 * m);
}

int orc_voxelize(const orc_set* g, int X, int Y, int Z, double* vol) {
  if (check_set(g) || X < 0 || Y < 0 || Z < 0) return -1;
  int64_t n = g->n;
  vox_proj* V = (vox_proj*)malloc(sizeof(vox_proj) * (size_t)(n > 0 ? n : 1));
  if (!V) return -2;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    world_cov w;
    world_covariance(g, i, &w);
    inv3(w.Sig, V[i].K);
  }
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
  for (int iz = 0; iz < Z; ++iz)
    for (int iy = 0; iy < Y; ++iy)
      for (int ix = 0; ix < X; ++ix) {
        double acc = 0;
        for (int64_t i = 0; i < n; ++i) acc += voxel_term(g, i, &V[i], ix + 0.5, iy + 0.5, iz + 0.5);
        vol[((int64_t)iz * Y + iy) * X + ix] = acc;
      }
  free(V);
  return 0;
}

int orc_voxelize_points(const orc_set* g, int64_t npts, const double* px, const double* py,
                        const double* pz, double* out) {
  if (check_set(g) || npts < 0) return -1;
  int64_t n = g->n;
  vox_proj* V = (vox_proj*)malloc(sizeof(vox_proj) * (size_t)(n > 0 ? n : 1));
  if (!V) return -2;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    world_cov w;
    world_covariance(g, i, &w);
    inv3(w.Sig, V[i].K);
  }
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t k = 0; k < npts; ++k) {
    double acc = 0;
    for (int64_t i = 0; i < n; ++i) acc += voxel_term(g, i, &V[i], px[k], py[k], pz[k]);
    out[k] = acc;
  }
  free(V);
  return 0;
}

int orc_voxelize_backward(const orc_set* g, int X, int Y, int Z, const double* dL_dV,
                          double* d_mu, double* d_scale, double* d_quat, double* d_alpha) {
  if (check_set(g) || X < 0 || Y < 0 || Z < 0) return -1;
  int64_t n = g->n;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n; ++i) {
    world_cov w;
    world_covariance(g, i, &w);
    double K[3][3];
    inv3(w.Sig, K);
    const double* mu = g->mu + 3 * i;
    double alpha = g->alpha[i];
    double galpha = 0, gmu[3] = {0, 0, 0}, gK[3][3];
    memset(gK, 0, sizeof(gK));
    for (int iz = 0; iz < Z; ++iz)
      for (int iy = 0; iy < Y; ++iy)
        for (int ix = 0; ix < X; ++ix) {
          double G = dL_dV[((int64_t)iz * Y + iy) * X + ix];
          if (G == 0.0) continue;
          double d[3] = {ix + 0.5 - mu[0], iy + 0.5 - mu[1], iz + 0.5 - mu[2]};
          double m = 0;
          for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) m += d[r] * K[r][c] * d[c];
          double E = exp(-0.5 * m);
          galpha += G * E;
          double ge = G * alpha * E;
          /* d(-1/2 d^T K d)/dmu = +1/2 (K + K^T) d ; d/dK = -1/2 d d^T */
          for (int r = 0; r < 3; ++r) {
            double s = 0;
            for (int c = 0; c < 3; ++c) s += 0.5 * (K[r][c] + K[c][r]) * d[c];
            gmu[r] += ge * s;
            for (int c = 0; c < 3; ++c) gK[r][c] += -0.5 * ge * d[r] * d[c];
          }
        }
    /* K = Sigma^-1: gSig = -K^T gK K^T */
    double gSig[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double s = 0;
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) s += K[k][r] * gK[k][l] * K[c][l];
        gSig[r][c] = -s;
      }
    double gs[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0};
    back_to_scale_quat(g, i, &w, gSig, gs, gq);
    for (int k = 0; k < 3; ++k) {
      d_mu[3 * i + k] = gmu[k];
      d_scale[3 * i + k] = gs[k];
    }
    for (int k = 0; k < 4; ++k) d_quat[4 * i + k] = gq[k];
    d_alpha[i] = galpha;
  }
  return 0;
}

/* ------------------------------------------------------------ work count */

static int64_t count_evals_rc(const orc_set* g, int S, const double* z, int H, int W,
                              double sigma_z, const double Rc[3][3], const double tc[3],
                              double eps) {
  if (check_set(g) || S < 0 || H < 0 || W < 0 || !(sigma_z > 0) || !(eps > 0 && eps < 1))
    return -1;
  const double k2 = 2.0 * log(1.0 / eps);
  int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
  for (int64_t i = 0; i < g->n; ++i) {
    world_cov w;
    world_covariance(g, i, &w);
    for (int s = 0; s < S; ++s) {
      slice_proj p;
      project(g, i, &w, Rc, tc, z[s], sigma_z, &p);
      if (!(p.op >= eps)) continue;
      /* per row: C00 dx^2 + 2 C01 dx dy + C11 dy^2 <= k2 is an interval in dx */
      for (int iy = 0; iy < H; ++iy) {
        double dy = iy + 0.5 - p.mue[1];
        double disc = p.C[0][1] * p.C[0][1] * dy * dy - p.C[0][0] * (p.C[1][1] * dy * dy - k2);
        if (disc < 0) continue;
        double sq = sqrt(disc);
        double lo = p.mue[0] + (-p.C[0][1] * dy - sq) / p.C[0][0];
        double hi = p.mue[0] + (-p.C[0][1] * dy + sq) / p.C[0][0];
        int64_t x0 = (int64_t)ceil(lo - 0.5), x1 = (int64_t)floor(hi - 0.5);
        if (x0 < 0) x0 = 0;
        if (x1 > W - 1) x1 = W - 1;
        if (x1 >= x0) total += x1 - x0 + 1;
      }
    }
  }
  return total;
}

/* ------------------------------------------- axis-aligned and general views */

int orc_render(const orc_set* g, int S, const double* z, int H, int W, double sigma_z,
               int axis, double* out) {
  double Rc[3][3], tc[3];
  if (axis_view(axis, Rc, tc)) return -1;
  return render_rc(g, S, z, H, W, sigma_z, Rc, tc, out);
}

int orc_render_view(const orc_set* g, const orc_view* view, int S, const double* z, int H,
                    int W, double sigma_z, double* out) {
  double Rc[3][3], tc[3];
  if (view_matrix(view, Rc, tc)) return -1;
  return render_rc(g, S, z, H, W, sigma_z, Rc, tc, out);
}

int orc_render_points(const orc_set* g, int S, const double* z, double sigma_z, int axis,
                      int64_t npts, const int* pt_slice, const double* pt_x,
                      const double* pt_y, double* out) {
  double Rc[3][3], tc[3];
  if (axis_view(axis, Rc, tc)) return -1;
  return render_points_rc(g, S, z, sigma_z, Rc, tc, npts, pt_slice, pt_x, pt_y, out);
}

int orc_render_points_view(const orc_set* g, const orc_view* view, int S, const double* z,
                           double sigma_z, int64_t npts, const int* pt_slice,
                           const double* pt_x, const double* pt_y, double* out) {
  double Rc[3][3], tc[3];
  if (view_matrix(view, Rc, tc)) return -1;
  return render_points_rc(g, S, z, sigma_z, Rc, tc, npts, pt_slice, pt_x, pt_y, out);
}

int orc_render_backward(const orc_set* g, int S, const double* z, int H, int W,
                        double sigma_z, int axis, const double* dL_dI, double* d_mu,
                        double* d_scale, double* d_quat, double* d_alpha) {
  double Rc[3][3], tc[3];
  if (axis_view(axis, Rc, tc)) return -1;
  return render_backward_rc(g, S, z, H, W, sigma_z, Rc, tc, dL_dI, d_mu, d_scale, d_quat,
                            d_alpha);
}

int orc_render_backward_view(const orc_set* g, const orc_view* view, int S, const double* z,
                             int H, int W, double sigma_z, const double* dL_dI, double* d_mu,
                             double* d_scale, double* d_quat, double* d_alpha) {
  double Rc[3][3], tc[3];
  if (view_matrix(view, Rc, tc)) return -1;
  return render_backward_rc(g, S, z, H, W, sigma_z, Rc, tc, dL_dI, d_mu, d_scale, d_quat,
                            d_alpha);
}

int64_t orc_count_evals(const orc_set* g, int S, const double* z, int H, int W, double sigma_z,
                        int axis, double eps) {
  double Rc[3][3], tc[3];
  if (axis_view(axis, Rc, tc)) return -1;
  return count_evals_rc(g, S, z, H, W, sigma_z, Rc, tc, eps);
}

int64_t orc_count_evals_view(const orc_set* g, const orc_view* view, int S, const double* z,
                             int H, int W, double sigma_z, double eps) {
  double Rc[3][3], tc[3];
  if (view_matrix(view, Rc, tc)) return -1;
  return count_evals_rc(g, S, z, H, W, sigma_z, Rc, tc, eps);
}

/* ------------------------------------------------------------------- loss */

double orc_mse(int64_t n, const double* I, const double* T, double* dL_dI) {
  double L = 0;
  for (int64_t k = 0; k < n; ++k) {
    double r = I[k] - T[k];
    L += r * r;
    if (dL_dI) dL_dI[k] = 2.0 * r / (double)n;
  }
  return n > 0 ? L / (double)n : 0.0;
}
