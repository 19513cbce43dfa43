/*
 * oracle.h -- FP64 CPU oracle of the finite-thickness slice projection operator
 * (GaussianPile, arXiv 2603.20611).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and oracle.c are used by the tests,
 * by __graft_entry__.smoke() and by the CPU-baseline leg of bench.py; the
 * product library never includes, links or calls them, and they share no code,
 * header, table or constant with the CUDA path.
 *
 * Everything is double precision and brute force: every pixel (or voxel) sums
 * over every Gaussian, nothing is culled.
 *
 * Conventions (the paper is silent on them):
 *   - quaternion q = (w, x, y, z), rotation from q/|q| (Sec. S1, "quatToMatrix");
 *   - Sigma = R S S^T R^T with S = diag(mod * s) (Sec. S1);
 *   - camera frame of a slice: mu_c = R_c mu + t, Sigma_c = R_c Sigma R_c^T
 *     (Sec. S1) with R_c the axis permutation below (or a general rotation,
 *     orc_view) and the translation shifted by -z_s e3, so that the focal
 *     plane is z_c = 0;
 *       axis 2: (x_c, y_c, z_c) = (x, y, z)
 *       axis 1: (x_c, y_c, z_c) = (x, z, y)
 *       axis 0: (x_c, y_c, z_c) = (y, z, x)
 *   - pixel (ix, iy) of an H x W slice sits at (x_c, y_c) = (ix + .5, iy + .5);
 *     images are [S][H][W] row-major (row = y_c);
 *   - voxel (ix, iy, iz) sits at (ix + .5, iy + .5, iz + .5); volumes are
 *     [Z][Y][X] row-major.
 * All functions return 0 on success and a negative value on bad arguments.
 */
#ifndef GP_ORACLE_H
#define GP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* n Gaussians, structure of arrays: mu[3n], scale[3n], quat[4n], alpha[n]. */
typedef struct {
  int64_t n;
  const double* mu;
  const double* scale;
  const double* quat;
  const double* alpha;
  double scale_mod;
} orc_set;

/* A general slice orientation (Sec. S1, view matrix [R_c | t]): R (row-major,
 * finite, orthonormal to within 1e-3) and t map world points to camera
 * coordinates x_c = R x + t; slice s of a stack is the plane z_c = z[s] and
 * pixel (ix, iy) sits at (x_c, y_c) = (ix + .5, iy + .5).  The axis-aligned
 * functions are the special case R = the permutation of the axis, t = 0. */
typedef struct {
  double R[9];
  double t[3];
} orc_view;

/* Eq. 10 on every pixel of S slices at plane positions z[S]. out: [S][H][W]. */
int orc_render(const orc_set* g, int S, const double* z, int H, int W,
               double sigma_z, int axis, double* out);

/* Eq. 10 at npts sample points: point k lies on slice pt_slice[k] at camera
 * coordinates (pt_x[k], pt_y[k]).  out[npts]. */
int orc_render_points(const orc_set* g, int S, const double* z, double sigma_z,
                      int axis, int64_t npts, const int* pt_slice,
                      const double* pt_x, const double* pt_y, double* out);

/* Gradient of L with respect to (mu, scale, quat, alpha) given dL/dI [S][H][W]
 * of the image orc_render produces.  Outputs are overwritten. */
int orc_render_backward(const orc_set* g, int S, const double* z, int H, int W,
                        double sigma_z, int axis, const double* dL_dI,
                        double* d_mu, double* d_scale, double* d_quat,
                        double* d_alpha);

/* The three functions above for a general view. */
int orc_render_view(const orc_set* g, const orc_view* view, int S, const double* z, int H,
                    int W, double sigma_z, double* out);
int orc_render_points_view(const orc_set* g, const orc_view* view, int S, const double* z,
                           double sigma_z, int64_t npts, const int* pt_slice,
                           const double* pt_x, const double* pt_y, double* out);
int orc_render_backward_view(const orc_set* g, const orc_view* view, int S, const double* z,
                             int H, int W, double sigma_z, const double* dL_dI, double* d_mu,
                             double* d_scale, double* d_quat, double* d_alpha);

/* Eq. 12: V(x) = sum_i alpha_i exp(-1/2 (x-mu_i)^T Sigma_i^-1 (x-mu_i)). */
int orc_voxelize(const orc_set* g, int X, int Y, int Z, double* vol);

/* Eq. 12 at npts points (px, py, pz). */
int orc_voxelize_points(const orc_set* g, int64_t npts, const double* px,
                        const double* py, const double* pz, double* out);

/* Gradient of L through orc_voxelize given dL/dV [Z][Y][X]. */
int orc_voxelize_backward(const orc_set* g, int X, int Y, int Z,
                          const double* dL_dV, double* d_mu, double* d_scale,
                          double* d_quat, double* d_alpha);

/* Number of (pixel, Gaussian) evaluations inside the culling region of a
 * render with bound eps: pairs (Gaussian, slice) with opacity_r >= eps, pixels
 * with d^T Sigma_2d^-1 d <= 2 ln(1/eps).  This is the algorithmic work of Eq. 10
 * under that culling (the oracle itself never culls). */
int64_t orc_count_evals(const orc_set* g, int S, const double* z, int H, int W,
                        double sigma_z, int axis, double eps);

/* orc_count_evals for a general view. */
int64_t orc_count_evals_view(const orc_set* g, const orc_view* view, int S, const double* z,
                             int H, int W, double sigma_z, double eps);

/* Mean squared error L = 1/n sum (I - T)^2 and its gradient 2 (I - T) / n. */
double orc_mse(int64_t n, const double* I, const double* T, double* dL_dI);

/* Number of OpenMP threads the oracle runs on. */
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
