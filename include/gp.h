/*
 * gp.h -- C ABI of the B300 (sm_103a) slice projection operator of GaussianPile
 * (arXiv 2603.20611): the finite-thickness Focus-Gaussian slice renderer, its
 * hand-written backward, the differentiable voxelizer, a batched launch and a
 * serving loop.
 *
 * The operator (Sec. 4.2, Eq. 6-10; Sec. S1).  For a slice plane at position
 * z_s along the slice axis, every 3-D Gaussian (mean mu, scale s, rotation
 * quaternion q, intensity alpha) with covariance Sigma = R S S^T R^T is weighted
 * by the Gaussian axial sensitivity h(t) = exp(-t^2 / 2 sigma_z^2) (Eq. 3) and
 * contributes, at pixel p of the slice,
 *      a~ exp(-1/2 d^T Sigma_2d^-1 d),   d = p - mu_2d,
 * with Sigma_2d, mu_2d the in-plane block of the Focus Gaussian (Eq. 6, 8) and
 * a~ = alpha opacity_r / sqrt(det Sigma_2d) (Eq. 7, 9).  Contributions add up
 * without occlusion (Eq. 10).  In closed form, with v = Sigma_cc + sigma_z^2
 * (c the slice axis, p the in-plane axes), delta = mu_c - z_s:
 *      Sigma_2d  = Sigma_pp - Sigma_pc Sigma_cp / v      (slice-invariant)
 *      mu_2d     = mu_p - Sigma_pc delta / v
 *      opacity_r = exp(-delta^2 / 2v).
 *
 * Conventions.
 *   - Gaussian parameters are fp32 structure-of-arrays in DEVICE memory, owned
 *     by the caller and never freed or written by the library: mu[3n],
 *     scale[3n] (linear, > 0), quat[4n] = (w, x, y, z) (normalised inside;
 *     16-byte aligned), alpha[n] (linear).  The covariance uses
 *     S = diag(scale_mod * s) (Sec. S1).
 *   - Slice axis `axis` = 2 (planes z = z_s; image columns x, rows y),
 *     1 (planes y = z_s; columns x, rows z) or 0 (planes x = z_s; columns y,
 *     rows z); any other orientation through gp_view (the *_view calls).
 *     Pixel (ix, iy) sits at (ix + 0.5, iy + 0.5) in the plane;
 *     voxel (ix, iy, iz) at (ix + .5, iy + .5, iz + .5).
 *   - Images are [S][H][W] fp32 row-major, volumes [Z][Y][X] fp32.
 *   - Every call is asynchronous on the caller's CUDA stream (`stream` is a
 *     cudaStream_t, NULL = the legacy default stream), except where noted.
 *     Plain render / backward / voxelize calls read back one pair count to
 *     size their sort buffers: on a context's first binning the host waits for
 *     it between the count and the emission; once the context holds pair
 *     buffers, the pairs are emitted and sorted into their capacity (at most a
 *     quarter above the context's last count) while the count is copied back
 *     on a context-owned side stream, and the call waits for that copy after
 *     queueing its rasteriser (a count that did not fit bins the call again
 *     and repeats the rasteriser before returning).  Either way the host
 *     returns once the binning's count is known; the rasteriser may still run.
 *   - Contributions are culled where they are provably below eps relative to
 *     their Gaussian: slices with opacity_r < eps are skipped, and only screen
 *     tiles that the ellipse d^T Sigma_2d^-1 d <= 2 ln(1/eps) touches are
 *     visited (the culling the paper leaves at "a small threshold", Sec. 4.2).
 *     Inside a visited tile every pixel is evaluated.
 *   - Errors never abort: each call returns a gp_status, and gp_last_error()
 *     gives a message.  Argument errors are detected before any launch.
 */
#ifndef GP_H
#define GP_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GP_API __attribute__((visibility("default")))
#else
#define GP_API
#endif

typedef int gp_status;
#define GP_OK 0
#define GP_PENDING 1          /* gp_serve_poll: request not finished yet */
#define GP_ERR_ARG (-1)       /* invalid argument (null pointer, bad size, ...) */
#define GP_ERR_OOM (-2)       /* device allocation failed or over the workspace limit */
#define GP_ERR_CUDA (-3)      /* a CUDA runtime call failed */
#define GP_ERR_TIMEOUT (-4)   /* a bounded wait ran out */
#define GP_ERR_OVERFLOW (-5)  /* a preplanned buffer was too small; re-plan */
#define GP_ERR_STATE (-6)     /* call not valid in the object's current state */
#define GP_ERR_CANCELLED (-7) /* gp_serve_poll result: the request was cancelled while queued */

typedef struct gp_ctx gp_ctx;

/* Exponential used by the rasterisers. */
#define GP_EXP_POLY 0  /* project-written exp2: range reduction + degree-6 polynomial on
                          the FP32 pipe (no ex2.approx); the default.  The backward
                          recomputes its per-pixel exponentials with a degree-4 polynomial
                          (relative error 3.6e-6; its gradients are held to 1e-3) */
#define GP_EXP_HW 1    /* the SFU ex2.approx instruction (benchmarked alternative) */
#define GP_EXP_POLY_PACKED 2  /* gp_exp2_eval only: GP_EXP_POLY in the packed two-value form
                                 the rasterisers use (bitwise equal to GP_EXP_POLY) */
#define GP_EXP_POLY_ROW 3     /* GP_EXP_POLY, with the Gaussian factored along each row of 8
                                 pixels: exp2 of the row's linear part at its larger end and of
                                 the per-pixel step, powers of the step by multiplication, and
                                 the quadratic part 2^(c q^2) once per Gaussian and tile, so a
                                 row costs two exp2 instead of eight (relative error of a few
                                 ulp per pixel instead of about 2).  Block-culled rasterisers
                                 only (fwd_px = bwd_px = 0); Gaussians narrower than about 0.3
                                 pixel fall back to one exp2 per pixel. */
#define GP_EXP_POLY_GRAD 4    /* gp_exp2_eval only: the backward's degree-4 exp2 */
#define GP_EXP_POLY_GRAD_PACKED 5  /* gp_exp2_eval only: GP_EXP_POLY_GRAD in the packed form the
                                      backward uses (bitwise equal to GP_EXP_POLY_GRAD) */

/* Form of the default rasterisers (fwd_px = bwd_px = 0), GP_EXP_POLY / GP_EXP_HW. */
#define GP_RASTER_AUTO 0   /* row units for the forward, and for the backward on voxelizer planes;
                              block-culled for the backward on slice planes (default) */
#define GP_RASTER_BLOCK 1  /* block-culled: four warps per 16 x 16 tile, each Gaussian evaluated
                              over the 8 x 8 blocks (forward) / 8 x 4 half-blocks (backward) its
                              culling ellipse touches */
#define GP_RASTER_ROWS 2   /* row units: one warp per tile, each Gaussian evaluated over the 8-pixel
                              row segments its culling ellipse touches */
#define GP_RASTER_PIXELS 3 /* (batch plans' report only) one thread per group of pixels of a tile,
                              every staged Gaussian evaluated at every pixel: the fwd_px / bwd_px
                              kernels */

typedef struct {
  float eps;              /* culling bound: truncated mass per pair <= eps (default 1e-6) */
  int deterministic;      /* 1: backward reduces per-pair partials in a fixed order
                             (bitwise repeatable); 0: warp-reduced atomics (default 0) */
  int exp_mode;           /* GP_EXP_POLY (default), GP_EXP_HW or GP_EXP_POLY_ROW */
  int tile;               /* screen tile side in pixels: 16 (default) or 8 */
  int fwd_px;             /* forward rasteriser: 0 (default) = block-culled kernel (16x16
                             tiles; 8x8 tiles use one pixel per thread), or the per-thread
                             kernel with this many pixels per thread (16: 1, 2, 4; 8: 1, 2) */
  int bwd_px;             /* backward rasteriser: 0 (default) = block-culled kernel, or the
                             per-thread kernel (16: 2, 4, 8 pixels per thread; 8: 2) */
  int64_t workspace_limit;/* max device bytes of library scratch, 0 = no limit.  A call that
                             would pass it (or whose cudaMalloc fails) returns GP_ERR_OOM
                             after freeing the context's whole workspace, so later calls
                             that fit still run. */
  int reuse_bins;         /* 1: gp_render_backward (gp_voxelize_backward) reuses the binning of
                             the immediately preceding gp_render_slices (gp_voxelize) on this
                             context when called with the same set pointers, n, scale_mod,
                             planes, image size, sigma_z and axis (grid); the caller guarantees
                             the parameter VALUES are unchanged in between (true inside one
                             forward/backward step).  0 (default): the backward always re-bins. */
  int raster;             /* GP_RASTER_AUTO (default), GP_RASTER_BLOCK or GP_RASTER_ROWS; the
                             row-factored exponential (GP_EXP_POLY_ROW) is block-culled only */
} gp_config;

/* Fills *cfg with the defaults above.  Returns GP_ERR_ARG if cfg is NULL. */
GP_API gp_status gp_config_default(gp_config* cfg);

/* Creates a context on CUDA device `device` (it becomes current on the calling
 * thread).  cfg may be NULL for defaults; GP_ERR_ARG for an invalid cfg.  The
 * context owns a grow-only device workspace pool (freed by gp_destroy).  A
 * context is not thread-safe: use one per host thread, or serialise calls. */
GP_API gp_status gp_create(gp_ctx** out, int device, const gp_config* cfg);

/* Frees the context and its workspace (after synchronising the device). */
GP_API gp_status gp_destroy(gp_ctx* ctx);

/* Message of the last error on ctx (static string if ctx is NULL).  Valid until
 * the next call on ctx. */
GP_API const char* gp_last_error(gp_ctx* ctx);

/* Library scratch currently held by ctx, in bytes. */
GP_API int64_t gp_workspace_bytes(gp_ctx* ctx);

/* Gaussian set: caller-owned device pointers (see conventions). n may be 0. */
typedef struct {
  const float* mu;
  const float* scale;
  const float* quat;
  const float* alpha;
  int64_t n;
  float scale_mod;       /* Sec. S1 "mod"; 1 for the plain S = diag(s) */
} gp_set;

/* Forward (Eq. 10): renders S slices at plane positions z[S] (HOST array) into
 * out (DEVICE, [S][H][W], fully overwritten).  sigma_z in (0, inf).
 * Returns GP_ERR_ARG for S < 0, H or W <= 0, bad sigma_z or axis, null
 * pointers, non-finite z, or S*H*W > 2^31; GP_ERR_OVERFLOW for more than 2^31
 * (Gaussian, slice, tile) pairs in one call. */
GP_API gp_status gp_render_slices(gp_ctx* ctx, const gp_set* set, const float* z, int S, int H,
                           int W, float sigma_z, int axis, float* out, void* stream);

/* Backward of gp_render_slices (Sec. 4.3; the chain of Sec. S2 re-derived in
 * closed form): given dL/dI (DEVICE, [S][H][W]), writes dL/dmu [3n],
 * dL/dscale [3n], dL/dquat [4n] (through the quaternion normalisation, 16-byte
 * aligned) and dL/dalpha [n] (DEVICE, overwritten).  Per-tile Gaussian lists
 * are recomputed, no per-pixel state is stored. */
GP_API gp_status gp_render_backward(gp_ctx* ctx, const gp_set* set, const float* z, int S, int H,
                             int W, float sigma_z, int axis, const float* dL_dI,
                             float* d_mu, float* d_scale, float* d_quat, float* d_alpha,
                             void* stream);

/* ------------------------------------------------------- oblique slices
 * A general slice orientation: the view matrix [R_c | t] of Sec. S1, which maps
 * a world point x to camera coordinates x_c = R_c x + t.  Slice s of a stack is
 * the plane z_c = z[s]; pixel (ix, iy) sits at (x_c, y_c) = (ix + .5, iy + .5).
 * R (row-major: row j is camera axis j in world coordinates) must be finite and
 * orthonormal to within 1e-3 (checked: GP_ERR_ARG otherwise), t finite.  All
 * planes of one call share R_c, so Sigma_2d stays slice-invariant and the
 * kernels are the axis-aligned ones; a different orientation is another call.
 * The axis-aligned calls are the special case R_c = the axis permutation
 * (gp_view_from_axis), t = 0, and give bitwise the same results as the view
 * calls with that view. */
typedef struct {
  float R[9];
  float t[3];
} gp_view;

/* Fills *view with the permutation view of a slice axis (0, 1, 2); GP_ERR_ARG otherwise. */
GP_API gp_status gp_view_from_axis(int axis, gp_view* view);

/* gp_render_slices / gp_render_backward / gp_count_evals for a general view
 * (HOST gp_view; NULL or invalid: GP_ERR_ARG).  Everything else as there. */
GP_API gp_status gp_render_slices_view(gp_ctx* ctx, const gp_set* set, const gp_view* view, const float* z,
                                       int S, int H, int W, float sigma_z, float* out, void* stream);
GP_API gp_status gp_render_backward_view(gp_ctx* ctx, const gp_set* set, const gp_view* view, const float* z,
                                         int S, int H, int W, float sigma_z, const float* dL_dI, float* d_mu,
                                         float* d_scale, float* d_quat, float* d_alpha, void* stream);
GP_API gp_status gp_count_evals_view(gp_ctx* ctx, const gp_set* set, const gp_view* view, const float* z, int S,
                                     int H, int W, float sigma_z, int64_t* evals);

/* Mean squared error of a rendered stack against target slices (the
 * benchmarked fit step's loss; the paper's own L1 + D-SSIM is
 * gp_l1_dssim_grad).  I: [S][H][W] DEVICE.  T: DEVICE target stack of at least
 * max(t_index)+1 slices of H*W.  t_index: HOST array of S slice indices into T,
 * or NULL for T[s] = slice s.  Writes dL/dI = 2 (I - T) / (S H W) (DEVICE) and,
 * if loss != NULL, L = mean (I - T)^2 into loss[0] (DEVICE, fp32). */
GP_API gp_status gp_mse_grad(gp_ctx* ctx, const float* I, const float* T, const int* t_index,
                      int S, int H, int W, float* dL_dI, float* loss, void* stream);

/* The paper's photometric loss (Eq. 11, lambda = 0.2 in Sec. 5.1):
 *     L = L1 + lambda (1 - SSIM),   L1 = mean |I - T|,
 * SSIM the mean over pixels and slices of the per-slice structural similarity
 * (Wang et al. 2004: 11 x 11 Gaussian window of standard deviation 1.5,
 * C1 = 0.01^2, C2 = 0.03^2 for data range 1, zero padding at the borders).
 * I, T, t_index and dL_dI as in gp_mse_grad; dL/dI is fully overwritten (the
 * L1 term takes sign(0) = 0).  If loss != NULL, writes (L, L1, mean SSIM) into
 * loss[0..2] (DEVICE, fp32; sums taken in double in a fixed order).  Scratch:
 * 12 bytes per pixel in the context's workspace.  GP_ERR_ARG for S < 0, H or W
 * <= 0, lambda < 0 or non-finite, NULL pointers, a negative index, S > 65535 or
 * S*H*W > 2^31.  Asynchronous on `stream`. */
GP_API gp_status gp_l1_dssim_grad(gp_ctx* ctx, const float* I, const float* T, const int* t_index, int S, int H,
                                  int W, float lambda, float* dL_dI, float* loss, void* stream);

/* Allocation-free variant of gp_mse_grad (the paper has no counterpart: this is a
 * deployment convenience).  For callers that must not allocate device memory:
 * processes whose device memory is already reserved by another allocator (a
 * framework's caching allocator or a fixed pool), where a fresh cudaMalloc can
 * fail although the pool has room, and latency-bound serving loops that cannot
 * pay for cudaMalloc / cudaFree, which synchronise the device.  It needs no
 * context and calls no allocating routine.
 *
 * Same arguments and results as gp_mse_grad (I, T, dL_dI, loss on the device,
 * t_index on the host or NULL), on the CURRENT device and the given stream.
 * Scratch: one fixed device array inside the library, 2^18 floats of per-block
 * partial sums plus 2^14 target indices (about 1.06 MiB, held by every GPU that
 * loads the library until the process exits).  Limits: S <= 2^18 slices, the
 * per-block partials of S slices of H*W pixels (S * ceil(H*W / 2048), at most
 * 4096 blocks per slice) <= 2^18, and S <= 2^14 when t_index is given; larger
 * calls return GP_ERR_OVERFLOW before anything runs.  GP_ERR_ARG for H or W
 * <= 0, S < 0, NULL pointers or a negative index; GP_ERR_CUDA if the scratch
 * address cannot be obtained.
 *
 * The first call on a device looks up the scratch's device address with
 * cudaGetSymbolAddress (once per device, thread-safe; a failed lookup returns
 * GP_ERR_CUDA and is not remembered, so the next call tries again); make that
 * first call before any stream capture.  Every call shares the one array, and each call
 * overwrites what it reads, so nothing carries over between calls; but calls
 * whose work overlaps on the GPU (different streams, or different host threads
 * without ordering) race on it and must be serialised by the caller. */
GP_API gp_status gp_mse_grad_noalloc(const float* I, const float* T, const int* t_index, int S,
                                     int H, int W, float* dL_dI, float* loss, void* stream);

/* Differentiable voxelizer (Sec. 4.3 "Differentiable Voxelization", Eq. 12):
 * V(x) = sum_i alpha_i exp(-1/2 (x - mu_i)^T Sigma_i^-1 (x - mu_i)) on the
 * X x Y x Z voxel grid (voxel centres at index + 1/2), written to vol (DEVICE,
 * [Z][Y][X], overwritten).  Rendered as the stack of the grid's z-planes
 * through the slice path: on a plane the term factors into alpha exp(-delta^2 /
 * 2 Sigma_zz) exp(-1/2 d^T Sigma_2d^-1 d) with Sigma_2d the conditional
 * covariance, i.e. the slice operator with sigma_z = 0 and amplitude alpha.
 * Each plane is culled by its section of the ellipsoid (x - mu)^T Sigma^-1
 * (x - mu) <= 2 ln(1/eps).  GP_ERR_ARG for X, Y or Z <= 0, more than 2^31
 * voxels or a NULL vol. */
GP_API gp_status gp_voxelize(gp_ctx* ctx, const gp_set* set, int X, int Y, int Z, float* vol,
                      void* stream);

/* Backward of gp_voxelize given dL/dV (DEVICE [Z][Y][X]); gradients as in
 * gp_render_backward (overwritten).  With reuse_bins it reuses the binning of
 * an immediately preceding gp_voxelize of the same set and grid. */
GP_API gp_status gp_voxelize_backward(gp_ctx* ctx, const gp_set* set, int X, int Y, int Z,
                               const float* dL_dV, float* d_mu, float* d_scale,
                               float* d_quat, float* d_alpha, void* stream);

/* Number of (voxel, Gaussian) evaluations inside the culling ellipsoid
 * (x - mu)^T Sigma^-1 (x - mu) <= 2 ln(1/eps), voxel centres in the X x Y x Z
 * grid: the algorithmic work of gp_voxelize (Eq. 12).  Synchronous. */
GP_API gp_status gp_count_vox_evals(gp_ctx* ctx, const gp_set* set, int X, int Y, int Z, int64_t* evals);

/* Pixels (or voxels) the context's default rasterisers (fwd_px = bwd_px = 0)
 * evaluate for a render or a voxelize, *fwd for the forward and *bwd for the
 * backward, with the same culling tests the kernels stage with (Sec. 4.2, the
 * eps reading above): the row-unit form evaluates 8 pixels per (Gaussian,
 * plane, screen tile, 8-pixel column band, pixel row) whose segment of pixel
 * centres the culling ellipse meets; the block-culled form 64 per 8 x 8 block
 * (forward) and 32 per 8 x 4 half-block (backward) the ellipse touches.
 * Divided by gp_count_evals / gp_count_vox_evals it gives the evaluations
 * spent per algorithmic one.  Synchronous.  GP_ERR_ARG as in the render calls. */
GP_API gp_status gp_count_evaluated_view(gp_ctx* ctx, const gp_set* set, const gp_view* view, const float* z,
                                         int S, int H, int W, float sigma_z, int64_t* fwd, int64_t* bwd);
GP_API gp_status gp_count_vox_evaluated(gp_ctx* ctx, const gp_set* set, int X, int Y, int Z, int64_t* fwd,
                                        int64_t* bwd);

/* Diagnostics of the last gp_render_slices / gp_render_backward / gp_voxelize
 * on ctx: number of (Gaussian, slice, tile) pairs binned and of pixel
 * evaluations issued (pairs x tile pixels). */
GP_API gp_status gp_last_counts(gp_ctx* ctx, int64_t* pairs, int64_t* issued_evals);

/* Number of Gaussian-pixel evaluations inside the culling ellipse
 * (d^T Sigma_2d^-1 d <= 2 ln(1/eps), opacity_r >= eps) of a render call with
 * these arguments: the algorithmic work of Eq. 10.  Synchronous. */
GP_API gp_status gp_count_evals(gp_ctx* ctx, const gp_set* set, const float* z, int S, int H,
                         int W, float sigma_z, int axis, int64_t* evals);

/* Test hook for the rasterisers' exponential: y[i] = 2^x[i] for n DEVICE floats
 * with the given mode (GP_EXP_POLY, GP_EXP_HW, GP_EXP_POLY_PACKED, GP_EXP_POLY_GRAD or
 * GP_EXP_POLY_GRAD_PACKED).  Inputs below -125 clamp. */
GP_API gp_status gp_exp2_eval(gp_ctx* ctx, const float* x, float* y, int64_t n, int mode,
                       void* stream);

/* ------------------------------------------------------------------ batching
 * Many Gaussian sets of uneven sizes, each with its own slice stack, image size,
 * sigma_z and axis, rendered and differentiated by ONE CUDA-graph launch (the
 * paper renders one stack at a time).  The plan
 * bins every item into one batch-wide key space and rasterises with
 * persistent kernels that take (item, slice, tile) work from a global counter.
 *
 * Per item (all pointers DEVICE except z):
 *   out     [S][H][W] forward image, or NULL;
 *   target  [S][H][W] MSE target: the plan computes loss (if `loss` != NULL),
 *           dL/dI = 2 (I - T) / (S H W) and, with d_mu != NULL, the backward;
 *   dL_dI   [S][H][W] upstream gradient, used when target is NULL;
 *   d_mu, d_scale, d_quat, d_alpha: gradient outputs (overwritten), or NULL.
 * The plan keeps the pointers; every run reads the current parameter values
 * and writes the outputs.  Pair buffers are sized at plan time with 25%
 * headroom; if a later run needs more (parameters moved a lot), every kernel
 * clamps to the capacity and gp_batch_wait returns GP_ERR_OVERFLOW: re-plan.
 * A plan belongs to its context (same device, not thread-safe). */
typedef struct {
  gp_set set;
  const float* z;   /* HOST [S] plane positions */
  int S, H, W;
  float sigma_z;
  int axis;
  float* out;
  const float* target;
  const float* dL_dI;
  float *d_mu, *d_scale, *d_quat, *d_alpha;
  float* loss;
  const gp_view* view;  /* HOST, copied at plan time; NULL = the view of `axis` */
} gp_batch_item;

typedef struct gp_plan gp_plan;

#define GP_BATCH_AUTOTUNE 1  /* time tile side (8/16) and staging chunks on this workload */

/* Builds the plan (allocates its buffers, counts pairs once, optionally
 * autotunes, captures the graph).  Synchronous.  GP_ERR_ARG for invalid items. */
GP_API gp_status gp_batch_plan(gp_ctx* ctx, const gp_batch_item* items, int n, int flags, gp_plan** out);
/* Enqueues the captured graph on `stream` (asynchronous). */
GP_API gp_status gp_batch_run(gp_plan* plan, void* stream);
/* Synchronises `stream`; GP_ERR_OVERFLOW if the last run outgrew the plan. */
GP_API gp_status gp_batch_wait(gp_plan* plan, void* stream);
/* Chosen configuration and memory of a plan. */
typedef struct {
  int64_t pair_capacity;   /* binned (Gaussian, slice, tile) pairs the plan's buffers hold */
  int64_t device_bytes;    /* device memory the plan owns */
  int tile;                /* screen tile side */
  int fwd_raster, bwd_raster;  /* GP_RASTER_BLOCK, GP_RASTER_ROWS or GP_RASTER_PIXELS */
  int fwd_chunk, bwd_chunk;    /* block-culled form: Gaussians per staging round (else 0) */
  int fwd_px, bwd_px;          /* per-thread form: pixels per thread (else 0) */
} gp_batch_config;
GP_API gp_status gp_batch_info(gp_plan* plan, gp_batch_config* out);
GP_API gp_status gp_batch_destroy(gp_plan* plan);

/* ---------------------------------------------------------------- codec
 * The paper's storage path (Sec. 4, "Quantization and compression"): Gaussians
 * in Morton (Z-order) of their quantised positions; positions normalised to
 * the bounding box at pos_bits (1..15, typically 14) bits per axis; scales
 * log-transformed and quantised to 12 bits over [ln min s, ln max s] (round to
 * nearest in the log domain); quaternions normalised, folded to w >= 0 and
 * quantised to 12 bits per component over [-1, 1]; intensities clamped to
 * [0, 1] and quantised to 12 bits; each of the 11 attribute streams (x y z,
 * s0 s1 s2, qw qx qy qz, alpha) holds the first code and then the differences
 * of consecutive codes, zigzag-mapped (d >= 0 -> 2d, d < 0 -> -2d - 1) to
 * uint16.  The entropy stage (LZMA) runs on the host over these streams.
 * Affine quantisations round with separately rounded fp32 operations,
 * code = floor((v - lo) * ((2^B - 1) / (hi - lo)) + 0.5) clamped; decoding
 * returns the Gaussians in Morton order. */
typedef struct {
  int64_t n;
  int pos_bits;
  float lo[3], hi[3];           /* position bounding box */
  double log_s_min, log_s_max;  /* scale range (natural logarithms) */
} gp_codec_header;

/* Encodes a set (DEVICE parameters; scale_mod is not applied) into streams
 * (DEVICE uint16 [11][n], caller-owned) and fills *header (HOST).  If order is
 * non-NULL (DEVICE uint32 [n]) it receives the input index of each encoded
 * Gaussian.  Synchronous (one readback of the bounding box).  GP_ERR_ARG for
 * pos_bits outside 1..15, NULL pointers, or a set with a non-finite parameter
 * or a scale <= 0. */
GP_API gp_status gp_encode(gp_ctx* ctx, const gp_set* set, int pos_bits, gp_codec_header* header,
                           uint16_t* streams, uint32_t* order, void* stream);
/* Decodes streams (DEVICE [11][n]) into mu [3n], scale [3n], quat [4n]
 * (16-byte aligned) and alpha [n] (DEVICE, caller-owned).  Asynchronous. */
GP_API gp_status gp_decode(gp_ctx* ctx, const gp_codec_header* header, const uint16_t* streams, float* mu,
                           float* scale, float* quat, float* alpha, void* stream);

/* ------------------------------------------------------------------- serving
 * A request loop over resident Gaussian sets (deployment form; the paper has no
 * server).  Requests -- one slice, a stack of slices, or a voxelize -- enter a
 * queue; worker threads, each with its own context (workspace) and CUDA
 * stream, take them as soon as a worker is free and the request's estimated
 * device memory fits the budget (free HBM minus a reserve, or a fixed budget),
 * so requests that arrive while others run overlap with them on the GPU.  A
 * worker taking a slice/stack request also takes every pending request for the
 * same set, view, image size and sigma_z (up to max_batch_slices planes) and
 * renders them in one call; results are bitwise the same alone and in a batch.
 * A worker taking a voxelize request also takes every pending voxelize request
 * for the same set and grid (up to max_batch_slices requests): they ask for the
 * same volume, which it voxelizes once and copies to each output.
 * Outputs are caller-owned device buffers that must stay valid until the
 * request completes.  submit / poll / stats / load may be called from any
 * thread; a request keeps a copy of its set's descriptor from its submit, so
 * sets may be registered while requests run. */
#define GP_REQ_SLICE 0     /* one plane: S must be 1 */
#define GP_REQ_STACK 1     /* S planes */
#define GP_REQ_VOXELIZE 2  /* X x Y x Z volume */

typedef struct {
  int workers;                 /* concurrent requests on the device (default 4) */
  int max_batch_slices;        /* planes per batched render (default 64) */
  int64_t hbm_budget_bytes;    /* fixed admission budget; 0 = free HBM minus reserve */
  int64_t hbm_reserve_bytes;   /* kept free when the budget follows free HBM (default 4 GiB) */
} gp_serve_cfg;

typedef struct {
  int kind;
  int set_id;
  const float* z;   /* HOST plane positions [S] (copied at submit) */
  int S, H, W;
  float sigma_z;
  int axis;
  int X, Y, Z;      /* voxelize */
  float* out;       /* DEVICE [S][H][W] or [Z][Y][X] */
  const gp_view* view;  /* HOST, copied at submit; NULL = the view of `axis` (slice / stack) */
  double timeout_ms;    /* queue deadline: a request not started within timeout_ms of its
                           submit is dropped with result status GP_ERR_TIMEOUT; 0 = none */
} gp_request;

typedef struct {
  gp_status status;
  double latency_ms;   /* submit -> completion */
  double queue_ms;     /* submit -> start on a worker */
  int batch_size;      /* requests rendered together */
} gp_result;

typedef struct {
  int64_t submitted, completed, failed, batches, admission_waits, pending, inflight_bytes;
  int64_t inflight_requests, max_inflight_requests;  /* admitted and not finished; its maximum */
  int64_t expired, cancelled;  /* dropped from the queue by their deadline / by gp_serve_cancel */
} gp_serve_stats;

typedef struct gp_server gp_server;

/* Starts the workers (cfg NULL = defaults) on ctx's device, with ctx's config. */
GP_API gp_status gp_serve_open(gp_ctx* ctx, const gp_serve_cfg* cfg, gp_server** out);
/* Registers a resident set (caller keeps its device memory valid); returns its id. */
GP_API gp_status gp_serve_load_set(gp_server* server, const gp_set* set, int* set_id);
/* Decodes an encoded set (gp_encode's header and DEVICE streams) into device
 * memory owned by the server (freed by gp_serve_close) and registers it;
 * returns its id.  Synchronous. */
GP_API gp_status gp_serve_load_encoded(gp_server* server, const gp_codec_header* header, const uint16_t* streams,
                                       float scale_mod, int* set_id);
/* Queues a request (validated here: GP_ERR_ARG) and returns its ticket. */
GP_API gp_status gp_serve_submit(gp_server* server, const gp_request* req, uint64_t* ticket);
/* Waits up to timeout_ms for the ticket: GP_OK with *out filled (once per
 * ticket), or GP_PENDING if it is still queued or running.  out->status is the
 * request's own outcome: GP_OK, an error of its run, GP_ERR_TIMEOUT (its queue
 * deadline passed before it started), GP_ERR_CANCELLED, or GP_ERR_STATE (still
 * queued when the server closed).  Requests past their deadline are dropped
 * by the workers and by poll / stats calls, without waiting for a worker. */
GP_API gp_status gp_serve_poll(gp_server* server, uint64_t ticket, int timeout_ms, gp_result* out);
/* Removes a request that is still queued; its poll result then has status
 * GP_ERR_CANCELLED.  GP_ERR_STATE if it has started or finished (it runs to
 * completion), GP_ERR_ARG for a ticket never issued. */
GP_API gp_status gp_serve_cancel(gp_server* server, uint64_t ticket);
GP_API gp_status gp_serve_stats_get(gp_server* server, gp_serve_stats* out);
/* Stops the workers after their current requests; still-queued requests are dropped. */
GP_API gp_status gp_serve_close(gp_server* server);

/* ------------------------------------------------------------- fit loop
 * The parameter update of the fit loop (Sec. 5.1: Adam for 30k iterations with
 * initial learning rates 6e-4 position, 2e-2 intensity, 2e-3 scale, 1e-3
 * rotation, each decaying exponentially to 0.1 of its initial value):
 *     lr_t = lr_0 * final_ratio^(k / total_steps),  k = min(t - 1, total_steps),
 *     m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
 *     theta <- theta - lr_t (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 * With log_scale_logit_alpha (default 1) the scale and the intensity are
 * optimised as log s and logit alpha (the Gaussian-splatting parameterisation
 * the paper builds on; the renderer still reads linear s and alpha, which the
 * step writes back), so s stays positive and alpha in (0, 1).  The position
 * rate is multiplied by mu_extent (rates relative to the scene extent). */
typedef struct {
  float lr_mu, lr_scale, lr_quat, lr_alpha;
  float mu_extent;          /* default 1 */
  float lr_final_ratio;     /* default 0.1 */
  int64_t total_steps;      /* default 30000 */
  float beta1, beta2, eps;  /* defaults 0.9, 0.999, 1e-15 */
  int log_scale_logit_alpha;
} gp_adam_cfg;

/* Fills *cfg with the defaults above (the paper's rates).  GP_ERR_ARG if NULL. */
GP_API gp_status gp_adam_default(gp_adam_cfg* cfg);
/* Floats of optimiser state for n Gaussians (DEVICE, caller-owned): 26 n,
 * laid out [26][n] -- first moments (11 rows: mu xyz, scale xyz, quat wxyz,
 * alpha), second moments (11 rows), raw log s (3 rows) and logit alpha. */
GP_API int64_t gp_adam_state_floats(int64_t n);
/* Zeroes the moments and sets the raw parameters from the current scale and
 * alpha (alpha clamped to [1e-6, 1 - 1e-6] before the logit).  Asynchronous. */
GP_API gp_status gp_adam_init(gp_ctx* ctx, const gp_adam_cfg* cfg, int64_t n, const float* scale,
                              const float* alpha, float* state, void* stream);
/* Step t (1, 2, ...): updates mu [3n], scale [3n], quat [4n] (16-byte aligned)
 * and alpha [n] in place (DEVICE) from the gradients d_* (DEVICE, as written by
 * gp_render_backward) and the state.  GP_ERR_ARG for t < 1, bad rates or NULL
 * pointers.  Asynchronous on `stream`. */
GP_API gp_status gp_adam_step(gp_ctx* ctx, const gp_adam_cfg* cfg, int64_t t, int64_t n, float* mu, float* scale,
                              float* quat, float* alpha, const float* d_mu, const float* d_scale,
                              const float* d_quat, const float* d_alpha, float* state, void* stream);

/* Phase timing.  When enabled, every call records a CUDA event pair on its
 * stream around each phase below; gp_timing_read synchronises those events,
 * returns the summed milliseconds and launch counts per phase since the last
 * read, and clears them.  Phases: */
#define GP_PHASE_BIN 0        /* K-pre, scan, K-emit, radix sort, K-range */
#define GP_PHASE_FWD 1        /* K-fwd rasteriser */
#define GP_PHASE_BWD 2        /* K-bwd rasteriser */
#define GP_PHASE_BWD_PRE 3    /* K-det (deterministic mode) and K-bwd-pre */
#define GP_PHASE_LOSS 4       /* K-loss */
#define GP_PHASE_VOX_FWD 5    /* voxelizer forward rasteriser */
#define GP_PHASE_VOX_BWD 6    /* voxelizer backward rasteriser + gradient finish */
#define GP_PHASE_OPT 7        /* gp_adam_step */
#define GP_NUM_PHASES 8
GP_API gp_status gp_timing_enable(gp_ctx* ctx, int enable);
/* Times only the phases whose bit (1 << GP_PHASE_*) is set in mask (0 = none);
 * each timed phase records two events per call, which cost the stream a few
 * microseconds.  GP_ERR_ARG for bits past GP_NUM_PHASES. */
GP_API gp_status gp_timing_enable_phases(gp_ctx* ctx, unsigned mask);
GP_API gp_status gp_timing_read(gp_ctx* ctx, double* ms /* [GP_NUM_PHASES] */,
                                int64_t* launches /* [GP_NUM_PHASES] */,
                                int64_t* calls /* [GP_NUM_PHASES], may be NULL */);

/* Total number of kernels this library has launched in the process (all
 * contexts), for accounting in benchmarks. */
GP_API int64_t gp_launch_count(void);

/* FP32-pipe throughput probe: every thread of a grid sized to fill the device
 * runs `iters` iterations of 8 independent FMA chains; out (DEVICE, one float
 * per thread of the grid, see gp_fma_probe_threads) receives the chain sums.
 * Used to measure the FP32 lane-instruction peak at the clocks in force. */
GP_API int64_t gp_fma_probe_threads(gp_ctx* ctx);
GP_API gp_status gp_fma_probe(gp_ctx* ctx, int iters, float* out, void* stream);
/* The same probe in one of four instruction forms: mode 0 = 8 scalar FFMA
 * chains (gp_fma_probe), 1 = 8 packed fp32x2 FFMA2 chains, 2 = 4 FFMA2 + 8 FFMA
 * chains, 3 = 8 chains of the SFU ex2.approx instruction (the SFU rate).
 * gp_fma_probe_lane_fmas(mode) gives the lane operations per thread and
 * iteration (8, 16, 16, 8; 0 for a bad mode).  GP_ERR_ARG for a bad mode,
 * iters <= 0 or a NULL out. */
GP_API gp_status gp_fma_probe_mode(gp_ctx* ctx, int mode, int iters, float* out, void* stream);
GP_API int gp_fma_probe_lane_fmas(int mode);

/* ------------------------------------------------ bounds-checked debug build
 * The library also builds as libgaussianpile_check.so (-DGP_CHECK), in place
 * of a memory sanitizer: its kernels check their shared- and global-memory
 * indices, skip an out-of-range access and record the first one per source
 * file, and gp_render_*, gp_voxelize* and gp_batch_wait then wait for their
 * stream and return GP_ERR_STATE with the file, check site and index in
 * gp_last_error.  gp_check_enabled() is 1 in that build and 0 in the default
 * one.  gp_check_selftest fails one check on purpose in a kernel that touches
 * no memory and returns what the checked build reports (GP_ERR_STATE naming
 * site 99, index 5); in the default build it launches nothing and returns
 * GP_ERR_STATE ("not a bounds-checked build"). */
GP_API int gp_check_enabled(void);
GP_API gp_status gp_check_selftest(gp_ctx* ctx, void* stream);

#ifdef __cplusplus
}
#endif
#endif
