/*
 * FP64 oracle for the MemGS splatting + voxel-merge hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is a plain, slow, obviously correct CPU
 * restatement of what the CUDA path computes.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant with the CUDA library and the CUDA library never calls it.
 *
 * Everything is evaluated in double precision from inputs that are exact copies of
 * the float32 parameters.  Sections followed:
 *   - 3D Gaussian map, projection and covariance: Sec. II-C, Eq. 1 and Eq. 2.
 *   - front-to-back colour and depth blending: Sec. II-E, Eq. 11, with the
 *     transmittance product read as prod_{j<i}(1 - alpha_j).
 *   - voxel merge: Sec. II-D, Eq. 3 (mask), Eq. 4 (squared Mahalanobis distance),
 *     the chi-square 0.05 / 3 dof critical value 7.815, Eq. 6 (merged mean),
 *     Eq. 7-9 (covariance as the 2-Wasserstein barycentre), Eq. 10 (solver
 *     initialisation), colour/opacity inherited from the older Gaussian.
 * The cutoffs (alpha >= 1/255, alpha <= 0.99, stop once T < 1e-4) and the tiling
 * conventions (16x16 tiles, 3-sigma square extent, 0.3 px^2 dilation, near plane)
 * are readings of the method that both sides implement.  The front-to-back order is
 * the float32 rounding of the camera-space depth, ties broken by Gaussian index: a
 * discrete decision taken from floating point is taken in the kernel's precision.
 *
 * All arrays are caller-owned, dense, row-major.  Functions return 0 on success and
 * a negative value on invalid arguments.  No function keeps state between calls.
 */
#ifndef MEMGS_ORACLE_H
#define MEMGS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double R[9];      /* world -> camera rotation, row-major */
  double t[3];      /* world -> camera translation */
  double fx, fy, cx, cy;
  double near_z;    /* Gaussians with camera z <= near_z are culled */
  int32_t width, height;
} orc_camera;

typedef struct {
  int64_t n;
  int32_t sh_degree;        /* 0..3, K = (deg+1)^2 coefficients per channel */
  const double* means;      /* [n][3] */
  const double* log_scales; /* [n][3] */
  const double* quats;      /* [n][4] (w,x,y,z), normalised inside */
  const double* opacity_logit; /* [n] */
  const double* sh;         /* [n][K][3] */
} orc_gaussians;

/* Margins below which a discrete decision is called a near-tie (pixel flagged). */
typedef struct {
  double alpha_rel;   /* |alpha*255 - 1| */
  double T_rel;       /* |T/1e-4 - 1| after a contribution */
  double depth_rel;   /* distance of a depth to a float32 rounding midpoint, relative,
                         for neighbouring contributors whose float32 keys are within 1 ulp */
  double extent_px;   /* distance of a tile-rect edge (u +- r) to a tile boundary, px */
  double radius_abs;  /* distance of 3*sqrt(lambda_max) to an integer */
  double near_rel;    /* |tz - near| / near */
  double clamp_rel;   /* |o*G - 0.99| / 0.99 (gradient switch) */
  double cond_rel;    /* added to alpha_rel per unit of |exponent| x conditioning c of the
                         projection: c = sqrt(gamma kappa) + kappa, kappa = lambda_max /
                         lambda_min of Sigma_I, gamma = (||T||_F^2 ||Sigma||_F + tr Sigma_I)
                         / lambda_min, T = J W.  Rounding the rotation, the scales and T
                         to float32 moves the exponent by up to ~c units of 2^-24 relative
                         (most for Gaussians long along the view ray); evaluating it moves
                         it by ~kappa.  The T margin grows by the root-sum-square of
                         alpha/(1-alpha) x the alpha margins so far. */
} orc_margins;

/* Per-Gaussian projection (Eq. 1-2, plus the tiling extent). */
typedef struct {
  double* mean2d;   /* [n][2] pixel coordinates u, v */
  double* conic;    /* [n][3] inverse of the dilated 2D covariance (A, B, C) */
  double* cov2d;    /* [n][3] dilated 2D covariance (a, b, c) */
  double* rgb;      /* [n][3] colour after the max(0, .) clamp */
  double* depth;    /* [n]    camera-space z */
  double* opacity;  /* [n]    sigmoid(logit) */
  int32_t* radius;  /* [n]    ceil(3 sqrt(lambda_max)); 0 when culled */
  int32_t* rect;    /* [n][4] inclusive tile rect x0,y0,x1,y1; x1<x0 when empty */
  int32_t* visible; /* [n]    1 when projected and the rect is non-empty */
} orc_projection;

int orc_project(const orc_gaussians* g, const orc_camera* cam, orc_projection* out);

/* Real orthonormal spherical harmonics up to degree 3 at a unit direction:
 * Y[k], k = l*l + l + m, and dY[k][3] the derivative of the polynomial form. */
int orc_sh_basis(int32_t degree, const double dir[3], double* Y, double* dY);

/* Forward render of one view.  Outputs are [H][W] planes (rgb is [3][H][W]).
 * n_contrib: 1 + index (within the pixel's sorted tile list) of the last contributor.
 * n_eval: list entries evaluated until the stop (or the list length).
 * flags: bit0 alpha cutoff, bit1 T stop, bit2 depth order, bit3 extent/near,
 *        bit4 opacity clamp near-tie.  tiles: optional list of tile ids to render
 *        (others are left untouched); n_tiles < 0 renders every tile.
 * decision_hash: hash of every pixel's contributor list (for finite differences). */
int orc_render(const orc_gaussians* g, const orc_camera* cam, const orc_margins* m,
               const int32_t* tiles, int32_t n_tiles,
               double* rgb, double* depth, double* alpha, double* T_final,
               int32_t* n_contrib, int32_t* n_eval, uint8_t* flags,
               uint64_t* decision_hash, int32_t n_threads);

/* Both outcomes of the near-tie decisions (needs margins).  Besides the image of
 * orc_render, per pixel: n_ties = the number of near-tie decisions that can change the
 * image (alpha cutoff, T stop, order of two neighbouring contributors, extent / near
 * plane; the opacity clamp is continuous in the image and is not counted), and alt_*
 * = the image with that decision taken the other way when n_ties == 1 (the same image
 * when n_ties == 0, NaN when n_ties >= 2).  A float32 renderer that takes the
 * decision either way matches one of the two. */
int orc_render_outcomes(const orc_gaussians* g, const orc_camera* cam, const orc_margins* m,
                        const int32_t* tiles, int32_t n_tiles,
                        double* rgb, double* depth, double* alpha, double* T_final,
                        int32_t* n_contrib, uint8_t* flags,
                        double* alt_rgb, double* alt_depth, double* alt_alpha, int32_t* n_ties,
                        int32_t n_threads);

/* Same image, computed pixel by pixel over all n Gaussians with the tile-rect
 * predicate and an explicit (depth, index) ordering; no binning. */
int orc_render_bruteforce(const orc_gaussians* g, const orc_camera* cam,
                          double* rgb, double* depth, double* alpha);

/* Reverse-mode gradient of L = sum(g_rgb*rgb) + sum(g_depth*depth) + sum(g_alpha*alpha)
 * for one view.  Any cotangent pointer may be NULL (zero).  Gradients are ADDED
 * into the outputs.  grad2d: optional [n][10] per-Gaussian screen-space gradient
 * (du, dv, dA, dB, dC, d_opacity, dr, dg, db, d_depth).  taint: optional [n], set
 * to 1 for Gaussians evaluated at a flagged pixel.  grad_stat / vis_count: optional
 * [n], += |dL/dmean| of this view and += 1 when visible (Eq. 3 statistic). */
typedef struct {
  double* means; double* log_scales; double* quats; double* opacity_logit; double* sh;
  double* grad2d; uint8_t* taint; double* grad_stat; double* vis_count;
  /* optional (all five or none), += like the gradients: the modelled float32 error
   * of each gradient element.  Each per-pixel term of a screen-space component is
   * taken in absolute value times the relative error it may carry in float32 (its
   * alpha margin, the pixel's accumulated T margin, and 32 x 2^-24 for the sums),
   * and the chain rule to the parameters is run in running-error arithmetic (sums
   * of absolute products).  It does not shrink where the exact terms cancel. */
  double* scale_means; double* scale_log_scales; double* scale_quats; double* scale_opacity_logit;
  double* scale_sh;
} orc_grads;

int orc_render_backward(const orc_gaussians* g, const orc_camera* cam, const orc_margins* m,
                        const int32_t* tiles, int32_t n_tiles,
                        const double* g_rgb, const double* g_depth, const double* g_alpha,
                        orc_grads* out, int32_t n_threads);

/* ---- voxel merge (Sec. II-D) ---- */
typedef struct {
  double chi2;               /* 7.815 */
  double grad_tau;           /* Eq. 3 tau, 1e-3 */
  int32_t kf_min, kf_max;    /* Eq. 3 keyframe window */
  const double* grad_stat;   /* [n] mean |dL/dmu| or NULL (all pass) */
  const int32_t* kf_id;      /* [n] keyframe index or NULL (all pass) */
  const double* vis_count;   /* [n] or NULL; non-NULL: grad_stat holds sums over the views
                                that drew each Gaussian and the mask tests the mean, taken
                                as the float32 quotient grad_stat / vis_count (0 when no view
                                drew it), the precision the kernel decides in */
  int32_t greedy;            /* 1: greedy disjoint pairs, 0: single minimum pair per voxel */
} orc_merge_params;

/* Voxel coordinates floor(mu/v) per axis, the quotient rounded to float32. */
int orc_voxel_keys(int64_t n, const double* means, double voxel, int32_t* keys);

/* Full merge.  Outputs have capacity n; *n_out receives the survivor count.
 * partner[n]: index of the merge partner or -1.  tie_flag[n] (optional): 1 when the
 * Gaussian is part of a near-tie (|d2 - chi2| < tie_rel*chi2, or two candidates of
 * its voxel that share a member with d2 within tie_rel of each other). */
int orc_voxel_merge(const orc_gaussians* g, const uint64_t* birth, double voxel,
                    const orc_merge_params* p,
                    double* out_means, double* out_log_scales, double* out_quats,
                    double* out_opacity_logit, double* out_sh, uint64_t* out_birth,
                    double* out_cov, /* [n_out][6] merged-or-copied covariance xx,xy,xz,yy,yz,zz */
                    int32_t* partner, int64_t* n_out, double tie_rel, uint8_t* tie_flag);

/* Eq. 9 closed form: equal-weight 2-Wasserstein barycentre of N(0,Si), N(0,Sj). */
int orc_w2_barycentre(const double Si[9], const double Sj[9], double Sk[9]);
/* Eq. 9 by L-BFGS over (q, s) from the Eq. 10 initialisation. Returns iterations. */
int orc_w2_lbfgs(const double qi[4], const double si[3], const double qj[4], const double sj[3],
                 double t, const double delta[3], double qk[4], double sk[3], double Sk[9],
                 double* final_objective);
/* Eq. 8: squared 2-Wasserstein distance between N(0,A) and N(0,B). */
double orc_w2_sq(const double A[9], const double B[9]);
/* Eq. 6 merged mean. */
int orc_merge_mean(const double Si[9], const double mi[3], const double Sj[9], const double mj[3],
                   double mk[3]);
/* Sigma = R(q) diag(s^2) R(q)^T. */
int orc_covariance(const double q[4], const double s[3], double S[9]);

/* Adam (bias-corrected), one step over n values, state updated in place. */
int orc_adam(int64_t n, double* param, const double* grad, double* m, double* v,
             double lr, double b1, double b2, double eps, int32_t step);

/* ---- mapping loss (Sec. II-E, Eq. 12) ----
 * Per view, rendered x and target y (planar [3][H][W]), depth d and target depth dt
 * ([H][W], dt NULL = no depth term):
 *   L = (1-lambda) mean|x-y| + lambda (1 - mean SSIM(x, y)) + w_depth mean_p [dt>0] |d-dt|
 * mean over the 3HW values (HW for depth).  SSIM per channel and pixel with the 11x11
 * Gaussian window (sigma 1.5, normalised), C1 = 0.01^2, C2 = 0.03^2, windows cut at the
 * image border with zero padding (the map has the image's size).  Per view the three
 * terms go to loss[3*v .. 3*v+2] = (L1 part, SSIM part, depth part), already weighted.
 * g_rgb / g_depth (optional) receive dL/dx and dL/dd (overwritten). */
int orc_mapping_loss(int32_t n_views, int32_t H, int32_t W, const double* x, const double* y,
                     const double* d, const double* dt, double lambda, double w_depth,
                     double* loss, double* g_rgb, double* g_depth);

/* Isotropic term (after MonoGS): w_iso / (3n) sum_i sum_k |s_ik - mean_k s_ik|, s = exp(log s).
 * *loss receives the value; grad_ls (optional) receives dL/dlog_scale ADDED to it. */
int orc_iso_loss(int64_t n, const double* log_scales, double w_iso, double* loss, double* grad_ls);

/* ---- Patch-Grid sampling (Sec. II-B) ----
 * The image is cut into patch x patch pixel patches (the last row / column of patches
 * clipped to the image).  A patch holding fewer than min_keypoints keypoints (of the
 * keypoints inside the image) receives grid x grid samples at the centres of an even
 * grid x grid split of the patch.  A sample's depth is the depth image's value at
 * (floor u, floor v) when that is > 0; otherwise the depth of the nearest keypoint
 * with a known depth (kp_depth > 0), nearest by the float32 value of
 * (ku - u)^2 + (kv - v)^2 evaluated as written (ties: smaller index); a sample with
 * neither is dropped.  Samples are back-projected (pinhole) and taken to the world
 * frame: x_w = R^T (x_c - t).  Output in patch order (row-major), then sample order.
 * kp_uv, kp_depth and depth_image are float32 (the precision the decisions use).
 * out [n][6] = (u, v, depth, xw, yw, zw); source [n] = 0 (depth image) / 1 (keypoint). */
int orc_patch_grid(const orc_camera* cam, int32_t n_kp, const float* kp_uv, const float* kp_depth,
                   const float* depth_image, int32_t patch, int32_t min_keypoints, int32_t grid,
                   double* out, int32_t* source, int64_t* n_out);

#ifdef __cplusplus
}
#endif
#endif
