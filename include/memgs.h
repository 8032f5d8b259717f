/*
 * memgs.h - C ABI of the GB300 (sm_103a) splatting + voxel-merge library.
 *
 * The library implements the data-parallel hot path of the MemGS mapping back-end:
 * the tile-based differentiable 3D Gaussian Splatting rasteriser (forward and
 * backward) of Sec. II-C / II-E and the voxel-space merge of Sec. II-D, plus the
 * optimiser step that consumes the gradients.  Every step runs in hand-written
 * CUDA kernels; there is no CPU fallback.
 *
 * Conventions for every entry point
 *   - Pointers are DEVICE pointers unless their name ends in _host.  The caller
 *     owns all memory; the library allocates nothing.  Scratch space is a caller
 *     workspace whose size comes from the matching *_workspace_size query.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous on it unless stated otherwise.
 *   - Return value: MGS_OK or an error code; mgs_last_error() gives a message
 *     (thread-local).  On an argument error nothing is launched.  No exception and
 *     no device trap crosses the ABI.
 *   - Layouts are dense, row-major, structure-of-arrays:
 *       means          f32 [n][3]  world frame
 *       log_scales     geom[n][3]  scale = exp(log_scale)
 *       quats          geom[n][4]  (w, x, y, z), need not be unit (normalised inside)
 *       opacity_logit  attr[n]     opacity = sigmoid(logit)
 *       sh             attr[n][K][3], K = (sh_degree+1)^2, real orthonormal SH basis
 *       birth          u64 [n]     insertion stamp, smaller = older (merge only)
 *     where geom and attr are each f32, f16 or bf16 (mgs_dtype); arithmetic is always
 *     f32.  Reduced-precision maps normally keep geom in f32: quantising the covariance
 *     parameters moves gradients by ~1e-2 relative, the appearance ones by <= 3.4e-3.
 *   - Camera: world->camera rotation R (row-major) and translation t; x right,
 *     y down, z forward; pixel (u, v) is evaluated at the point (u, v).
 */
#ifndef MEMGS_H
#define MEMGS_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MGS_MAX_VIEWS 32
#define MGS_TILE 16

typedef enum {
  MGS_OK = 0,
  MGS_ERR_INVALID = 1,     /* bad argument: nothing was launched */
  MGS_ERR_WORKSPACE = 2,   /* workspace too small: nothing was written to outputs */
  MGS_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  MGS_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
  MGS_ERR_UNSUPPORTED = 5  /* size or mode outside what the kernels handle */
} mgs_status;

typedef enum { MGS_F32 = 0, MGS_F16 = 1, MGS_BF16 = 2 } mgs_dtype;

typedef struct {
  int64_t n;
  int32_t sh_degree;   /* 0..3 */
  int32_t attr_dtype;  /* mgs_dtype of opacity_logit and sh */
  int32_t geom_dtype;  /* mgs_dtype of log_scales */
  int32_t quat_dtype;  /* mgs_dtype of quats */
  const float* means;
  const void* log_scales;
  const void* quats;
  const void* opacity_logit;
  const void* sh;
  const uint64_t* birth; /* may be NULL except for mgs_voxel_merge */
} mgs_gaussians;

typedef struct {
  int64_t n;           /* capacity on input; unused on output (see n_out_host) */
  int32_t sh_degree;
  int32_t attr_dtype;
  int32_t geom_dtype;
  int32_t quat_dtype;
  float* means;
  void* log_scales;
  void* quats;
  void* opacity_logit;
  void* sh;
  uint64_t* birth;
} mgs_gaussians_mut;

typedef struct {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height;
  float near_z;        /* Gaussians with camera-space z <= near_z are culled (0.2) */
  int32_t reserved;
} mgs_camera;

/* One view's image planes: rgb f32 [3][H][W], depth f32 [H][W], alpha f32 [H][W]. */
typedef struct {
  float* rgb;
  float* depth;
  float* alpha;
} mgs_image;

/* Gradient accumulators, f32, same layouts as the parameters (always f32).
 * grad_stat / vis_count (optional, [n]) collect the Eq. 3 statistic: per view in
 * which the Gaussian is drawn, += |dL/dmean| and += 1.
 * overwrite (read by mgs_render_backward only): 0 adds the call's gradients to the
 * arrays; nonzero stores them, zeros for Gaussians drawn in no view (the arrays need
 * no clearing before the call, which saves a read and a write of every element);
 * grad_stat / vis_count are added to either way. */
typedef struct {
  float* means;
  float* log_scales;
  float* quats;
  float* opacity_logit;
  float* sh;
  float* grad_stat;
  float* vis_count;
  int32_t overwrite;
  int32_t reserved;
} mgs_grads;

/* ------------------------------------------------------------------------------
 * Rasteriser.  Sec. II-C Eq. 1 (projection mu_I = pi(T_CW mu_W), Sigma_I = J W Sigma
 * W^T J^T), Eq. 2 (Sigma = R S S^T R^T) and Sec. II-E Eq. 11 (front-to-back colour
 * and depth blending, product read as prod_{j<i}(1 - alpha_j)).
 * Per pixel, Gaussians are taken in order of (float32 camera depth, index); a
 * Gaussian is skipped when alpha = min(0.99, o exp(-d^T Sigma_I^-1 d / 2)) < 1/255
 * and the pixel stops after the Gaussian that takes its transmittance below 1e-4.
 * Sigma_I is dilated by 0.3 px^2, the Jacobian is taken at the ray clamped to 1.3x
 * the half field of view, and a Gaussian covers the 16x16 tiles that meet the square
 * of half-width ceil(3 sqrt(lambda_max)) around mu_I.  Outputs: rgb (black
 * background), depth = sum_i d_i w_i with d_i the camera-space z of the mean (not
 * normalised), alpha = 1 - T_final.
 * ------------------------------------------------------------------------------ */

/* Bytes of workspace for rendering n Gaussians into n_views views with room for
 * key_capacity (Gaussian, tile) pairs.  Returns 0 on invalid arguments. */
size_t mgs_render_workspace_size(int64_t n, const mgs_camera* cams_host, int32_t n_views,
                                 int64_t key_capacity);

/* Forward render of n_views views (1..MGS_MAX_VIEWS, resolutions may differ) in one
 * pass: per-Gaussian projection for all views, one depth sort, one tile sort, one
 * blend launch over every (view, tile).  cams_host / out_host: host arrays of
 * n_views entries; out_host[v] planes are device pointers.  The workspace keeps the
 * state the backward pass needs and must not be modified until then.
 * *n_keys_host (optional) receives the number of (Gaussian, tile) pairs.  If they
 * exceed the workspace's capacity, returns MGS_ERR_WORKSPACE without touching the
 * outputs; grow the workspace for *n_keys_host keys and call again.
 * Synchronises `stream` once (to read the key count). */
mgs_status mgs_render(const mgs_gaussians* g, const mgs_camera* cams_host, int32_t n_views,
                      const mgs_image* out_host, void* workspace, size_t workspace_bytes,
                      int64_t* n_keys_host, void* stream);

/* mgs_render without the host synchronisation: the launches are sized for the
 * workspace's key capacity and read the actual counts from device memory.  If the keys
 * exceed the capacity, nothing is emitted or blended (the images come out empty) and
 * the status says so.  status_pinned (optional, page-locked host memory of 2 int64):
 * receives {number of (Gaussian, tile) keys, 1 if they exceeded the capacity else 0}
 * once the stream has reached the end of the call; read it after synchronising with
 * the stream (or an event recorded after the call).  Everything else as mgs_render,
 * including the state mgs_render_backward reads.  Asynchronous. */
mgs_status mgs_render_async(const mgs_gaussians* g, const mgs_camera* cams_host, int32_t n_views,
                            const mgs_image* out_host, void* workspace, size_t workspace_bytes,
                            int64_t* status_pinned, void* stream);

/* Forward render of views that each name their own map (Sec. II-E rasteriser, serving
 * several resident maps at once): view v is rendered from maps_host[map_of_view_host[v]]
 * (0 <= index < n_maps; map_of_view_host is a host array of n_views entries).  One
 * projection launch per run of consecutive views that share a map, then, for all views
 * together, one depth sort, one key emission, one tile sort and one blend launch over
 * every (view, tile).  Each view's image is bit-identical to rendering it alone with
 * mgs_render.  Together the views' maps may hold fewer than 2^32 Gaussians (counted once
 * per view).  Workspace, key capacity, *n_keys_host, errors and the synchronisation are
 * as for mgs_render; the workspace does not support mgs_render_backward (one map only).
 * Not in the paper: the serving form of its rasteriser. */
size_t mgs_render_multi_workspace_size(const mgs_gaussians* maps_host, int32_t n_maps,
                                       const int32_t* map_of_view_host, const mgs_camera* cams_host,
                                       int32_t n_views, int64_t key_capacity);
mgs_status mgs_render_multi(const mgs_gaussians* maps_host, int32_t n_maps, const int32_t* map_of_view_host,
                            const mgs_camera* cams_host, int32_t n_views, const mgs_image* out_host,
                            void* workspace, size_t workspace_bytes, int64_t* n_keys_host, void* stream);

/* Reverse pass of the last mgs_render / mgs_render_async on `workspace` (same g, cams,
 * n_views).  dL_host[v] gives dL/drgb, dL/ddepth, dL/dalpha planes of view v (any plane
 * may be NULL = zero).  Gradients of all views are ADDED to `grads` (f32), or stored when
 * grads->overwrite is nonzero.  It may be called more than once for the same render
 * (each call computes that render's gradients afresh).  Asynchronous. */
mgs_status mgs_render_backward(const mgs_gaussians* g, const mgs_camera* cams_host,
                               int32_t n_views, const mgs_image* dL_host, void* workspace,
                               size_t workspace_bytes, const mgs_grads* grads, void* stream);

/* Per-Gaussian projection of one view into caller arrays (debugging / inspection):
 * mean2d f32[n][2], conic f32[n][3], rgb f32[n][3], depth f32[n], radius i32[n],
 * rect i32[n][4] (inclusive tile rect; x1 < x0 when not drawn).  Any pointer may be NULL. */
mgs_status mgs_project(const mgs_gaussians* g, const mgs_camera* cam_host, float* mean2d,
                       float* conic, float* rgb, float* depth, int32_t* radius, int32_t* rect,
                       void* stream);

/* ------------------------------------------------------------------------------
 * Voxel merge, Sec. II-D.  Eq. 3 mask: eligible iff the mean gradient norm (grad_stat,
 * or grad_stat / vis_count) < grad_tau and kf_min <= kf_id <= kf_max (a NULL array
 * makes its test pass).  Eligible Gaussians
 * are grouped by voxel floor(mu / voxel_size) (float32 quotient, origin at 0).  In a
 * voxel every pair (i older than j) gets Eq. 4's d^2 = (mu_j-mu_i)^T Sigma_i^-1
 * (mu_j-mu_i); pairs with d^2 < chi2 (7.815, chi-square 0.05 with 3 dof) are similar.
 * greedy=1: repeatedly merge the unmatched pair of smallest (d^2, birth_i, birth_j);
 * greedy=0: only the smallest pair of each voxel.  A merged pair keeps G_i's slot:
 * mean by Eq. 6, covariance the equal-weight 2-Wasserstein barycentre (the minimiser
 * of Eq. 9: in closed form, or by L-BFGS with solver = 1), stored as (quaternion with
 * w >= 0, scales descending),
 * opacity, SH and birth copied from the older G_i; G_j is dropped.  Survivors keep
 * the input order.
 * ------------------------------------------------------------------------------ */
typedef struct {
  float chi2;              /* 7.815 */
  float grad_tau;          /* 1e-3 */
  int32_t kf_min, kf_max;
  const float* grad_stat;  /* [n] or NULL */
  const int32_t* kf_id;    /* [n] or NULL */
  const float* vis_count;  /* [n] or NULL.  Non-NULL: grad_stat holds sums of |dL/dmu| over
                              the views that drew each Gaussian and vis_count the number of
                              those views (both as mgs_render_backward accumulates them over
                              a keyframe window); the mask tests the mean, the float32
                              quotient grad_stat / vis_count (0 for a Gaussian drawn in no
                              view), against grad_tau.  NULL: grad_stat is the mean itself. */
  int32_t greedy;          /* 1 or 0 */
  int32_t solver;          /* merged covariance: 0 = the closed-form minimiser of Eq. 9;
                              1 = the paper's route, L-BFGS over (q, s) from the Eq. 10
                              start (slerp t = 0.5, mean scale + (0.001, 0.002, 0.003)),
                              float32, memory 6, line search on the directional
                              derivative, at most 200 iterations */
} mgs_merge_params;

/* Counters of the calling thread's last successful mgs_voxel_merge: out[0] = merged
 * pairs, out[1] = L-BFGS iterations summed over the pairs (0 with solver 0).  Not part
 * of the paper. */
void mgs_merge_stats(int64_t out[2]);

size_t mgs_voxel_merge_workspace_size(int64_t n);

/* out: capacity >= in->n, same sh_degree, attr_dtype and geom_dtype.  partner (optional, [n]):
 * index of the merge partner or -1.  voxel (optional, i32 [n][3]): voxel coordinates
 * of eligible Gaussians (INT32_MIN for ineligible ones).  Voxels of any number of
 * members.  Synchronises `stream` and writes the survivor count to *n_out_host.  Voxel
 * coordinates must fit in 21 bits signed (|mu / voxel_size| < 2^20) and the occupied
 * voxels' box in 31 key bits, else nothing merges (out is a copy) and the call returns
 * MGS_ERR_UNSUPPORTED. */
mgs_status mgs_voxel_merge(const mgs_gaussians* in, float voxel_size, const mgs_merge_params* p,
                           const mgs_gaussians_mut* out, int32_t* partner, int32_t* voxel,
                           int64_t* n_out_host, void* workspace, size_t workspace_bytes,
                           void* stream);
/* mgs_voxel_merge without the host synchronisation (every launch is sized from n and
 * reads its counts from device memory).  status_pinned (optional, page-locked host
 * memory of 2 int32): receives {survivor count, flags} once the stream has reached the
 * end of the call; flags bit 0: a voxel coordinate outside +-2^20, bit 2: nothing
 * merged because of it or of a box needing more than 31 key bits.  mgs_merge_stats
 * does not cover this form.  Asynchronous. */
mgs_status mgs_voxel_merge_async(const mgs_gaussians* in, float voxel_size, const mgs_merge_params* p,
                                 const mgs_gaussians_mut* out, int32_t* partner, int32_t* voxel,
                                 int32_t* status_pinned, void* workspace, size_t workspace_bytes,
                                 void* stream);

/* ------------------------------------------------------------------------------
 * Optimiser: Adam with bias correction over every parameter array of `params`
 * (one streaming launch over all arrays; the optimiser is not named in the paper, Sec. II-E; Adam is this
 * library's choice).  m and v are f32 state arrays shaped like the parameters
 * (same mgs_gaussians_mut layout, f32 pointers in m_state / v_state), 16-byte
 * aligned like the parameter and gradient arrays (every f32 array: a misaligned
 * one returns MGS_ERR_INVALID before anything runs).  Parameters
 * stored in f16/bf16 (either group) are updated in f32 and rounded back.  step >= 1.  zero_grads = 1
 * clears each gradient element after it is consumed (the next backward pass
 * accumulates from zero without a separate clearing pass).  Asynchronous.
 * ------------------------------------------------------------------------------ */
mgs_status mgs_adam_step(const mgs_gaussians_mut* params, const mgs_grads* grads,
                         const mgs_grads* m_state, const mgs_grads* v_state, float lr, float beta1,
                         float beta2, float eps, int32_t step, int32_t zero_grads, void* stream);

/* ------------------------------------------------------------------------------
 * Mapping loss of Sec. II-E, Eq. 12, per view v (all views width x height):
 *   L_v = (1 - lambda) mean|x - y| + lambda (1 - mean SSIM(x, y))
 *         + w_depth mean_p [dt(p) > 0] |d(p) - dt(p)|          (depth residual, RGB-D)
 * x = rendered[v].rgb, y = target[v].rgb (planar f32 [3][H][W]), d = rendered[v].depth,
 * dt = target[v].depth (f32 [H][W]; NULL: no depth term).  Means over the 3HW colour
 * values and the HW pixels.  SSIM per channel and pixel with the 11x11 Gaussian window
 * (sigma 1.5, normalised), C1 = 0.01^2, C2 = 0.03^2, windows cut by the image border
 * (zero padding).  The paper gives no lambda (0.2 is the usual choice).
 * grad[v].rgb receives dL_v/dx (written, not accumulated), grad[v].depth (optional)
 * dL_v/dd; they are the cotangents mgs_render_backward takes.  loss: device f32
 * [n_views][3] = (L1 part, SSIM part, depth part), each already weighted, written.
 * lambda = 0 skips the SSIM windows altogether (the plain L1 form; SSIM part 0).
 * 1 <= n_views <= MGS_MAX_VIEWS.  Deterministic (fixed-order sums).  Asynchronous.
 * ------------------------------------------------------------------------------ */
size_t mgs_mapping_loss_workspace_size(int32_t n_views, int32_t width, int32_t height);
mgs_status mgs_mapping_loss(int32_t n_views, int32_t width, int32_t height, const mgs_image* rendered,
                            const mgs_image* target, const mgs_image* grad, float lambda_ssim,
                            float w_depth, float* loss, void* workspace, size_t workspace_bytes,
                            void* stream);

/* Isotropic term of Eq. 12 (the paper follows MonoGS and gives no formula):
 *   L_iso = w_iso / (3n) sum_i sum_k |s_ik - mean_k s_ik|,  s = exp(log_scales).
 * grads (optional): dL_iso/dlog_scales ADDED to grads->log_scales.  loss: device f32,
 * written.  Asynchronous. */
size_t mgs_iso_loss_workspace_size(int64_t n);
mgs_status mgs_iso_loss(const mgs_gaussians* g, float w_iso, const mgs_grads* grads, float* loss,
                        void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------------
 * Patch-Grid sampling, Sec. II-B: initial points for new Gaussians in the patches of a
 * keyframe that hold too few keypoints.  The image is cut into patch x patch pixel
 * patches (the last row / column clipped to the image).  A patch holding fewer than
 * min_keypoints of the keypoints that lie inside the image receives grid x grid samples
 * at the centres of an even grid x grid split of the patch.  A sample's depth is
 * depth_image[floor v][floor u] when that is > 0, else the depth of the nearest
 * keypoint with kp_depth > 0 (float32 squared pixel distance, ties: smaller index); a
 * sample with neither is dropped.  Samples are back-projected with the pinhole camera
 * and taken to the world frame (x_w = R^T (x_c - t)).
 * kp_uv: device f32 [n_keypoints][2]; kp_depth: device f32 [n_keypoints] or NULL;
 * depth_image: device f32 [height][width] or NULL.  out: device f32 [capacity][6] =
 * (u, v, depth, x, y, z world), in patch order then sample order; source (optional,
 * i32 [capacity]): 0 depth image, 1 keypoint.  Synchronises `stream` and writes the
 * sample count to *n_out_host; MGS_ERR_WORKSPACE when it exceeds capacity (nothing
 * beyond capacity is written).  mgs_patch_grid_capacity gives the largest count.
 * ------------------------------------------------------------------------------ */
typedef struct {
  int32_t patch;          /* patch edge, px */
  int32_t min_keypoints;  /* patches with fewer keypoints are sampled */
  int32_t grid;           /* grid x grid samples per sampled patch */
  int32_t reserved;
} mgs_pg_params;

size_t mgs_patch_grid_workspace_size(int32_t width, int32_t height, const mgs_pg_params* p);
int64_t mgs_patch_grid_capacity(int32_t width, int32_t height, const mgs_pg_params* p);
mgs_status mgs_patch_grid_sample(const mgs_camera* cam, int32_t n_keypoints, const float* kp_uv,
                                 const float* kp_depth, const float* depth_image, const mgs_pg_params* p,
                                 float* out, int32_t* source, int64_t capacity, int64_t* n_out_host,
                                 void* workspace, size_t workspace_bytes, void* stream);

/* L1 loss helper for mapping steps: grad[i] = scale * sign(pred[i] - target[i]) and
 * *loss += scale * sum |pred - target| (loss is a device f32 accumulator). */
mgs_status mgs_l1_loss_grad(const float* pred, const float* target, int64_t n, float scale,
                            float* grad, float* loss, void* stream);

/* ------------------------------------------------------------------------------
 * Device radix sort used by the rasteriser, exposed for testing: stable LSD sort
 * of (key, value) u32 pairs on bits [begin_bit, end_bit).  keys/vals are sorted in
 * place (the workspace holds the ping-pong buffers).  vals may be NULL: the values
 * are then the input positions 0..n-1 and are written to vals_out.
 * ------------------------------------------------------------------------------ */
size_t mgs_sort_workspace_size(int64_t n);
mgs_status mgs_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* vals_out, int64_t n,
                          int32_t begin_bit, int32_t end_bit, void* workspace,
                          size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------------
 * Render serving with continuous batching (not in the paper: the serving form of the
 * Sec. II-E rasteriser).  Resident scene maps are registered once; requests (scene,
 * camera, output planes) are submitted at any time.  When a worker slot is free, a
 * dispatcher thread admits the oldest pending requests, of any scene and resolution,
 * up to max_batch_views of them and as many as their workspace fits in free memory of
 * the caller's device arena (first-fit; the server allocates no device memory), and
 * renders them with one mgs_render_multi call: one blend launch over the (view, tile)
 * items of all of them.  Each slot has its own stream and thread, so batches overlap
 * on the device.  Results are bit-identical to rendering each request alone (the
 * forward pass is deterministic).  The gaussians and output
 * buffers must stay valid until the request completes; destroying the server drops
 * requests not yet admitted.
 * ------------------------------------------------------------------------------ */
typedef struct mgs_server mgs_server;
typedef struct {
  int32_t n_slots;          /* concurrent batches (1..64) */
  int32_t max_batch_views;  /* 1..MGS_MAX_VIEWS */
  int32_t device;           /* CUDA device ordinal */
  int32_t reserved;
  void* arena;              /* caller-owned device memory for workspaces */
  size_t arena_bytes;
} mgs_server_config;

mgs_status mgs_server_create(const mgs_server_config* cfg, mgs_server** out_host);
mgs_status mgs_server_add_scene(mgs_server* s, const mgs_gaussians* g, int32_t* scene_id_host);
/* t_submit: arrival time on mgs_server_clock() (<= 0: now); tag: caller's request id. */
mgs_status mgs_server_submit(mgs_server* s, int32_t scene_id, const mgs_camera* cam_host,
                             const mgs_image* out_host, int64_t tag, double t_submit);
/* Completed requests (up to max; waits up to wait_s seconds for the first one):
 * arrival, admission and completion times in seconds, and the mgs_status of each. */
int32_t mgs_server_poll(mgs_server* s, int32_t max, int64_t* tags_host, double* t_submit_host,
                        double* t_start_host, double* t_done_host, int32_t* status_host,
                        double wait_s);
double mgs_server_clock(void);
/* Counters since creation: out[0] render launches, out[1] requests served by them,
 * out[2] largest number of requests in one launch, out[3] launches holding more than
 * one scene. */
mgs_status mgs_server_stats(mgs_server* s, int64_t out_host[4]);
mgs_status mgs_server_destroy(mgs_server* s);

/* ------------------------------------------------------------------------------
 * Diagnostics (not part of the method).
 * mgs_launch_count: kernels launched by this library in this process so far.
 * mgs_profile_enable(1) clears the per-kernel totals and starts bracketing each of
 * the library's kernel groups with CUDA events on its stream; mgs_profile_read
 * waits for the pending events and returns up to max_kinds entries: name (32 bytes
 * each, NUL-terminated), total milliseconds and launch count.  Returns the number
 * of kinds.
 * mgs_render_stats: counting pass over the saved state of the last mgs_render on
 * `workspace` (same g, cams, n_views), stats_host[9]: [0] (pixel, entry) pairs the
 * forward evaluated, [1] contributing pairs (alpha >= 1/255), [2] pairs the backward
 * walks, [3] (Gaussian, tile) keys, [4]/[5] forward/backward pairs padded to each
 * tile's longest pixel list (x 256 pixels), [6]/[7] the same padded per warp of the
 * blend kernels (forward: 8x8-pixel blocks, backward: 8x4), [8] drawn (view, Gaussian)
 * items.
 * Synchronises `stream`.
 * ------------------------------------------------------------------------------ */
uint64_t mgs_launch_count(void);
void mgs_profile_enable(int32_t on);
int32_t mgs_profile_read(int32_t max_kinds, char* names, double* ms_total, int64_t* launches);
mgs_status mgs_render_stats(const mgs_gaussians* g, const mgs_camera* cams_host, int32_t n_views,
                            void* workspace, size_t workspace_bytes, uint64_t* stats_host,
                            void* stream);

/* ------------------------------------------------------------------------------
 * Sort without allocation.  The paper has no counterpart; this entry point serves
 * callers that cannot call cudaMalloc (or hand a workspace to every call): hosts that
 * reserve all device memory in their own pool up front, plugins given no allocator,
 * and latency-critical loops where a device allocation would synchronise the device
 * and stall work on other streams.  Same result as mgs_sort_pairs, with the scratch
 * in a statically sized device array inside the library: n <= MGS_SORT_NOALLOC_MAX
 * (1,048,576 pairs; about 13 MB held on every GPU that loads the library until the
 * process exits).  Larger n returns MGS_ERR_UNSUPPORTED.  It calls no cudaMalloc or
 * cudaFree.  The first call on a device looks up the array's device address (once
 * per device, with that device current); make that first call before any stream
 * capture.  Every call shares the one array: calls that overlap on the GPU (other
 * streams, other host threads) race, so serialise them.  Asynchronous on `stream`.
 * ------------------------------------------------------------------------------ */
#define MGS_SORT_NOALLOC_MAX (1 << 20)
mgs_status mgs_sort_pairs_noalloc(uint32_t* keys, uint32_t* vals, uint32_t* vals_out, int64_t n,
                                  int32_t begin_bit, int32_t end_bit, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* mgs_last_error(void);

/* Library version, e.g. "memgs 0.1 sm_103a". */
const char* mgs_version(void);

#ifdef __cplusplus
}
#endif
#endif
