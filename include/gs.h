/*
 * gs.h - C ABI of the GB300 multi-view Gaussian-splatting library
 * (libgsraster.so, built from paper_2510_26358_gb300/csrc).
 *
 * The library renders B cameras of one shared set of 3-D Gaussians and
 * back-propagates to every Gaussian parameter and to each camera's SE(3)
 * pose, as the multi-view mapping of AgriGS-SLAM describes (Sec. III-B,
 * Eqs. 2-4: a single shared splat set, per-camera EWA projection
 * Sigma' = J W Sigma W^T J^T; Sec. III-C, Eqs. 6-8: photometric and
 * probabilistic LiDAR depth losses whose gradients also refine the poses).
 *
 * Conventions
 *  - Every pointer marked (device) is CUDA device memory owned by the caller.
 *    The library owns only the workspace, which gs_workspace_create allocates
 *    once; no other call allocates, frees or synchronises.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). All work of a call is enqueued on it, in order.
 *  - Gaussians are float32 structure-of-arrays: means [N][3], log_scales
 *    [N][3], quats [N][4] as (w,x,y,z) (normalised inside), opacity_logits
 *    [N], sh [N][K][3] with K = (sh_degree+1)^2 (real orthonormal basis,
 *    ordered by l then m = -l..l, no Condon-Shortley phase).
 *  - Submaps: the Gaussian array is partitioned by submap_offsets [S+1];
 *    camera v renders only the Gaussians of its submap.
 *  - Cameras: OpenCV axes (x right, y down, z forward); T_cw is the row-major
 *    3x4 world->camera transform [R | t]. Pixel (i,j) is sampled at its centre.
 *  - Images are planar float32, views concatenated: view v's RGB occupies
 *    rgb[3*pix_off[v] .. 3*pix_off[v] + 3*W*H) as [3][H][W]; depth and alpha
 *    occupy [pix_off[v] .. pix_off[v] + W*H) as [H][W]; pix_off[v] is the sum
 *    of W*H over the views before v.
 *  - Gradients are accumulated (+=) into the caller's buffers, or written
 *    (gs_grads.overwrite).
 *  - Errors: argument errors return at once and enqueue nothing. Conditions
 *    found on the device (instance capacity exceeded, a bounded device wait
 *    that ran out) set a flag in the workspace that lasts until the next
 *    gs_bin_sort; after a capacity overflow the kernels that follow work on
 *    empty lists (blank images, zero gradients).  gs_workspace_status reports
 *    the flags.  Nothing traps or aborts.
 */
#ifndef GS_H
#define GS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_MAX_VIEWS 64
#define GS_MAX_SUBMAPS 64

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1, /* a pointer, size or configuration value is out of range */
    GS_ERR_CAPACITY = 2,    /* more (view, Gaussian, tile) instances than the workspace holds */
    GS_ERR_CUDA = 3,        /* a CUDA runtime call failed (message: gs_last_error) */
    GS_ERR_STATE = 4,       /* calls out of order (e.g. gs_render_fwd before gs_bin_sort) */
    GS_ERR_TIMEOUT = 5      /* a bounded device-side wait ran out (the step's results are not valid) */
} gs_status;

/* One pinhole camera (80 bytes). */
typedef struct {
    int32_t width, height; /* image size in pixels, 1..16384 */
    int32_t submap;        /* index of the submap this camera renders */
    int32_t reserved;      /* must be 0 */
    float fx, fy, cx, cy;  /* focal lengths and principal point, pixels */
    float T_cw[12];        /* row-major [R | t], world -> camera */
} gs_camera;

/* Renderer constants (the paper leaves them to standard 3DGS). */
typedef struct {
    int32_t tile_w, tile_h; /* tile size in pixels: 8x8, 16x16, 16x32 or 32x16 */
    int32_t batch_depth;    /* Gaussians staged per shared-memory batch: 32..256, multiple of 32 */
    int32_t depth_mode;     /* gs_depth_loss: 0 = L1 |D - z|, 1 = KL of Eq. (7) with fixed sigma_U */
    float near_z;           /* pairs with view-space z <= near_z are culled (0.2 m) */
    float dilation;         /* added to the diagonal of Sigma' (0.3 px^2) */
    float alpha_min;        /* fragments with alpha < alpha_min are skipped (1/255) */
    float alpha_max;        /* alpha = min(alpha_max, o*exp(-d^T Sigma'^-1 d / 2)) (0.99) */
    float t_min;            /* a fragment that would take T below t_min ends the pixel (1e-4) */
    float jac_clamp;        /* tangent clamp of the projection Jacobian, x max(cx,W-cx)/fx (1.3) */
    float ext_rel_pad;      /* relative padding of the support extent used for tiles (1e-3) */
    float ext_abs_pad;      /* absolute padding of that extent, pixels (1e-2) */
    float sigma_L;          /* LiDAR standard deviation of Eq. (7), metres (0.05) */
    float sigma_U;          /* rendered-depth standard deviation of Eq. (7), metres (0.05) */
    float lambda_L;         /* weight lambda_L of Eq. (7) (1) */
    float reserved;         /* must be 0 */
} gs_config;

/* Gaussian parameters (device, float32, C-contiguous). */
typedef struct {
    const float *means, *log_scales, *quats, *opacity_logits, *sh;
    int64_t n; /* must equal submap_offsets[n_submaps] given at workspace creation */
} gs_gaussians;

/* Gradient outputs (device). pose, densify_acc and densify_cnt may be NULL.
 * densify_acc[g] gets ||dL/d(u,v)|| (pixels) and densify_cnt[g] 1 for every
 * view in which Gaussian g is visible (the densification statistic of Sec.
 * III-B).  overwrite = 0: every output is accumulated (+=) into the caller's
 * values; overwrite = 1: every output is written (=), zeros for the rows of
 * Gaussians that no view sees, so the buffers need no clearing before the
 * call (one write of each row instead of a clear and a read-modify-write). */
typedef struct {
    float *means, *log_scales, *quats, *opacity_logits, *sh;
    float *pose;        /* [n_views][6]: dL/d(rho, phi) of the left perturbation exp(xi^) T_cw */
    float *densify_acc; /* [N] */
    int32_t *densify_cnt; /* [N] */
    int32_t overwrite;  /* 0 accumulate, 1 write */
    int32_t reserved;   /* must be 0 */
} gs_grads;

typedef struct gs_workspace gs_workspace;

/* Fill *cfg with the defaults quoted above (16x16 tiles, depth 256, L1 depth loss). */
void gs_config_default(gs_config *cfg);

/* Create a workspace for a fixed camera geometry and submap partition.
 * cams (host, n_views entries, 1..GS_MAX_VIEWS): sizes and submap ids are
 *   fixed here; intrinsics and poses are read from the device copy given to
 *   each call, so poses may change between calls (and CUDA-graph replays).
 * submap_offsets (host, n_submaps+1 entries, 1..GS_MAX_SUBMAPS, nondecreasing,
 *   offsets[0] = 0).
 * sh_degree 0..3. inst_capacity: maximum (view, Gaussian, tile) instances per
 * iteration (gs_workspace_status reports the number needed).
 * Allocates all device memory the other calls use (on the current device). */
gs_status gs_workspace_create(const gs_camera *cams, int32_t n_views, const int64_t *submap_offsets,
                              int32_t n_submaps, int32_t sh_degree, const gs_config *cfg,
                              int64_t inst_capacity, gs_workspace **out);
void gs_workspace_destroy(gs_workspace *ws);

/* Per-camera projection (Eqs. 3-4): for every (view, Gaussian) pair of the
 * same submap, Sigma = R S S^T R^T from the normalised quaternion and
 * exp(log_scale), p = W mu + t, near-plane cull, Sigma' = J W Sigma W^T J^T
 * + dilation*I, its inverse, opacity sigmoid(omega), the extent of the
 * alpha >= alpha_min ellipse and the tiles it covers, and the SH colour seen
 * from the camera centre.  cams_dev: (device) n_views gs_camera, same sizes
 * and submaps as at creation. */
gs_status gs_project(gs_workspace *ws, const gs_gaussians *g, const gs_camera *cams_dev, void *stream);

/* Binning: one instance per (visible pair, covered tile), ordered by the
 * 64-bit key (global tile id << 32 | float bits of the view depth), ties by
 * (view, Gaussian index); per-tile [start, end) ranges. Stable on-device
 * radix sorts (depth of the visible pairs, then tile id of the instances).
 * A tile of the pair's rectangle is covered iff the box of its pixel centres,
 * grown by ext_abs_pad, meets the ellipse d^T Sigma'^-1 d <= 2 ln(o /
 * alpha_min) (1 + ext_rel_pad)^2; the rectangle's other tiles are emitted
 * with tile id 0xFFFFFFFF, sort after every list and belong to no range
 * (the instance count and capacity cover the whole rectangles). */
gs_status gs_bin_sort(gs_workspace *ws, void *stream);

/* Front-to-back alpha compositing of every tile's list into rgb (device,
 * planar, 3*N_pix), depth (device, N_pix: sum of alpha*T*z, not normalised)
 * and alpha (device, N_pix: 1 - T).  Keeps, per pixel, the number of list
 * entries up to the last blended fragment and the final T for the backward. */
gs_status gs_render_fwd(gs_workspace *ws, float *rgb, float *depth, float *alpha, void *stream);

/* gs_render_fwd that also renders each pixel's depth distribution, the
 * renderer's N(mu_u, sigma_u^2) of Eq. (7) (Sec. III-C): with the blending
 * weights w = alpha T of the pixel's fragments and W = sum w,
 * depth_mean (device, N_pix) = sum w z / W and depth_var (device, N_pix) =
 * sum w (z - mean)^2 / W, both 0 where nothing blends.  They are accumulated
 * front to back by a weighted Welford update in depths relative to the first
 * blended fragment's, so that their rounding scales with the spread of the
 * depths, not with the depth.  alpha is written as W (1 - T in exact
 * arithmetic).  Keeps (mean, var, 1/W) per pixel for gs_render_bwd_var. */
gs_status gs_render_fwd_var(gs_workspace *ws, float *rgb, float *depth, float *alpha, float *depth_mean,
                            float *depth_var, void *stream);

/* LiDAR depth consistency (Eq. 7).  lidar (device, [n_pts][4] float32 rows
 * u, v, z, view): pixel (floor u, floor v) of view `view`; a point is valid if
 * it lies inside the image, z > near_z and alpha > 0 there.  depth_mode 0:
 * mean |D - z|; 1: mean KL(N(z, sigma_L^2) || N(D, sigma_U^2)).  Times
 * lambda_L.  loss (device, 1 float) receives the value; dL_ddepth (device,
 * N_pix, nullable) is accumulated with dL/dD.  Zero valid points give 0. */
gs_status gs_depth_loss(gs_workspace *ws, const float *depth, const float *alpha, const float *lidar,
                        int64_t n_pts, float *loss, float *dL_ddepth, void *stream);

/* Eq. (7) with the rendered distribution: the same valid points (alpha > 0)
 * and lambda_L as gs_depth_loss, mean KL(N(z, sigma_L^2) || N(mu_u,
 * sigma_u^2)) with mu_u = depth_mean and sigma_u^2 = max(depth_var, 0) +
 * sigma_U^2 (sigma_U is the floor of the predicted spread); depth_mode is not
 * used.  alpha, depth_mean, depth_var (device, N_pix) from gs_render_fwd_var;
 * dL_dmean and dL_dvar (device, N_pix, each nullable) are accumulated (a
 * clamped variance passes no gradient). */
gs_status gs_depth_loss_var(gs_workspace *ws, const float *alpha, const float *depth_mean,
                            const float *depth_var, const float *lidar, int64_t n_pts, float *loss,
                            float *dL_dmean, float *dL_dvar, void *stream);

/* L1 photometric term of Eq. (6) (with the SSIM weight lambda = 0):
 * loss = mean |rgb - target| over 3*N_pix values, dL_drgb += sign(rgb -
 * target) / (3*N_pix) (nullable). rgb, target, dL_drgb: (device) planar. */
gs_status gs_image_l1(gs_workspace *ws, const float *rgb, const float *target, float *loss,
                      float *dL_drgb, void *stream);

/* gs_image_l1 with 8-bit target images, as cameras deliver them: target
 * (device, 3*N_pix bytes, planar like rgb) holds values t in 0..255 that
 * stand for t / 255 (rounded as a float32 division rounds it), so that a
 * keyframe uploads a quarter of the float bytes.  Loss and gradient equal
 * gs_image_l1's on the float targets t / 255, bit for bit. */
gs_status gs_image_l1_u8(gs_workspace *ws, const float *rgb, const uint8_t *target, float *loss,
                         float *dL_drgb, void *stream);

/* The photometric loss of Eq. (6) (Sec. III-C):
 * (1 - lambda) mean |rgb - target| + lambda (1 - mean SSIM).  SSIM per channel
 * plane of every view, 11x11 Gaussian window of sigma 1.5 (normalised), zero
 * padding outside the image, C1 = 0.01^2, C2 = 0.03^2 (unit dynamic range),
 * averaged over the 3*N_pix values.  rgb, target, dL_drgb: (device) planar as
 * the renderer's output; loss (device, 3 floats) receives the total, the L1
 * term and 1 - SSIM; dL_drgb (nullable) is accumulated.  lambda in [0, 1]
 * (the paper leaves it open; 3DGS uses 0.2), GS_ERR_INVALID_ARG otherwise. */
gs_status gs_image_loss(gs_workspace *ws, const float *rgb, const float *target, float lambda, float *loss,
                        float *dL_drgb, void *stream);

/* Backward of gs_render_fwd and gs_project: walks each tile's list back to
 * front from the last blended fragment, recomputing alpha, reduces each
 * Gaussian's contributions across the warp before one atomic per component,
 * then chains to the parameters and, through the projection, to each
 * camera's pose twist.  dL_drgb, dL_ddepth (device, planar like the outputs),
 * dL_dalpha (device, nullable).  g and cams_dev must be those of the
 * preceding gs_project.  The image-space gradient rows the backward adds into
 * are cleared by gs_project (next to the records it writes); only a further
 * backward of the same projection launches a clearing kernel of its own.  (A
 * CUDA graph that holds the first backward after a projection but not the
 * projection itself does not clear those rows when it is replayed.) */
gs_status gs_render_bwd(gs_workspace *ws, const gs_gaussians *g, const gs_camera *cams_dev,
                        const float *dL_drgb, const float *dL_ddepth, const float *dL_dalpha,
                        const gs_grads *out, void *stream);

/* gs_render_bwd that also takes the adjoints of the depth mean and variance,
 * dL_dmean and dL_dvar (device, N_pix, each nullable).  The last forward
 * must have been gs_render_fwd_var (GS_ERR_STATE otherwise). */
gs_status gs_render_bwd_var(gs_workspace *ws, const gs_gaussians *g, const gs_camera *cams_dev,
                            const float *dL_drgb, const float *dL_ddepth, const float *dL_dalpha,
                            const float *dL_dmean, const float *dL_dvar, const gs_grads *out,
                            void *stream);

/* Synchronise `stream` and report device-side conditions: returns
 * GS_ERR_TIMEOUT if a bounded device-side wait ran out since the last
 * gs_bin_sort (the outputs of that step are not valid), else GS_ERR_CAPACITY
 * if the last gs_bin_sort needed more instances than the capacity. Any out
 * pointer may be NULL. */
gs_status gs_workspace_status(gs_workspace *ws, void *stream, int64_t *n_instances, int64_t *n_visible);

/* Sizes of the workspace: info[0] n_pairs, [1] n_tiles, [2] n_pix, [3]
 * inst_capacity, [4] n_views, [5] N, [6] bytes of device memory held,
 * [7] kernels this workspace's calls have enqueued so far. */
gs_status gs_workspace_info(gs_workspace *ws, int64_t *info, int32_t n_info);

/* Copy an internal buffer to `dst` (device) for inspection; bytes must equal
 * the buffer size reported through *bytes when dst is NULL.
 * which: 0 records [n_pairs][12] f32, 1 pair depth keys [n_pairs] u32,
 * 2 tile rectangles [n_pairs][4] i16 (records and rectangles are written for
 * the visible pairs only, those whose depth key is not 0xFFFFFFFF; the
 * others hold whatever an earlier projection left), 3 sorted instance tile ids [capacity]
 * u32 (0xFFFFFFFF, last, for a rectangle tile that is not covered), 4 sorted
 * instance pair ids [capacity] u32, 5 tile ranges [n_tiles][2]
 * u32, 6 per-pixel list count up to the last blended fragment [N_pix] u32,
 * 7 per-pixel final T [N_pix] f32, 8 image-space gradients [n_pairs][10] f32,
 * 9 per-pixel depth (mean, var, 1/W, 0) of gs_render_fwd_var [N_pix][4] f32. */
gs_status gs_workspace_copy(gs_workspace *ws, int32_t which, void *dst, int64_t *bytes, void *stream);

/* gs_image_l1 for callers that cannot allocate device memory (the paper has
 * no counterpart).  Some callers may not call cudaMalloc: a hard real-time mapping loop whose
 * memory is fixed at start-up (cudaMalloc can block and synchronise the
 * device), or code embedded in a host program that only hands over its
 * buffers.  This call needs no workspace and allocates nothing: its only
 * scratch is a file-scope device array of GS_IMAGE_L1_NOALLOC_BLOCKS doubles
 * (8 KiB) that every GPU which loads the library holds until exit.
 * rgb, target (device, n floats), loss (device, 1 float) receives
 * mean |rgb - target| (0 when n = 0), dL_drgb (device, n floats, nullable)
 * is accumulated with sign(rgb - target)/n.
 * n beyond GS_IMAGE_L1_NOALLOC_BLOCKS * GS_IMAGE_L1_NOALLOC_CHUNK returns
 * GS_ERR_INVALID_ARG without launching anything.  The first call on a device
 * (made with that device current) resolves the array's address once; make
 * it before any stream capture.  After a device reset (cudaDeviceReset) the
 * next call resolves it again, so that call too belongs outside a capture.
 * All calls share the array: calls whose kernels overlap on the GPU race on
 * it. */
#define GS_IMAGE_L1_NOALLOC_BLOCKS 1024
#define GS_IMAGE_L1_NOALLOC_CHUNK 65536
gs_status gs_image_l1_noalloc(const float *rgb, const float *target, int64_t n, float *loss,
                              float *dL_drgb, void *stream);

/* ------------------------------------------------------------------------ */
/* Map lifecycle and optimiser step (Sec. III-B, "Gaussian Splats Lifecycle */
/* Operations"; the paper names no optimiser, Adam is this library's).       */
/* ------------------------------------------------------------------------ */

/* Mutable Gaussian parameter arrays (device, float32, the layouts of
 * gs_gaussians).  Also used for gradients and optimiser moments. */
typedef struct {
    float *means, *log_scales, *quats, *opacity_logits, *sh;
} gs_param_arrays;

#define GS_LC_PRUNE 1   /* drop splats with o < prune_opacity, s > prune_scale_max or s < prune_scale_min */
#define GS_LC_DENSIFY 2 /* mean image-space gradient > densify_grad: split if s > split_scale, clone if s <= clone_scale */
#define GS_LC_RESET 4   /* prune_opacity < o < reset_opacity and reset_scale_min < s < reset_scale_max: o = reset_opacity */

/* Lifecycle thresholds.  s is the largest axis scale exp(log_scale); o the
 * opacity sigmoid(logit).  Every comparison is made on the stored logit or
 * log-scale against the threshold moved to that domain (float32).  The paper
 * gives prune_opacity 0.01, prune_scale_max 0.3 m, prune_scale_min 5e-5 m;
 * densify_grad (gamma_g), split_scale (kappa), clone_scale (2 s_init),
 * reset_opacity, reset_scale_min/max (s_min, s_max) are left to the caller. */
typedef struct {
    int32_t ops;          /* GS_LC_* bits */
    float prune_opacity, prune_scale_max, prune_scale_min;
    float densify_grad;   /* on the mean of ||dL/d(u,v)|| (pixels) over the counted views */
    float split_scale, clone_scale;
    float split_shrink;   /* children's scales = parent's / split_shrink (1.6) */
    float reset_opacity, reset_scale_min, reset_scale_max;
} gs_lifecycle_params;

typedef struct gs_lifecycle gs_lifecycle;

/* Scratch for up to max_in input splats and max_submaps submaps (allocates). */
gs_status gs_lifecycle_create(int64_t max_in, int32_t max_submaps, gs_lifecycle **out);
void gs_lifecycle_destroy(gs_lifecycle *lc);

/* One lifecycle pass over n_in splats in order.  Per splat: prune drops it;
 * otherwise the opacity reset applies, then densification: a split writes two
 * children mu + R(q) diag(exp(log_scale)) z_k (z_k = split_normals[j][k][0..2],
 * standard-normal samples the caller draws) with log_scale - ln(split_shrink)
 * and the parent's quaternion, opacity and SH; a clone writes the splat and an
 * exact copy after it.  The outputs keep the input order, so each submap stays
 * contiguous: submap_offsets_out (device, n_submaps+1) receives the new
 * partition and n_out (device, 1, nullable) the number of output splats.
 * in_m/in_v/out_m/out_v (all or none): Adam moments, carried for surviving
 * splats and zero for copies and children.  densify_acc/densify_cnt (device,
 * n_in; the gs_grads statistic) and split_normals (device, [n_in][2][3]) are
 * needed with GS_LC_DENSIFY.  submap_offsets_in (device, n_submaps+1).
 * Outputs must not alias inputs.  If the outputs need more than out_capacity
 * rows nothing is written and gs_lifecycle_status returns GS_ERR_CAPACITY. */
gs_status gs_lifecycle_run(gs_lifecycle *lc, const gs_lifecycle_params *p, int32_t sh_degree, int64_t n_in,
                           int32_t n_submaps, const int64_t *submap_offsets_in, const gs_param_arrays *in,
                           const gs_param_arrays *in_m, const gs_param_arrays *in_v, const float *densify_acc,
                           const int32_t *densify_cnt, const float *split_normals, const gs_param_arrays *out,
                           const gs_param_arrays *out_m, const gs_param_arrays *out_v, int64_t out_capacity,
                           int64_t *submap_offsets_out, int64_t *n_out, void *stream);

/* Synchronise `stream`; *n_needed (nullable) = outputs the last run needed;
 * GS_ERR_CAPACITY if they exceeded its capacity. */
gs_status gs_lifecycle_status(gs_lifecycle *lc, void *stream, int64_t *n_needed);

/* Adam step on n splats: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps), with one
 * learning rate per array (means, log_scales, quats, opacity_logits, sh). */
typedef struct {
    float lr[5];
    float beta1, beta2, eps;
    int32_t step; /* 1-based */
} gs_adam_params;
gs_status gs_adam_step(const gs_param_arrays *param, const gs_param_arrays *grad, const gs_param_arrays *m,
                       const gs_param_arrays *v, int64_t n, int32_t sh_degree, const gs_adam_params *p,
                       void *stream);

/* ------------------------------------------------------------------------ */
/* Voxel-hash insertion (Sec. III-B, Eq. 5) and the LRU active set          */
/* ("Memory Management").                                                    */
/* ------------------------------------------------------------------------ */

/* Eq. (5) keys: k = floor(x/v) P1 + floor(y/v) P2 + floor(z/v) P3 in unsigned
 * 64-bit arithmetic (wrap-around), P1..P3 = 73856093, 19349663, 83492791
 * (Teschner et al.; the paper gives none), x/v divided in float32 before the
 * floor; the all-ones key is folded onto its predecessor.  xyz (device,
 * n rows of `stride` floats, x y z first), keys (device, n). */
gs_status gs_voxel_keys(const float *xyz, int64_t n, int32_t stride, float voxel, uint64_t *keys, void *stream);

typedef struct gs_voxel gs_voxel;

/* Scratch for batches of up to max_points points and for LRU selection and
 * partitions of up to max_items splats (allocates). */
gs_status gs_voxel_create(int64_t max_points, int64_t max_items, gs_voxel **out);
void gs_voxel_destroy(gs_voxel *vx);

typedef struct {
    float voxel;   /* v of Eq. (5), metres */
    float s_init;  /* scale of a new splat (isotropic), metres */
    float o_init;  /* opacity of a new splat, (0, 1) */
    int32_t frame; /* written to last_used of the splats the batch touches */
} gs_insert_params;

/* Inserts a batch of fused points (device, [n_points][6]: x y z r g b).
 * Device splats whose key (splat_keys, device, n_splats) equals a point's key
 * get last_used (device, n_splats) = frame; host-resident splats whose key
 * (host_keys, device, n_host) equals a point's key get reload[h] = 1 (0
 * otherwise); every voxel of the batch known to neither creates one splat from
 * its first point in input order: mean = the point, log-scales ln(s_init),
 * quaternion (1,0,0,0), opacity o_init, SH DC = (rgb - 1/2) / Y00, other SH
 * coefficients 0.  New splats are written in point order to new_splats and
 * their keys to new_keys (device, new_capacity rows); *n_new (device,
 * nullable) receives their number.  More than new_capacity writes none of
 * them: gs_voxel_status reports GS_ERR_CAPACITY. */
gs_status gs_voxel_insert(gs_voxel *vx, const gs_insert_params *p, const float *points, int64_t n_points,
                          const uint64_t *splat_keys, int32_t *last_used, int64_t n_splats,
                          const uint64_t *host_keys, int32_t *reload, int64_t n_host, int32_t sh_degree,
                          const gs_param_arrays *new_splats, uint64_t *new_keys, int64_t new_capacity,
                          int64_t *n_new, void *stream);

/* Synchronise; *n_new (nullable) = splats the last insert created or needed. */
gs_status gs_voxel_status(gs_voxel *vx, void *stream, int64_t *n_new);

/* LRU offload selection: with n > tau splats, flags (device, n) = 1 for the
 * n - tau smallest (last_used, index) pairs, 0 for the others. */
gs_status gs_active_select(gs_voxel *vx, const int32_t *last_used, int64_t n, int64_t tau, int32_t *flags,
                           void *stream);

/* Stable partition of n splat rows by flags (device, n): rows with flag 0 go
 * in order to `kept`, rows with flag 1 in order to `moved`, with their keys and
 * last_used (each pair nullable).  Any output may be host memory that the
 * device can address (pinned, mapped): offloading to the CPU store and
 * reloading from it are partitions.  counts (device, 2, nullable) receives
 * (kept, moved). */
gs_status gs_partition(gs_voxel *vx, const int32_t *flags, int64_t n, int32_t sh_degree, const gs_param_arrays *in,
                       const uint64_t *in_keys, const int32_t *in_last_used, const gs_param_arrays *kept,
                       uint64_t *kept_keys, int32_t *kept_last_used, const gs_param_arrays *moved,
                       uint64_t *moved_keys, int32_t *moved_last_used, int64_t *counts, void *stream);

/* Self-test of the bound on device-side waits (the TMA staging of the SSIM
 * kernels waits on an mbarrier for at most a second): one block waits on a
 * barrier that no copy will ever complete for limit_ns (1 .. 2e9), then sets
 * the workspace's time-out flag and writes *result (device int32) = 1.
 * gs_workspace_status then reports GS_ERR_TIMEOUT until the next gs_bin_sort. */
gs_status gs_selftest_wait_timeout(gs_workspace *ws, int64_t limit_ns, int32_t *result, void *stream);

/* Sets count (0..16) device buffers to zero in one launch: ptrs[i] (device)
 * of bytes[i] bytes (host arrays).  For the gradient buffers, which the
 * backward accumulates into. */
gs_status gs_zero_buffers(void *const *ptrs, const int64_t *bytes, int32_t count, void *stream);

/* Optional per-stage timing. With profiling on, each call records CUDA
 * events on its stream around every stage below (do not enable it while
 * capturing a CUDA graph); gs_workspace_stage_ms synchronises on the events
 * and writes the last duration of each stage in milliseconds (-1 if the
 * stage has not run since profiling was enabled). */
enum {
    GS_STAGE_PROJECT = 0,    /* gs_project */
    GS_STAGE_COMPACT = 1,    /* visible-pair compaction */
    GS_STAGE_DEPTH_SORT = 2, /* radix sort of visible pairs by depth */
    GS_STAGE_EMIT = 3,       /* instance counting, capacity check, emission */
    GS_STAGE_TILE_SORT = 4,  /* radix sort of instances by tile */
    GS_STAGE_RANGES = 5,     /* per-tile ranges */
    GS_STAGE_RASTER_FWD = 6, /* forward compositing */
    GS_STAGE_IMAGE_L1 = 7,   /* gs_image_l1 */
    GS_STAGE_DEPTH_LOSS = 8, /* gs_depth_loss */
    GS_STAGE_ZERO_GRAD = 9,  /* clearing the image-space gradients */
    GS_STAGE_RASTER_BWD = 10, /* backward compositing */
    GS_STAGE_PROJECT_BWD = 11, /* projection adjoint and pose reduction */
    GS_STAGE_IMAGE_SSIM = 12, /* SSIM forward and backward of gs_image_loss */
    GS_NUM_STAGES = 13
};
gs_status gs_workspace_set_profiling(gs_workspace *ws, int32_t on);
gs_status gs_workspace_stage_ms(gs_workspace *ws, float *ms, int32_t n);

/* ------------------------------------------------------------------------ */
/* Measurement (the paper times nothing on this path: these calls give the  */
/* rates and counts the benchmark's rooflines are quoted against; neither   */
/* runs inside the mapping step).                                            */
/* ------------------------------------------------------------------------ */

/* Arithmetic-rate probe: blocks x 256 threads each run `iters` rounds of 8
 * independent dependency chains of one instruction: kind 0 FP32 FMA (2
 * FLOP), 1 packed f32x2 FMA (4 FLOP), 2 MUFU ex2.approx, 3 MUFU rcp.approx.
 * The caller times the launch; operations = blocks * 256 * iters * 8.
 * sink (device, 1 float) is written only in a case that never occurs.
 * Enqueued on `stream`; GS_ERR_INVALID_ARG for kind outside 0..3 or
 * blocks, iters < 1. */
gs_status gs_alu_probe(int32_t kind, int32_t blocks, int32_t iters, float *sink, void *stream);

/* Fragment counts of the last forward (call after gs_render_fwd; GS_ERR_STATE
 * before): every pixel's tile list is walked up to the count the forward
 * kept, with the rasterisers' own alpha evaluation, and counts (host, 4
 * int64) receives [0] (pixel, entry) pairs walked, [1] of those blended
 * (alpha >= alpha_min), [2] (tile, entry) pairs walked (the longest count of
 * each tile), [3] (tile, entry) pairs that some pixel of the tile blends.
 * Synchronises `stream`. */
gs_status gs_workspace_fragment_counts(gs_workspace *ws, int64_t *counts, void *stream);

const char *gs_status_string(gs_status s);
/* Text of the last CUDA error seen by this thread's calls ("" if none). */
const char *gs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
