/*
 * gs.h -- C ABI of libgs, a differentiable 3D Gaussian Splatting rasterizer for NVIDIA GB300
 * (sm_103a), forward and backward, with SE(3) pose gradients, batched over many views of many
 * scenes (agents' submaps), plus the fused losses and the in-kernel Adam step of the mapping loop.
 *
 * What it computes.  MAGS-SLAM optimises each agent's Gaussian submap against a sliding window of
 * keyframes through "differentiably rendered RGB and depth" (Sec. III-A, mapping loss Eq. 4) and,
 * after fusion, refines Gaussians together with per-keyframe pose deltas (Sec. III-C, refinement
 * loss Eq. 23).  Keyframe poses are world-to-camera (Sec. III-B, lifting relation Eq. 15); a
 * Gaussian carries a centre, per-axis scale, rotation, opacity and colour, with covariance
 * R diag(s)^2 R^T (Eq. 19).  The paper cites the 3DGS rasterizer for the rendering itself and fixes
 * none of its internals; the readings this library implements are:
 *   - EWA projection with 0.3 px dilation, radius = ceil(3 sqrt(lambda_max)), near-plane cull;
 *   - 16x16 pixel tiles, one 64-bit key (global tile << 32 | float bits of camera depth) per
 *     (view, Gaussian, touched tile), stably sorted (ties: ascending flattened (view, Gaussian));
 *   - per pixel (sample at x + 0.5, y + 0.5), front to back: sigma = 1/2 d^T conic d,
 *     alpha = min(alpha_max, o exp(-sigma)), skip alpha < alpha_min, stop before blending when
 *     T (1 - alpha) < t_min; outputs RGB (+ T_final bg), unnormalised depth, alpha = 1 - T_final;
 *   - culling, binning and every skip / stop decision in FP32 with a fixed operation order and a
 *     library-defined FP32 exponential (Cody-Waite reduction, degree-7 Taylor), so that any other
 *     implementation of the same decision chain takes the same branches bit for bit.
 *
 * Conventions.
 *   - Every function returns int: GS_OK (0) or a negative GS_ERR_* code; no exceptions cross the
 *     ABI.  gs_error_string() names a code.
 *   - Every data pointer is a DEVICE pointer owned by the caller (except where marked "host").
 *     The library allocates no device memory in any call: scratch lives in a caller-allocated
 *     workspace of gs_workspace_size() bytes (256-byte aligned), initialised by gs_workspace_init().
 *   - Every call is ordered on the caller's CUDA stream (`stream`, a cudaStream_t; NULL = the legacy
 *     default stream) and none synchronises the host, except gs_check_status().  The sequence
 *     project -> bin_sort -> render_fwd -> loss -> render_bwd -> pose_grad -> adam contains no host
 *     synchronisation and may be captured in a CUDA graph.
 *   - Data-dependent failures (key capacity exceeded, a bounded wait that timed out) are recorded in
 *     a status block inside the workspace; gs_check_status() synchronises the stream and reports
 *     the first one.  Argument errors are reported immediately and launch nothing.
 *   - Arrays are row-major float32 unless stated.  N = rows of the concatenated Gaussian arrays of
 *     all scenes; V = views; P = number of (view, Gaussian) pairs = sum over views of the Gaussian
 *     count of the view's scene; images are [V, 3, H, W] (planar RGB) and [V, H, W].
 */
#ifndef GS_H_
#define GS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = -1,   /* a pointer, size or parameter is out of range            */
    GS_ERR_CAPACITY = -2,      /* more duplicated keys than key_capacity (required K kept) */
    GS_ERR_TIMEOUT = -3,       /* a bounded device-side wait gave up                      */
    GS_ERR_CUDA = -4,          /* a CUDA launch or runtime call failed                     */
    GS_ERR_DEVICE_FAULT = -5,  /* a device-side consistency check failed                   */
    GS_ERR_TOO_LARGE = -6,     /* input larger than a fixed-size static scratch area holds   */
};

#define GS_MAX_VIEWS 1024

/* Pinhole camera with world-to-camera pose p_c = R p_w + t (R row-major); camera x right,
 * y down, z forward.  Intrinsics in pixels.  64 bytes. */
typedef struct gs_camera {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
} gs_camera;

/* Binning algorithms of gs_bin_sort.  Both produce the same lists bit for bit: every tile's
 * entries ordered by (depth bits, flattened pair index).
 *   GS_SORT_ONESWEEP (default): scan of tiles_touched, keys (tile << 32 | depth bits) in emission
 *     order and the digit histograms of every pass (one kernel), then a stable LSD onesweep radix
 *     sort over all keys (8-bit digits, decoupled look-back).
 *   GS_SORT_TILE_BUCKET: gs_project counts the keys of every tile, a scan of the G counts gives
 *     each tile its slice, emission drops each key into its tile's slice by atomic slot taking
 *     (order inside the slice arbitrary), and each tile's slice is sorted by (depth bits, pair
 *     index) in shared memory (a warp per slice of at most 128 entries, a CTA per longer slice,
 *     slices longer than 4096 entries as sorted runs merged in global memory).  No global sort,
 *     but one atomic per key twice; measured slower than the onesweep path on GB300 except for
 *     small single-view problems. */
enum { GS_SORT_TILE_BUCKET = 0, GS_SORT_ONESWEEP = 1 };

/* Rasterizer constants.  gs_default_params() gives tile 16x16, near 0.2, dilation 0.3,
 * radius_sigmas 3, alpha_max 0.99, alpha_min 1/255 (float division), t_min 1e-4, bg 0,
 * sort_mode GS_SORT_ONESWEEP, batch_records 0.  Supported tiles: 16x16, 16x8, 32x16. */
typedef struct gs_params {
    int32_t tile_w, tile_h;
    float near_plane;
    float dilation;
    float radius_sigmas;
    float alpha_max;
    float alpha_min;
    float t_min;
    float bg[3];
    int32_t sort_mode;                 /* GS_SORT_ONESWEEP or GS_SORT_TILE_BUCKET */
    int32_t batch_records;             /* list entries staged per TMA batch by the compositing kernels:
                                          0 = min(256, tile pixels); else 64, 128 or 256, at most the
                                          tile's pixel count (a tuning knob: results do not change) */
} gs_params;

/* One rendering problem: V views of one or more scenes (agents' submaps) whose Gaussians are
 * concatenated row-wise.  View v renders rows [view_gauss_begin[v], +view_gauss_count[v]).
 * All views share width x height (the agents share one camera model, Sec. VI). */
typedef struct gs_problem {
    int32_t num_views;                 /* V, 1..GS_MAX_VIEWS                          */
    int32_t width, height;             /* image size, pixels                          */
    int32_t visible_capacity;          /* slots for projection records and 2-D gradients in the
                                          workspace; 0 = the pair count (always enough).  A slot is
                                          taken by every (view, Gaussian) pair that the
                                          projection's conservative pre-test cannot reject: its
                                          visible pairs and a few it then finds invisible.  Too
                                          few slots record GS_ERR_CAPACITY and drop the visible
                                          pairs beyond them (K is then counted without their
                                          keys); gs_read_stats reports the slots needed. */
    int64_t num_gaussians;             /* N                                           */
    const int64_t *view_gauss_begin;   /* host [V]                                    */
    const int64_t *view_gauss_count;   /* host [V]                                    */
    const gs_camera *cameras;          /* device [V]                                  */
    int64_t key_capacity;              /* max duplicated keys K the workspace holds   */
    gs_params params;
} gs_problem;

/* Gaussian parameters, device, [N,3] means, [N,3] log-scales (natural log of the per-axis
 * standard deviation), [N,4] quaternions (w,x,y,z; normalised internally), [N] opacities already
 * in (0,1), [N,3] RGB colours. */
typedef struct gs_gaussians {
    const float *means, *log_scales, *quats, *opacities, *colors;
} gs_gaussians;

/* Forward outputs (device): rgb [V,3,H,W], depth [V,H,W] (sum of z alpha T, background 0),
 * alpha [V,H,W] = 1 - T_final, final_T [V,H,W], last_idx [V,H,W] int32 = 1 + position (within
 * the pixel's tile list) of the last blended Gaussian, 0 if none.  final_T and last_idx are what
 * the backward pass needs; rgb, depth, alpha may be NULL. */
typedef struct gs_image {
    float *rgb, *depth, *alpha, *final_T;
    int32_t *last_idx;
} gs_image;

/* Upstream gradients (device): dL/drgb [V,3,H,W], dL/ddepth [V,H,W], dL/dalpha [V,H,W]; NULL = 0. */
typedef struct gs_image_grad {
    const float *d_rgb, *d_depth, *d_alpha;
} gs_image_grad;

/* Gaussian gradients (device), same shapes as gs_gaussians; ACCUMULATED (+=), so the caller
 * zeroes them (or lets gs_adam_step do it) before a backward pass. */
typedef struct gs_grads {
    float *means, *log_scales, *quats, *opacities, *colors;
} gs_grads;

/* Device pointers into an initialised workspace, for inspection and tests.  Sizes: proj [P,12]
 * float (mean_x, mean_y, conic_A, conic_B | conic_C, opacity, depth, radius | r, g, b, sigma_cut);
 * tiles_touched [P] uint32 (counts; inclusive prefix sums after a GS_SORT_ONESWEEP gs_bin_sort);
 * sorted_keys [K] uint64 (tile << 32 | depth bits);
 * sorted_vals [K] uint32 (flattened pair index p = pair_offset[v] + i); tile_ranges [G,2] uint32
 * with G = V * ceil(W/tile_w) * ceil(H/tile_h); grad2d [P,12] float (dL/d mean_x, mean_y,
 * conic A, B, C, opacity, depth, r, g, b, 0, 0); num_keys -> uint32 K. */
typedef struct gs_ws_view {
    float *proj;                       /* [visible_capacity, 12] projection records, by slot */
    uint32_t *tiles_touched;
    uint64_t *sorted_keys;
    uint32_t *sorted_vals;             /* flattened (view, Gaussian) pair indices */
    uint32_t *tile_ranges;
    float *grad2d;                     /* [visible_capacity, 12] 2-D gradients, by slot */
    uint32_t *num_keys;
    int64_t num_pairs;                 /* P */
    int64_t num_tiles;                 /* G */
    int32_t sort_passes;               /* 8-bit LSD passes of the onesweep sort */
    int32_t reserved;
    uint32_t *pair_slot;               /* [P] slot of each visible pair, 0xffffffff if culled */
    int64_t visible_capacity;          /* slots in proj and grad2d */
    uint32_t *claim_count;             /* [32] items in each claim class */
    uint32_t *claim_list;              /* [32, G] the (view, tile) items of each claim class k in
                                          claim_list[k*G .. k*G + claim_count[k]); class k holds
                                          lists of n entries with 2 min(floor(log2 n), 15) + (the
                                          bit below the leading one) = 31 - k.  The compositing
                                          kernels claim class 0 (longest lists) first. */
} gs_ws_view;

/* Statistics of the last calls, read by gs_read_stats (synchronises the stream). */
typedef struct gs_stats {
    int64_t num_keys;                  /* K of the last gs_bin_sort                           */
    int64_t fwd_pairs;                 /* (pixel, list entry) pairs evaluated by the forward
                                          launches since the last gs_bin_sort                 */
    int64_t bwd_pairs;                 /* (pixel, list entry) pairs walked by the backward
                                          launches since the last gs_bin_sort                 */
    int64_t num_visible;               /* slots the last gs_project took: its visible pairs and
                                          the candidates its pre-test kept but its decision
                                          chain culled (also beyond visible_capacity: the
                                          capacity a retry needs)                             */
} gs_stats;

const char *gs_error_string(int code);

/* Library version and the device architecture it was compiled for (e.g. 1030 = sm_103a). */
int gs_version(int *major, int *minor, int *arch);

void gs_default_params(gs_params *out);

/* Workspace bytes for a problem (host only, no CUDA call). */
int gs_workspace_size(const gs_problem *pb, size_t *bytes);

/* Writes the per-view tables into the workspace and clears its status block.  Call once after
 * allocating the workspace and again whenever view_gauss_begin / view_gauss_count change.  The
 * work counters in the status block return to zero at the end of every launch that uses them, so
 * calls need no clearing in between; one workspace serves one stream of calls at a time. */
int gs_workspace_init(const gs_problem *pb, void *ws, void *stream);

/* Fills *out with device pointers into the workspace (host only). */
int gs_workspace_view(const gs_problem *pb, void *ws, gs_ws_view *out);

/* Synchronises `stream`, then returns the first recorded device status (GS_OK,
 * GS_ERR_CAPACITY with *required_keys = K needed, or GS_ERR_TIMEOUT) and clears it.
 * required_keys may be NULL. */
int gs_check_status(const gs_problem *pb, void *ws, void *stream, int64_t *required_keys);

/* Synchronises `stream` and reads the statistics counters. */
int gs_read_stats(const gs_problem *pb, void *ws, void *stream, gs_stats *out);

/* Workspace guard blocks (no counterpart in the paper; a check of the library itself): 256-byte
 * blocks of a fixed byte pattern, written by gs_workspace_init, follow every workspace buffer that
 * kernels index with data (projection records, tile counts, both key and value buffers, the tile
 * ranges and lists, the records in list order, the 2-D gradients, the pose partials, the pair
 * slots, the claim-class lists).  This call
 * synchronises `stream` and returns GS_OK when every block is intact, else GS_ERR_DEVICE_FAULT with
 * *first_bad (may be NULL) = the index of the first changed block in that order. */
int gs_check_guards(const gs_problem *pb, void *ws, void *stream, int32_t *first_bad);

/* 1 in the bounds-checked build of the library (libgs_checked.so, compiled with GS_CHECKED=1):
 * there every index a kernel takes from data (a record's pair index, a key's tile, a tile range,
 * a scatter position, a bilinear tap) is compared with its buffer's length first, and a violation
 * records GS_ERR_DEVICE_FAULT (read by gs_check_status) and skips the access instead of making it.
 * 0 in the release build (libgs.so), where these comparisons are compiled out. */
int32_t gs_checked_build(void);

/* EWA projection of every (view, Gaussian) pair (Eq. 19 covariance form, world-to-camera poses
 * of Eq. 15): camera transform, 2-D conic with dilation, radius, tile rectangle, touched-tile
 * count; writes proj and tiles_touched in the workspace (and, with GS_SORT_TILE_BUCKET, the key
 * count of every tile). */
int gs_project(const gs_problem *pb, const gs_gaussians *g, void *ws, void *stream);

/* Tile binning (params.sort_mode selects the algorithm, see GS_SORT_*): per-tile lists ordered by
 * (depth bits, flattened pair index), their [start, end) ranges, the sorted keys/values and the
 * projection records in list order, and the order in which the compositing kernels claim the
 * (view, tile) work items: longer lists first (no counterpart in the paper: scheduling only, no
 * result depends on it), so that a persistent launch does not end on a long tile claimed last.
 * K > key_capacity records GS_ERR_CAPACITY (keys beyond capacity dropped). */
int gs_bin_sort(const gs_problem *pb, void *ws, void *stream);

/* Front-to-back compositing of every (view, tile) of the problem in one persistent launch.
 * g supplies nothing here but is kept for symmetry (colours were captured by gs_project). */
int gs_render_fwd(const gs_problem *pb, void *ws, const gs_image *out, void *stream);

/* Targets and outputs of the L1 terms of the mapping loss (Eq. 4), as gs_loss_l1 defines them:
 * L = w_rgb mean|rgb - rgb_t| + w_depth mean|depth - depth_t| (sign(0) = 0); d_rgb [V,3,H,W] and
 * d_depth [V,H,W] receive dL/drgb and dL/ddepth, *loss (device double) receives L.  depth_t and
 * d_depth may be NULL when w_depth = 0. */
typedef struct gs_l1_target {
    const float *rgb_t, *depth_t;
    float w_rgb, w_depth;
    float *d_rgb, *d_depth;
    double *loss;
} gs_l1_target;

/* gs_render_fwd with the L1 terms fused into its per-pixel epilogue: the same outputs as
 * gs_render_fwd followed by gs_loss_l1 on its rgb and depth (which may then be NULL in *out),
 * without a second pass over the images.  The loss is summed in a different order than
 * gs_loss_l1 (per warp, then one double atomic per warp). */
int gs_render_fwd_l1(const gs_problem *pb, void *ws, const gs_image *out, const gs_l1_target *l1, void *stream);

/* Adjoint of the compositing, back to front from final_T and last_idx (no per-pixel lists),
 * followed by the projection adjoint: accumulates dL/d(means, log_scales, quats, opacities,
 * colors) into `grads` (+=) and leaves per-view pose partial sums in the workspace.  It is
 * gs_render_bwd_composite followed by gs_project_bwd. */
int gs_render_bwd(const gs_problem *pb, const gs_gaussians *g, void *ws, const gs_image *fwd,
                  const gs_image_grad *dimg, const gs_grads *grads, void *stream);

/* The compositing adjoint alone: the 10 per-(view, Gaussian) 2-D gradients (mean2D, conic,
 * opacity, depth, colour) summed over every pixel into the workspace (they were zeroed for the
 * visible pairs by gs_bin_sort).  dimg: dL/d rgb [V,3,H,W], dL/d depth [V,H,W], dL/d alpha
 * [V,H,W], each may be NULL (zero). */
int gs_render_bwd_composite(const gs_problem *pb, void *ws, const gs_image *fwd, const gs_image_grad *dimg,
                            void *stream);

/* The projection adjoint alone (after gs_render_bwd_composite): chains the 2-D gradients through
 * the projection to the Gaussian parameters, accumulated (+=) into `grads` and summed over the
 * views of each Gaussian, and leaves per-view pose partial sums in the workspace for
 * gs_pose_grad. */
int gs_project_bwd(const gs_problem *pb, const gs_gaussians *g, void *ws, const gs_grads *grads, void *stream);

/* dL/d xi for each view, xi = (rho, phi) the left perturbation T <- Exp(xi) T of the world-to-camera
 * pose at xi = 0 (the per-keyframe pose delta of Sec. III-C): pose_grad [V,6] (rho_x, rho_y, rho_z,
 * phi_x, phi_y, phi_z), overwritten, summed deterministically from the partials of gs_render_bwd. */
int gs_pose_grad(const gs_problem *pb, void *ws, float *pose_grad, void *stream);

/* Photometric + depth L1 terms of the mapping loss (Eq. 4): L = w_rgb mean|rgb - rgb_t| +
 * w_depth mean|depth - depth_t| over `views` views of width x height.  Writes d_rgb [V,3,H,W],
 * d_depth [V,H,W] (d_depth / depth / depth_t may be NULL when w_depth = 0) and writes L to
 * *loss (device double, overwritten).  sign(0) = 0.  1 <= views <= 65535. */
int gs_loss_l1(int32_t views, int32_t width, int32_t height, const float *rgb, const float *rgb_t,
               const float *depth, const float *depth_t, float w_rgb, float w_depth,
               float *d_rgb, float *d_depth, double *loss, void *stream);

/* Normal term of the mapping loss (Eq. 4: lambda_n L_normal, lambda_n = 1e-2 in the paper), the
 * cosine loss between the depth-induced normal N_hat and a given normal prior N_bar:
 * L = weight * (1 / (V H W)) * sum over valid pixels of |1 - N_hat . N_bar|.  P = D r with
 * r = ((x + 0.5 - cx) / fx, (y + 0.5 - cy) / fy, 1); t_x = P(x+1, y) - P(x-1, y),
 * t_y = P(x, y+1) - P(x, y-1); N_hat = (t_y x t_x) / |t_y x t_x| (facing the camera for a surface
 * seen from the front).  Valid: not on the image border, depth positive and finite at the pixel
 * and its four neighbours, |t_y x t_x| > 0.  sign(0) = 0.
 *   depth [V,H,W] (the rendered depth), prior [V,3,H,W] unit normals in each view's camera frame,
 *   cams [V] device cameras (only the intrinsics are read).  ADDS L to *loss (device double) and
 *   dL/d depth to d_depth [V,H,W] (so it follows gs_loss_l1 / gs_render_fwd_l1, which write
 *   them).  One kernel (a warp walks down a strip of 30 columns, the neighbours' terms passed by
 *   warp shuffles and kept in registers), no scratch memory, no synchronisation. */
int gs_loss_normal(int32_t views, int32_t width, int32_t height, const float *depth, const float *prior,
                   const gs_camera *cams, float weight, float *d_depth, double *loss, void *stream);

/* L = w_l1 mean|rgb - rgb_t| + w_ssim (1 - SSIM(rgb, rgb_t)) (Eq. 23's photometric and
 * structural terms): 11x11 Gaussian window, sigma 1.5, zero padding, C1 = 0.01^2, C2 = 0.03^2,
 * mean over views, channels, pixels.  Writes d_rgb and writes L to *loss (overwritten).
 * `scratch` is a device buffer of gs_ssim_scratch_size() bytes, 256-byte aligned. */
size_t gs_ssim_scratch_size(int32_t views, int32_t width, int32_t height);
int gs_loss_l1_ssim(int32_t views, int32_t width, int32_t height, const float *rgb, const float *rgb_t,
                    float w_l1, float w_ssim, float *d_rgb, double *loss, void *scratch, void *stream);

/* The same loss and gradient as gs_loss_l1_ssim, for callers that cannot allocate device memory:
 * for example a tracking / mapping front-end that claims a fixed device-memory budget at start-up
 * and may not grow it afterwards, or a host program whose allocator belongs to another component
 * (cudaMalloc can also stall every stream on the device, which a real-time loop cannot afford).
 * The paper has no counterpart to this entry point; it exists only for such callers.
 *
 * Instead of a caller-provided scratch buffer it uses a fixed area inside the library: a static
 * device array of 256 + 3 * 4 * GS_SSIM_NOALLOC_MAX_PLANE bytes (about 12 MiB) that every GPU which
 * loads libgs keeps until the process exits.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.  The caller still provides rgb, rgb_t, d_rgb and loss as for gs_loss_l1_ssim.
 *  - Limit: width * height <= GS_SSIM_NOALLOC_MAX_PLANE pixels per image plane (any number of
 *    views); larger images are rejected with GS_ERR_TOO_LARGE before anything is launched.
 *  - Set-up: a call made outside stream capture (with its device current) looks up the device
 *    address of the static area, every time, so the address stays right after a device reset
 *    reloads the library's module; a call made during stream capture reuses the address of the
 *    last call outside capture on that device, so make one call on a device before capturing.
 *  - Sharing: every call on a device uses the same area and leaves its last contents there; the
 *    call clears what must start at zero itself.  Calls whose executions overlap on the GPU (on
 *    different streams, or from different host threads) race on the area and give wrong results:
 *    order them on one stream or synchronise between them.
 * The image planes are processed one after another, so it launches 2 kernels per plane plus 2. */
#define GS_SSIM_NOALLOC_MAX_PLANE (1 << 20)
int gs_loss_l1_ssim_noalloc(int32_t views, int32_t width, int32_t height, const float *rgb, const float *rgb_t,
                            float w_l1, float w_ssim, float *d_rgb, double *loss, void *stream);

/* One bias-corrected Adam step over all Gaussian parameters (beta1 0.9, beta2 0.999, eps 1e-15)
 * with per-group learning rates lr[5] = {means, log_scales, quats, opacity_logits, colors}.
 * The opacity group steps logit(o): its gradient is dL/do * o (1 - o), and `opacities` is
 * rewritten as sigmoid(logit).  `step` is a device int32 incremented by the kernel (bias
 * correction uses the incremented value).  Moments m, v hold 14 N floats each, group-major in the
 * parameters' own layout: [N,3] means, [N,3] log_scales, [N,4] quats, [N] logits, [N,3] colors.
 * If zero_grads != 0 the gradients are cleared. */
typedef struct gs_adam_state {
    float *means, *log_scales, *quats, *opacity_logits, *opacities, *colors;
    float *m, *v;
    int32_t *step;
} gs_adam_state;
int gs_adam_step(int64_t n, const gs_adam_state *st, const gs_grads *grads, const float lr[5],
                 int32_t zero_grads, void *stream);

/* gs_adam_step with the isotropy regulariser of the mapping loss (Eq. 4: lambda_s L_iso,
 * L_iso = sum_i sum_axes |s_i - mean(s_i)| over each Gaussian's per-axis scales s = exp(log-scale),
 * lambda_s = 10 in the paper) added to the log-scale gradients inside the same pass.  iso_loss
 * (device double, may be NULL) receives lambda_s L_iso at the pre-step parameters. */
int gs_adam_step_reg(int64_t n, const gs_adam_state *st, const gs_grads *grads, const float lr[5], float iso_weight,
                     int32_t zero_grads, double *iso_loss, void *stream);

/* ---- joint pose-Gaussian refinement after fusion (Sec. III-C) ---- */

/* Mutable Gaussian arrays, same shapes as gs_gaussians. */
typedef struct gs_gaussian_arrays {
    float *means, *log_scales, *quats, *opacities, *colors;
} gs_gaussian_arrays;

/* Refinement loss of Eq. 23 on the exposure-compensated render I~_v = exp(a_v) I^_v + b_v of each
 * view (per-keyframe log-gain and bias, Sec. III-C):
 *   L = w_l1 L1(I~, I) + w_ssim (1 - SSIM(I~, I)) + w_depth L1(D^, D-)
 * (the paper's alpha' = 1.75, lambda = 0.2, beta = 0.25; its normal term needs a monocular normal
 * prior and is not computed).  SSIM as in gs_loss_l1_ssim, on I~.  expo [V,2] = (a_v, b_v).
 * Writes d_rgb = dL/dI^ [V,3,H,W], d_depth = dL/dD^ [V,H,W] (depth, depth_t, d_depth may all be
 * NULL), d_expo = dL/d(a_v, b_v) [V,2] (may be NULL) and L to *loss (double), all overwritten.
 * scratch: gs_refine_scratch_size() bytes, 256-byte aligned. */
size_t gs_refine_scratch_size(int32_t views, int32_t width, int32_t height);
int gs_loss_refine(int32_t views, int32_t width, int32_t height, const float *rgb, const float *rgb_t,
                   const float *depth, const float *depth_t, const float *expo, float w_l1, float w_ssim,
                   float w_depth, float *d_rgb, float *d_depth, float *d_expo, double *loss, void *scratch,
                   void *stream);

/* Pruning of the refined map (Sec. III-C removes Gaussians with opacity below 0.005): copies the
 * Gaussians of `in` with opacity >= threshold, in their original order, to `out` (capacity n rows,
 * must not alias `in`) and writes their number to *kept (device int64).  scratch:
 * gs_prune_scratch_size(n) bytes, 256-byte aligned.  n < 2^30. */
size_t gs_prune_scratch_size(int64_t n);
int gs_prune(int64_t n, const gs_gaussians *in, float threshold, const gs_gaussian_arrays *out, int64_t *kept,
             void *scratch, void *stream);

/* One bias-corrected Adam step (beta1 0.9, beta2 0.999, eps 1e-15) on each view's pose delta and
 * exposure (the per-keyframe delta xi_k and (a_k, b_k) of Sec. III-C): gradients pose_grad [V,6]
 * (from gs_pose_grad) and expo_grad [V,2] (from gs_loss_refine); moments m, v [V,8]; the pose part
 * of the step is applied to the world-to-camera pose as T <- Exp(delta) T (SE(3) exponential),
 * the exposure part is added to expo [V,2].  `step` (device int32) is incremented. */
typedef struct gs_view_adam_state {
    gs_camera *cameras;
    float *expo, *m, *v;
    int32_t *step;
} gs_view_adam_state;
int gs_view_adam_step(int32_t views, const gs_view_adam_state *st, const float *pose_grad, const float *expo_grad,
                      float lr_pose, float lr_expo, void *stream);

/* ---- occupancy-aware fusion of aligned submaps (Sec. III-C, Eqs. 19-22) ---- */

/* Sim(3) correction: rotation as a quaternion (w,x,y,z) (normalised internally), translation t,
 * scale s > 0. */
typedef struct gs_sim3 {
    float q[4];
    float t[3];
    float s;
} gs_sim3;

/* Eq. 19: out = C applied to n Gaussians: mu' = s R mu + t, Sigma' = s^2 R Sigma R^T (rotation
 * q' = q_R (x) q, log-scales + ln s), opacity and colour unchanged.  C is a host pointer; out may
 * alias in. */
int gs_sim3_apply(int64_t n, const gs_gaussians *in, const gs_sim3 *C, const gs_gaussian_arrays *out, void *stream);

/* Voxel sets: open-addressing hash sets of 64-bit voxel keys.  A voxel index is
 * kappa(x) = floor(x / voxel) per axis (FP32 division), packed 21 bits per axis with offset 2^20
 * (indices clamped to [-2^20, 2^20)).  A set occupies gs_voxset_bytes(capacity) bytes of device
 * memory (256-byte aligned); capacity is a power of two >= 2 and should be about twice the number
 * of distinct voxels.  A full table records GS_ERR_CAPACITY, a box or ray beyond the supported
 * extent (64 voxels per axis per Gaussian, 65536 voxels per ray) records GS_ERR_INVALID_ARG; both
 * are read by gs_voxset_status. */
size_t gs_voxset_bytes(int64_t capacity);
int gs_voxset_clear(void *set, int64_t capacity, void *stream);
int gs_voxset_status(void *set, void *stream, int64_t *count, int64_t capacity);

/* Eq. 20: inserts the occupied voxels of n target Gaussians, every voxel of the box
 * [kappa(mu - k s), kappa(mu + k s)] with s = exp(log-scales) per axis. */
int gs_voxset_add_boxes(void *set, int64_t capacity, int64_t n, const float *means, const float *log_scales, float k,
                        float voxel, void *stream);

/* Eq. 21: inserts the free voxels carved by keyframe depth maps: for every stride-th pixel (row and
 * column) of each view with depth d > 0 (camera z, [V,H,W]), every voxel crossed by the segment from
 * the camera centre to the back-projected point, excluding the end point (t in [0, 1)). */
int gs_voxset_add_rays(void *set, int64_t capacity, int32_t views, int32_t width, int32_t height,
                       const gs_camera *cams, const float *depth, int32_t stride, float voxel, void *stream);

/* Eq. 22: keep[i] = 1 iff kappa(means[i]) is in neither set (free_set may be NULL). */
int gs_voxset_keep(int64_t n, const float *means, void *occ, int64_t occ_capacity, void *free_set,
                   int64_t free_capacity, float voxel, uint8_t *keep, void *stream);

/* ---- Anchor-image photometric residuals of the submap pose graph (Sec. III-B, Eq. 12) ----
 *
 * For an inter-agent edge with a source anchor keyframe s and a target anchor keyframe a (images,
 * z-depth maps and world-to-camera cameras given in their own submaps' coordinates) and the two
 * submap corrections C_src, C_tgt (gs_sim3: x -> s R(q) x + t), every anchor pixel u of s (every
 * stride-th row and column) gives three residuals (one per colour channel)
 *   r(u) = I_s(u) - I_a(pi_a(C_tgt^-1 C_src p_s(u))),   p_s(u) = R_s^T (d(u) K_s^-1 [u + 0.5, 1] - t_s),
 * with I_a sampled bilinearly at pi_a - 0.5 (pixel centres at +0.5).  U_e, the in-frame,
 * finite-depth anchor-pixel set, holds the pixels with 0 < d < inf, camera-space depth in the
 * target above near_plane and all four bilinear taps inside the target image; membership and the
 * bilinear cell follow one fixed FP32 operation sequence (deterministic, reproducible).
 * Jacobians are taken w.r.t. left Sim(3) twists xi = (rho, phi, sigma) (translation, rotation,
 * log-scale) of the global frame, C <- Exp(xi) C, for the source (columns 0-6) and target
 * (columns 7-13) corrections.  With Huber weights omega (threshold huber_delta on each scalar
 * residual) and n = |U_e|, each edge returns
 *   cost = (w_e / n) sum rho(r),  H = (w_e / n) sum omega J^T J (14 x 14),  g = (w_e / n) sum omega J^T r,
 * the robust Gauss-Newton blocks of the edge's term of the graph cost (the cost gradient is 2 g);
 * an empty U_e gives zeros. */
typedef struct gs_pho_edge {
    int32_t src_image, tgt_image;      /* anchor keyframes: indices into images/depths/cameras */
    int32_t src_corr, tgt_corr;        /* indices into the correction array */
    float weight;                      /* w_e of the edge */
    float reserved[3];
} gs_pho_edge;

typedef struct gs_pho_params {
    int32_t stride;                    /* anchor pixels on every stride-th row and column, >= 1 */
    float huber_delta;                 /* Huber threshold per scalar residual (default 9/255) */
    float near_plane;                  /* target camera-space depth must exceed this (default 0.2) */
    int32_t reserved;
} gs_pho_params;

gs_pho_params gs_default_pho_params(void);

/* Device scratch for gs_pho_residual (per-block partial sums), in bytes. */
size_t gs_pho_scratch_size(int32_t num_edges);

/* num_edges edges (device array, 32 B each); images [M, 3, H, W] and depths [M, H, W] FP32 planar
 * (device); cameras [M] and corrections [num_corr] device arrays; params a host pointer.
 * Outputs (device): cost [E] double, count [E] int64 (|U_e|, or -1 for an edge whose indices are
 * out of range, whose other outputs are then zero), H [E, 14, 14] double (row-major), g [E, 14]
 * double.  scratch: gs_pho_scratch_size(num_edges) bytes of device memory (any contents).
 * Results are deterministic (fixed reduction order).  GS_ERR_INVALID_ARG for null pointers,
 * stride < 1, num_edges outside [0, 65535], empty images or too small a scratch. */
int gs_pho_residual(int32_t num_edges, const gs_pho_edge *edges, int32_t num_images, int32_t width, int32_t height,
                    const float *images, const float *depths, const gs_camera *cameras, int32_t num_corr,
                    const gs_sim3 *corrections, const gs_pho_params *params, double *cost, int64_t *count,
                    double *H, double *g, void *scratch, size_t scratch_bytes, void *stream);

/* Zeroes the five gradient arrays of n Gaussians (one stream-ordered kernel launch). */
int gs_grads_zero(int64_t n, const gs_grads *grads, void *stream);

/* Number of kernels this library has launched in the calling process since it was loaded
 * (host-side counter; graph replays are not counted). */
int64_t gs_launch_count(void);

/* ---- test hooks (no counterpart in the paper; they exist to check the library itself) ---- */

/* y_spec[i] = the library's FP32 decision-chain exponential of x[i]; y_cuda[i] = CUDA's expf(x[i])
 * (either output may be NULL).  n elements, device arrays. */
int gs_debug_expf(const float *x, float *y_spec, float *y_cuda, int64_t n, void *stream);

/* Bounded-wait check of the decoupled look-back: runs the inclusive scan over n ones in `scratch`
 * (device, gs_debug_scan_scratch_size(n) bytes) with partition `silent_partition` never
 * publishing its count (-1: normal run) and a short spin limit (about a millisecond), then
 * synchronises and returns the recorded status: GS_ERR_TIMEOUT when a successor gave up waiting,
 * GS_OK otherwise.  *total receives the scan total (n on a normal run). */
size_t gs_debug_scan_scratch_size(int64_t n);
int gs_debug_scan_timeout(void *scratch, int64_t n, int32_t silent_partition, void *stream, int64_t *total);


#ifdef __cplusplus
}
#endif
#endif /* GS_H_ */
