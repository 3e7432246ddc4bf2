/* vtsplat: differentiable splatting of view-tied isotropic 3D Gaussians on
 * GB300 (sm_103a).  C ABI.
 *
 * The operations follow VTGaussian-SLAM (arXiv 2506.02741):
 *   - a Gaussian has only a colour c (3), an opacity o and an isotropic
 *     radius r, and is tied to one valid depth pixel of one view; its centre
 *     is that pixel back-projected with the view's pose (Sec. 3.2);
 *   - a section groups the Gaussians of N consecutive views (Sec. 3.2);
 *   - splat(gaussians, pose) renders colour and depth (Eq. 1 text) and the
 *     silhouette used to find uncovered pixels (Sec. 3.4);
 *   - tracking differentiates the render with respect to the camera pose,
 *     mapping with respect to colour, opacity and radius (Sec. 3.3, Eq. 1;
 *     Sec. 3.4, Eq. 2).
 * The splatting definition implemented here (per target pixel (u, v) at
 * normalised position p = ((u-cx)/fx, (v-cy)/fy), Gaussian centre x = (x,y,z)
 * in the target camera):
 *   q = ((p_x z - x)^2 + (p_y z - y)^2) / r^2, ahat = o exp(-q/2),
 *   included iff z_key >= 0.1, q <= 9 and ahat >= 1/255, alpha = min(0.99, ahat),
 *   front to back by (z_key, id), stop before a Gaussian that would make the
 *   transmittance T < 1e-4;  C = sum w c, D = sum w z, S = sum w, w = alpha T.
 * id = (section index, position in the section); z_key = FP32 camera depth
 * of the centre computed with a fixed operation order.
 *
 * Conventions for every entry point:
 *   - Pointers marked "device" are CUDA global memory on the current device,
 *     owned by the caller; the library never frees or keeps them beyond the
 *     call (except that vt_render_backward reads the buffers of the
 *     preceding vt_render on the same context, which must still be alive).
 *   - Structs passed by pointer (vt_section arrays, vt_grads arrays) are host
 *     memory, read during the call only.
 *   - All work is enqueued on `stream` (a cudaStream_t; NULL = legacy
 *     default stream) and is asynchronous; no call synchronises the stream
 *     except vt_ctx_sync_status and the inspection hooks vt_ctx_debug_copy
 *     and vt_ctx_debug_pixel_lists, which say so.
 *   - Poses are camera-to-world 3x4 [R | t] as 12 doubles: R row-major, then t.
 *   - Images are float32, planar: rgb is 3 x H x W (channel-major), depth and
 *     silhouette H x W.
 *   - Errors are returned as vt_status; vt_last_error() gives a message for
 *     the calling thread.  Argument errors are found on the host before any
 *     launch.  A shortage of instance capacity is found on the device: the
 *     call returns VT_OK, the results of that render are undefined, and
 *     vt_ctx_sync_status reports VT_ERR_CAPACITY with the size needed.
 */
#ifndef VTSPLAT_H
#define VTSPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *vt_stream; /* same type as cudaStream_t */
typedef struct CUevent_st *vt_event;   /* same type as cudaEvent_t */

typedef enum {
    VT_OK = 0,
    VT_ERR_INVALID_ARG = 1, /* a size, pointer or value is out of range */
    VT_ERR_OOM = 2,         /* device memory for the workspace could not be allocated */
    VT_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
    VT_ERR_CAPACITY = 4,    /* more tile instances than the workspace holds */
    VT_ERR_TIMEOUT = 5,     /* a bounded wait expired */
    VT_ERR_STATE = 6        /* backward without a matching render */
} vt_status;

typedef struct {
    float fx, fy, cx, cy; /* pinhole intrinsics in pixels */
} vt_intrinsics;

typedef enum {
    VT_F32 = 0, /* colour, opacity, radius stored as float32 */
    VT_F16 = 1  /* stored as IEEE half; all arithmetic stays float32 */
} vt_precision;

/* One section (Sec. 3.2): the Gaussians tied to the valid depth pixels of
 * n_views views of one camera.  Every pointer is device memory. */
typedef struct {
    int32_t n_views, W, H;  /* views share size W x H and intrinsics K */
    vt_intrinsics K;
    const double *poses;    /* n_views x 12 camera-to-world */
    const float *depth;     /* n_views x H x W metres; <= 0 or non-finite = no Gaussian */
    int64_t n;              /* number of Gaussians */
    const uint32_t *src;    /* n: (view*H + v)*W + u, strictly increasing (canonical id order) */
    vt_precision prec;
    const void *colour;     /* n x 3 */
    const void *opacity;    /* n, activated value in (0, 1] */
        const void *radius;     /* n, activated value > 0 (metres, a standard deviation);
                               unused (may be NULL) for ellipsoids */
    /* Ellipsoids (the anisotropic variant of the ablation on the Gaussians'
     * attributes, Sec. 4): with scale != NULL every Gaussian of the section
     * is the ellipsoid R(q) diag(s^2) R(q)^T, expressed in the camera frame
     * of its source view (it moves with that view), and is splatted with
     * the local affine (EWA) projection at its centre:
     *   Sigma_2D = J M R(q) diag(s^2) R(q)^T M^T J^T + 0.3 I (pixels^2),
     *   M = R^T R_k, J = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]],
     *   q = d^T Sigma_2D^-1 d for the pixel offset d from the projected
     *   centre; inclusion, clamp, order and termination as for the spheres. */
    const void *scale;      /* n x 3 standard deviations (metres, > 0) or NULL */
    const void *rot;        /* n x 4 quaternions (w, x, y, z), normalised on use;
                               required with scale */
} vt_section;

/* Per-section gradient buffers (device, accumulated with +=).  A NULL
 * pointer skips that gradient; a section whose attribute pointers are NULL
 * is frozen (only the learnable section gets gradients, Sec. 3.2 / Eq. 2). */
typedef struct {
    float *d_colour;       /* n x 3, float32 */
    float *d_opacity;      /* n, float32 */
    float *d_radius;       /* n, float32 */
    double *d_view_twist;  /* n_views x 6 (VT_GRAD_VIEWS): dL/d(rho, phi) of each source
                              view's pose P_k for the right perturbation P_k Exp(xi) */
    double *d_view_mat;    /* n_views x 12 (VT_GRAD_VIEWS): dL/dR_k (row-major), dL/dt_k */
    float *d_depth;        /* n, float32 (VT_GRAD_VIEWS): dL/dD of each Gaussian's depth,
                              i.e. of its position along its pixel's ray (the movable
                              Gaussians of the supplementary); apply by editing the
                                                            section's depth map at src */
    float *d_scale;        /* n x 3, float32 (ellipsoid sections, VT_GRAD_ATTR) */
    float *d_rot;          /* n x 4, float32 (ellipsoid sections, VT_GRAD_ATTR): with
                              respect to the stored (unnormalised) quaternion */
} vt_grads;

typedef enum {
    VT_GRAD_ATTR = 1,  /* colour, opacity, radius (mapping, Eq. 2) */
    VT_GRAD_POSE = 2,  /* target camera pose (tracking, Eq. 1) */
    VT_GRAD_VIEWS = 4  /* source-view poses through the centres mu = R_k X_c + t_k
                          (head-frame bundle adjustment, Sec. 3.4), and each
                          Gaussian's depth along its ray */
} vt_grad_mode;

/* Opaque render context: the library-owned workspace (projected Gaussians,
 * tile lists, per-pixel state) kept from a render for its backward. */
typedef struct vt_ctx vt_ctx;

/* Create / destroy a context on the current CUDA device.  Destroy frees the
 * workspace after the work queued on the context's last stream. */
vt_status vt_ctx_create(vt_ctx **ctx);
void vt_ctx_destroy(vt_ctx *ctx);

/* Reserve workspace for renders of up to n_gaussians Gaussians into W x H
 * images with up to n_instances (Gaussian, tile) pairs, so that later calls
 * allocate nothing (needed before capturing renders in a CUDA graph).
 * n_instances <= 0 picks 4 * n_gaussians + 65536.  Allocates on `stream`. */
vt_status vt_ctx_reserve(vt_ctx *ctx, int64_t n_gaussians, int32_t W, int32_t H,
                         int64_t n_instances, vt_stream stream);

/* Workspace bytes a reserve of those sizes needs. */
size_t vt_workspace_bytes(int64_t n_gaussians, int32_t W, int32_t H, int64_t n_instances);

/* Synchronises `stream`, then reports the status word of the last render on
 * this context: VT_OK, or VT_ERR_CAPACITY with *needed_instances set to the
 * count that render required (reserve at least that much and render again).
 * needed_instances may be NULL. */
vt_status vt_ctx_sync_status(vt_ctx *ctx, vt_stream stream, int64_t *needed_instances);

/* Back-projection (Sec. 3.2): the world centre mu = R (D K^-1 [u v 1]^T) + t
 * of every valid depth pixel, in raster order.  depth: device H x W;
 * pose12: device; centres: device float32 3 x cap (x,y,z interleaved);
 * pix: device uint32 cap (v*W + u); n_out: device int64, receives the number
 * of valid pixels (entries beyond cap are counted but not written). */
vt_status vt_backproject(const float *depth, int32_t W, int32_t H, vt_intrinsics K,
                         const double *pose12, float *centres, uint32_t *pix, int64_t cap,
                         int64_t *n_out, vt_stream stream);

/* Allocation-free variant of vt_backproject (the paper has no counterpart:
 * this is a deployment aid).  Same arguments, same results.  For callers
 * that cannot let the library allocate device memory: code recorded into a
 * CUDA graph without a memory pool, real-time loops that must not call the
 * CUDA allocator after start-up, hosts that give all device memory to their
 * own allocator.  The scratch it needs (per-block counts and offsets) lives
 * in a fixed 512 KiB array inside the library, present on every GPU that
 * loads it until the process exits; the call allocates nothing.
 *   - Depth maps are limited to W * H <= 2^24 pixels; larger ones return
 *     VT_ERR_INVALID_ARG (use vt_backproject), and both sides to 65535, as
 *     for every entry point.
 *   - A call made while `stream` is not being captured looks up the array's
 *     device address on the current device (with that device current) and
 *     caches it; calls during a stream capture use the cached address, so
 *     make the first call on a device before any stream capture (a call
 *     during capture with nothing cached returns VT_ERR_STATE).  After a
 *     device reset, make one call outside capture again before capturing.
 *   - All calls share the one array: calls that may overlap on the GPU (on
 *     different streams, or from different threads) race and must be
 *     serialised by the caller.  No state carries over from one call to the
 *     next. */
vt_status vt_backproject_noalloc(const float *depth, int32_t W, int32_t H, vt_intrinsics K,
                                 const double *pose12, float *centres, uint32_t *pix,
                                 int64_t cap, int64_t *n_out, vt_stream stream);

/* Section initialisation (Sec. 3.2 and supplementary r = D/f): one Gaussian
 * per valid depth pixel of n_views views, in canonical order, with
 * colour = V(u, v), opacity = 0.9 and radius = D / fx.  depth: device
 * n_views x H x W; rgb: device n_views x 3 x H x W float32 in [0, 1];
 * outputs (device, capacity cap): src, colour (cap x 3), opacity, radius in
 * precision `prec`; n_out (device int64) receives the count. */
vt_status vt_section_init(const float *depth, const float *rgb, int32_t n_views, int32_t W,
                          int32_t H, vt_intrinsics K, vt_precision prec, uint32_t *src,
                          void *colour, void *opacity, void *radius, int64_t cap,
                          int64_t *n_out, vt_stream stream);

/* Complement initialisation of a regular frame (Sec. 3.4: the section is
 * splatted into a silhouette at the frame's pose and Gaussians are
 * initialised where it leaves the frame uncovered): one Gaussian per pixel
 * with valid depth and silhouette < sil_max (0.5 in the paper's setting),
 * colour = V(u, v), opacity 0.9, radius = D / fx, in raster order.  depth,
 * silhouette (H x W) and rgb (3 x H x W): device float32 of the new frame.
 * The frame becomes view number `view` of the section, so src = view * W * H +
 * v * W + u; the caller appends the outputs (device, capacity cap; count to
 * n_out, a device int64) to the section's arrays and the frame's depth and
 * pose to its views.  Allocates stream-ordered scratch of 8 bytes per 256
 * pixels. */
vt_status vt_section_complement(const float *depth, const float *rgb, const float *silhouette,
                                int32_t W, int32_t H, vt_intrinsics K, float sil_max,
                                int32_t view, vt_precision prec, uint32_t *src, void *colour,
                                void *opacity, void *radius, int64_t cap, int64_t *n_out,
                                vt_stream stream);

/* Render sections [secs, secs + n_secs) (their concatenation, as in the
 * multi-section render of Sec. 3.4) from the camera pose12 (device, 12
 * doubles) with intrinsics K into W x H images.  rgb (3 x H x W), depth and
 * silhouette (H x W) are device float32; any of them may be NULL.  The
  * context keeps what vt_render_backward needs.  W and H are at most 65535
 * (VT_ERR_INVALID_ARG beyond).  The sections of one render are either all
 * spheres or all ellipsoids (VT_ERR_INVALID_ARG otherwise). */
vt_status vt_render(vt_ctx *ctx, const vt_section *secs, int32_t n_secs, const double *pose12,
                    vt_intrinsics K, int32_t W, int32_t H, float *rgb, float *depth,
                    float *silhouette, vt_stream stream);

/* Backward of the last vt_render on ctx for L with upstream gradients
 * dL_drgb (3 x H x W), dL_ddepth, dL_dsil (H x W; each device, NULL = 0).
 * mode is a combination of vt_grad_mode bits.
  *   VT_GRAD_ATTR: grads[s] (host array of n_secs entries) receive
 *     dL/dcolour, dL/dopacity, dL/dradius of section s (+=, float32); for
 *     ellipsoids d_scale and d_rot instead of d_radius.
 *   VT_GRAD_VIEWS: grads[s].d_view_twist / d_view_mat (device doubles, +=)
 *     receive the gradients with respect to the poses of section s's source
 *     views (sections with both NULL are skipped): per Gaussian dL/dx of its
 *     centre (float32 accumulation), then per view FP64 sums
 *     dL/dR_k = R sum g X_c^T, dL/dt_k = R sum g, dL/drho_k = R_k^T R sum g,
 *     dL/dphi_k = sum X_c x (R_k^T R g), X_c = D ((u-cx)/fx, (v-cy)/fy, 1);
 *     grads[s].d_depth (device float32, +=, may be NULL) receives
 *     dL/dD = (R g) . (R_k X_c / D) per Gaussian.
 *   VT_GRAD_POSE: d_twist (device, 6 doubles) += dL/d(rho, phi) for the
 *     right perturbation P exp(xi), xi = (rho, phi); d_mat (device, 12
 *     doubles) += dL/dR (row-major) and dL/dt.  The pose sums are reduced in
  *     FP64 in a fixed order (bit-reproducible).  For ellipsoids the pose
 *     gradient also runs through the covariance: dL/dR adds
 *     R Sigma_c (G + G^T) per Gaussian, G = dL/dSigma_c.
 * For ellipsoids the per-pair terms are accumulated per Gaussian (float32
 * atomics) and a per-Gaussian pass chains them to the scale, the quaternion
 * and the pose; VT_GRAD_VIEWS is not available for them (VT_ERR_INVALID_ARG).
 * The included sets and their order are those of the render (piecewise
 * constant).  Returns VT_ERR_STATE when ctx holds no render. */
vt_status vt_render_backward(vt_ctx *ctx, const float *dL_drgb, const float *dL_ddepth,
                             const float *dL_dsil, int32_t mode, const vt_grads *grads,
                             double *d_twist, double *d_mat, vt_stream stream);

/* ---- Loss inputs: visibility check (Sec. 3.3) and the masked L1 terms of
 * Eq. 1 (tracking) and Eq. 2 (mapping). ---------------------------------- */

/* One view of a section for the visibility check. */
typedef struct {
    const float *depth;       /* device, H x W metres; <= 0 or non-finite = invalid */
    int32_t W, H;
    vt_intrinsics K;
    const double *pose12;     /* device, 12 doubles, camera-to-world */
} vt_view;

#define VT_MAX_VIS_VIEWS 8

/* Visibility check (Sec. 3.3): visible[p] (device uint8, H x W) = 1 iff the
 * valid depth pixel p of `depth` (device, H x W), back-projected with
 * intrinsics K and pose12 (device), lands in front of and inside one of
 * views[0, n_views) (host array, 1 <= n_views <= VT_MAX_VIS_VIEWS) at a depth
 * within rel_tol (the paper's 1%: 0.01) of that view's depth map bilinearly
 * interpolated at the projection (all four neighbours valid); else 0.  The
 * paper takes the union over a section's head, middle and last frames.
 * Pixels sit at integer coordinates.  The arithmetic is FP64 in a fixed
 * order without contraction, so the decisions equal those of a plain FP64
 * evaluation of the same formula. */
vt_status vt_visibility(const float *depth, int32_t W, int32_t H, vt_intrinsics K,
                        const double *pose12, const vt_view *views, int32_t n_views,
                        double rel_tol, uint8_t *visible, vt_stream stream);

/* Overlap-section selection (Sec. 3.3): the head frame's depth (device,
 * H x W), back-projected with its initial pose12 (device), checked against
 * each view of views[0, n_views) separately with the test of vt_visibility;
 * counts[k] (device uint32, overwritten) = number of valid pixels visible to
 * view k; *n_valid (device uint32, overwritten, may be NULL) = number of valid
 * pixels.  The paper keeps the candidate views (every N1 = 5th frame) whose
 * visible fraction exceeds gamma (0.24-0.26). */
vt_status vt_visibility_counts(const float *depth, int32_t W, int32_t H, vt_intrinsics K,
                               const double *pose12, const vt_view *views, int32_t n_views,
                               double rel_tol, uint32_t *counts, uint32_t *n_valid,
                               vt_stream stream);

/* Weights and masks of the masked L1 loss. */
typedef struct {
    double w_rgb;             /* alpha of Eq. 1, rho of Eq. 2 */
    double w_depth;           /* beta of Eq. 1, sigma of Eq. 2 */
    float sil_min;            /* covered iff silhouette > sil_min; < 0: no coverage mask */
    int32_t rgb_needs_depth;  /* 1: the colour term is also masked by valid observed depth */
} vt_l1_weights;

/* Masked L1 loss and its image gradient, P = W H:
 *   L = w_rgb / (3P) sum_{p,c} m_c(p) |rgb - obs_rgb| + w_depth / P sum_p m_d(p) |depth - obs_depth|
 *   m_d = valid observed depth AND covered AND visible,
 *   m_c = covered AND visible [AND valid observed depth if rgb_needs_depth],
 *   covered = silhouette > sil_min (always when sil_min < 0; silhouette may
 *   then be NULL), visible = visible[p] != 0 (always when visible is NULL).
 * Eq. 1: (alpha, beta, 0.99, 1) with the visibility mask of vt_visibility;
 * Eq. 2 L1 terms: (rho, sigma, -1, 0).  All images are device float32
 * (rgb 3 x H x W, the others H x W).  d_rgb and d_depth (device float32, may
 * be NULL) are overwritten with dL/drgb = w_rgb / (3P) m_c sign(rgb -
 * obs_rgb) and dL/ddepth = w_depth / P m_d sign(depth - obs_depth), sign(0)
 * = 0; loss (device, one double, may be NULL) receives L, summed in FP64 in a
 * fixed order.  ctx provides scratch only (its last render is untouched);
 * size it with vt_ctx_reserve before capturing a graph. */
vt_status vt_masked_l1(vt_ctx *ctx, int32_t W, int32_t H, const float *rgb, const float *depth,
                       const float *silhouette, const float *obs_rgb, const float *obs_depth,
                       const uint8_t *visible, vt_l1_weights w, float *d_rgb, float *d_depth,
                       double *loss, vt_stream stream);

/* ---- Batched work items ----------------------------------------------------
 * Many independent requests processed together, for serving: each item
 * renders one section from its own camera (vt_render of that section alone)
 * and a tracking item adds the Eq. 1 masked L1 loss against its observation
 * and the gradient with respect to its camera pose (vt_masked_l1 and
 * vt_render_backward with VT_GRAD_POSE).  Every stage -- view set-up,
 * projection, tile binning, the per-tile sorts, compositing, the loss, the
 * pose backward and the final sums -- runs as one launch over the
 * Gaussians, tiles or pixels of all items (item ranges concatenated), so a
 * batch costs the same ~15 launches whatever its size.  The items are read
 * on the device from a work-item table that vt_batch_set writes into pinned
 * host memory and vt_batch_launch uploads first; the launch sequence can
 * therefore be captured once in a CUDA graph and replayed for every later
 * batch of the context.  The paper describes no serving system: this
 * follows the serving pattern of the benchmark spec.  Per item the results
 * equal those of the single-render calls, except that the loss and the pose
 * sums are reduced in another fixed order.  A context reserved for batches
 * keeps no single render: a batch launch invalidates vt_render state. */

#define VT_MAX_BATCH_ITEMS 64

typedef struct {
    int32_t section;        /* index into the section array of vt_batch_set (spheres only) */
    int32_t track;          /* 0: render (forward only); 1: tracking iteration */
    int32_t W, H;           /* image size, each <= 65535 */
    vt_intrinsics K;
    const double *pose12;   /* device, 12 doubles, camera-to-world */
    float *image;           /* device, 5 x H x W float32, written: rgb planes, depth,
                               silhouette */
    const float *obs;       /* device, 4 x H x W float32 (track): observed rgb planes and
                               depth (<= 0 or non-finite = no depth) */
    double *result;         /* device, 19 doubles (track), overwritten: the loss, dL/dtwist
                               (rho, phi), dL/dR (row-major), dL/dt */
} vt_batch_item;

/* Device bytes a batch reserve of these capacities takes (see vt_batch_reserve),
 * with per-pixel lists of list_cap entries. */
size_t vt_batch_workspace_bytes(int64_t max_gaussians, int64_t max_pixels, int64_t max_tiles,
                                int64_t max_instances, int64_t max_views, int64_t max_table_rows,
                                int32_t list_cap);

/* Reserve ctx for batches whose totals over the items stay within
 * max_gaussians (section sizes), max_pixels (W H), max_tiles (16 x 16 tiles),
 * max_instances ((Gaussian, tile) pairs), max_views (source views) and
 * max_table_rows (views x (W + H) of the sections' view sizes).  Per-pixel
 * lists of the context's list capacity are kept for the tracking items'
 * backward when they fit the workspace budget (else their tiles are
 * replayed).  Allocates on stream; call before capturing a launch. */
vt_status vt_batch_reserve(vt_ctx *ctx, int64_t max_gaussians, int64_t max_pixels,
                           int64_t max_tiles, int64_t max_instances, int64_t max_views,
                           int64_t max_table_rows, vt_stream stream);

/* Stage a batch (host only, no launch): validates the sections (device
 * pointers, as for vt_render; host array, n_secs in [1, 64]) and items (host
 * array, n_items in [1, VT_MAX_BATCH_ITEMS]) and writes the work-item table
 * into the context's pinned staging.  w: the Eq. 1 weights and masks of the
 * tracking items (vt_masked_l1; visibility is not used).  Returns
 * VT_ERR_CAPACITY, staging nothing, when the batch exceeds the reserved
 * totals (the instance count is checked on the device: see
 * vt_ctx_sync_status).  Waits for the upload of the previous eager launch
 * of ctx; when launches are replayed from a captured graph, stage the next
 * batch only after the previous replay has completed. */
vt_status vt_batch_set(vt_ctx *ctx, const vt_section *secs, int32_t n_secs,
                       const vt_batch_item *items, int32_t n_items, vt_l1_weights w);

/* Enqueue on stream the upload of the staged table and the batch's
 * launches.  obs_ready (may be NULL): an event the tracking items'
 * observations are complete at (e.g. recorded after their uploads on a copy
 * stream); the stream waits for it only before the loss stage, so the
 * uploads overlap the render stages.  Pass NULL when capturing.  Outside a stream capture the grids are sized to the staged
 * batch (one block per unit of work, so that concurrent batches on streams
 * of different priority share the SMs block by block); inside a capture
 * they are persistent grids sized by the SM count that read the work from
 * the uploaded table, so the captured graph serves every later batch.  Results are in the items' image and result
 * buffers when the stream reaches that point; vt_ctx_sync_status reports
 * VT_ERR_CAPACITY if the batch had more tile instances than reserved (its
 * results are then undefined). */
vt_status vt_batch_launch(vt_ctx *ctx, vt_stream stream, vt_event obs_ready);

/* SSIM term of Eq. 2 (Sec. 3.4 mapping loss: tau L_S(V, V'), L_S the SSIM
 * loss; tau = 0.2 in Sec. 4).  L_S = 1 - mean SSIM over the pixels and the
 * three channels of rgb (rendered) against obs_rgb (observed), both device
 * float32 3 x H x W; SSIM per channel with an 11 x 11 Gaussian window
 * (sigma 1.5, weights normalised to 1, zero padding) and C1 = 0.01^2,
 * C2 = 0.03^2.  loss (device, one double, may be NULL) is overwritten with
 * weight * L_S (FP64 sum in a fixed order); d_rgb (device float32
 * 3 x H x W, may be NULL) is ACCUMULATED (+=) with weight * dL_S/drgb, so it
 * adds to the gradient vt_masked_l1 wrote.  ctx holds the scratch (60 bytes
 * per pixel), allocated on the first call of a size: call once before
 * capturing a graph. */
vt_status vt_ssim(vt_ctx *ctx, int32_t W, int32_t H, const float *rgb, const float *obs_rgb,
                  double weight, float *d_rgb, double *loss, vt_stream stream);

/* One Adam step on the camera pose (Sec. 3.3 tracking optimises the pose of
 * the latest frame; the supplementary gives Adam learning rates lr_rot and
 * lr_trans).  With the twist gradient g = d_twist (device, 6 doubles, as
 * accumulated by vt_render_backward) and state (device, 15 doubles: m[6],
 * v[6], step count t, b1^t, b2^t; zero-initialised, zero again to restart):
 *   t += 1, m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 *   s = lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
 *   pose12 (device) <- pose12 Exp(-s)  (right perturbation, xi = (rho, phi)),
 * and d_twist is zeroed for the next backward.  lr (host, 6 doubles) holds
 * the rates for rho (translation) then phi (rotation).  FP64, one thread.
 * ctx may be NULL; when given it only records the launch (vt_ctx_timing,
 * vt_ctx_launch_count). */
vt_status vt_pose_adam(vt_ctx *ctx, double *pose12, double *d_twist, double *state,
                       const double *lr, double beta1, double beta2, double eps,
                       vt_stream stream);

/* Adam hyper-parameters of the mapping step: learning rates of the five
 * parameter planes (c0, c1, c2, logit o, log r; the supplementary gives
 * colour 0.0025, opacity 0.05, radius 0.005) and the moment decays. */
typedef struct {
    float lr[5];
    float beta1, beta2, eps;
} vt_adam_params;

/* One Adam step on the attributes of the n Gaussians of a section being
 * mapped (Sec. 3.4 learns colour, opacity and radius), taken on FP32
 * parameters theta = (c0, c1, c2, logit o, log r) (a reading: the paper
 * gives the rates, not the parametrisation):
 *   g = (dL/dc, dL/do o (1 - o), dL/dr r)     (chain rule at the current theta)
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   theta -= lr m / (1 - b1^t) / (sqrt(v) / sqrt(1 - b2^t) + eps),
 * then the activated values (c, sigmoid, exp) are written to the section's
 * storage colour (n x 3), opacity, radius in precision prec, and the
 * gradients d_colour (n x 3), d_opacity, d_radius (device float32, as
 * accumulated by vt_render_backward) are zeroed.  theta, m, v: device
 * float32, 5 planes of n (plane k = parameter k of every Gaussian); m and v
 * start at zero.  step: device, 3 doubles, zero-initialised: the step count
 * t (incremented here) and the two bias corrections.  ctx may be NULL; when
 * given it only records the launches. */
vt_status vt_attr_adam(vt_ctx *ctx, int64_t n, float *theta, float *m, float *v, double *step,
                       float *d_colour, float *d_opacity, float *d_radius, vt_precision prec,
                       void *colour, void *opacity, void *radius, vt_adam_params p,
                       vt_stream stream);

/* Optimiser state of the mapping step (vt_attr_adam) from a section's
 * storage: theta (device float32, 5 planes of n) = (c0, c1, c2, logit o,
 * log r) with o clamped to [1e-4, 1 - 1e-4] first (o = 1 has no finite
 * logit); m and v (5 planes) zeroed; step (device, 3 doubles) zeroed.  With
 * scale != NULL (ellipsoid section) the state of vt_shape_adam instead:
 * theta = (log s0, log s1, log s2, q0, q1, q2, q3), m and v 7 planes of n.
 * colour, opacity, radius, scale, rot: device arrays of the section in
 * precision prec (radius unused with scale; colour and opacity unused with
 * scale).  This is the parametrisation of the design's optimiser reading
 * (the paper gives the rates, not the parametrisation).  ctx may be NULL;
 * when given it only records the launch. */
vt_status vt_adam_init(vt_ctx *ctx, int64_t n, vt_precision prec, const void *colour,
                       const void *opacity, const void *radius, const void *scale,
                       const void *rot, float *theta, float *m, float *v, double *step,
                       vt_stream stream);

/* Ellipsoid shape step of the mapping optimiser (the anisotropic variant of
 * the attribute ablation, Sec. 4): Adam on theta = (log s0, log s1, log s2,
 * q0, q1, q2, q3) with rate lr_scale for the log scales and lr_rot for the
 * quaternion components (the 3D Gaussian splatting convention; the
 * quaternion is stored unnormalised and normalised where it is used):
 *   g = (dL/ds s, dL/dq),  m, v and the bias corrections as vt_attr_adam,
 * then scale = exp(log s) (n x 3) and rot = q (n x 4) are written in
 * precision prec and d_scale (n x 3), d_rot (n x 4) (device float32, as
 * accumulated by vt_render_backward) are zeroed.  theta, m, v: device
 * float32, 7 planes of n; step: device, 3 doubles (its own counter,
 * incremented here).  ctx may be NULL; when given it only records the
 * launches. */
typedef struct {
    float lr_scale, lr_rot, beta1, beta2, eps;
} vt_shape_adam_params;

vt_status vt_shape_adam(vt_ctx *ctx, int64_t n, float *theta, float *m, float *v, double *step,
                        float *d_scale, float *d_rot, vt_precision prec, void *scale, void *rot,
                        vt_shape_adam_params p, vt_stream stream);

/* Per-kernel timing of the context's launches with CUDA events on the
 * launching stream (enable != 0).  vt_ctx_timing synchronises the stream
 * and writes, for up to n_max kernels, their names (static strings), the
 * number of launches and the summed milliseconds since the last reset;
 * returns the number of kernels. */
vt_status vt_ctx_set_timing(vt_ctx *ctx, int32_t enable);
int32_t vt_ctx_timing(vt_ctx *ctx, vt_stream stream, const char **names, int64_t *launches,
                      double *ms, int32_t n_max, int32_t reset);

/* Number of kernels launched by the library on this context since it was
 * created (host-side counter). */
int64_t vt_ctx_launch_count(const vt_ctx *ctx);

/* Per-pixel lists.  By default every render keeps, for each pixel, the ids
 * of the first `cap` Gaussians it added and the transmittance in front of
 * each (8 * cap bytes per pixel, cap = 256),
 * so that the backward walks each pixel's own Gaussians; pixels that add
 * more, and renders where the lists do not fit the workspace budget, fall
 * back to replaying the tile lists (same results).  cap = 0 never keeps
 * lists.  Takes effect at the next vt_render. */
vt_status vt_ctx_set_list_capacity(vt_ctx *ctx, int32_t cap);

/* Upper bound in bytes on the context's workspace; 0 = unbounded.  When the
 * per-pixel lists of a render would exceed it, that render keeps none. */
vt_status vt_ctx_set_workspace_budget(vt_ctx *ctx, size_t bytes);

/* Device bytes the context currently holds. */
size_t vt_ctx_workspace_bytes(const vt_ctx *ctx);

/* 1 if the last render on ctx kept per-pixel lists, else 0. */
int32_t vt_ctx_used_lists(const vt_ctx *ctx);

/* Test and inspection hook: synchronises `stream` and copies an internal
 * array of the last render to host memory dst (bytes <= capacity).
 * what: 0 = depth keys (float32 x n, 0 for culled), 1 = tile offsets
 * (uint32 x tiles+1), 2 = sorted tile lists (uint32 x instances, Gaussian
 * ids), 3 = per-pixel list end (uint32 x H*W, relative to the tile start),
 * 4 = per-pixel count of added Gaussians (uint32 x H*W), 5 = per-pixel final
 * transmittance (float32 x H*W).  Returns the number of bytes copied, or a
 * negative vt_status. */
int64_t vt_ctx_debug_copy(vt_ctx *ctx, int32_t what, void *dst, int64_t capacity,
                          vt_stream stream);

/* Test and inspection hook: synchronises `stream` and copies the per-pixel
 * lists the last render on ctx kept (vt_ctx_set_list_capacity) for the
 * pixels of the rectangle [x0, x0 + w) x [y0, y0 + h) to host memory, pixels
 * row-major: counts[y * w + x] (host uint32, w * h) = the number of Gaussians
 * the pixel added; ids[(y * w + x) * cap + j] (host uint32, w * h * cap) =
 * the id (section index and position, as the concatenation of the render's
 * sections) of its j-th added Gaussian front to back and T_front (host
 * float32, same layout, may be NULL) the transmittance in front of it, for
 * j < min(count, cap, kept); other entries are left untouched.  *kept (may
 * be NULL) receives the context's list capacity: a pixel whose count
 * exceeds it has only its first `kept` entries recorded.  Returns
 * VT_ERR_STATE when the last render kept no lists, VT_ERR_INVALID_ARG for a
 * rectangle outside the image.  (Used by the tests to compare each pixel's
 * decisions with the oracle's.) */
vt_status vt_ctx_debug_pixel_lists(vt_ctx *ctx, int32_t x0, int32_t y0, int32_t w, int32_t h,
                                   int32_t cap, uint32_t *ids, float *T_front, uint32_t *counts,
                                   int32_t *kept, vt_stream stream);

/* Message of the last error on the calling thread ("" if none). */
const char *vt_last_error(void);

/* Library version string. */
const char *vt_version(void);

#ifdef __cplusplus
}
#endif
#endif
