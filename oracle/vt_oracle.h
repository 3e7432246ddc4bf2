/* Plain FP64 CPU oracle of view-tied isotropic Gaussian splatting.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load or call this library.  It shares
 * no code with the CUDA path.
 *
 * What it computes (paper Sec. 3.2, Eq. 1 text, supplementary Eq. for r):
 * every Gaussian is tied to one valid depth pixel of a source view and has a
 * colour c, an opacity o and an isotropic radius r (a standard deviation in
 * metres).  Its centre is the back-projection of that depth pixel with the
 * source view's pose.  A target camera (pose, intrinsics, W x H) is rendered
 * per pixel by front-to-back alpha compositing with
 *     q     = ((px*z - x)^2 + (py*z - y)^2) / r^2     (isotropic footprint)
 *     ahat  = o * exp(-q/2),  included iff q <= 9 and ahat >= 1/255
 *     alpha = min(0.99, ahat),
 * ordered by (z_key, id) and stopped before the Gaussian whose inclusion
 * would drop the transmittance below 1e-4.  Outputs: colour, depth
 * (sum w*z) and silhouette (sum w).  Thresholds are the FP32 constants the
 * kernels compare against (1.0f/255.0f, 0.99f, 1e-4f, z_near 0.1f).
 */
#ifndef VT_ORACLE_H
#define VT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t n_views, W, H;
    float fx, fy, cx, cy;        /* source-view intrinsics (shared by the section) */
    const double *poses;         /* n_views x 12: R row-major (camera-to-world), then t */
    const float *depth;          /* n_views x H x W, metres; <=0 or non-finite = invalid */
    int64_t n;                   /* number of Gaussians */
    const uint32_t *src;         /* n: (view*H + v)*W + u, strictly increasing */
    const double *colour;        /* n x 3 */
    const double *opacity;       /* n */
    const double *radius;        /* n */
} orc_section;

typedef struct {
    double pose[12];             /* target camera-to-world: R row-major then t */
    float fx, fy, cx, cy;
    int32_t W, H;
} orc_camera;

typedef struct {
    double *rgb;                 /* 3 x H x W */
    double *depth;               /* H x W */
    double *sil;                 /* H x W */
    double *T_final;             /* H x W */
    int32_t *n_added;            /* H x W */
    double *margin;              /* H x W: smallest relative distance of an inclusion test
                                    (q <= 9, ahat >= 1/255) to its threshold */
    double *margin_T;            /* H x W: same for the termination test T' < 1e-4 */
    double *margin_clamp;        /* H x W: same for the clamp ahat vs 0.99 (gradient only) */
    int64_t *lists;              /* H x W x list_cap ids added front to back, -1 padded (may be NULL) */
    int32_t list_cap;
} orc_image;

typedef struct {
    const double *g_rgb;         /* 3 x H x W (NULL = 0) */
    const double *g_depth;       /* H x W (NULL = 0) */
    const double *g_sil;         /* H x W (NULL = 0) */
} orc_upstream;

typedef struct {
    double **d_colour;           /* per section, n x 3 (entries may be NULL) */
    double **d_opacity;          /* per section, n */
    double **d_radius;           /* per section, n */
    double **a_colour;           /* optional, per section n x 3: sum over pixels of the
                                    componentwise magnitude of each term (|gC w| for colour) */
    double **a_opacity;          /* optional: the same for opacity (sum of |products| of the
                                    dL/dalpha formula times dalpha/do) */
    double **a_radius;           /* optional: the same for radius */
    double **d_x;                /* optional, per section n x 3: dL/dx of each Gaussian's
                                    centre in the target camera frame (summed over pixels);
                                    the source-view pose gradients follow from it */
    double **a_x;                /* optional, per section n x 3: componentwise magnitude of
                                    the terms of d_x (as a_colour for colour) */
    double twist[6];             /* dL/d(rho, phi) for P(xi) = P * Exp(xi) */
    double mat[12];              /* dL/dR (row-major 3x3) then dL/dt */
    double twist_noise[6];       /* sqrt(sum over pixels of n_p m_p^2), n_p the pixel's added
                                    Gaussians and m_p the componentwise magnitude of its
                                    contribution to the component: the scale of the rounding
                                    noise of an evaluation that sums each pixel's terms in a
                                    short float format and the pixels in a long one */
    double mat_noise[12];        /* the same for mat */
} orc_grads;

void orc_set_threads(int n);
int orc_get_threads(void);

/* FP32 depth keys of every Gaussian for the target pose; valid[i]=0 marks a
 * Gaussian with invalid depth or z_key < 0.1f. */
void orc_zkeys(const orc_section *sec, const orc_camera *cam, float *zkey, uint8_t *valid);

/* Render; binned = 0 evaluates every Gaussian at every pixel (brute force),
 * binned = 1 takes candidates from 16x16 pixel bins of conservative disc
 * boxes.  Returns 0 on success. */
int orc_render(const orc_section *secs, int n_secs, const orc_camera *cam, int binned,
               orc_image *out);

/* Gradients of L = <g_rgb, rgb> + <g_depth, depth> + <g_sil, sil>; the
 * included sets and their order are held fixed.  Accumulates (+=) into the
 * per-Gaussian arrays; twist and mat are overwritten. */
int orc_backward(const orc_section *secs, int n_secs, const orc_camera *cam, int binned,
                 const orc_upstream *up, orc_grads *g);

/* ---- compositing along given decisions -------------------------------- */

/* Per-pixel lists of added Gaussians, front to back, as another
 * implementation of the method reports them: ids[(v*W + u)*cap + j] for
 * j < count[v*W + u]; ids are positions in the concatenation of the
 * sections (the ids of orc_image.lists). */
typedef struct {
    const int64_t *ids;
    const int32_t *count;
    int32_t cap;
} orc_lists;

/* Verdict on each pixel's list. */
typedef struct {
    int32_t *status;      /* H x W: 0 = the definition's list, up to decisions that lie within
                             the given relative margins of their thresholds; 1 = no list of
                             the definition at all (keys not strictly increasing, an id out of
                             range, culled or outside the pixel's band q <= 9.009); 2 = a
                             decision differs from its FP64 outcome by more than the margins */
    int32_t *flips;       /* H x W: decisions taken otherwise than in FP64 */
    double *flip_margin;  /* H x W: largest relative margin among them (0 if none) */
} orc_verdict;

/* Where an inclusion test (q <= 9, ahat >= 1/255) or the termination test
 * (T' < 1e-4) lies within the rounding of a lower precision of its
 * threshold, both outcomes are correct results.  For every pixel this
 * checks that the given list differs from the FP64 decisions only at
 * decisions within tau_incl (inclusion, relative) or tau_T (termination,
 * relative) of their thresholds -- before the list's last entry every
 * candidate is added or excluded, after it the walk stops at a candidate
 * whose inclusion ends it, or excludes it -- and composites along the given
 * list in FP64: rgb, depth, sil, T_final and n_added (= count) of out;
 * the margin fields of out are not written.  Always binned.  Returns 0. */
int orc_render_lists(const orc_section *secs, int n_secs, const orc_camera *cam,
                     const orc_lists *L, double tau_incl, double tau_T, orc_image *out,
                     orc_verdict *vd);

/* orc_backward with each pixel's added Gaussians taken from L instead of
 * from the FP64 decisions (alpha, q and the pose terms still in FP64).
 * Returns 2 if an id is out of range or culled, else 0. */
int orc_backward_lists(const orc_section *secs, int n_secs, const orc_camera *cam,
                       const orc_lists *L, const orc_upstream *up, orc_grads *g);

/* Centres of the Gaussians of one depth map: mu = R (D * K^-1 [u v 1]) + t
 * for every valid pixel in raster order.  Returns the count. */
int64_t orc_backproject(const float *depth, int32_t W, int32_t H, float fx, float fy,
                        float cx, float cy, const double *pose12, double *centres,
                        uint32_t *pix);

/* Section initialisation from RGB-D views: one Gaussian per valid depth
 * pixel, colour = V(u,v), opacity = 0.9, radius = D / fx.  Returns n. */
int64_t orc_section_init(const float *depth, const float *rgb, int32_t n_views, int32_t W,
                         int32_t H, float fx, uint32_t *src, double *colour,
                         double *opacity, double *radius);

/* Complement initialisation of a regular frame (Sec. 3.4): one Gaussian per
 * pixel of the frame with valid depth whose silhouette (the section rendered
 * from the frame's pose) is below sil_max; the frame is view `view`, so
 * src = view * W * H + pixel.  Returns n. */
int64_t orc_section_complement(const float *depth, const float *rgb, const float *sil,
                               int32_t W, int32_t H, float fx, float sil_max, int32_t view,
                               uint32_t *src, double *colour, double *opacity, double *radius);

/* ---- loss inputs (vt_oracle_loss.c) ---------------------------------- */

typedef struct {
    const float *depth;          /* H x W, metres; <=0 or non-finite = invalid */
    int32_t W, H;
    float fx, fy, cx, cy;
    double pose[12];             /* camera-to-world: R row-major then t */
} orc_view;

/* Visibility check (Sec. 3.3): visible[p] = 1 iff the valid depth pixel p of
 * the current frame, back-projected with `pose`, projects in front of and
 * inside at least one of the views with a depth within rel_tol (0.01) of the
 * view's bilinearly interpolated depth (all four neighbours valid). */
void orc_visibility(const float *depth, int32_t W, int32_t H, float fx, float fy, float cx,
                    float cy, const double *pose, const orc_view *views, int32_t n_views,
                    double rel_tol, uint8_t *visible);

typedef struct {
    double w_rgb;                /* alpha (Eq. 1) or rho (Eq. 2) */
    double w_depth;              /* beta (Eq. 1) or sigma (Eq. 2) */
    double sil_min;              /* covered iff silhouette > sil_min (an FP32 value, widened);
                                    < 0: no coverage mask */
    int32_t rgb_needs_depth;     /* 1: the colour term is masked by valid observed depth too */
} orc_l1_weights;

/* L = w_rgb / (3P) sum m_c |V' - V| + w_depth / P sum m_d |D' - D| and its
 * gradient (d_rgb 3 x H x W, d_depth H x W; either may be NULL). */
double orc_masked_l1(int32_t W, int32_t H, const float *rgb, const float *depth, const float *sil,
                     const float *obs_rgb, const float *obs_depth, const uint8_t *visible,
                     orc_l1_weights w, double *d_rgb, double *d_depth);

#ifdef __cplusplus
}
#endif
#endif
