/* Plain FP64 CPU oracle of the tracking / mapping loss inputs.
 *
 * TEST INFRASTRUCTURE ONLY (see vt_oracle.h).
 *
 * orc_visibility: the visibility check of Sec. 3.3 ("Visibility Check"): a
 * 3D point is visible to a view when its depth in that view lies within 1%
 * of the view's depth map interpolated at the point's projection; the mask of
 * a section is the union over its head, middle and last frames.  The points
 * are the valid depth pixels of the current frame back-projected with its
 * pose.  Readings: pixel (u, v) sits at integer coordinates (as everywhere in
 * this oracle), "interpolated" is bilinear over the four neighbouring pixels,
 * all four of which must hold valid depth, and a projection must lie inside
 * [0, W-1] x [0, H-1] in front of the camera.
 *
 * orc_masked_l1: the L1 terms of Eq. 1 (tracking: alpha W |V - V'| +
 * beta W |D - D'|, W = valid observed depth, covered by the render
 * (silhouette > sil_min) and visible) and of Eq. 2 (mapping:
 * rho |V - V'| + sigma U |D - D'|, U = valid observed depth), each sum taken
 * over pixels (and channels) and divided by the pixel count (and 3 for
 * colour), with their gradient with respect to the rendered images.
 *
 * Every operation is written in the order the definition reads, in double
 * precision, with no contraction (-ffp-contract=off).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "vt_oracle.h"

static int valid_depth(float d) { return isfinite(d) && d > 0.0f; }

/* Depth of view V bilinearly interpolated at (x, y); returns 0 when the
 * point falls outside the image or a neighbour lacks valid depth. */
static int interp_depth(const orc_view *V, double x, double y, double *out) {
    if (!(x >= 0.0 && x <= (double)(V->W - 1) && y >= 0.0 && y <= (double)(V->H - 1))) return 0;
    const int i0 = (int)floor(x), j0 = (int)floor(y);
    const int i1 = i0 + 1 < V->W ? i0 + 1 : V->W - 1;
    const int j1 = j0 + 1 < V->H ? j0 + 1 : V->H - 1;
    const double fx = x - (double)i0, fy = y - (double)j0;
    const float d00 = V->depth[(int64_t)j0 * V->W + i0], d10 = V->depth[(int64_t)j0 * V->W + i1];
    const float d01 = V->depth[(int64_t)j1 * V->W + i0], d11 = V->depth[(int64_t)j1 * V->W + i1];
    if (!valid_depth(d00) || !valid_depth(d10) || !valid_depth(d01) || !valid_depth(d11)) return 0;
    const double top = (double)d00 * (1.0 - fx) + (double)d10 * fx;
    const double bot = (double)d01 * (1.0 - fx) + (double)d11 * fx;
    *out = top * (1.0 - fy) + bot * fy;
    return 1;
}

void orc_visibility(const float *depth, int32_t W, int32_t H, float fx, float fy, float cx,
                    float cy, const double *pose, const orc_view *views, int32_t n_views,
                    double rel_tol, uint8_t *visible) {
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            const int64_t p = (int64_t)v * W + u;
            const float D = depth[p];
            uint8_t vis = 0;
            if (valid_depth(D)) {
                /* camera-space point, then world: X = R Xc + t */
                const double a = ((double)u - (double)cx) / (double)fx;
                const double b = ((double)v - (double)cy) / (double)fy;
                const double xc[3] = {(double)D * a, (double)D * b, (double)D};
                double X[3];
                for (int i = 0; i < 3; ++i)
                    X[i] = pose[3 * i + 0] * xc[0] + pose[3 * i + 1] * xc[1] +
                           pose[3 * i + 2] * xc[2] + pose[9 + i];
                for (int k = 0; k < n_views && !vis; ++k) {
                    const orc_view *V = &views[k];
                    const double *Pk = V->pose;
                    const double d[3] = {X[0] - Pk[9], X[1] - Pk[10], X[2] - Pk[11]};
                    double x[3];   /* R_k^T (X - t_k) */
                    for (int j = 0; j < 3; ++j)
                        x[j] = Pk[0 * 3 + j] * d[0] + Pk[1 * 3 + j] * d[1] + Pk[2 * 3 + j] * d[2];
                    if (!(x[2] > 0.0)) continue;
                    const double px = (double)V->fx * (x[0] / x[2]) + (double)V->cx;
                    const double py = (double)V->fy * (x[1] / x[2]) + (double)V->cy;
                    double Dk;
                    if (!interp_depth(V, px, py, &Dk)) continue;
                    if (fabs(x[2] - Dk) <= rel_tol * Dk) vis = 1;
                }
            }
            visible[p] = vis;
        }
}

static double sgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

double orc_masked_l1(int32_t W, int32_t H, const float *rgb, const float *depth, const float *sil,
                     const float *obs_rgb, const float *obs_depth, const uint8_t *visible,
                     orc_l1_weights w, double *d_rgb, double *d_depth) {
    const int64_t P = (int64_t)W * H;
    const double sc = w.w_rgb / (3.0 * (double)P), sd = w.w_depth / (double)P;
    double sum_c = 0.0, sum_d = 0.0;
    for (int64_t p = 0; p < P; ++p) {
        const int valid = valid_depth(obs_depth[p]);
        const int covered = !(w.sil_min >= 0.0) || (double)sil[p] > w.sil_min;
        const int vis = visible == NULL || visible[p] != 0;
        const int m_d = valid && covered && vis;
        const int m_c = covered && vis && (!w.rgb_needs_depth || valid);
        for (int c = 0; c < 3; ++c) {
            const double e = (double)rgb[c * P + p] - (double)obs_rgb[c * P + p];
            if (m_c) sum_c += fabs(e);
            if (d_rgb) d_rgb[c * P + p] = m_c ? sc * sgn(e) : 0.0;
        }
        const double e = (double)depth[p] - (double)obs_depth[p];
        if (m_d) sum_d += fabs(e);
        if (d_depth) d_depth[p] = m_d ? sd * sgn(e) : 0.0;
    }
    return sc * sum_c + sd * sum_d;
}
