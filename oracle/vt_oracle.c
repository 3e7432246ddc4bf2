/* Plain FP64 CPU oracle of view-tied isotropic Gaussian splatting.
 *
 * TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark are its only users.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Every function follows a passage of the paper (VTGaussian-SLAM):
 *   - Gaussian = colour, isotropic radius, opacity (Sec. 3.2, "View-tied
 *     Gaussians"); its centre is the back-projected depth pixel of its view
 *     (Sec. 3.2), so positions are never stored.
 *   - initial radius r = D / f (supplementary, Implementation Details).
 *   - splat(gaussians, pose) -> RGB, depth (Eq. 1 text, Sec. 3.3) and the
 *     silhouette used for the 0.5 coverage test (Sec. 3.4, Sec. 4).
 * The rasterisation constants (3-sigma cutoff, alpha = o exp(-d^2 / 2r^2)
 * clamped at 0.99 and skipped below 1/255, termination at T < 1e-4, stable
 * depth order) are the ones the benchmark spec fixes; the readings of the
 * points the paper leaves open are listed in the design notes and repeated
 * inline where they matter.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no fast-math):
 * the FP32 depth key below must round every operation separately.
 */
#include "vt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Thresholds as the FP32 constants the kernels compare against. */
#define ORC_Q_MAX 9.0                    /* 3-sigma disc: q <= 9          */
#define ORC_A_MIN ((double)(1.0f / 255.0f))
#define ORC_A_CLAMP ((double)0.99f)
#define ORC_T_MIN ((double)1e-4f)
#define ORC_ZNEAR 0.1f
#define ORC_BAND 1.001                   /* candidates up to q <= 9*1.001 carry a margin */
#define ORC_BIN 16

static int g_threads = 0;

void orc_set_threads(int n) { g_threads = n; }

int orc_get_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

static int valid_depth(float d) { return isfinite(d) && d > 0.0f; }

/* ------------------------------------------------------------------------ */
/* Depth key: z of the centre in the target camera, in FP32 with a fixed
 * operation order (reading of "stable depth order": the order key is this
 * FP32 value, ties broken by the Gaussian id).  Composite transform
 * M = R^T R_k, m = R^T (t_k - t) is formed in FP64 in the order written and
 * rounded to FP32; then a = (u - cx)/fx, b = (v - cy)/fy, X = D a, Y = D b,
 * z = ((M20 X + M21 Y) + M22 D) + m2, each operation rounded to FP32. */
static void composite(const double *P, const double *Pk, double M[9], double m[3]) {
    const double *R = P, *t = P + 9, *Rk = Pk, *tk = Pk + 9;
    double d0 = tk[0] - t[0], d1 = tk[1] - t[1], d2 = tk[2] - t[2];
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) {
            double s = R[0 * 3 + a] * Rk[0 * 3 + b];
            s = s + R[1 * 3 + a] * Rk[1 * 3 + b];
            s = s + R[2 * 3 + a] * Rk[2 * 3 + b];
            M[a * 3 + b] = s;
        }
        double s = R[0 * 3 + a] * d0;
        s = s + R[1 * 3 + a] * d1;
        s = s + R[2 * 3 + a] * d2;
        m[a] = s;
    }
}

static float zkey_fp32(const float Mf[9], const float mf[3], float D, int u, int v,
                       float fx, float fy, float cx, float cy) {
    float a = ((float)u - cx) / fx;
    float b = ((float)v - cy) / fy;
    float X = D * a;
    float Y = D * b;
    float z = Mf[6] * X;
    z = z + Mf[7] * Y;
    z = z + Mf[8] * D;
    z = z + mf[2];
    return z;
}

/* ------------------------------------------------------------------------ */
/* Per-Gaussian quantities that do not depend on the pixel. */
typedef struct {
    double x[3];      /* centre in the target camera: R^T (mu - t) */
    double d[3];      /* mu - t */
    double c[3], o, r;
    float zkey;
    int valid;
    int32_t sec;
    int64_t local, id;
} gpre;

static int64_t total_n(const orc_section *secs, int n_secs) {
    int64_t n = 0;
    for (int s = 0; s < n_secs; ++s) n += secs[s].n;
    return n;
}

static void prepare(const orc_section *secs, int n_secs, const orc_camera *cam, gpre *g) {
    const double *R = cam->pose, *t = cam->pose + 9;
    int64_t base = 0;
    for (int s = 0; s < n_secs; ++s) {
        const orc_section *S = &secs[s];
        int64_t plane = (int64_t)S->W * S->H;
        float *Mf = (float *)malloc(sizeof(float) * 12 * (size_t)(S->n_views > 0 ? S->n_views : 1));
        for (int k = 0; k < S->n_views; ++k) {
            double M[9], m[3];
            composite(cam->pose, S->poses + 12 * k, M, m);
            for (int i = 0; i < 9; ++i) Mf[12 * k + i] = (float)M[i];
            for (int i = 0; i < 3; ++i) Mf[12 * k + 9 + i] = (float)m[i];
        }
#pragma omp parallel for schedule(static) num_threads(orc_get_threads())
        for (int64_t i = 0; i < S->n; ++i) {
            gpre *G = &g[base + i];
            uint32_t src = S->src[i];
            int k = (int)(src / plane);
            int64_t pix = src % plane;
            int u = (int)(pix % S->W), v = (int)(pix / S->W);
            float D = S->depth[src];
            G->sec = s;
            G->local = i;
            G->id = base + i;
            G->c[0] = S->colour[3 * i + 0];
            G->c[1] = S->colour[3 * i + 1];
            G->c[2] = S->colour[3 * i + 2];
            G->o = S->opacity[i];
            G->r = S->radius[i];
            G->valid = 0;
            G->zkey = 0.0f;
            if (!valid_depth(D)) continue;
            G->zkey = zkey_fp32(Mf + 12 * k, Mf + 12 * k + 9, D, u, v, S->fx, S->fy, S->cx, S->cy);
            if (!(G->zkey >= ORC_ZNEAR)) continue;
            /* centre by back-projection with the source pose (Sec. 3.2) */
            const double *Rk = S->poses + 12 * k, *tk = Rk + 9;
            double Xc[3] = {(double)D * (((double)u - S->cx) / S->fx),
                            (double)D * (((double)v - S->cy) / S->fy), (double)D};
            double mu[3];
            for (int a = 0; a < 3; ++a)
                mu[a] = Rk[3 * a + 0] * Xc[0] + Rk[3 * a + 1] * Xc[1] + Rk[3 * a + 2] * Xc[2] + tk[a];
            for (int a = 0; a < 3; ++a) G->d[a] = mu[a] - t[a];
            for (int a = 0; a < 3; ++a)
                G->x[a] = R[0 * 3 + a] * G->d[0] + R[1 * 3 + a] * G->d[1] + R[2 * 3 + a] * G->d[2];
            G->valid = 1;
        }
        free(Mf);
        base += S->n;
    }
}

void orc_zkeys(const orc_section *sec, const orc_camera *cam, float *zkey, uint8_t *valid) {
    int64_t n = sec->n;
    gpre *g = (gpre *)malloc(sizeof(gpre) * (size_t)(n > 0 ? n : 1));
    prepare(sec, 1, cam, g);
    for (int64_t i = 0; i < n; ++i) {
        zkey[i] = g[i].zkey;
        valid[i] = (uint8_t)g[i].valid;
    }
    free(g);
}

/* ------------------------------------------------------------------------ */
/* Candidate bins (binned form only): a Gaussian is listed in every 16x16 bin
 * touched by the pixel box of its disc q <= 9*1.001, which contains every
 * pixel where it can be included or carry a margin. */
typedef struct {
    int nbx, nby;
    int64_t *start;   /* nbx*nby + 1 */
    int64_t *items;
} bins_t;

static int disc_box(const gpre *G, const orc_camera *cam, int *u0, int *u1, int *v0, int *v1) {
    double z = G->x[2];
    double uc = cam->fx * (G->x[0] / z) + cam->cx;
    double vc = cam->fy * (G->x[1] / z) + cam->cy;
    double s = sqrt(ORC_Q_MAX * ORC_BAND) * G->r / z;
    double ex = s * cam->fx * (1.0 + 1e-9) + 1e-9, ey = s * cam->fy * (1.0 + 1e-9) + 1e-9;
    double a0 = ceil(uc - ex), a1 = floor(uc + ex), b0 = ceil(vc - ey), b1 = floor(vc + ey);
    if (a0 < 0) a0 = 0;
    if (b0 < 0) b0 = 0;
    if (a1 > cam->W - 1) a1 = cam->W - 1;
    if (b1 > cam->H - 1) b1 = cam->H - 1;
    if (!(a0 <= a1 && b0 <= b1)) return 0;
    *u0 = (int)a0; *u1 = (int)a1; *v0 = (int)b0; *v1 = (int)b1;
    return 1;
}

static void build_bins(const gpre *g, int64_t n, const orc_camera *cam, bins_t *B) {
    B->nbx = (cam->W + ORC_BIN - 1) / ORC_BIN;
    B->nby = (cam->H + ORC_BIN - 1) / ORC_BIN;
    int64_t nb = (int64_t)B->nbx * B->nby;
    B->start = (int64_t *)calloc((size_t)nb + 1, sizeof(int64_t));
    int64_t *cnt = (int64_t *)calloc((size_t)nb + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int u0, u1, v0, v1;
        if (!g[i].valid || !disc_box(&g[i], cam, &u0, &u1, &v0, &v1)) continue;
        for (int by = v0 / ORC_BIN; by <= v1 / ORC_BIN; ++by)
            for (int bx = u0 / ORC_BIN; bx <= u1 / ORC_BIN; ++bx) cnt[(int64_t)by * B->nbx + bx]++;
    }
    for (int64_t b = 0; b < nb; ++b) B->start[b + 1] = B->start[b] + cnt[b];
    B->items = (int64_t *)malloc(sizeof(int64_t) * (size_t)(B->start[nb] > 0 ? B->start[nb] : 1));
    memset(cnt, 0, sizeof(int64_t) * (size_t)nb);
    for (int64_t i = 0; i < n; ++i) {   /* id order inside every bin */
        int u0, u1, v0, v1;
        if (!g[i].valid || !disc_box(&g[i], cam, &u0, &u1, &v0, &v1)) continue;
        for (int by = v0 / ORC_BIN; by <= v1 / ORC_BIN; ++by)
            for (int bx = u0 / ORC_BIN; bx <= u1 / ORC_BIN; ++bx) {
                int64_t b = (int64_t)by * B->nbx + bx;
                B->items[B->start[b] + cnt[b]++] = i;
            }
    }
    free(cnt);
}

static void free_bins(bins_t *B) {
    free(B->start);
    free(B->items);
}

/* ------------------------------------------------------------------------ */
/* One pixel: collect the included Gaussians, order them, walk front to back. */
typedef struct {
    float zkey;
    int64_t id, gi;
    double q, ahat, G, alpha, ex, ey;
} inc_t;

typedef struct {
    inc_t *buf;
    int64_t cap;
} scratch_t;

static int cmp_inc(const void *a, const void *b) {
    const inc_t *x = (const inc_t *)a, *y = (const inc_t *)b;
    if (x->zkey < y->zkey) return -1;
    if (x->zkey > y->zkey) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

static double mind(double a, double b) { return a < b ? a : b; }

/* Returns the number of included candidates (sorted in sc->buf) and the
 * smallest margin of the inclusion decisions. */
static int64_t collect(const gpre *g, const int64_t *cand, int64_t ncand, double px, double py,
                       scratch_t *sc, double *margin, double *mclamp) {
    int64_t m = 0;
    for (int64_t j = 0; j < ncand; ++j) {
        int64_t i = cand ? cand[j] : j;
        const gpre *G = &g[i];
        if (!G->valid) continue;
        double ex = px * G->x[2] - G->x[0];
        double ey = py * G->x[2] - G->x[1];
        double q = (ex * ex + ey * ey) / (G->r * G->r);
        if (!(q <= ORC_Q_MAX * ORC_BAND)) continue;
        *margin = mind(*margin, fabs(q - ORC_Q_MAX) / ORC_Q_MAX);
        if (!(q <= ORC_Q_MAX)) continue;
        double Gv = exp(-0.5 * q);
        double ahat = G->o * Gv;
        *margin = mind(*margin, fabs(ahat - ORC_A_MIN) / ORC_A_MIN);
        if (!(ahat >= ORC_A_MIN)) continue;
        *mclamp = mind(*mclamp, fabs(ahat - ORC_A_CLAMP) / ORC_A_CLAMP);
        if (m == sc->cap) {
            sc->cap = sc->cap ? 2 * sc->cap : 256;
            sc->buf = (inc_t *)realloc(sc->buf, sizeof(inc_t) * (size_t)sc->cap);
        }
        inc_t *e = &sc->buf[m++];
        e->zkey = G->zkey;
        e->id = G->id;
        e->gi = i;
        e->q = q;
        e->ahat = ahat;
        e->G = Gv;
        e->alpha = ahat < ORC_A_CLAMP ? ahat : ORC_A_CLAMP;
        e->ex = ex;
        e->ey = ey;
    }
    qsort(sc->buf, (size_t)m, sizeof(inc_t), cmp_inc);
    return m;
}

/* Front-to-back walk; returns how many of the sorted candidates are added.
 * Stops before the Gaussian whose inclusion would make T < 1e-4. */
static int64_t walk(const inc_t *e, int64_t m, double *T_out, double *margin) {
    double T = 1.0;
    int64_t k = 0;
    for (; k < m; ++k) {
        double Tn = T * (1.0 - e[k].alpha);
        *margin = mind(*margin, fabs(Tn - ORC_T_MIN) / ORC_T_MIN);
        if (Tn < ORC_T_MIN) break;
        T = Tn;
    }
    *T_out = T;
    return k;
}

static void pixel_coords(const orc_camera *cam, int u, int v, double *px, double *py) {
    /* reading: pixel (u, v) is evaluated at the integer position, no +0.5 */
    *px = ((double)u - cam->cx) / cam->fx;
    *py = ((double)v - cam->cy) / cam->fy;
}

int orc_render(const orc_section *secs, int n_secs, const orc_camera *cam, int binned,
               orc_image *out) {
    int64_t n = total_n(secs, n_secs);
    gpre *g = (gpre *)malloc(sizeof(gpre) * (size_t)(n > 0 ? n : 1));
    if (!g) return 1;
    prepare(secs, n_secs, cam, g);
    bins_t B = {0};
    if (binned) build_bins(g, n, cam, &B);
    int64_t HW = (int64_t)cam->W * cam->H;
#pragma omp parallel num_threads(orc_get_threads())
    {
        scratch_t sc = {0};
#pragma omp for schedule(dynamic, 1)
        for (int v = 0; v < cam->H; ++v) {
            for (int u = 0; u < cam->W; ++u) {
                int64_t p = (int64_t)v * cam->W + u;
                double px, py, margin = INFINITY, mT = INFINITY, mc = INFINITY, T;
                pixel_coords(cam, u, v, &px, &py);
                const int64_t *cand = NULL;
                int64_t ncand = n;
                if (binned) {
                    int64_t b = (int64_t)(v / ORC_BIN) * B.nbx + u / ORC_BIN;
                    cand = B.items + B.start[b];
                    ncand = B.start[b + 1] - B.start[b];
                }
                int64_t m = collect(g, cand, ncand, px, py, &sc, &margin, &mc);
                int64_t k = walk(sc.buf, m, &T, &mT);
                double C[3] = {0, 0, 0}, Dp = 0, S = 0, Tw = 1.0;
                for (int64_t j = 0; j < k; ++j) {
                    const gpre *G = &g[sc.buf[j].gi];
                    double w = sc.buf[j].alpha * Tw;
                    C[0] += w * G->c[0];
                    C[1] += w * G->c[1];
                    C[2] += w * G->c[2];
                    Dp += w * G->x[2];
                    S += w;
                    Tw = Tw * (1.0 - sc.buf[j].alpha);
                }
                if (out->rgb) {
                    out->rgb[p] = C[0];
                    out->rgb[HW + p] = C[1];
                    out->rgb[2 * HW + p] = C[2];
                }
                if (out->depth) out->depth[p] = Dp;
                if (out->sil) out->sil[p] = S;
                if (out->T_final) out->T_final[p] = T;
                if (out->n_added) out->n_added[p] = (int32_t)k;
                if (out->margin) out->margin[p] = margin;
                if (out->margin_T) out->margin_T[p] = mT;
                if (out->margin_clamp) out->margin_clamp[p] = mc;
                if (out->lists) {
                    for (int32_t j = 0; j < out->list_cap; ++j)
                        out->lists[p * out->list_cap + j] = j < k ? sc.buf[j].id : -1;
                }
            }
        }
        free(sc.buf);
    }
    if (binned) free_bins(&B);
    free(g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Backward of L = <gC, C> + <gD, D'> + <gS, S> with the included sets held
 * fixed.  With A_i, B_i the colour / depth sums of the Gaussians behind i:
 *   dL/dc_i     = gC w_i
 *   dL/dalpha_i = T_i (gC.c_i + gD z_i) - (gC.A_i + gD B_i)/(1-alpha_i)
 *                 + gS T_final/(1-alpha_i)
 *   alpha = o exp(-q/2) below the clamp (else constant), q as above,
 *   plus the direct depth term dL/dz_i += gD w_i.
 * Pose: x_i = R^T (mu_i - t); with P(xi) = P Exp(xi) the centre moves by
 * dx = -rho - phi x x, so dL/drho = -sum g_i and dL/dphi = sum g_i x x_i;
 * dL/dR_ba = sum (mu - t)_b g_a and dL/dt = -R sum g_i. */
static void atomic_add(double *p, double v) {
#pragma omp atomic
    *p += v;
}

/* Pose sums of a thread (or of the whole image). */
typedef struct {
    double tw[6], mt[12], nz[18];
} pose_sums;

/* Gradient terms of one pixel whose added Gaussians are e[0..k) front to
 * back (alpha, q, ahat, exp(-q/2) and the offsets e_x, e_y filled in) with
 * final transmittance Tfin; Tb and wb are scratch of k doubles. */
static void pixel_grads(const gpre *g, const double *R, double px, double py, const double gC[3],
                        double gD, double gS, const inc_t *e_all, int64_t k, double Tfin,
                        double *Tb, double *wb, orc_grads *gr, pose_sums *ps) {
    double T = 1.0;
    for (int64_t j = 0; j < k; ++j) {   /* transmittance before each, weights */
        Tb[j] = T;
        wb[j] = e_all[j].alpha * T;
        T = T * (1.0 - e_all[j].alpha);
    }
    double A[3] = {0, 0, 0}, Bd = 0;    /* sums over the Gaussians behind */
    double pm[18] = {0};                 /* componentwise pose magnitudes */
    for (int64_t j = k - 1; j >= 0; --j) {
        const inc_t *e = &e_all[j];
        const gpre *G = &g[e->gi];
        double w = wb[j], al = e->alpha, z = G->x[2];
        double dal = Tb[j] * (gC[0] * G->c[0] + gC[1] * G->c[1] + gC[2] * G->c[2] + gD * z) -
                     (gC[0] * A[0] + gC[1] * A[1] + gC[2] * A[2] + gD * Bd) / (1.0 - al) +
                     gS * Tfin / (1.0 - al);
        double dq = 0.0, dop = 0.0;
        if (e->ahat < ORC_A_CLAMP) {
            dop = dal * e->G;
            dq = dal * (-0.5 * e->ahat);
        }
        double r = G->r;
        double dr = dq * (-2.0 * e->q / r);
        double gx = dq * (-2.0 * e->ex / (r * r));
        double gy = dq * (-2.0 * e->ey / (r * r));
        double gz = dq * (2.0 * (px * e->ex + py * e->ey) / (r * r)) + gD * w;
        double **dcol = gr->d_colour, **dop_ = gr->d_opacity, **drad = gr->d_radius;
        if (dcol && dcol[G->sec]) {
            atomic_add(&dcol[G->sec][3 * G->local + 0], gC[0] * w);
            atomic_add(&dcol[G->sec][3 * G->local + 1], gC[1] * w);
            atomic_add(&dcol[G->sec][3 * G->local + 2], gC[2] * w);
        }
        if (dop_ && dop_[G->sec]) atomic_add(&dop_[G->sec][G->local], dop);
        if (drad && drad[G->sec]) atomic_add(&drad[G->sec][G->local], dr);
        /* Componentwise magnitude of every per-pixel term: the sum of the
         * absolute values of the products the derivative formula adds,
         * which bounds the floating-point error of evaluating the term
         * (the term itself can cancel to far less). */
        double mal = Tb[j] * (fabs(gC[0] * G->c[0]) + fabs(gC[1] * G->c[1]) +
                              fabs(gC[2] * G->c[2]) + fabs(gD * z)) +
                     (fabs(gC[0] * A[0]) + fabs(gC[1] * A[1]) + fabs(gC[2] * A[2]) +
                      fabs(gD * Bd) + fabs(gS * Tfin)) / (1.0 - al);
        if (gr->a_colour && gr->a_colour[G->sec])
            for (int c = 0; c < 3; ++c)
                atomic_add(&gr->a_colour[G->sec][3 * G->local + c], fabs(gC[c] * w));
        if (e->ahat < ORC_A_CLAMP) {
            if (gr->a_opacity && gr->a_opacity[G->sec])
                atomic_add(&gr->a_opacity[G->sec][G->local], mal * e->G);
            if (gr->a_radius && gr->a_radius[G->sec])
                atomic_add(&gr->a_radius[G->sec][G->local], mal * 0.5 * e->ahat * 2.0 * e->q / r);
        }
        double gv[3] = {gx, gy, gz};
        const double *x = G->x;
        if (gr->d_x && gr->d_x[G->sec])
            for (int a = 0; a < 3; ++a) atomic_add(&gr->d_x[G->sec][3 * G->local + a], gv[a]);
        if (gr->a_x && gr->a_x[G->sec]) {
            /* |dq| <= ahat / 2 mal below the clamp, 0 above */
            const double mq = e->ahat < ORC_A_CLAMP ? 0.5 * e->ahat * mal : 0.0;
            const double ax[3] = {mq * 2.0 * fabs(e->ex) / (r * r), mq * 2.0 * fabs(e->ey) / (r * r),
                                  mq * 2.0 * (fabs(px * e->ex) + fabs(py * e->ey)) / (r * r) +
                                      fabs(gD * w)};
            for (int a = 0; a < 3; ++a) atomic_add(&gr->a_x[G->sec][3 * G->local + a], ax[a]);
        }
        ps->tw[0] -= gx;
        ps->tw[1] -= gy;
        ps->tw[2] -= gz;
        ps->tw[3] += gv[1] * x[2] - gv[2] * x[1];
        ps->tw[4] += gv[2] * x[0] - gv[0] * x[2];
        ps->tw[5] += gv[0] * x[1] - gv[1] * x[0];
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) ps->mt[3 * b + a] += G->d[b] * gv[a];
        for (int b = 0; b < 3; ++b)
            ps->mt[9 + b] -= R[3 * b + 0] * gx + R[3 * b + 1] * gy + R[3 * b + 2] * gz;
        /* magnitudes: |g| per axis from its products, then the same
         * sums as above with every product taken absolute */
        double ag[3] = {fabs(gx), fabs(gy),
                        fabs(dq * 2.0 * px * e->ex / (r * r)) +
                            fabs(dq * 2.0 * py * e->ey / (r * r)) + fabs(gD * w)};
        pm[0] += ag[0];
        pm[1] += ag[1];
        pm[2] += ag[2];
        pm[3] += ag[1] * fabs(x[2]) + ag[2] * fabs(x[1]);
        pm[4] += ag[2] * fabs(x[0]) + ag[0] * fabs(x[2]);
        pm[5] += ag[0] * fabs(x[1]) + ag[1] * fabs(x[0]);
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) pm[6 + 3 * b + a] += fabs(G->d[b]) * ag[a];
        for (int b = 0; b < 3; ++b)
            pm[15 + b] += fabs(R[3 * b + 0]) * ag[0] + fabs(R[3 * b + 1]) * ag[1] +
                          fabs(R[3 * b + 2]) * ag[2];
        A[0] += w * G->c[0];
        A[1] += w * G->c[1];
        A[2] += w * G->c[2];
        Bd += w * z;
    }
    for (int i = 0; i < 18; ++i) ps->nz[i] += (double)k * pm[i] * pm[i];
}

static int upstream_at(const orc_upstream *up, int64_t HW, int64_t p, double gC[3], double *gD,
                       double *gS) {
    gC[0] = gC[1] = gC[2] = 0.0;
    *gD = *gS = 0.0;
    if (up->g_rgb) {
        gC[0] = up->g_rgb[p];
        gC[1] = up->g_rgb[HW + p];
        gC[2] = up->g_rgb[2 * HW + p];
    }
    if (up->g_depth) *gD = up->g_depth[p];
    if (up->g_sil) *gS = up->g_sil[p];
    return !(gC[0] == 0 && gC[1] == 0 && gC[2] == 0 && *gD == 0 && *gS == 0);
}

static void finish_grads(const pose_sums *tot, orc_grads *gr) {
    memcpy(gr->twist, tot->tw, sizeof tot->tw);
    memcpy(gr->mat, tot->mt, sizeof tot->mt);
    for (int i = 0; i < 6; ++i) gr->twist_noise[i] = sqrt(tot->nz[i]);
    for (int i = 0; i < 12; ++i) gr->mat_noise[i] = sqrt(tot->nz[6 + i]);
}

static void add_sums(pose_sums *tot, const pose_sums *ps) {
    for (int i = 0; i < 6; ++i) tot->tw[i] += ps->tw[i];
    for (int i = 0; i < 12; ++i) tot->mt[i] += ps->mt[i];
    for (int i = 0; i < 18; ++i) tot->nz[i] += ps->nz[i];
}

static void grow(double **Tb, double **wb, int64_t *cap, int64_t k) {
    if (k <= *cap) return;
    *cap = k;
    *Tb = (double *)realloc(*Tb, sizeof(double) * (size_t)k);
    *wb = (double *)realloc(*wb, sizeof(double) * (size_t)k);
}

int orc_backward(const orc_section *secs, int n_secs, const orc_camera *cam, int binned,
                 const orc_upstream *up, orc_grads *gr) {
    int64_t n = total_n(secs, n_secs);
    gpre *g = (gpre *)malloc(sizeof(gpre) * (size_t)(n > 0 ? n : 1));
    if (!g) return 1;
    prepare(secs, n_secs, cam, g);
    bins_t B = {0};
    if (binned) build_bins(g, n, cam, &B);
    int64_t HW = (int64_t)cam->W * cam->H;
    pose_sums tot = {{0}};
#pragma omp parallel num_threads(orc_get_threads())
    {
        scratch_t sc = {0};
        pose_sums ps = {{0}};
        double *Tb = NULL, *wb = NULL;
        int64_t wcap = 0;
#pragma omp for schedule(dynamic, 1)
        for (int v = 0; v < cam->H; ++v) {
            for (int u = 0; u < cam->W; ++u) {
                int64_t p = (int64_t)v * cam->W + u;
                double gC[3], gD, gS;
                if (!upstream_at(up, HW, p, gC, &gD, &gS)) continue;
                double px, py, margin = INFINITY, mc = INFINITY, Tfin;
                pixel_coords(cam, u, v, &px, &py);
                const int64_t *cand = NULL;
                int64_t ncand = n;
                if (binned) {
                    int64_t b = (int64_t)(v / ORC_BIN) * B.nbx + u / ORC_BIN;
                    cand = B.items + B.start[b];
                    ncand = B.start[b + 1] - B.start[b];
                }
                int64_t m = collect(g, cand, ncand, px, py, &sc, &margin, &mc);
                int64_t k = walk(sc.buf, m, &Tfin, &margin);
                grow(&Tb, &wb, &wcap, k);
                pixel_grads(g, cam->pose, px, py, gC, gD, gS, sc.buf, k, Tfin, Tb, wb, gr, &ps);
            }
        }
#pragma omp critical
        add_sums(&tot, &ps);
        free(sc.buf);
        free(Tb);
        free(wb);
    }
    finish_grads(&tot, gr);
    if (binned) free_bins(&B);
    free(g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Compositing along given decisions.  Where a decision of the definition
 * (an inclusion test, the termination test) lies within the rounding of
 * another precision of its threshold, both outcomes are correct results of
 * the method.  orc_render_lists takes the per-pixel lists of added Gaussians
 * another implementation reports, checks that they differ from the FP64
 * decisions only at such decisions, and composites along them in FP64, so
 * that the values can be compared at every pixel. */

/* One candidate of a pixel: every valid Gaussian of its bin whose q lies in
 * the band q <= 9 * 1.001, with its FP64 decision and the relative margin a
 * flip of that decision needs. */
typedef struct {
    float zkey;
    int64_t id;
    double alpha, m_in;
    int inc;
} cand_t;

static int cmp_cand(const void *a, const void *b) {
    const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
    if (x->zkey < y->zkey) return -1;
    if (x->zkey > y->zkey) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* key order of two Gaussians: (z_key, id) */
static int key_less(const gpre *a, const gpre *b) {
    return a->zkey < b->zkey || (a->zkey == b->zkey && a->id < b->id);
}

/* FP64 quantities of Gaussian G at the pixel (px, py). */
static void pair_eval(const gpre *G, double px, double py, inc_t *e) {
    e->zkey = G->zkey;
    e->id = G->id;
    e->ex = px * G->x[2] - G->x[0];
    e->ey = py * G->x[2] - G->x[1];
    e->q = (e->ex * e->ex + e->ey * e->ey) / (G->r * G->r);
    e->G = exp(-0.5 * e->q);
    e->ahat = G->o * e->G;
    e->alpha = e->ahat < ORC_A_CLAMP ? e->ahat : ORC_A_CLAMP;
}

/* Inclusion decision of a pair and the relative margin a flip needs: an
 * included pair flips when either test does (the smaller margin), an
 * excluded one only when every failing test does (the larger). */
static int inclusion(const inc_t *e, double *m_in) {
    const double mq = fabs(e->q - ORC_Q_MAX) / ORC_Q_MAX;
    const double ma = fabs(e->ahat - ORC_A_MIN) / ORC_A_MIN;
    const int pq = e->q <= ORC_Q_MAX, pa = e->ahat >= ORC_A_MIN;
    if (pq && pa) {
        *m_in = mind(mq, ma);
        return 1;
    }
    *m_in = (pq ? 0.0 : mq) > (pa ? 0.0 : ma) ? (pq ? 0.0 : mq) : (pa ? 0.0 : ma);
    return 0;
}

static void note_flip(int32_t *flips, double *fmax, double m) {
    ++*flips;
    if (m > *fmax) *fmax = m;
}

int orc_render_lists(const orc_section *secs, int n_secs, const orc_camera *cam,
                     const orc_lists *L, double tau_incl, double tau_T, orc_image *out,
                     orc_verdict *vd) {
    int64_t n = total_n(secs, n_secs);
    gpre *g = (gpre *)malloc(sizeof(gpre) * (size_t)(n > 0 ? n : 1));
    if (!g) return 1;
    prepare(secs, n_secs, cam, g);
    bins_t B = {0};
    build_bins(g, n, cam, &B);
    int64_t HW = (int64_t)cam->W * cam->H;
#pragma omp parallel num_threads(orc_get_threads())
    {
        cand_t *cb = NULL;
        int64_t ccap = 0;
#pragma omp for schedule(dynamic, 1)
        for (int v = 0; v < cam->H; ++v) {
            for (int u = 0; u < cam->W; ++u) {
                const int64_t p = (int64_t)v * cam->W + u;
                const int64_t *ids = L->ids + p * (int64_t)L->cap;
                const int32_t cnt = L->count[p];
                double px, py;
                pixel_coords(cam, u, v, &px, &py);
                int32_t status = 0, flips = 0;
                double fmax = 0.0;
                /* the list itself: ids in range, valid, strictly increasing keys */
                if (cnt < 0 || cnt > L->cap) status = 1;
                for (int32_t j = 0; j < cnt && !status; ++j) {
                    if (ids[j] < 0 || ids[j] >= n || !g[ids[j]].valid) status = 1;
                    else if (j > 0 && !key_less(&g[ids[j - 1]], &g[ids[j]])) status = 1;
                }
                /* composite along the list in FP64 */
                double C[3] = {0, 0, 0}, Dp = 0, S = 0, T = 1.0;
                for (int32_t j = 0; j < cnt && !status; ++j) {
                    const gpre *G = &g[ids[j]];
                    inc_t e;
                    pair_eval(G, px, py, &e);
                    const double w = e.alpha * T;
                    C[0] += w * G->c[0];
                    C[1] += w * G->c[1];
                    C[2] += w * G->c[2];
                    Dp += w * G->x[2];
                    S += w;
                    T = T * (1.0 - e.alpha);
                }
                /* candidates of the pixel in key order */
                const int64_t b = (int64_t)(v / ORC_BIN) * B.nbx + u / ORC_BIN;
                const int64_t nb = B.start[b + 1] - B.start[b];
                int64_t m = 0;
                if (nb > ccap) {
                    ccap = nb;
                    cb = (cand_t *)realloc(cb, sizeof(cand_t) * (size_t)ccap);
                }
                for (int64_t j = 0; j < nb && !status; ++j) {
                    const gpre *G = &g[B.items[B.start[b] + j]];
                    if (!G->valid) continue;
                    inc_t e;
                    pair_eval(G, px, py, &e);
                    if (!(e.q <= ORC_Q_MAX * ORC_BAND)) continue;
                    cand_t *c = &cb[m++];
                    c->zkey = G->zkey;
                    c->id = G->id;
                    c->alpha = e.alpha;
                    c->inc = inclusion(&e, &c->m_in);
                }
                if (!status) qsort(cb, (size_t)m, sizeof(cand_t), cmp_cand);
                /* walk the candidates: before the list's last entry every
                 * candidate is either added (listed) or excluded; after it the
                 * walk has either terminated at a candidate or excluded it */
                double Tw = 1.0;
                int32_t next = 0;
                for (int64_t j = 0; j < m && !status; ++j) {
                    const cand_t *c = &cb[j];
                    const double Tn = Tw * (1.0 - c->alpha);
                    const double mT = fabs(Tn - ORC_T_MIN) / ORC_T_MIN;
                    if (next < cnt) {
                        if (c->id == ids[next]) {          /* added */
                            if (!c->inc) {
                                if (c->m_in < tau_incl) note_flip(&flips, &fmax, c->m_in);
                                else status = 2;
                            }
                            if (Tn < ORC_T_MIN) {
                                if (mT < tau_T) note_flip(&flips, &fmax, mT);
                                else status = 2;
                            }
                            Tw = Tn;
                            ++next;
                        } else if (c->inc) {               /* excluded, though included in FP64 */
                            if (c->m_in < tau_incl) note_flip(&flips, &fmax, c->m_in);
                            else status = 2;
                        }
                        continue;
                    }
                    /* after the list: terminate here, or exclude and go on */
                    const int incl_ok = c->inc || c->m_in < tau_incl;
                    const int term_ok = Tn < ORC_T_MIN || mT < tau_T;
                    if (incl_ok && term_ok) {
                        if (!c->inc) note_flip(&flips, &fmax, c->m_in);
                        if (!(Tn < ORC_T_MIN)) note_flip(&flips, &fmax, mT);
                        break;
                    }
                    if (!c->inc) continue;
                    if (c->m_in < tau_incl) note_flip(&flips, &fmax, c->m_in);
                    else status = 2;
                }
                if (!status && next < cnt) status = 1;   /* a listed id is not a candidate */
                if (out->rgb) {
                    out->rgb[p] = C[0];
                    out->rgb[HW + p] = C[1];
                    out->rgb[2 * HW + p] = C[2];
                }
                if (out->depth) out->depth[p] = Dp;
                if (out->sil) out->sil[p] = S;
                if (out->T_final) out->T_final[p] = T;
                if (out->n_added) out->n_added[p] = cnt;
                if (vd->status) vd->status[p] = status;
                if (vd->flips) vd->flips[p] = flips;
                if (vd->flip_margin) vd->flip_margin[p] = fmax;
            }
        }
        free(cb);
    }
    free_bins(&B);
    free(g);
    return 0;
}

int orc_backward_lists(const orc_section *secs, int n_secs, const orc_camera *cam,
                       const orc_lists *L, const orc_upstream *up, orc_grads *gr) {
    int64_t n = total_n(secs, n_secs);
    gpre *g = (gpre *)malloc(sizeof(gpre) * (size_t)(n > 0 ? n : 1));
    if (!g) return 1;
    prepare(secs, n_secs, cam, g);
    for (int64_t p = 0; p < (int64_t)cam->W * cam->H; ++p) {
        if (L->count[p] < 0 || L->count[p] > L->cap) { free(g); return 2; }
        for (int32_t j = 0; j < L->count[p]; ++j) {
            const int64_t id = L->ids[p * (int64_t)L->cap + j];
            if (id < 0 || id >= n || !g[id].valid) { free(g); return 2; }
        }
    }
    int64_t HW = (int64_t)cam->W * cam->H;
    pose_sums tot = {{0}};
#pragma omp parallel num_threads(orc_get_threads())
    {
        pose_sums ps = {{0}};
        inc_t *eb = NULL;
        double *Tb = NULL, *wb = NULL;
        int64_t ecap = 0, wcap = 0;
#pragma omp for schedule(dynamic, 1)
        for (int v = 0; v < cam->H; ++v) {
            for (int u = 0; u < cam->W; ++u) {
                int64_t p = (int64_t)v * cam->W + u;
                double gC[3], gD, gS;
                if (!upstream_at(up, HW, p, gC, &gD, &gS)) continue;
                double px, py;
                pixel_coords(cam, u, v, &px, &py);
                const int64_t k = L->count[p];
                if (k > ecap) {
                    ecap = k;
                    eb = (inc_t *)realloc(eb, sizeof(inc_t) * (size_t)ecap);
                }
                double Tfin = 1.0;
                for (int64_t j = 0; j < k; ++j) {
                    const int64_t id = L->ids[p * (int64_t)L->cap + j];
                    pair_eval(&g[id], px, py, &eb[j]);
                    eb[j].gi = id;
                    Tfin = Tfin * (1.0 - eb[j].alpha);
                }
                grow(&Tb, &wb, &wcap, k);
                pixel_grads(g, cam->pose, px, py, gC, gD, gS, eb, k, Tfin, Tb, wb, gr, &ps);
            }
        }
#pragma omp critical
        add_sums(&tot, &ps);
        free(eb);
        free(Tb);
        free(wb);
    }
    finish_grads(&tot, gr);
    free(g);
    return 0;
}

/* ------------------------------------------------------------------------ */
int64_t orc_backproject(const float *depth, int32_t W, int32_t H, float fx, float fy, float cx,
                        float cy, const double *P, double *centres, uint32_t *pix) {
    int64_t n = 0;
    for (int v = 0; v < H; ++v)
        for (int u = 0; u < W; ++u) {
            float D = depth[(int64_t)v * W + u];
            if (!valid_depth(D)) continue;
            double Xc[3] = {(double)D * (((double)u - cx) / fx), (double)D * (((double)v - cy) / fy),
                            (double)D};
            for (int a = 0; a < 3; ++a)
                centres[3 * n + a] = P[3 * a + 0] * Xc[0] + P[3 * a + 1] * Xc[1] + P[3 * a + 2] * Xc[2] + P[9 + a];
            pix[n] = (uint32_t)((int64_t)v * W + u);
            ++n;
        }
    return n;
}

int64_t orc_section_init(const float *depth, const float *rgb, int32_t n_views, int32_t W,
                         int32_t H, float fx, uint32_t *src, double *colour, double *opacity,
                         double *radius) {
    int64_t plane = (int64_t)W * H, n = 0;
    for (int k = 0; k < n_views; ++k)
        for (int64_t p = 0; p < plane; ++p) {
            float D = depth[k * plane + p];
            if (!valid_depth(D)) continue;
            src[n] = (uint32_t)(k * plane + p);
            for (int c = 0; c < 3; ++c) colour[3 * n + c] = rgb[(k * 3 + c) * plane + p];
            opacity[n] = 0.9;
            radius[n] = (double)D / (double)fx;   /* r = D / f, f = fx */
            ++n;
        }
    return n;
}

int64_t orc_section_complement(const float *depth, const float *rgb, const float *sil,
                               int32_t W, int32_t H, float fx, float sil_max, int32_t view,
                               uint32_t *src, double *colour, double *opacity, double *radius) {
    int64_t plane = (int64_t)W * H, n = 0;
    for (int64_t p = 0; p < plane; ++p) {
        float D = depth[p];
        if (!valid_depth(D) || !(sil[p] < sil_max)) continue;   /* covered: no new Gaussian */
        src[n] = (uint32_t)((int64_t)view * plane + p);
        for (int c = 0; c < 3; ++c) colour[3 * n + c] = rgb[c * plane + p];
        opacity[n] = 0.9;
        radius[n] = (double)D / (double)fx;
        ++n;
    }
    return n;
}
