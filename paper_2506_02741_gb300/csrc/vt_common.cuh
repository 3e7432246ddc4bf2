// Shared device definitions of the vtsplat CUDA library (sm_103a).
//
// Layout of the workspace a render keeps (all in HBM, library-owned):
//   geo[g]   : float4 x 2 per Gaussian  {iu, fu, iv, fv} {kx', ky', 1/r, o}
//   app[g]   : float4 per Gaussian      {c0, c1, c2, z}
//   info[g]  : uint4 per Gaussian       {tx0 | ty0<<16, tx1 | ty1<<16, zkey bits, n_tiles}
//   bucket   : uint64 per instance      (zkey << 32 | gid), unsorted per tile
//   sorted   : uint32 per instance      Gaussian ids, per tile in (zkey, gid) order
//   per pixel: list end, count added, final transmittance, and (optional)
//              (id, transmittance in front) of each Gaussian it added,
//              8 B each, pixel-major, plist_cap per pixel
// The projected centre of a Gaussian in pixels is iu + fu (integer part and
// a float remainder), accurate to ~1e-7 px, because footprints are only
// about one pixel wide while centres lie hundreds of pixels from the origin.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vtsplat.h"

namespace vt {

constexpr int kTile = 16;          // tile edge in pixels
constexpr int kBlockPix = 256;     // threads of a compositing block (one per pixel)
constexpr int kBatch = 256;        // Gaussians staged in shared memory per step
constexpr int kMaxSecs = 16;       // sections per render
constexpr float kQMax = 9.0f;      // 3-sigma disc
constexpr float kZNear = 0.1f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaClamp = 0.99f;
constexpr float kTMin = 1e-4f;

// Status flags written on the device.
constexpr int kFlagCapacity = 1;

struct SecDesc {
    const double *poses;    // n_views x 12 camera-to-world
    const float *depth;
    const uint32_t *src;
    const void *colour, *opacity, *radius;
    const void *scale, *rot;                  // ellipsoids (NULL: spheres)
    float *d_colour, *d_opacity, *d_radius;  // backward only
    float *d_scale, *d_rot;                   // backward only (ellipsoids)
    double *d_view_twist, *d_view_mat;        // backward only (source-view poses)
    float *d_depth;                           // backward only (depth along the ray)
    int64_t gbase, n;       // global id range [gbase, gbase + n)
    int64_t tab_base;       // first table row of view 0
    int32_t view_base;      // first ViewXf of this section
    int32_t n_views, W, H, prec;
    float fx, fy, cx, cy;
};

struct SecTable {
    int32_t n;
    int64_t n_total;
    SecDesc s[kMaxSecs];
};

struct Camera {
    float fx, fy, cx, cy;
    int32_t W, H, tiles_x, tiles_y;
};

// Per source view, per render: FP32 composite transform for the depth key
// and the float-float offsets of the projection numerators.
struct ViewXf {
    float Mf[12];            // R^T R_k (row-major) then R^T (t_k - t), rounded to FP32
    float2 mu, mv, mz;       // fx m0 + cx m2, fy m1 + cy m2, m2 (float-float)
    float pad[2];
};

// One table row: three float-float values (u numerator, v numerator, z).
struct __align__(16) TabRow {
    float2 a, b, c;
    float kf;    // FP32 (u - cx)/fx (column rows) or (v - cy)/fy (row rows) of the depth key
    float pad;
};

struct Status {
    int32_t flags;
    int32_t pad;
    unsigned long long n_instances;
    unsigned long long n_overflow_tiles;
    uint32_t sort_next[2];   // work counters of the long-list sorts (reset by the tile scan)
    uint32_t n_long, pad2;   // tiles listed in long_tiles by the tile scan
};

// Lists longer than this are sorted by the long-list launches (on chip up to
// 13,312 entries, beyond in global memory); the tile scan lists their tiles.
constexpr int kSortLongMin = 6000;

// ---------------------------------------------------------------------------
// Batched launches (vt_batch_*): many independent work items -- one section
// rendered from one camera each, a tracking item adding the Eq. 1 masked L1
// loss and the pose gradient -- processed by one launch per stage over all
// items (grids sized to the batch, or persistent grids inside a graph
// capture).  The work-item table lives in device memory (uploaded from pinned
// host memory at the start of the launch sequence), so one captured launch
// sequence serves any mix of items within the reserved capacity.  The index
// spaces are concatenated over the items: Gaussians and pixels (each item's
// range starts at a multiple of 256, so a block of 256 never holds two
// items), tiles, views and per-view table rows.
constexpr int kMaxItems = 64;
constexpr int kBatchResult = 19;   // loss, dL/dtwist (6), dL/dR (9), dL/dt (3)

struct BatchItem {
    Camera cam;
    const double *pose;          // 12 doubles, camera-to-world
    float *image;                // 5 x H x W: rgb planes, depth, silhouette
    const float *obs;            // 4 x H x W: observed rgb planes and depth (track)
    double *result;              // kBatchResult doubles (track)
    int64_t gbase, n;            // Gaussians [gbase, gbase + n)
    int64_t pbase;               // first pixel of the per-pixel arrays
    int64_t tab_base;            // first per-view table row
    int32_t tbase, vbase;        // first tile, first view
    int32_t sec, track;          // section (index into BatchTable::sec), tracking item?
};

struct BatchTable {
    int32_t n_items, n_secs;
    int32_t n_tiles, n_views;    // totals
    int64_t n_gauss, n_pix;      // ends of the last item's (padded) ranges
    double w_rgb, w_depth;       // Eq. 1 weights (alpha, beta)
    float sil_min;               // covered iff silhouette > sil_min
    int32_t rgb_needs_depth;
    uint32_t ctr[4];             // work counters of the persistent stages (zero on upload)
    BatchItem it[kMaxItems];
    SecDesc sec[kMaxItems];      // gbase, view_base, tab_base unused (per item instead)
};

// Last item whose range starts at or before x (binary search; items in order).
template <typename F>
__device__ __forceinline__ int batch_find(int n, F start_of, int64_t x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start_of(mid) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int item_of_gauss(const BatchTable &B, int64_t g) {
    return batch_find(B.n_items, [&](int i) { return B.it[i].gbase; }, g);
}
__device__ __forceinline__ int item_of_tile(const BatchTable &B, int64_t t) {
    return batch_find(B.n_items, [&](int i) { return (int64_t)B.it[i].tbase; }, t);
}
__device__ __forceinline__ int item_of_view(const BatchTable &B, int64_t v) {
    return batch_find(B.n_items, [&](int i) { return (int64_t)B.it[i].vbase; }, v);
}
__device__ __forceinline__ int item_of_pixel(const BatchTable &B, int64_t p) {
    return batch_find(B.n_items, [&](int i) { return B.it[i].pbase; }, p);
}

// The item of a position in a grid-stride loop, remembered between
// iterations: positions grow, so the search runs only when one leaves the
// current item's range [lo, hi).
struct ItemCursor {
    int it = -1;
    int64_t lo = 0, hi = 0;
    template <typename F>
    __device__ __forceinline__ int at(const BatchTable &B, F start_of, int64_t x) {
        if (it < 0 || x < lo || x >= hi) {
            it = batch_find(B.n_items, start_of, x);
            lo = start_of(it);
            hi = it + 1 < B.n_items ? start_of(it + 1) : INT64_MAX;
        }
        return it;
    }
};

// ---------------------------------------------------------------------------
// float-float ("double-single") arithmetic: Knuth's TwoSum, Dekker's
// FastTwoSum and the FMA-based exact product.  Every operation uses the
// explicit round-to-nearest intrinsics so that no contraction or
// reassociation can break the error-free transformations.

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = ff_two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return ff_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return ff_fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ff_fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_from_double(double d) {
    float hi = __double2float_rn(d);
    float lo = __double2float_rn(__dsub_rn(d, (double)hi));
    return {hi, lo};
}

__device__ __forceinline__ ff ff_div(ff a, ff b) {
    float q1 = __fdiv_rn(a.hi, b.hi);
    ff p = ff_mul_f(b, q1);
    ff r = ff_add(a, ff{-p.hi, -p.lo});
    float q2 = __fdiv_rn(r.hi, b.hi);
    return ff_fast_two_sum(q1, q2);
}

__device__ __forceinline__ ff ff_from(float2 v) { return {v.x, v.y}; }

// ---------------------------------------------------------------------------
// Shared per-pair footprint, in base-2 exponent form: with kx' = -kx log2(e)/2
// and ky' likewise (kx = (z / (fx r))^2 etc., so q = du^2 kx + dv^2 ky),
//   t = du^2 kx' + dv^2 ky' = -q log2(e) / 2,   exp(-q/2) = 2^t.
// A pair is included iff t >= t_min = max(-4.5 log2(e), -log2(255 o)), i.e.
// q <= 9 and o exp(-q/2) >= 1/255.  Explicit rounding makes the forward and
// backward kernels take bit-identical decisions.
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kTScale = -0.5f * kLog2e;          // t = q * kTScale
constexpr float kQFromT = -2.0f * 0.69314718055994531f;   // q = t * kQFromT
constexpr float kLn2 = 0.69314718055994531f;
constexpr float kLowPass = 0.3f;                   // EWA low-pass added to Sigma_2D (px^2)

// The pixel offsets du = (px - iu) - fu, dv = (py - iv) - fv take one
// rounding each (the integer differences are exact in FP32).
__device__ __forceinline__ float pair_t(float du, float dv, float kxs, float kys) {
    return __fmaf_rn(__fmul_rn(du, kxs), du, __fmul_rn(__fmul_rn(dv, kys), dv));
}
// Offsets and exponent of pixel (px, py) for a Gaussian record g0/g1.
__device__ __forceinline__ float pair_t_at(int px, int py, const float4 &g0, const float4 &g1,
                                           float &du, float &dv) {
    du = __fsub_rn((float)(px - __float_as_int(g0.x)), g0.y);
    dv = __fsub_rn((float)(py - __float_as_int(g0.z)), g0.w);
    return pair_t(du, dv, g1.x, g1.y);
}
// Ellipsoids: the record holds (a', b', c') = kTScale (Q00, 2 Q01, Q11) of
// the conic Q = Sigma_2D^-1, and t = a' du^2 + b' du dv + c' dv^2; the
// sphere form is the special case b' = 0 term by term.
__device__ __forceinline__ float pair_t_aniso(float du, float dv, float a, float b, float c) {
    return __fmaf_rn(__fmul_rn(du, a), du,
                     __fmaf_rn(__fmul_rn(du, b), dv, __fmul_rn(__fmul_rn(dv, c), dv)));
}
__device__ __forceinline__ float pair_t_at_aniso(int px, int py, const float4 &g0,
                                                 const float4 &g1, float &du, float &dv) {
    du = __fsub_rn((float)(px - __float_as_int(g0.x)), g0.y);
    dv = __fsub_rn((float)(py - __float_as_int(g0.z)), g0.w);
    return pair_t_aniso(du, dv, g1.x, g1.y, g1.z);
}

// 2^t with the hardware approximation (t in [-6.5, 0]: no subnormals).
__device__ __forceinline__ float exp2_approx(float t) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(t));
    return y;
}

// log2(x) with the hardware approximation (x >= 1 here).
__device__ __forceinline__ float log2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Inclusion threshold on t for opacity o (both cuts: q <= 9 and
// o exp(-q/2) >= 1/255); every kernel derives it with this function, so the
// decisions agree bit for bit.
__device__ __forceinline__ float t_min_of(float o) {
    return fmaxf(kQMax * kTScale, -log2_approx(__fmul_rn(255.f, o)));
}

// Conservative test: can a pixel of the block (columns 0..lxmax and rows
// 0..lymax from the block origin) pass t >= t_min for a Gaussian at offsets
// du0 ~ bx0 - uc, dv0 ~ by0 - vc from the origin?  The nearest pixel is taken
// 1e-3 px nearer and the threshold loosened by 1e-4 relative so that rounding
// never drops a pixel the per-pixel test includes.
__device__ __forceinline__ bool block_touches(float du0, float dv0, float kxs, float kys,
                                              float tmin, float lxmax, float lymax) {
    const float dx = fmaxf(fmaxf(du0, -du0 - lxmax) - 1e-3f, 0.f);
    const float dy = fmaxf(fmaxf(dv0, -dv0 - lymax) - 1e-3f, 0.f);
    return dx * dx * kxs + dy * dy * kys >= tmin * 1.0001f - 1e-6f;
}

// Which of the eight 8x4 pixel blocks of tile (tx, ty) (block w at
// ((w & 1) * 8, (w >> 1) * 4)) can a pixel of pass t >= t_min for the
// Gaussian with records (g0, g1): bit w set (block_touches per block; blocks
// outside the image get 0).  Written next to each sorted tile entry so that a
// warp of the compositor only visits the entries of its own block.
__device__ __forceinline__ uint32_t tile_block_mask(float4 g0, float4 g1, int tx, int ty,
                                                    const Camera &cam) {
    // the block_touches test with the column and row terms formed once: two
    // block columns (x offsets 0, 8) and four block rows (y offsets 0, 4, 8, 12)
    const float tl = t_min_of(g1.w) * 1.0001f - 1e-6f;
    float ex[2], ey[4];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int bx0 = tx * kTile + 8 * c;
        const float du0 = (float)(bx0 - __float_as_int(g0.x)) - g0.y;
        const float dx = fmaxf(fmaxf(du0, -du0 - (float)min(7, cam.W - 1 - bx0)) - 1e-3f, 0.f);
        ex[c] = bx0 < cam.W ? dx * dx * g1.x : -INFINITY;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int by0 = ty * kTile + 4 * r;
        const float dv0 = (float)(by0 - __float_as_int(g0.z)) - g0.w;
        const float dy = fmaxf(fmaxf(dv0, -dv0 - (float)min(3, cam.H - 1 - by0)) - 1e-3f, 0.f);
        ey[r] = by0 < cam.H ? dy * dy * g1.y : -INFINITY;
    }
    uint32_t m = 0u;
#pragma unroll
    for (int w = 0; w < 8; ++w)
        if (ex[w & 1] + ey[w >> 1] >= tl) m |= 1u << w;
    return m;
}

// Attribute loads in either storage precision.
__device__ __forceinline__ float ld_attr(const void *p, int prec, int64_t i) {
    if (prec == VT_F16) return __half2float(reinterpret_cast<const __half *>(p)[i]);
    return reinterpret_cast<const float *>(p)[i];
}

__device__ __forceinline__ int find_section(const SecTable &T, int64_t gid) {
    int s = 0;
#pragma unroll 1
    for (int k = 1; k < T.n; ++k)
        if (gid >= T.s[k].gbase) s = k;
    return s;
}

// ---------------------------------------------------------------------------
// Kernel entry points (defined in the .cu files, launched from vt_api.cu).

__global__ void k_setup(SecTable T, Camera cam, const double *pose12, ViewXf *views, TabRow *tab,
                        double *pose_copy);
__global__ void k_preprocess(SecTable T, Camera cam, const ViewXf *views, const TabRow *tab,
                             float4 *geo, float4 *app, uint4 *info, uint32_t *tile_count);
__global__ void k_preprocess_aniso(SecTable T, Camera cam, const ViewXf *views,
                                   const TabRow *tab, float4 *geo, float4 *app, uint4 *info,
                                   uint32_t *tile_count);
__global__ void k_scan_tiles(const uint32_t *tile_count, int n_tiles, uint32_t *tile_off,
                             uint32_t *tile_cursor, Status *st, unsigned long long cap,
                             uint32_t *long_tiles);
__global__ void k_emit(int64_t n, const uint4 *info, Camera cam, uint32_t *tile_cursor,
                       unsigned long long *bucket, uint8_t *bmask_u, const Status *st);
// Per-tile depth sort, one kernel per list-length class (vt_raster.cu).
#define VT_DECLARE_SORT(name)                                                                    \
    __global__ void name(const uint32_t *tile_off, int n_tiles, unsigned long long *bucket,     \
                         unsigned long long *alt, const uint8_t *bmask_u, uint32_t *sorted,     \
                         uint8_t *bmask, const float4 *geo, Camera cam, Status *st, int smem_n, \
                         int lo, int hi, const uint32_t *long_tiles);
VT_DECLARE_SORT(k_sort_tiles)
VT_DECLARE_SORT(k_sort_tiles_mid)
VT_DECLARE_SORT(k_sort_tiles_large)
VT_DECLARE_SORT(k_sort_tiles_long)
VT_DECLARE_SORT(k_sort_tiles_xl)
#undef VT_DECLARE_SORT
__global__ void k_composite_fwd(Camera cam, const uint32_t *tile_off, const uint32_t *sorted,
                                const uint8_t *bmask, const float4 *geo, const float4 *app,
                                float *rgb, float *depth, float *sil, uint32_t *pix_last,
                                uint32_t *pix_nadd, float *pix_T, uint2 *plist, int plist_cap,
                                uint32_t *blk_ovf, const Status *st);
__global__ void k_composite_fwd_aniso(Camera cam, const uint32_t *tile_off,
                                      const uint32_t *sorted, const uint8_t *bmask,
                                      const float4 *geo, const float4 *app, float *rgb,
                                      float *depth, float *sil, uint32_t *pix_last,
                                      uint32_t *pix_nadd, float *pix_T, uint2 *plist,
                                      int plist_cap, uint32_t *blk_ovf, const Status *st);
__global__ void k_composite_bwd(SecTable T, Camera cam, const uint32_t *tile_off,
                                const uint32_t *sorted, const float4 *geo, const float4 *app,
                                const uint32_t *pix_last, const float *pix_T,
                                const float *g_rgb, const float *g_depth, const float *g_sil,
                                int mode, double *pose_partials, const uint32_t *tile_mask,
                                float4 *acc4, float *accr, float4 *accg, const Status *st);
__global__ void k_composite_bwd_list(SecTable T, Camera cam, const float4 *geo,
                                     const float4 *app, const uint32_t *pix_nadd,
                                     const float *pix_T, const uint2 *plist, int plist_cap,
                                     const uint32_t *blk_ovf, const float *g_rgb,
                                     const float *g_depth, const float *g_sil, int mode,
                                     double *pose_partials, float4 *acc4, float *accr,
                                     float4 *accg, const Status *st);
__global__ void k_composite_bwd_list_pose(SecTable T, Camera cam, const float4 *geo,
                                          const float4 *app, const uint32_t *pix_nadd,
                                          const float *pix_T, const uint2 *plist, int plist_cap,
                                          const uint32_t *blk_ovf, const float *g_rgb,
                                          const float *g_depth, const float *g_sil, int mode,
                                          double *pose_partials, float4 *acc4, float *accr,
                                          float4 *accg, const Status *st);
__global__ void k_composite_bwd_list_posemat(SecTable T, Camera cam, const float4 *geo,
                                             const float4 *app, const uint32_t *pix_nadd,
                                             const float *pix_T, const uint2 *plist,
                                             int plist_cap, const uint32_t *blk_ovf,
                                             const float *g_rgb, const float *g_depth,
                                             const float *g_sil, int mode, double *pose_partials,
                                             float4 *acc4, float *accr, float4 *accg,
                                             const Status *st);
__global__ void k_composite_bwd_list_aniso(SecTable T, Camera cam, const float4 *geo,
                                           const float4 *app, const uint32_t *pix_nadd,
                                           const float *pix_T, const uint2 *plist, int plist_cap,
                                           const uint32_t *blk_ovf, const float *g_rgb,
                                           const float *g_depth, const float *g_sil, int mode,
                                           double *pose_partials, float4 *acc4, float *accr,
                                           float4 *accg, float2 *accm, const Status *st);
__global__ void k_composite_bwd_aniso(SecTable T, Camera cam, const uint32_t *tile_off,
                                      const uint32_t *sorted, const float4 *geo,
                                      const float4 *app, const uint32_t *pix_last,
                                      const float *pix_T, const float *g_rgb,
                                      const float *g_depth, const float *g_sil, int mode,
                                      const uint32_t *tile_mask, float4 *acc4, float4 *accg,
                                      float2 *accm, const Status *st);
// Ellipsoids, per Gaussian: accumulated conic / centre terms -> scale,
// quaternion and FP64 pose partials (one per block).
__global__ void k_aniso_chain(SecTable T, Camera cam, const ViewXf *views, const float4 *geo,
                              const float4 *app, const float4 *accg, const float2 *accm,
                              int want_pose, int want_attr, double *pose_partials);
__global__ void k_composite_bwd_list_views(SecTable T, Camera cam, const float4 *geo,
                                           const float4 *app, const uint32_t *pix_nadd,
                                           const float *pix_T, const uint2 *plist, int plist_cap,
                                           const uint32_t *blk_ovf, const float *g_rgb,
                                           const float *g_depth, const float *g_sil, int mode,
                                           double *pose_partials, float4 *acc4, float *accr,
                                           float4 *accg, const Status *st);
constexpr int kViewChunks = 64;   // blocks per source view in k_view_grads
__global__ void k_view_grads(SecTable T, const float4 *accg, const double *pose_copy,
                             double *partials);
__global__ void k_view_finalize(SecTable T, const double *pose_copy, const double *partials,
                                int n_views);
__global__ void k_attr_scatter(SecTable T, const float4 *acc4, const float *accr);

// Batched launches (see BatchTable): one launch per stage over all items.
__global__ void kb_setup(const BatchTable *B, ViewXf *views, TabRow *tab, double *pose_copy,
                         uint32_t *tile_count);
__global__ void kb_preprocess(const BatchTable *B, const ViewXf *views, const TabRow *tab,
                              float4 *geo, float4 *app, uint4 *info, uint32_t *tile_count);
__global__ void kb_scan_tiles(const BatchTable *B, const uint32_t *tile_count, uint32_t *tile_off,
                              uint32_t *tile_cursor, Status *st, unsigned long long cap,
                              uint32_t *long_tiles);
__global__ void kb_emit(const BatchTable *B, const uint4 *info, uint32_t *tile_cursor,
                        unsigned long long *bucket, uint8_t *bmask_u, const Status *st);
#define VT_DECLARE_SORT_B(name)                                                                  \
    __global__ void name(const BatchTable *B, const uint32_t *tile_off,                          \
                         unsigned long long *bucket, unsigned long long *alt,                    \
                         const uint8_t *bmask_u, uint32_t *sorted, uint8_t *bmask,               \
                         const float4 *geo, Status *st, int smem_n, int lo, int hi,      \
                         const uint32_t *long_tiles);
VT_DECLARE_SORT_B(kb_sort_tiles)
VT_DECLARE_SORT_B(kb_sort_tiles_mid)
VT_DECLARE_SORT_B(kb_sort_tiles_large)
VT_DECLARE_SORT_B(kb_sort_tiles_long)
VT_DECLARE_SORT_B(kb_sort_tiles_xl)
#undef VT_DECLARE_SORT_B
__global__ void kb_composite_fwd(const BatchTable *B, uint32_t *ctr, const uint32_t *tile_off,
                                 const uint32_t *sorted, const uint8_t *bmask, const float4 *geo,
                                 const float4 *app, uint32_t *pix_last, uint32_t *pix_nadd,
                                 float *pix_T, uint2 *plist, int plist_cap, uint32_t *blk_ovf,
                                 const Status *st);
__global__ void kb_masked_l1(const BatchTable *B, float *grads, double *l1_part);
__global__ void kb_composite_bwd_list_pose(const BatchTable *B, uint32_t *ctr, const float4 *geo,
                                           const float4 *app, const uint32_t *pix_nadd,
                                           const float *pix_T, const uint2 *plist, int plist_cap,
                                           const uint32_t *blk_ovf, const float *grads,
                                           double *pose_partials, const Status *st);
__global__ void kb_composite_bwd_pose(const BatchTable *B, const uint32_t *tile_off,
                                      const uint32_t *sorted, const float4 *geo,
                                      const float4 *app, const uint32_t *pix_last,
                                      const float *pix_T, const uint32_t *blk_ovf,
                                      const float *grads, double *pose_partials,
                                      const Status *st);
__global__ void kb_finalize(const BatchTable *B, const double *l1_part,
                            const double *pose_partials, const double *pose_copy);

// Loss inputs (vt_loss.cu).
struct VisView {
    const float *depth;
    int W, H;
    float fx, fy, cx, cy;
    const double *pose;
};
struct VisViews {
    int n;
    VisView v[VT_MAX_VIS_VIEWS];
};
__global__ void k_visibility(const float *depth, int W, int H, float fx, float fy, float cx,
                             float cy, const double *pose, VisViews views, double rel_tol,
                             uint8_t *visible);
__global__ void k_visibility_counts(const float *depth, int W, int H, float fx, float fy,
                                    float cx, float cy, const double *pose, VisViews views,
                                    double rel_tol, uint32_t *counts, uint32_t *n_valid);
__global__ void k_masked_l1(int64_t P, const float *rgb, const float *depth, const float *sil,
                            const float *obs_rgb, const float *obs_depth, const uint8_t *visible,
                            float sil_min, int rgb_needs_depth, float gc, float gd, float *d_rgb,
                            float *d_depth, double *partials);
__global__ void k_sum_partials(const double *partials, int n_blocks, double wc, double wd,
                               double *loss);

// Tracking optimiser step (vt_pose.cu).
struct PoseAdamParams {
    double lr[6];
    double beta1, beta2, eps;
};
__global__ void k_pose_adam(double *pose, double *d_twist, double *state, PoseAdamParams prm);

// SSIM term (vt_ssim.cu): the 11 normalised 1-D window weights.
constexpr int kSsimTileW = 32, kSsimTileH = 32;   // SSIM output tile (256 threads)
struct SsimWindow {
    float g[11];
};
__global__ void k_ssim_fwd(int W, int H, const float *x, const float *y, SsimWindow win,
                           float *maps, double *partials);
__global__ void k_ssim_bwd(int W, int H, const float *x, const float *y, SsimWindow win,
                           const float *maps, float scale, float *d_x);

// Mapping optimiser step (vt_pose.cu).
struct AttrAdamParams {
    float lr[5];
    float beta1, beta2, eps;
};
struct ShapeAdamParams {
    float lr_scale, lr_rot, beta1, beta2, eps;
};
__global__ void k_shape_adam(int64_t n, float *theta, float *m, float *v, const double *step,
                             float *d_scale, float *d_rot, int prec, void *scale, void *rot,
                             ShapeAdamParams prm);
__global__ void k_adam_step_count(double *step, double beta1, double beta2);
__global__ void k_attr_adam(int64_t n, float *theta, float *m, float *v, const double *step,
                            float *d_colour, float *d_opacity, float *d_radius, int prec,
                            void *colour, void *opacity, void *radius, AttrAdamParams prm);
__global__ void k_adam_init(int64_t n, int prec, const void *colour, const void *opacity,
                            const void *radius, const void *scale, const void *rot, float *theta,
                            float *m, float *v);
__global__ void k_pose_finalize(const double *partials, int n_parts, const double *pose_copy,
                                double *d_twist, double *d_mat);
__global__ void k_count_valid(const float *depth, int64_t total, uint32_t *block_counts);
__global__ void k_count_yield(const float *depth, int64_t total, const float *sil,
                              float sil_max, uint32_t *block_counts);
__global__ void k_scan_counts(const uint32_t *counts, int64_t n, uint32_t *offs,
                              long long *n_out);
__global__ void k_backproject(const float *depth, int W, int H, vt_intrinsics K,
                              const double *pose12, const uint32_t *offs, float *centres,
                              uint32_t *pix, int64_t cap);
__global__ void k_section_init(const float *depth, const float *rgb, const float *sil,
                               float sil_max, int64_t plane, int64_t total, float fx, int prec,
                               const uint32_t *offs, uint32_t src_base, uint32_t *src,
                               void *colour, void *opacity, void *radius, int64_t cap);

constexpr int kInitBlock = 256;

}  // namespace vt
