// Loss inputs of tracking and mapping: the visibility check of Sec. 3.3 and
// the masked L1 terms of Eq. 1 / Eq. 2 with their image gradient, fused into
// one pass over the pixels.  Both kernels are HBM-bound: one thread per pixel,
// coalesced planar loads and stores.
#include "vt_common.cuh"

namespace vt {

__device__ __forceinline__ bool valid_depth(float d) { return isfinite(d) && d > 0.f; }

// FP64 with explicit rounding (no contraction), in the order of the plain
// definition: ((a0 x0 + a1 x1) + a2 x2).
__device__ __forceinline__ double dot3(double a0, double x0, double a1, double x1, double a2,
                                       double x2) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a0, x0), __dmul_rn(a1, x1)), __dmul_rn(a2, x2));
}

// Bilinear depth of view V at (x, y); false outside the image or when one of
// the four neighbours lacks valid depth.
__device__ __forceinline__ bool interp_depth(const VisView &V, double x, double y, double &out) {
    if (!(x >= 0.0 && x <= (double)(V.W - 1) && y >= 0.0 && y <= (double)(V.H - 1)))
        return false;
    const int i0 = (int)floor(x), j0 = (int)floor(y);
    const int i1 = min(i0 + 1, V.W - 1), j1 = min(j0 + 1, V.H - 1);
    const double fx = __dsub_rn(x, (double)i0), fy = __dsub_rn(y, (double)j0);
    const float d00 = V.depth[(size_t)j0 * V.W + i0], d10 = V.depth[(size_t)j0 * V.W + i1];
    const float d01 = V.depth[(size_t)j1 * V.W + i0], d11 = V.depth[(size_t)j1 * V.W + i1];
    if (!valid_depth(d00) || !valid_depth(d10) || !valid_depth(d01) || !valid_depth(d11))
        return false;
    const double gx = __dsub_rn(1.0, fx), gy = __dsub_rn(1.0, fy);
    const double top = __dadd_rn(__dmul_rn((double)d00, gx), __dmul_rn((double)d10, fx));
    const double bot = __dadd_rn(__dmul_rn((double)d01, gx), __dmul_rn((double)d11, fx));
    out = __dadd_rn(__dmul_rn(top, gy), __dmul_rn(bot, fy));
    return true;
}

// World point of pixel p of the current frame (false for invalid depth).
__device__ __forceinline__ bool world_point(const float *depth, int W, int64_t p, float fx,
                                            float fy, float cx, float cy, const double *pose,
                                            double X[3]) {
    const int v = (int)(p / W), u = (int)(p - (int64_t)v * W);
    const float D = depth[p];
    if (!valid_depth(D)) return false;
    const double a = __ddiv_rn(__dsub_rn((double)u, (double)cx), (double)fx);
    const double b = __ddiv_rn(__dsub_rn((double)v, (double)cy), (double)fy);
    const double xc0 = __dmul_rn((double)D, a), xc1 = __dmul_rn((double)D, b), xc2 = (double)D;
#pragma unroll
    for (int i = 0; i < 3; ++i)
        X[i] = __dadd_rn(dot3(pose[3 * i], xc0, pose[3 * i + 1], xc1, pose[3 * i + 2], xc2),
                         pose[9 + i]);
    return true;
}

// Is world point X visible to view V: in front, projecting inside, and within
// rel_tol of the view's interpolated depth.
__device__ __forceinline__ bool visible_to(const VisView &V, const double X[3], double rel_tol) {
    const double *Pk = V.pose;
    const double d0 = __dsub_rn(X[0], Pk[9]), d1 = __dsub_rn(X[1], Pk[10]),
                 d2 = __dsub_rn(X[2], Pk[11]);
    const double x0 = dot3(Pk[0], d0, Pk[3], d1, Pk[6], d2);
    const double x1 = dot3(Pk[1], d0, Pk[4], d1, Pk[7], d2);
    const double x2 = dot3(Pk[2], d0, Pk[5], d1, Pk[8], d2);
    if (!(x2 > 0.0)) return false;
    const double px = __dadd_rn(__dmul_rn((double)V.fx, __ddiv_rn(x0, x2)), (double)V.cx);
    const double py = __dadd_rn(__dmul_rn((double)V.fy, __ddiv_rn(x1, x2)), (double)V.cy);
    double Dk;
    if (!interp_depth(V, px, py, Dk)) return false;
    return fabs(__dsub_rn(x2, Dk)) <= __dmul_rn(rel_tol, Dk);
}

// One thread per pixel of the current frame: back-project with its pose,
// then for each view transform into the view, project, interpolate the
// view's depth and test |z - D~| <= rel_tol D~ (union over views).
__global__ void __launch_bounds__(256) k_visibility(const float *depth, int W, int H, float fx,
                                                    float fy, float cx, float cy,
                                                    const double *pose, VisViews views,
                                                    double rel_tol, uint8_t *visible) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)W * H) return;
    double X[3];
    uint8_t vis = 0;
    if (world_point(depth, W, p, fx, fy, cx, cy, pose, X))
        for (int k = 0; k < views.n && !vis; ++k) vis = visible_to(views.v[k], X, rel_tol);
    visible[p] = vis;
}

// Overlap selection (Sec. 3.3): for every view separately, the number of
// valid pixels of the current frame visible to it (counts[k]), and the
// number of valid pixels (*n_valid).  Warp-aggregated integer atomics.
__global__ void __launch_bounds__(256) k_visibility_counts(const float *depth, int W, int H,
                                                           float fx, float fy, float cx,
                                                           float cy, const double *pose,
                                                           VisViews views, double rel_tol,
                                                           uint32_t *counts, uint32_t *n_valid) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    double X[3];
    const bool ok = p < (int64_t)W * H && world_point(depth, W, p, fx, fy, cx, cy, pose, X);
    const unsigned vb = __ballot_sync(0xffffffffu, ok);
    if (lane == 0 && vb && n_valid) atomicAdd(n_valid, (uint32_t)__popc(vb));
    for (int k = 0; k < views.n; ++k) {
        const unsigned b = __ballot_sync(0xffffffffu, ok && visible_to(views.v[k], X, rel_tol));
        if (lane == 0 && b) atomicAdd(&counts[k], (uint32_t)__popc(b));
    }
}

__device__ __forceinline__ float sign_of(float e) { return e > 0.f ? 1.f : (e < 0.f ? -1.f : 0.f); }

// |a - b| exactly, as a float-float: TwoSum gives a - b = s + e exactly, and
// the rounded difference s carries the sign of the exact one (s = 0 only
// when a = b).  A non-finite input makes the sum non-finite.
__device__ __forceinline__ ff abs_diff(float a, float b) {
    const ff d = ff_two_sum(a, -b);
    return d.hi < 0.f ? ff{-d.hi, -d.lo} : d;
}

__device__ __forceinline__ ff shfl_xor_ff(ff a, int o) {
    return ff{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// One thread per pixel: masks, |residuals| and the gradient of the masked L1
// loss.  The residuals are exact float-floats, summed over the pixel's
// channels and the warp in float-float (non-negative terms: ~2^-47 relative
// per addition) and over the block's eight warps in FP64; per block the two
// sums (colour, depth) go to partials[2 b + i].  FP64 arithmetic is a narrow
// pipe on this part, so no per-pixel step uses it.
// Pixel p of an image of P pixels (one block of 256 threads); the block's
// two sums go to part[0, 1] (if part != NULL).
__device__ __forceinline__ void masked_l1_block(int64_t P, int64_t p, const float *rgb,
                                                const float *depth, const float *sil,
                                                const float *obs_rgb, const float *obs_depth,
                                                const uint8_t *visible, float sil_min,
                                                int rgb_needs_depth, float gc, float gd,
                                                float *d_rgb, float *d_depth, double *part) {
    __shared__ double s_sum[2][8];
    const double *partials = part;
    ff sc{0.f, 0.f}, sd{0.f, 0.f};
    if (p < P) {
        const bool valid = valid_depth(obs_depth[p]);
        const bool covered = !(sil_min >= 0.f) || sil[p] > sil_min;
        const bool vis = visible == nullptr || visible[p] != 0;
        const bool m_d = valid && covered && vis;
        const bool m_c = covered && vis && (!rgb_needs_depth || valid);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float r = rgb[c * P + p], o = obs_rgb[c * P + p];
            if (m_c) sc = ff_add(sc, abs_diff(r, o));
            if (d_rgb) d_rgb[c * P + p] = m_c ? gc * sign_of(r - o) : 0.f;
        }
        const float r = depth[p], o = obs_depth[p];
        if (m_d) sd = abs_diff(r, o);
        if (d_depth) d_depth[p] = m_d ? gd * sign_of(r - o) : 0.f;
    }
    if (!partials) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sc = ff_add(sc, shfl_xor_ff(sc, o));
        sd = ff_add(sd, shfl_xor_ff(sd, o));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_sum[0][warp] = (double)sc.hi + (double)sc.lo;
        s_sum[1][warp] = (double)sd.hi + (double)sd.lo;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += s_sum[threadIdx.x][w];
        part[threadIdx.x] = t;
    }
    __syncthreads();   // s_sum is reused by the block's next pixels
}

__global__ void __launch_bounds__(256) k_masked_l1(int64_t P, const float *rgb, const float *depth,
                                                   const float *sil, const float *obs_rgb,
                                                   const float *obs_depth, const uint8_t *visible,
                                                   float sil_min, int rgb_needs_depth, float gc,
                                                   float gd, float *d_rgb, float *d_depth,
                                                   double *partials) {
    masked_l1_block(P, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, rgb, depth, sil, obs_rgb,
                    obs_depth, visible, sil_min, rgb_needs_depth, gc, gd, d_rgb, d_depth,
                    partials ? partials + 2 * blockIdx.x : nullptr);
}

// Batched form: the pixels of every tracking item in blocks of 256 (an
// item's pixels start at a multiple of 256), Eq. 1 masks and weights of the
// batch, the item's rendered planes from its image and the observed ones
// from obs; the image gradient goes to grads (4 x P from 4 pbase: rgb,
// depth) and the block sums to l1_part[2 b].
__global__ void __launch_bounds__(256) kb_masked_l1(const BatchTable *Bp, float *grads,
                                                    double *l1_part) {
    const BatchTable &B = *Bp;
    ItemCursor cur;
    const auto pstart = [&](int i) { return B.it[i].pbase; };
    for (int64_t b = blockIdx.x; b * 256 < B.n_pix; b += gridDim.x) {
        const BatchItem &I = B.it[cur.at(B, pstart, b * 256)];
        if (!I.track) continue;
        const int64_t P = (int64_t)I.cam.W * I.cam.H;
        const double wc = B.w_rgb / (3.0 * (double)P), wd = B.w_depth / (double)P;
        float *g = grads + 4 * I.pbase;
        masked_l1_block(P, b * 256 + threadIdx.x - I.pbase, I.image, I.image + 3 * P,
                        I.image + 4 * P, I.obs, I.obs + 3 * P, nullptr, B.sil_min,
                        B.rgb_needs_depth, (float)wc, (float)wd, g, g + 3 * P, l1_part + 2 * b);
    }
}

// One block: fixed-order sums of the per-block partials (strided per thread,
// then the warp by shuffles, then the warps in order), then
// L = wc * sum_c + wd * sum_d.
__global__ void __launch_bounds__(256) k_sum_partials(const double *partials, int n_blocks,
                                                      double wc, double wd, double *loss) {
    __shared__ double s[2][8];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n_blocks; i += blockDim.x) {
        a += partials[2 * i];
        b += partials[2 * i + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s[0][warp] = a;
        s[1][warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, B = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            A += s[0][w];
            B += s[1][w];
        }
        *loss = __dadd_rn(__dmul_rn(wc, A), __dmul_rn(wd, B));
    }
}

}  // namespace vt
