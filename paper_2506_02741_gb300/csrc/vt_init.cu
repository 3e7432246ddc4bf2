// Section building (Sec. 3.2): ordered compaction of the valid depth pixels
// of one or more views into Gaussians, and the back-projection of depth maps
// into world centres.  Three launches: per-block counts, one-block scan,
// per-block ordered write.
#include "vt_common.cuh"

namespace vt {

constexpr unsigned kAll = 0xffffffffu;

__device__ __forceinline__ bool depth_ok(float d) { return isfinite(d) && d > 0.f; }

// Rank of this thread among the valid threads of its block (block order).
__device__ __forceinline__ uint32_t block_rank(bool valid) {
    __shared__ uint32_t wc[kInitBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned b = __ballot_sync(kAll, valid);
    if (lane == 0) wc[warp] = __popc(b);
    __syncthreads();
    uint32_t base = 0;
    for (int w = 0; w < warp; ++w) base += wc[w];
    return base + __popc(b & ((1u << lane) - 1u));
}

// A pixel yields a Gaussian when its depth is valid and, when a silhouette is
// given (complement initialisation, Sec. 3.4), the current render leaves it
// uncovered (silhouette < sil_max).
__device__ __forceinline__ bool yields(const float *depth, const float *sil, float sil_max,
                                       int64_t i, float &D) {
    D = depth[i];
    return depth_ok(D) && (sil == nullptr || sil[i] < sil_max);
}

__global__ void __launch_bounds__(kInitBlock) k_count_valid(const float *depth, int64_t total,
                                                            uint32_t *block_counts) {
    const int64_t i = (int64_t)blockIdx.x * kInitBlock + threadIdx.x;
    const bool v = i < total && depth_ok(depth[i]);
    const int n = __syncthreads_count(v);
    if (threadIdx.x == 0) block_counts[blockIdx.x] = (uint32_t)n;
}

// Per-block counts of the pixels that yield a Gaussian (valid depth and, with
// a silhouette, uncovered).
__global__ void __launch_bounds__(kInitBlock) k_count_yield(const float *depth, int64_t total,
                                                            const float *sil, float sil_max,
                                                            uint32_t *block_counts) {
    const int64_t i = (int64_t)blockIdx.x * kInitBlock + threadIdx.x;
    float D;
    const bool v = i < total && yields(depth, sil, sil_max, i, D);
    const int n = __syncthreads_count(v);
    if (threadIdx.x == 0) block_counts[blockIdx.x] = (uint32_t)n;
}

__global__ void __launch_bounds__(1024) k_scan_counts(const uint32_t *counts, int64_t n,
                                                      uint32_t *offs, long long *n_out) {
    __shared__ unsigned long long ws[32];
    __shared__ unsigned long long carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t i = base + tid;
        const unsigned long long c = i < n ? counts[i] : 0ull;
        unsigned long long x = c;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kAll, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = ws[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(kAll, w, o);
                if (lane >= o) w += y;
            }
            ws[lane] = w;
        }
        __syncthreads();
        const unsigned long long excl = carry + (warp ? ws[warp - 1] : 0ull) + x - c;
        if (i < n) offs[i] = (uint32_t)excl;
        __syncthreads();
        if (tid == 1023) carry = excl + c;
        __syncthreads();
    }
    if (tid == 0 && n_out) *n_out = (long long)carry;
}

// mu = R (D ((u - cx)/fx, (v - cy)/fy, 1)) + t for every valid pixel, in
// raster order, computed in FP64 and stored as float32.
__global__ void __launch_bounds__(kInitBlock) k_backproject(const float *depth, int W, int H,
                                                            vt_intrinsics K,
                                                            const double *pose12,
                                                            const uint32_t *offs, float *centres,
                                                            uint32_t *pix, int64_t cap) {
    const int64_t i = (int64_t)blockIdx.x * kInitBlock + threadIdx.x;
    const int64_t total = (int64_t)W * H;
    const float D = i < total ? depth[i] : 0.f;
    const bool v = i < total && depth_ok(D);
    const int64_t pos = (int64_t)offs[blockIdx.x] + block_rank(v);
    if (!v || pos >= cap) return;
    const int u = (int)(i % W), vv = (int)(i / W);
    const double Xc = (double)D * (((double)u - K.cx) / K.fx);
    const double Yc = (double)D * (((double)vv - K.cy) / K.fy);
    const double Zc = (double)D;
    const double *R = pose12, *t = pose12 + 9;
    for (int a = 0; a < 3; ++a)
        centres[3 * pos + a] = (float)(R[3 * a] * Xc + R[3 * a + 1] * Yc + R[3 * a + 2] * Zc + t[a]);
    pix[pos] = (uint32_t)i;
}

// One Gaussian per yielding pixel of all views, in (view, pixel) order:
// colour = V(u, v), opacity = 0.9, radius = D / fx; src = src_base + index.
__global__ void __launch_bounds__(kInitBlock) k_section_init(
    const float *depth, const float *rgb, const float *sil, float sil_max, int64_t plane,
    int64_t total, float fx, int prec, const uint32_t *offs, uint32_t src_base, uint32_t *src,
    void *colour, void *opacity, void *radius, int64_t cap) {
    const int64_t i = (int64_t)blockIdx.x * kInitBlock + threadIdx.x;
    float D = 0.f;
    const bool v = i < total && yields(depth, sil, sil_max, i, D);
    const int64_t pos = (int64_t)offs[blockIdx.x] + block_rank(v);
    if (!v || pos >= cap) return;
    const int64_t view = i / plane, p = i - view * plane;
    const float r = __fdiv_rn(D, fx);
    src[pos] = src_base + (uint32_t)i;
    for (int ch = 0; ch < 3; ++ch) {
        const float c = rgb[(view * 3 + ch) * plane + p];
        if (prec == VT_F16)
            reinterpret_cast<__half *>(colour)[3 * pos + ch] = __float2half_rn(c);
        else
            reinterpret_cast<float *>(colour)[3 * pos + ch] = c;
    }
    if (prec == VT_F16) {
        reinterpret_cast<__half *>(opacity)[pos] = __float2half_rn(0.9f);
        reinterpret_cast<__half *>(radius)[pos] = __float2half_rn(r);
    } else {
        reinterpret_cast<float *>(opacity)[pos] = 0.9f;
        reinterpret_cast<float *>(radius)[pos] = r;
    }
}

}  // namespace vt
