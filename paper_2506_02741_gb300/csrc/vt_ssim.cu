// SSIM term of Eq. 2 (Sec. 3.4 mapping loss: tau L_S(V, V'), L_S the SSIM
// loss) and its gradient with respect to the rendered colour image.
//
// L_S = 1 - mean SSIM over pixels and channels; SSIM per channel with an
// 11 x 11 Gaussian window (sigma 1.5, zero padding) and C1 = 0.01^2,
// C2 = 0.03^2.  Two kernels over 32 x 32 pixel tiles with a 5-pixel halo
// staged in shared memory, each evaluating the 121-tap window directly:
//   k_ssim_fwd: the five local moments, the SSIM map and its partial
//     derivatives S_mu, S_s, S_c (stored with mu_x, mu_y per pixel), and
//     per-block FP64 sums of SSIM for the loss;
//   k_ssim_bwd: dSSIM/dx(q) = sum_p G(p - q) [S_mu(p) + 2 S_s(p) (x(q) -
//     mu_x(p)) + S_c(p) (y(q) - mu_y(p))], scaled into the caller's gradient.
// The window is not split into two 1-D passes on purpose: around every
// output pixel the moments are taken of x - x(q) and y - y(q), and the
// gradient terms of x(q) - mu_x(p), so that no sum cancels (E[x^2] - mu^2 and
// the two halves of the gradient cancel to ~1e-3 in FP32 on smooth patches
// next to edges when a whole tile shares one reference value).
#include "vt_common.cuh"

namespace vt {

constexpr int kSR = 5;                        // window radius
constexpr int kSW = 2 * kSR + 1;              // window width
constexpr int kSTW = kSsimTileW, kSTH = kSsimTileH;
constexpr int kRows = kSTH / 8;               // output rows per thread (8 threads per column)
constexpr int kSRW = kSTW + 2 * kSR, kSRH = kSTH + 2 * kSR;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;
static_assert(kSTW == 32 && kSTH % 8 == 0, "one warp per tile row band of 32 columns");

// Loads plane[region] (0 outside the image) into dst.
__device__ __forceinline__ void load_region(float (*dst)[kSRW], const float *plane, int W, int H,
                                            int ox, int oy) {
    for (int i = threadIdx.x; i < kSRH * kSRW; i += blockDim.x) {
        const int r = i / kSRW, q = i - r * kSRW;
        const int gx = ox - kSR + q, gy = oy - kSR + r;
        dst[r][q] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? plane[(int64_t)gy * W + gx] : 0.f;
    }
}

// Each thread evaluates kRows vertically adjacent pixels of its column: a
// staged value at window row rr serves every output k with 0 <= rr - k <
// 11, so each output still visits its 121 taps row by row in the same order
// while the shared-memory loads are shared.
__global__ void __launch_bounds__(256, 3) k_ssim_fwd(int W, int H, const float *x, const float *y,
                                                  SsimWindow win, float *maps,
                                                  double *partials) {
    __shared__ float sx[kSRH][kSRW], sy[kSRH][kSRW];
    __shared__ float w2[kSW][kSW];
    __shared__ double red[2][8];
    const int tid = threadIdx.x;
    const int ox = blockIdx.x * kSTW, oy = blockIdx.y * kSTH;
    const int64_t P = (int64_t)W * H;
    const int tx = tid % kSTW, y0 = (tid / kSTW) * kRows;
    const int px = ox + tx;
    if (tid < kSW * kSW) w2[tid / kSW][tid % kSW] = win.g[tid / kSW] * win.g[tid % kSW];
    double sum_s = 0.0, cnt = 0.0;
    for (int c = 0; c < 3; ++c) {
        load_region(sx, x + c * P, W, H, ox, oy);
        load_region(sy, y + c * P, W, H, ox, oy);
        __syncthreads();
        float a[kRows], b[kRows], su[kRows], sv[kRows], suu[kRows], svv[kRows], suv[kRows];
#pragma unroll
        for (int k = 0; k < kRows; ++k) {
            a[k] = sx[y0 + k + kSR][tx + kSR];
            b[k] = sy[y0 + k + kSR][tx + kSR];
            su[k] = sv[k] = suu[k] = svv[k] = suv[k] = 0.f;
        }
#pragma unroll
        for (int rr = 0; rr < kSW + kRows - 1; ++rr) {
#pragma unroll
            for (int dx = 0; dx < kSW; ++dx) {
                const float xv = sx[y0 + rr][tx + dx], yv = sy[y0 + rr][tx + dx];
#pragma unroll
                for (int k = 0; k < kRows; ++k) {
                    const int dy = rr - k;
                    if (dy < 0 || dy >= kSW) continue;
                    const float w = w2[dy][dx];
                    const float u = xv - a[k], v = yv - b[k];
                    const float wu = w * u, wv = w * v;
                    su[k] += wu;
                    sv[k] += wv;
                    suu[k] = fmaf(wu, u, suu[k]);
                    svv[k] = fmaf(wv, v, svv[k]);
                    suv[k] = fmaf(wu, v, suv[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kRows; ++k) {
            const int py = oy + y0 + k;
            if (px >= W || py >= H) continue;
            const float s_x = suu[k] - su[k] * su[k], s_y = svv[k] - sv[k] * sv[k];
            const float s_xy = suv[k] - su[k] * sv[k];
            const float mu_x = a[k] + su[k], mu_y = b[k] + sv[k];
            const float A = 2.f * mu_x * mu_y + kC1, B = 2.f * s_xy + kC2;
            const float Cm = mu_x * mu_x + mu_y * mu_y + kC1, D = s_x + s_y + kC2;
            const float icd = 1.f / (Cm * D);
            const float S = A * B * icd;
            float *mp = maps + c * P + (int64_t)py * W + px;
            mp[0 * 3 * P] = 2.f * mu_y * B * icd - 2.f * mu_x * S / Cm;   // S_mu
            mp[1 * 3 * P] = -S / D;                                         // S_s
            mp[2 * 3 * P] = 2.f * A * icd;                                  // S_c
            mp[3 * 3 * P] = mu_x;
            mp[4 * 3 * P] = mu_y;
            sum_s += (double)S;
            cnt += 1.0;
        }
        __syncthreads();   // shared memory is reused by the next channel
    }
    if (!partials) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum_s += __shfl_xor_sync(0xffffffffu, sum_s, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = sum_s;
        red[1][tid >> 5] = cnt;
    }
    __syncthreads();
    if (tid < 2) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[tid][w];
        const int b = blockIdx.y * gridDim.x + blockIdx.x;
        partials[2 * b + tid] = t;
    }
}

__global__ void __launch_bounds__(256) k_ssim_bwd(int W, int H, const float *x, const float *y,
                                                  SsimWindow win, const float *maps, float scale,
                                                  float *d_x) {
    __shared__ float sm_mu[kSRH][kSRW], sm_s[kSRH][kSRW], sm_c[kSRH][kSRW];
    __shared__ float sm_mx[kSRH][kSRW], sm_my[kSRH][kSRW];
    __shared__ float w2[kSW][kSW];
    const int tid = threadIdx.x;
    const int ox = blockIdx.x * kSTW, oy = blockIdx.y * kSTH;
    const int64_t P = (int64_t)W * H;
    const int tx = tid % kSTW, y0 = (tid / kSTW) * kRows;
    const int px = ox + tx;
    if (tid < kSW * kSW) w2[tid / kSW][tid % kSW] = win.g[tid / kSW] * win.g[tid % kSW];
    for (int c = 0; c < 3; ++c) {
        const float *mc = maps + c * P;
        load_region(sm_mu, mc, W, H, ox, oy);
        load_region(sm_s, mc + 3 * P, W, H, ox, oy);
        load_region(sm_c, mc + 6 * P, W, H, ox, oy);
        load_region(sm_mx, mc + 9 * P, W, H, ox, oy);
        load_region(sm_my, mc + 12 * P, W, H, ox, oy);
        __syncthreads();
        float xq[kRows], yq[kRows], g[kRows];
#pragma unroll
        for (int k = 0; k < kRows; ++k) {
            const int py = oy + y0 + k;
            const bool inside = px < W && py < H;
            const int64_t pc = inside ? (int64_t)py * W + px : 0;
            xq[k] = inside ? x[c * P + pc] : 0.f;
            yq[k] = inside ? y[c * P + pc] : 0.f;
            g[k] = 0.f;
        }
#pragma unroll
        for (int rr = 0; rr < kSW + kRows - 1; ++rr) {
#pragma unroll
            for (int dx = 0; dx < kSW; ++dx) {
                const int r = y0 + rr, q = tx + dx;
                const float mu = sm_mu[r][q], ss = sm_s[r][q], sc = sm_c[r][q];
                const float mx = sm_mx[r][q], my = sm_my[r][q];
#pragma unroll
                for (int k = 0; k < kRows; ++k) {
                    const int dy = rr - k;
                    if (dy < 0 || dy >= kSW) continue;
                    const float t = mu + 2.f * ss * (xq[k] - mx) + sc * (yq[k] - my);
                    g[k] = fmaf(w2[dy][dx], t, g[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kRows; ++k) {
            const int py = oy + y0 + k;
            if (px < W && py < H) d_x[c * P + (int64_t)py * W + px] += scale * g[k];
        }
        __syncthreads();
    }
}

}  // namespace vt
