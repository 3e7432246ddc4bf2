// SSIM term of Eq. 2 (Sec. 3.4 mapping loss: tau L_S(V, V'), L_S the SSIM
// loss) and its gradient with respect to the rendered colour image.
//
// L_S = 1 - mean SSIM over pixels and channels; SSIM per channel with an
// 11 x 11 Gaussian window (sigma 1.5, zero padding) and C1 = 0.01^2,
// C2 = 0.03^2.  Two kernels over 32 x 8 pixel tiles with a 5-pixel halo
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
constexpr int kSTW = 32, kSTH = 8;            // tile
constexpr int kSRW = kSTW + 2 * kSR, kSRH = kSTH + 2 * kSR;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

// Loads plane[region] (0 outside the image) into dst.
__device__ __forceinline__ void load_region(float (*dst)[kSRW], const float *plane, int W, int H,
                                            int ox, int oy) {
    for (int i = threadIdx.x; i < kSRH * kSRW; i += blockDim.x) {
        const int r = i / kSRW, q = i - r * kSRW;
        const int gx = ox - kSR + q, gy = oy - kSR + r;
        dst[r][q] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? plane[(int64_t)gy * W + gx] : 0.f;
    }
}

__global__ void __launch_bounds__(256) k_ssim_fwd(int W, int H, const float *x, const float *y,
                                                  SsimWindow win, float *maps,
                                                  double *partials) {
    __shared__ float sx[kSRH][kSRW], sy[kSRH][kSRW];
    __shared__ float w2[kSW][kSW];
    __shared__ double red[2][8];
    const int tid = threadIdx.x;
    const int ox = blockIdx.x * kSTW, oy = blockIdx.y * kSTH;
    const int64_t P = (int64_t)W * H;
    const int tx = tid % kSTW, ty = tid / kSTW;
    const int px = ox + tx, py = oy + ty;
    const bool inside = px < W && py < H;
    if (tid < kSW * kSW) w2[tid / kSW][tid % kSW] = win.g[tid / kSW] * win.g[tid % kSW];
    double sum_s = 0.0, cnt = 0.0;
    for (int c = 0; c < 3; ++c) {
        load_region(sx, x + c * P, W, H, ox, oy);
        load_region(sy, y + c * P, W, H, ox, oy);
        __syncthreads();
        const float a = sx[ty + kSR][tx + kSR], b = sy[ty + kSR][tx + kSR];
        float su = 0.f, sv = 0.f, suu = 0.f, svv = 0.f, suv = 0.f;
        for (int dy = 0; dy < kSW; ++dy) {
#pragma unroll
            for (int dx = 0; dx < kSW; ++dx) {
                const float w = w2[dy][dx];
                const float u = sx[ty + dy][tx + dx] - a, v = sy[ty + dy][tx + dx] - b;
                const float wu = w * u, wv = w * v;
                su += wu;
                sv += wv;
                suu = fmaf(wu, u, suu);
                svv = fmaf(wv, v, svv);
                suv = fmaf(wu, v, suv);
            }
        }
        if (inside) {
            const float s_x = suu - su * su, s_y = svv - sv * sv, s_xy = suv - su * sv;
            const float mu_x = a + su, mu_y = b + sv;
            const float A = 2.f * mu_x * mu_y + kC1, B = 2.f * s_xy + kC2;
            const float Cm = mu_x * mu_x + mu_y * mu_y + kC1, D = s_x + s_y + kC2;
            const float icd = 1.f / (Cm * D);
            const float S = A * B * icd;
            const int64_t p = (int64_t)py * W + px;
            float *mp = maps + c * P + p;
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
    const int tx = tid % kSTW, ty = tid / kSTW;
    const int px = ox + tx, py = oy + ty;
    const bool inside = px < W && py < H;
    const int64_t pc = inside ? (int64_t)py * W + px : 0;
    if (tid < kSW * kSW) w2[tid / kSW][tid % kSW] = win.g[tid / kSW] * win.g[tid % kSW];
    for (int c = 0; c < 3; ++c) {
        const float *mc = maps + c * P;
        load_region(sm_mu, mc, W, H, ox, oy);
        load_region(sm_s, mc + 3 * P, W, H, ox, oy);
        load_region(sm_c, mc + 6 * P, W, H, ox, oy);
        load_region(sm_mx, mc + 9 * P, W, H, ox, oy);
        load_region(sm_my, mc + 12 * P, W, H, ox, oy);
        __syncthreads();
        const float xq = inside ? x[c * P + pc] : 0.f, yq = inside ? y[c * P + pc] : 0.f;
        float g = 0.f;
        for (int dy = 0; dy < kSW; ++dy) {
#pragma unroll
            for (int dx = 0; dx < kSW; ++dx) {
                const int r = ty + dy, q = tx + dx;
                const float t = sm_mu[r][q] + 2.f * sm_s[r][q] * (xq - sm_mx[r][q]) +
                                sm_c[r][q] * (yq - sm_my[r][q]);
                g = fmaf(w2[dy][dx], t, g);
            }
        }
        if (inside) d_x[c * P + pc] += scale * g;
        __syncthreads();
    }
}

}  // namespace vt
