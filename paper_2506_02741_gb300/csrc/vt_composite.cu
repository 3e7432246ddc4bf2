// Per-tile front-to-back compositing (forward) and its back-to-front replay
// (backward).  One block of 256 threads per 16x16 tile, one thread per pixel;
// warp w owns the 8x4 pixel block ((w & 1) * 8, (w >> 1) * 4) of the tile.
// Gaussians of the tile's depth-sorted list are staged in shared memory in
// batches of 256; before evaluating a Gaussian for its 32 pixels a warp
// checks, one Gaussian per lane, whether the Gaussian's 3-sigma disc touches
// its 8x4 block, and only visits the ones that do.  sm_103a; no tensor cores.
#include "vt_common.cuh"

namespace vt {

constexpr unsigned kFullMask = 0xffffffffu;

// Conservative test: does the disc q <= 9 of a Gaussian (centre iu + fu,
// iv + fv, coefficients kx, ky) touch the pixel rectangle [x0,x1] x [y0,y1]?
// The distance is shrunk by 1e-3 px so that rounding of the float centre
// never drops a pixel the exact per-pixel test would include.
__device__ __forceinline__ bool disc_touches(const float4 &g0, const float4 &g1, float x0, float x1,
                                             float y0, float y1) {
    const float uc = (float)__float_as_int(g0.x) + g0.y;
    const float vc = (float)__float_as_int(g0.z) + g0.w;
    const float dx = fmaxf(fmaxf(x0 - uc, uc - x1) - 1e-3f, 0.f);
    const float dy = fmaxf(fmaxf(y0 - vc, vc - y1) - 1e-3f, 0.f);
    return dx * dx * g1.x + dy * dy * g1.y <= kQMax;
}

__global__ void __launch_bounds__(kBlockPix) k_composite_fwd(
    Camera cam, const uint32_t *tile_off, const uint32_t *sorted, const float4 *geo,
    const float4 *app, float *rgb, float *depth, float *sil, uint32_t *pix_last,
    uint32_t *pix_nadd, float *pix_T, const Status *st) {
    __shared__ float4 s_g0[kBatch], s_g1[kBatch], s_a[kBatch];
    if (st->flags) return;
    const int tile = blockIdx.x;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx0 = tx * kTile + (warp & 1) * 8, by0 = ty * kTile + (warp >> 1) * 4;
    const int px = bx0 + (lane & 7), py = by0 + (lane >> 3);
    const bool inside = px < cam.W && py < cam.H;
    const float rx0 = (float)bx0, rx1 = (float)min(bx0 + 7, cam.W - 1);
    const float ry0 = (float)by0, ry1 = (float)min(by0 + 3, cam.H - 1);
    const uint32_t start = tile_off[tile], end = tile_off[tile + 1];

    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, dd = 0.f, ss = 0.f;
    uint32_t last = 0, nadd = 0;
    bool done = !inside;
    for (uint32_t b0 = start; b0 < end; b0 += kBatch) {
        if (__syncthreads_and(done)) break;
        const uint32_t i = b0 + threadIdx.x;
        if (i < end) {
            const uint32_t g = sorted[i];
            s_g0[threadIdx.x] = geo[2 * (size_t)g];
            s_g1[threadIdx.x] = geo[2 * (size_t)g + 1];
            s_a[threadIdx.x] = app[g];
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)kBatch, end - b0);
        bool wdone = __all_sync(kFullMask, done);
        for (int j0 = 0; j0 < nb && !wdone; j0 += 32) {
            const int jj = j0 + lane;
            bool rel = false;
            if (jj < nb) rel = disc_touches(s_g0[jj], s_g1[jj], rx0, rx1, ry0, ry1);
            unsigned mask = __ballot_sync(kFullMask, rel);
            while (mask) {
                const int j = j0 + __ffs(mask) - 1;
                mask &= mask - 1;
                if (done) continue;
                const float4 g0 = s_g0[j], g1 = s_g1[j];
                float du, dv;
                const float q = pair_q(px, py, g0, g1, du, dv);
                if (!(q <= kQMax)) continue;
                const float ah = __fmul_rn(g1.w, pair_gauss(q));
                if (!(ah >= kAlphaMin)) continue;
                const float al = fminf(ah, kAlphaClamp);
                const float Tn = __fmul_rn(T, __fsub_rn(1.f, al));
                if (Tn < kTMin) {
                    done = true;
                    continue;
                }
                const float w = __fmul_rn(al, T);
                const float4 a = s_a[j];
                c0 = __fmaf_rn(w, a.x, c0);
                c1 = __fmaf_rn(w, a.y, c1);
                c2 = __fmaf_rn(w, a.z, c2);
                dd = __fmaf_rn(w, g1.z, dd);
                ss = __fadd_rn(ss, w);
                T = Tn;
                last = b0 - start + (uint32_t)j + 1u;
                ++nadd;
            }
            wdone = __all_sync(kFullMask, done);
        }
        __syncthreads();
    }
    if (inside) {
        const size_t p = (size_t)py * cam.W + px, HW = (size_t)cam.W * cam.H;
        if (rgb) {
            rgb[p] = c0;
            rgb[HW + p] = c1;
            rgb[2 * HW + p] = c2;
        }
        if (depth) depth[p] = dd;
        if (sil) sil[p] = ss;
        pix_last[p] = last;
        pix_nadd[p] = nadd;
        pix_T[p] = T;
    }
}

// ---------------------------------------------------------------------------
// Backward.  For a pixel with upstream gradients (gC, gD, gS), walking its
// added Gaussians from the last one forward with T_i = T_{i+1} / (1 - alpha_i)
// and the sums A, B of w c and w z behind the current one:
//   dL/dc_i     = gC w_i
//   dL/dalpha_i = T_i (gC.c_i + gD z_i) - (gC.A + gD B - gS T_final) / (1 - alpha_i)
// Evaluated as written in FP32, T_i z_i and B / (1 - alpha_i) cancel almost
// completely when the Gaussians lie on one surface (depths agree to ~1e-3),
// so the sums are kept relative to the pixel's last added Gaussian (c_r, z_r):
// with S = sum_{j>i} w_j, A' = sum w_j (c_j - c_r), B' = sum w_j (z_j - z_r)
// and T_{i+1} = S + T_final the same derivative is
//   [gC.(c_i T_final + (c_i - c_r) S - A') + gD (z_i T_final + (z_i - z_r) S - B')
//    + gS T_final] / (1 - alpha_i),
// whose terms are all of the size of the result.
//   below the clamp: dL/do = dL/dalpha exp(-q/2),  dL/dq = -ahat/2 dL/dalpha
//   dL/dr = dL/dq (-2q/r)
//   camera-space centre: with e = (p_x z - x, p_y z - y) = z (du/fx, dv/fy),
//   dq/dx = -2 e_x / r^2, dq/dy = -2 e_y / r^2, dq/dz = 2 (p_x e_x + p_y e_y) / r^2,
//   plus the direct depth term dL/dz += gD w_i.
// Colour/opacity/radius gradients are summed over the warp with shuffles and
// added to the section's buffers with one float atomic per value; the pose
// needs only A = sum x g^T and s = sum g, kept per lane in FP32, summed over
// the warp and the block in FP64 and written as one partial per tile.

struct PoseAcc {
    float a[12];  // a[3*i + j] = sum x_i g_j ; a[9 + j] = sum g_j
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
    return v;
}

__global__ void __launch_bounds__(kBlockPix) k_composite_bwd(
    SecTable Tab, Camera cam, const uint32_t *tile_off, const uint32_t *sorted, const float4 *geo,
    const float4 *app, const uint32_t *pix_last, const float *pix_T, const float *g_rgb,
    const float *g_depth, const float *g_sil, int mode, double *pose_partials, const Status *st) {
    __shared__ float4 s_g0[kBatch], s_g1[kBatch], s_a[kBatch];
    __shared__ float2 s_xy[kBatch];
    __shared__ uint32_t s_gid[kBatch];
    __shared__ double s_pose[kBlockPix / 32][12];
    __shared__ uint32_t s_last;
    if (st->flags) return;
    const int tile = blockIdx.x;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx0 = tx * kTile + (warp & 1) * 8, by0 = ty * kTile + (warp >> 1) * 4;
    const int px = bx0 + (lane & 7), py = by0 + (lane >> 3);
    const bool inside = px < cam.W && py < cam.H;
    const float rx0 = (float)bx0, rx1 = (float)min(bx0 + 7, cam.W - 1);
    const float ry0 = (float)by0, ry1 = (float)min(by0 + 3, cam.H - 1);
    const uint32_t start = tile_off[tile];
    const bool want_attr = (mode & VT_GRAD_ATTR) != 0, want_pose = (mode & VT_GRAD_POSE) != 0;

    const size_t HW = (size_t)cam.W * cam.H;
    const size_t p = inside ? (size_t)py * cam.W + px : 0;
    uint32_t my_last = inside ? pix_last[p] : 0u;
    const float Tfin = inside ? pix_T[p] : 1.f;
    float gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gD = 0.f, gS = 0.f;
    if (inside) {
        if (g_rgb) {
            gC0 = g_rgb[p];
            gC1 = g_rgb[HW + p];
            gC2 = g_rgb[2 * HW + p];
        }
        if (g_depth) gD = g_depth[p];
        if (g_sil) gS = g_sil[p];
    }
    if (gC0 == 0.f && gC1 == 0.f && gC2 == 0.f && gD == 0.f && gS == 0.f) my_last = 0;
    const float pxn = ((float)px - cam.cx) / cam.fx, pyn = ((float)py - cam.cy) / cam.fy;
    const float ifx = 1.f / cam.fx, ify = 1.f / cam.fy;

    if (threadIdx.x == 0) s_last = 0;
    __syncthreads();
    const uint32_t wl = __reduce_max_sync(kFullMask, my_last);
    if (lane == 0 && wl) atomicMax(&s_last, wl);
    __syncthreads();
    const uint32_t tile_last = s_last;

    float T = Tfin, A0 = 0.f, A1 = 0.f, A2 = 0.f, Bd = 0.f, Sb = 0.f;
    float cr0 = 0.f, cr1 = 0.f, cr2 = 0.f, zr = 0.f;
    bool have_ref = false;
    PoseAcc acc;
#pragma unroll
    for (int i = 0; i < 12; ++i) acc.a[i] = 0.f;

    if (tile_last > 0) {
        for (int b0 = (int)((tile_last - 1) / kBatch) * kBatch; b0 >= 0; b0 -= kBatch) {
            const int nb = (int)min((uint32_t)kBatch, tile_last - (uint32_t)b0);
            if ((int)threadIdx.x < nb) {
                const uint32_t g = sorted[start + b0 + threadIdx.x];
                const float4 g0 = geo[2 * (size_t)g], g1 = geo[2 * (size_t)g + 1];
                s_g0[threadIdx.x] = g0;
                s_g1[threadIdx.x] = g1;
                s_a[threadIdx.x] = app[g];
                s_gid[threadIdx.x] = g;
                const float uc = (float)__float_as_int(g0.x) + g0.y;
                const float vc = (float)__float_as_int(g0.z) + g0.w;
                s_xy[threadIdx.x] = make_float2(g1.z * (uc - cam.cx) * ifx,
                                                g1.z * (vc - cam.cy) * ify);
            }
            __syncthreads();
            if (wl > (uint32_t)b0) {
                for (int j0 = ((nb - 1) >> 5) << 5; j0 >= 0; j0 -= 32) {
                    const int jj = j0 + lane;
                    bool rel = false;
                    if (jj < nb && (uint32_t)(b0 + jj) < wl)
                        rel = disc_touches(s_g0[jj], s_g1[jj], rx0, rx1, ry0, ry1);
                    unsigned mask = __ballot_sync(kFullMask, rel);
                    while (mask) {
                        const int bit = 31 - __clz(mask);
                        mask &= ~(1u << bit);
                        const int j = j0 + bit;
                        const uint32_t idx = (uint32_t)(b0 + j);
                        float dc0 = 0.f, dc1 = 0.f, dc2 = 0.f, dop = 0.f, drd = 0.f;
                        bool contrib = false;
                        if (idx < my_last) {
                            const float4 g0 = s_g0[j], g1 = s_g1[j];
                            float du, dv;
                            const float q = pair_q(px, py, g0, g1, du, dv);
                            if (q <= kQMax) {
                                const float G = pair_gauss(q);
                                const float ah = __fmul_rn(g1.w, G);
                                if (ah >= kAlphaMin) {
                                    contrib = true;
                                    const float al = fminf(ah, kAlphaClamp);
                                    const float om = 1.f - al;
                                    const float Ti = T / om;
                                    const float w = al * Ti;
                                    const float4 a = s_a[j];
                                    const float z = g1.z, r = a.w;
                                    if (!have_ref) {
                                        have_ref = true;
                                        cr0 = a.x;
                                        cr1 = a.y;
                                        cr2 = a.z;
                                        zr = z;
                                    }
                                    const float e0 = a.x - cr0, e1 = a.y - cr1, e2 = a.z - cr2,
                                                ez = z - zr;
                                    const float num =
                                        gC0 * (a.x * Tfin + e0 * Sb - A0) +
                                        gC1 * (a.y * Tfin + e1 * Sb - A1) +
                                        gC2 * (a.z * Tfin + e2 * Sb - A2) +
                                        gD * (z * Tfin + ez * Sb - Bd) + gS * Tfin;
                                    const float dal = num / om;
                                    dc0 = gC0 * w;
                                    dc1 = gC1 * w;
                                    dc2 = gC2 * w;
                                    float dq = 0.f;
                                    if (ah < kAlphaClamp) {
                                        dop = dal * G;
                                        dq = -0.5f * ah * dal;
                                    }
                                    drd = dq * (-2.f * q / r);
                                    if (want_pose) {
                                        const float ir2 = 1.f / (r * r);
                                        const float ex = z * du * ifx, ey = z * dv * ify;
                                        const float gx = dq * (-2.f * ex * ir2);
                                        const float gy = dq * (-2.f * ey * ir2);
                                        const float gz =
                                            dq * (2.f * (pxn * ex + pyn * ey) * ir2) + gD * w;
                                        const float2 xy = s_xy[j];
                                        const float X[3] = {xy.x, xy.y, z}, Gv[3] = {gx, gy, gz};
#pragma unroll
                                        for (int a_ = 0; a_ < 3; ++a_)
#pragma unroll
                                            for (int b_ = 0; b_ < 3; ++b_)
                                                acc.a[3 * a_ + b_] =
                                                    __fmaf_rn(X[a_], Gv[b_], acc.a[3 * a_ + b_]);
                                        acc.a[9] += gx;
                                        acc.a[10] += gy;
                                        acc.a[11] += gz;
                                    }
                                    A0 = __fmaf_rn(w, e0, A0);
                                    A1 = __fmaf_rn(w, e1, A1);
                                    A2 = __fmaf_rn(w, e2, A2);
                                    Bd = __fmaf_rn(w, ez, Bd);
                                    Sb += w;
                                    T = Ti;
                                }
                            }
                        }
                        if (want_attr && __any_sync(kFullMask, contrib)) {
                            dc0 = warp_sum(dc0);
                            dc1 = warp_sum(dc1);
                            dc2 = warp_sum(dc2);
                            dop = warp_sum(dop);
                            drd = warp_sum(drd);
                            if (lane == 0) {
                                const int64_t g = s_gid[j];
                                const int s = find_section(Tab, g);
                                const SecDesc &S = Tab.s[s];
                                const int64_t li = g - S.gbase;
                                if (S.d_colour) {
                                    atomicAdd(S.d_colour + 3 * li + 0, dc0);
                                    atomicAdd(S.d_colour + 3 * li + 1, dc1);
                                    atomicAdd(S.d_colour + 3 * li + 2, dc2);
                                }
                                if (S.d_opacity) atomicAdd(S.d_opacity + li, dop);
                                if (S.d_radius) atomicAdd(S.d_radius + li, drd);
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    if (want_pose) {
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            const double v = warp_sum_d((double)acc.a[i]);
            if (lane == 0) s_pose[warp][i] = v;
        }
        __syncthreads();
        if (threadIdx.x < 12) {
            double v = 0.0;
            for (int w = 0; w < kBlockPix / 32; ++w) v += s_pose[w][threadIdx.x];
            pose_partials[(size_t)tile * 12 + threadIdx.x] = v;
        }
    }
}

// Fixed-order FP64 sum of the per-tile partials, then
//   twist: dL/drho = -s,  dL/dphi = (A21 - A12, A02 - A20, A10 - A01)
//   matrix: dL/dR = R A,  dL/dt = -R s          (A_ab = sum x_a g_b)
// accumulated (+=) into the outputs.
__global__ void __launch_bounds__(384) k_pose_finalize(const double *partials, int n_parts,
                                                       const double *pose_copy, double *d_twist,
                                                       double *d_mat) {
    __shared__ double tot[12];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double v = 0.0;
    for (int i = lane; i < n_parts; i += 32) v += partials[(size_t)i * 12 + warp];
    v = warp_sum_d(v);
    if (lane == 0) tot[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double *A = tot, *s = tot + 9, *R = pose_copy;
        if (d_twist) {
            d_twist[0] -= s[0];
            d_twist[1] -= s[1];
            d_twist[2] -= s[2];
            d_twist[3] += A[2 * 3 + 1] - A[1 * 3 + 2];
            d_twist[4] += A[0 * 3 + 2] - A[2 * 3 + 0];
            d_twist[5] += A[1 * 3 + 0] - A[0 * 3 + 1];
        }
        if (d_mat) {
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) {
                    double x = 0.0;
                    for (int c = 0; c < 3; ++c) x += R[b * 3 + c] * A[c * 3 + a];
                    d_mat[b * 3 + a] += x;
                }
            for (int b = 0; b < 3; ++b)
                d_mat[9 + b] -= R[b * 3 + 0] * s[0] + R[b * 3 + 1] * s[1] + R[b * 3 + 2] * s[2];
        }
    }
}

}  // namespace vt
