// Front-to-back compositing (forward) and its back-to-front replay
// (backward).  The image is cut into 16x16 tiles and each tile into eight 8x4
// pixel blocks, one warp and one pixel per lane each; block w of a tile has
// its origin at ((w & 1) * 8, (w >> 1) * 4).  A warp walks the depth-sorted
// list of its tile; before evaluating a Gaussian for its 32 pixels it checks,
// one Gaussian per lane, whether any pixel of its block can pass the
// inclusion test, and only visits the ones that can.  sm_103a; no tensor
// cores (the per-pair work is a handful of scalar operations).
//
// Every pair's exponent t, inclusion decision and alpha come from the same
// FP32 operations (pair_t_at) in the forward and both backward kernels.
#include "vt_common.cuh"

namespace vt {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kWarps = kBlockPix / 32;

// Conservative set of the pixels of an 8x4 block (bit lx + 8 ly, columns
// 0..lxmax, rows 0..lymax) that can pass t >= t_min for a Gaussian at offsets
// du0 ~ bx0 - uc, dv0 ~ by0 - vc: row by row, kx' (du0 + lx)^2 >= t_min -
// ky' (dv0 + ly)^2 bounds |du0 + lx|.  The threshold is loosened by 1e-4
// relative and the half-width widened by 1e-3 px, which covers the rounding of
// the exact per-pixel test and of the approximate reciprocal and square root.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ uint32_t pixel_mask(float du0, float dv0, float kxs, float kys,
                                               float tmin, int lxmax, int lymax) {
    const float tl = tmin * 1.0001f - 1e-6f;
    const float ikx = rcp_approx(kxs);   // kx' < 0
    uint32_t m = 0u;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float dv = dv0 + (float)r;
        const float s = (tl - kys * dv * dv) * ikx;   // bound on (du0 + lx)^2
        if (r <= lymax && s >= 0.f) {
            const float w = sqrt_approx(s) * 1.0001f + 1e-3f;
            const int lo = max(0, (int)ceilf(-du0 - w));
            const int hi = min(lxmax, (int)floorf(w - du0));
            if (lo <= hi) m |= ((0xFFu >> (7 - hi)) & (0xFFu << lo)) << (8 * r);
        }
    }
    return m;
}

// 32 x 32 bit transpose across a warp: on return bit j of lane i's word is
// bit i of lane j's input word (five butterfly stages).
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
    const uint32_t M[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int w = 16 >> s;
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, w);
        x = (lane & w) ? ((x & ~M[s]) | ((y & ~M[s]) >> w)) : ((x & M[s]) | ((y & M[s]) << w));
    }
    return x;
}

// OR of the list-overflow flags of the eight blocks of a tile.
__device__ __forceinline__ bool tile_flagged(const uint32_t *blk_ovf, int tile) {
    const uint4 *f = reinterpret_cast<const uint4 *>(blk_ovf + (size_t)tile * kWarps);
    const uint4 a = f[0], b = f[1];
    return (a.x | a.y | a.z | a.w | b.x | b.y | b.z | b.w) != 0u;
}

// Forward.  One block of eight warps per tile; the warps never synchronise,
// so a warp whose pixels saturate early retires instead of waiting for the
// rest of its tile (the eight warps of a tile still share its records in L1:
// handing pixel blocks to warps from a global work counter, which spreads a
// tile's blocks over several SMs, measured slower).  A warp only visits the
// list entries whose block mask (written by the sort) has its block's bit:
// it classifies the masks 128 entries at a time into a warp-private ring of
// list indices and takes them out in batches of 32, in list order.  For a
// batch the lanes load the records (one batch ahead; the ids two batches
// ahead), build each Gaussian's pixel set in the block, stage the batch in
// warp-private shared memory ({bx0 - iu, by0 - iv, fu, fv}, {kx', ky', t_min,
// o}, {c, z}, id, list index) and walk the relevant ones in order.  Adding
// the lane's column lx to bx0 - iu gives px - iu exactly, so du = (px - iu) -
// fu is bit-identical to pair_t_at.  The warp leaves the block once all its
// pixels have terminated.  With plist != NULL every pixel also records the id
// of every Gaussian it added together with the transmittance in front of it
// (up to plist_cap entries, pixel-major), which the backward replays instead
// of the tile list; blk_ovf[item] flags blocks where a pixel added more
// (always 1 without lists).
constexpr int kQueue = 256;   // ring of list indices per warp (>= 31 + 128)

__global__ void __launch_bounds__(kBlockPix) k_composite_fwd(
    Camera cam, const uint32_t *tile_off, const uint32_t *sorted, const uint8_t *bmask,
    const float4 *geo, const float4 *app, float *rgb, float *depth, float *sil,
    uint32_t *pix_last, uint32_t *pix_nadd, float *pix_T, uint2 *plist, int plist_cap,
    uint32_t *blk_ovf, const Status *st) {
    __shared__ float4 s_f[kWarps][32], s_k[kWarps][32], s_c[kWarps][32];
    __shared__ uint32_t s_gid[kWarps][32], s_idx[kWarps][32];
    __shared__ uint32_t s_q[kWarps][kQueue];
    if (st->flags) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lx = lane & 7, ly = lane >> 3;
    const float lxf = (float)lx, lyf = (float)ly;
    float4 (&fs)[32] = s_f[warp];
    float4 (&ks)[32] = s_k[warp];
    float4 (&cs)[32] = s_c[warp];
    uint32_t (&ids)[32] = s_gid[warp];
    uint32_t (&lidx)[32] = s_idx[warp];
    uint32_t (&q)[kQueue] = s_q[warp];
    const size_t HW = (size_t)cam.W * cam.H;

    const int item = blockIdx.x * kWarps + warp;
    const int tile = blockIdx.x, sub = warp;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int bx0 = tx * kTile + (sub & 1) * 8, by0 = ty * kTile + (sub >> 1) * 4;
    const int px = bx0 + lx, py = by0 + ly;
    const bool inside = px < cam.W && py < cam.H;
    const int lxmaxi = min(7, cam.W - 1 - bx0), lymaxi = min(3, cam.H - 1 - by0);
    const uint32_t start = tile_off[tile];
    const int n = (int)(tile_off[tile + 1] - start);
    const size_t p = inside ? (size_t)py * cam.W + px : 0;
    uint2 *mylist = (plist && inside) ? plist + p * (size_t)plist_cap : nullptr;
    const uint32_t cap = mylist ? (uint32_t)plist_cap : 0u;
    const uint32_t my_bit = 1u << sub, lt_mask = (1u << lane) - 1u;

    // Ring of this block's list indices: head qh, length qn; scan = next list
    // index to classify, mw = the block masks of entries scan + lane + 32 j
    // (byte j), loaded one window ahead.
    uint32_t qh = 0, qn = 0, mw = 0;
    int scan = 0;
    auto load_window = [&]() {
        mw = 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int e = scan + 32 * j + lane;
            if (e < n) mw |= (uint32_t)bmask[start + e] << (8 * j);
        }
    };
    auto take = [&](uint32_t &idx, int &cnt) {
        while (qn < 32u && scan < n) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const bool mine = (mw >> (8 * j)) & my_bit;
                const unsigned rel = __ballot_sync(kFullMask, mine);
                if (mine) q[(qh + qn + __popc(rel & lt_mask)) & (kQueue - 1)] = scan + 32 * j + lane;
                qn += __popc(rel);
            }
            scan += 128;
            load_window();
        }
        __syncwarp();
        cnt = (int)min(qn, 32u);
        idx = lane < cnt ? q[(qh + lane) & (kQueue - 1)] : 0u;
        qh += cnt;
        qn -= cnt;
    };

    float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, dd = 0.f, ss = 0.f;
    uint32_t last = 0, nadd = 0;
    bool done = !inside;
    // Two-stage prefetch: the ids of batch r + 2 and the records of batch
    // r + 1 are in flight while batch r is composited.
    uint32_t idx_n = 0, idx_nn = 0, gid_n = 0, gid_nn = 0;
    int cnt_n = 0, cnt_nn = 0;
    float4 g0n = make_float4(0.f, 0.f, 0.f, 0.f), g1n = g0n, an = g0n;
    if (!__all_sync(kFullMask, done)) {
        load_window();
        take(idx_n, cnt_n);
        if (lane < cnt_n) {
            gid_n = sorted[start + idx_n];
            g0n = geo[2 * (size_t)gid_n];
            g1n = geo[2 * (size_t)gid_n + 1];
            an = app[gid_n];
        }
        take(idx_nn, cnt_nn);
        if (lane < cnt_nn) gid_nn = sorted[start + idx_nn];
    }
    for (;;) {
        const int cnt = cnt_n;
        if (cnt == 0 || __all_sync(kFullMask, done)) break;
        const uint32_t gid = gid_n, idx = idx_n;
        const float4 g0 = g0n, g1 = g1n, a = an;
        idx_n = idx_nn;
        cnt_n = cnt_nn;
        gid_n = gid_nn;
        if (lane < cnt_n) {   // records of the next batch
            g0n = geo[2 * (size_t)gid_n];
            g1n = geo[2 * (size_t)gid_n + 1];
            an = app[gid_n];
        }
        take(idx_nn, cnt_nn);
        if (lane < cnt_nn) gid_nn = sorted[start + idx_nn];
        const float ku = (float)(bx0 - __float_as_int(g0.x));
        const float kv = (float)(by0 - __float_as_int(g0.z));
        const float tmin = t_min_of(g1.w);
        const uint32_t pm =
            lane < cnt ? pixel_mask(ku - g0.y, kv - g0.w, g1.x, g1.y, tmin, lxmaxi, lymaxi) : 0u;
        if (!__any_sync(kFullMask, pm != 0u)) continue;
        __syncwarp();
        fs[lane] = make_float4(ku, kv, g0.y, g0.w);
        ks[lane] = make_float4(g1.x, g1.y, tmin, g1.w);
        cs[lane] = a;
        ids[lane] = gid;
        lidx[lane] = idx;
        // this pixel's candidates of the batch, in list order (bit j = entry j)
        uint32_t cand = transpose32(pm, lane);
        __syncwarp();
        if (done) cand = 0u;
        // each lane walks its own candidates: lanes work on different
        // Gaussians at once, and the warp takes as many steps as the busiest
        // pixel has candidates
        while (__any_sync(kFullMask, cand != 0u)) {
            if (!cand) continue;
            const int j = __ffs(cand) - 1;
            cand &= cand - 1u;
            const float4 f = fs[j], k = ks[j];
            const float t = pair_t(__fsub_rn(__fadd_rn(f.x, lxf), f.z),
                                   __fsub_rn(__fadd_rn(f.y, lyf), f.w), k.x, k.y);
            if (!(t >= k.z)) continue;
            const float al = fminf(__fmul_rn(k.w, exp2_approx(t)), kAlphaClamp);
            const float Tn = __fmaf_rn(-al, T, T);   // T (1 - alpha), one rounding
            if (Tn < kTMin) {
                done = true;
                cand = 0u;
                continue;
            }
            const float w = __fmul_rn(al, T);
            const float4 c = cs[j];
            c0 = __fmaf_rn(w, c.x, c0);
            c1 = __fmaf_rn(w, c.y, c1);
            c2 = __fmaf_rn(w, c.z, c2);
            dd = __fmaf_rn(w, c.w, dd);
            ss = __fadd_rn(ss, w);
            if (nadd < cap) mylist[nadd] = make_uint2(ids[j], __float_as_uint(T));
            T = Tn;
            last = lidx[j] + 1u;
            ++nadd;
        }
    }
    if (inside) {
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
    const bool ovf = __any_sync(kFullMask, nadd > cap);
    if (lane == 0) blk_ovf[item] = plist ? (uint32_t)ovf : 1u;
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

struct PoseAcc {
    float a[12];  // a[3*i + j] = sum x_i g_j ; a[9 + j] = sum g_j
};

// Per-pixel state of the back-to-front walk (see the derivation above).
struct BwdPixel {
    float gC0, gC1, gC2, gD, gS, Tfin, pxn, pyn;
    float T, A0, A1, A2, Bd, Sb, cr0, cr1, cr2, zr;
    bool have_ref;
};

__device__ __forceinline__ void bwd_pixel_init(BwdPixel &P, float Tfin, float gC0, float gC1,
                                               float gC2, float gD, float gS, int px, int py,
                                               const Camera &cam) {
    P.gC0 = gC0;
    P.gC1 = gC1;
    P.gC2 = gC2;
    P.gD = gD;
    P.gS = gS;
    P.Tfin = Tfin;
    P.pxn = ((float)px - cam.cx) / cam.fx;
    P.pyn = ((float)py - cam.cy) / cam.fy;
    P.T = Tfin;
    P.A0 = P.A1 = P.A2 = P.Bd = P.Sb = 0.f;
    P.cr0 = P.cr1 = P.cr2 = P.zr = 0.f;
    P.have_ref = false;
}

// One added Gaussian of the pixel, visited back to front (g0, g1: footprint
// record with 1/r in g1.z, a: colour and depth z, t: exponent of pair_t,
// G = 2^t, ah = o G).  Returns its colour / opacity / radius gradient terms
// and adds its pose terms to acc.  Ti_fwd >= 0 is the forward's transmittance in front
// of this Gaussian (recorded in the per-pixel list); otherwise it is
// recovered by division, which accumulates the rounding of every Gaussian
// behind.
__device__ __forceinline__ void bwd_pair(BwdPixel &P, const float4 &g0, const float4 &g1,
                                         const float4 &a, float t, float du, float dv, float G,
                                         float ah, const Camera &cam, bool want_pose, PoseAcc &acc,
                                         float &dc0, float &dc1, float &dc2, float &dop,
                                         float &drd, bool want_geo, float &gxo, float &gyo,
                                         float &gzo, float Ti_fwd = -1.f) {
    const float ifx = 1.f / cam.fx, ify = 1.f / cam.fy;
    const float al = fminf(ah, kAlphaClamp);
    const float om = 1.f - al;
    const float Ti = Ti_fwd >= 0.f ? Ti_fwd : P.T / om;
    const float w = al * Ti;
    const float z = a.w, q = t * kQFromT;
    const float ir = g1.z, ir2 = ir * ir;
    if (!P.have_ref) {
        P.have_ref = true;
        P.cr0 = a.x;
        P.cr1 = a.y;
        P.cr2 = a.z;
        P.zr = z;
    }
    const float e0 = a.x - P.cr0, e1 = a.y - P.cr1, e2 = a.z - P.cr2, ez = z - P.zr;
    const float num = P.gC0 * (a.x * P.Tfin + e0 * P.Sb - P.A0) +
                      P.gC1 * (a.y * P.Tfin + e1 * P.Sb - P.A1) +
                      P.gC2 * (a.z * P.Tfin + e2 * P.Sb - P.A2) +
                      P.gD * (z * P.Tfin + ez * P.Sb - P.Bd) + P.gS * P.Tfin;
    const float dal = num / om;
    dc0 = P.gC0 * w;
    dc1 = P.gC1 * w;
    dc2 = P.gC2 * w;
    float dq = 0.f;
    dop = 0.f;
    if (ah < kAlphaClamp) {
        dop = dal * G;
        dq = -0.5f * ah * dal;
    }
    drd = dq * (-2.f * q * ir);
    gxo = gyo = gzo = 0.f;
    if (want_pose || want_geo) {
        const float ex = z * du * ifx, ey = z * dv * ify;
        const float gx = dq * (-2.f * ex * ir2);
        const float gy = dq * (-2.f * ey * ir2);
        const float gz = dq * (2.f * (P.pxn * ex + P.pyn * ey) * ir2) + P.gD * w;
        gxo = gx;
        gyo = gy;
        gzo = gz;
    }
    if (want_pose) {
        const float gx = gxo, gy = gyo, gz = gzo;
        const float uc = (float)__float_as_int(g0.x) + g0.y;
        const float vc = (float)__float_as_int(g0.z) + g0.w;
        const float X[3] = {z * (uc - cam.cx) * ifx, z * (vc - cam.cy) * ify, z};
        const float Gv[3] = {gx, gy, gz};
#pragma unroll
        for (int a_ = 0; a_ < 3; ++a_)
#pragma unroll
            for (int b_ = 0; b_ < 3; ++b_)
                acc.a[3 * a_ + b_] = __fmaf_rn(X[a_], Gv[b_], acc.a[3 * a_ + b_]);
        acc.a[9] += gx;
        acc.a[10] += gy;
        acc.a[11] += gz;
    }
    P.A0 = __fmaf_rn(w, e0, P.A0);
    P.A1 = __fmaf_rn(w, e1, P.A1);
    P.A2 = __fmaf_rn(w, e2, P.A2);
    P.Bd = __fmaf_rn(w, ez, P.Bd);
    P.Sb += w;
    P.T = Ti;
}

// Per-Gaussian gradient terms go to workspace accumulators indexed by
// Gaussian id: one 16-byte vector atomic for (colour, opacity), one for the
// radius instead of five scalar ones (k_attr_scatter then adds them to the
// caller's per-section buffers), and with source-view gradients one for dL/dx
// of the centre (k_view_grads reduces them per view).  Gaussians of sections
// that want neither are skipped.
__device__ __forceinline__ void add_pair_grads(const SecTable &Tab, int64_t g, bool want_attr,
                                               bool want_views, float dc0, float dc1, float dc2,
                                               float dop, float drd, float gx, float gy,
                                               float gz, float4 *acc4, float *accr,
                                               float4 *accg) {
    const SecDesc &S = Tab.s[find_section(Tab, g)];
    if (want_attr && (S.d_colour || S.d_opacity || S.d_radius)) {
        atomicAdd(acc4 + g, make_float4(dc0, dc1, dc2, dop));
        atomicAdd(accr + g, drd);
    }
    if (want_views && (S.d_view_twist || S.d_view_mat || S.d_depth))
        atomicAdd(accg + g, make_float4(gx, gy, gz, 0.f));
}

__global__ void __launch_bounds__(256) k_attr_scatter(SecTable Tab, const float4 *acc4,
                                                      const float *accr) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= Tab.n_total) return;
    const SecDesc &S = Tab.s[find_section(Tab, g)];
    if (!S.d_colour && !S.d_opacity && !S.d_radius) return;
    const int64_t li = g - S.gbase;
    const float4 v = acc4[g];
    if (S.d_colour) {
        S.d_colour[3 * li + 0] += v.x;
        S.d_colour[3 * li + 1] += v.y;
        S.d_colour[3 * li + 2] += v.z;
    }
    if (S.d_opacity) S.d_opacity[li] += v.w;
    if (S.d_radius) S.d_radius[li] += accr[g];
}

// Block sum of the per-lane pose terms in FP64, in a fixed order, written as
// the tile's partial.
__device__ __forceinline__ void write_pose_partial(const PoseAcc &acc, double (*s_pose)[12],
                                                   double *pose_partials, int tile) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
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

// Tile replay: the block walks its tile's list from the largest list end of
// its pixels back to the front in shared-memory batches; each warp visits the
// Gaussians whose disc touches its 8x4 block.  Used when no per-pixel lists
// were kept (memory budget) and for tiles whose lists overflowed (tile_mask:
// only tiles with tile_mask[t] != 0; NULL = all tiles).
__global__ void __launch_bounds__(kBlockPix) k_composite_bwd(
    SecTable Tab, Camera cam, const uint32_t *tile_off, const uint32_t *sorted, const float4 *geo,
    const float4 *app, const uint32_t *pix_last, const float *pix_T,
    const float *g_rgb, const float *g_depth, const float *g_sil, int mode,
    double *pose_partials, const uint32_t *tile_mask, float4 *acc4, float *accr, float4 *accg,
    const Status *st) {
    __shared__ float4 s_g0[kBatch], s_g1[kBatch], s_a[kBatch];
    __shared__ float s_tmin[kBatch];
    __shared__ uint32_t s_gid[kBatch];
    __shared__ double s_pose[kBlockPix / 32][12];
    __shared__ uint32_t s_last;
    if (st->flags) return;
    const int tile = blockIdx.x;
    if (tile_mask && !tile_flagged(tile_mask, tile)) return;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx0 = tx * kTile + (warp & 1) * 8, by0 = ty * kTile + (warp >> 1) * 4;
    const int px = bx0 + (lane & 7), py = by0 + (lane >> 3);
    const bool inside = px < cam.W && py < cam.H;
    const float lxmax = (float)min(7, cam.W - 1 - bx0);
    const float lymax = (float)min(3, cam.H - 1 - by0);
    const uint32_t start = tile_off[tile];
    const bool want_attr = (mode & VT_GRAD_ATTR) != 0, want_pose = (mode & VT_GRAD_POSE) != 0;
    const bool want_views = (mode & VT_GRAD_VIEWS) != 0;

    const size_t HW = (size_t)cam.W * cam.H;
    const size_t p = inside ? (size_t)py * cam.W + px : 0;
    uint32_t my_last = inside ? pix_last[p] : 0u;
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
    BwdPixel P;
    bwd_pixel_init(P, inside ? pix_T[p] : 1.f, gC0, gC1, gC2, gD, gS, px, py, cam);

    if (threadIdx.x == 0) s_last = 0;
    __syncthreads();
    const uint32_t wl = __reduce_max_sync(kFullMask, my_last);
    if (lane == 0 && wl) atomicMax(&s_last, wl);
    __syncthreads();
    const uint32_t tile_last = s_last;

    PoseAcc acc;
#pragma unroll
    for (int i = 0; i < 12; ++i) acc.a[i] = 0.f;

    if (tile_last > 0) {
        for (int b0 = (int)((tile_last - 1) / kBatch) * kBatch; b0 >= 0; b0 -= kBatch) {
            const int nb = (int)min((uint32_t)kBatch, tile_last - (uint32_t)b0);
            if ((int)threadIdx.x < nb) {
                const uint32_t g = sorted[start + b0 + threadIdx.x];
                s_g0[threadIdx.x] = geo[2 * (size_t)g];
                const float4 h1 = geo[2 * (size_t)g + 1];
                s_g1[threadIdx.x] = h1;
                s_tmin[threadIdx.x] = t_min_of(h1.w);
                s_a[threadIdx.x] = app[g];
                s_gid[threadIdx.x] = g;
            }
            __syncthreads();
            if (wl > (uint32_t)b0) {
                for (int j0 = ((nb - 1) >> 5) << 5; j0 >= 0; j0 -= 32) {
                    const int jj = j0 + lane;
                    bool rel = false;
                    if (jj < nb && (uint32_t)(b0 + jj) < wl) {
                        const float4 h0 = s_g0[jj], h1 = s_g1[jj];
                        rel = block_touches((float)(bx0 - __float_as_int(h0.x)) - h0.y,
                                            (float)(by0 - __float_as_int(h0.z)) - h0.w, h1.x,
                                            h1.y, s_tmin[jj], lxmax, lymax);
                    }
                    unsigned mask = __ballot_sync(kFullMask, rel);
                    while (mask) {
                        const int bit = 31 - __clz(mask);
                        mask &= ~(1u << bit);
                        const int j = j0 + bit;
                        float dc0 = 0.f, dc1 = 0.f, dc2 = 0.f, dop = 0.f, drd = 0.f;
                        float gx = 0.f, gy = 0.f, gz = 0.f;
                        bool contrib = false;
                        if ((uint32_t)(b0 + j) < my_last) {
                            const float4 g0 = s_g0[j], g1 = s_g1[j];
                            float du, dv;
                            const float t = pair_t_at(px, py, g0, g1, du, dv);
                            if (t >= s_tmin[j]) {
                                const float G = exp2_approx(t);
                                const float ah = __fmul_rn(g1.w, G);
                                contrib = true;
                                bwd_pair(P, g0, g1, s_a[j], t, du, dv, G, ah, cam, want_pose,
                                         acc, dc0, dc1, dc2, dop, drd, want_views, gx, gy, gz);
                            }
                        }
                        if ((want_attr || want_views) && __any_sync(kFullMask, contrib)) {
                            dc0 = warp_sum(dc0);
                            dc1 = warp_sum(dc1);
                            dc2 = warp_sum(dc2);
                            dop = warp_sum(dop);
                            drd = warp_sum(drd);
                            gx = warp_sum(gx);
                            gy = warp_sum(gy);
                            gz = warp_sum(gz);
                            if (lane == 0)
                                add_pair_grads(Tab, s_gid[j], want_attr, want_views, dc0, dc1,
                                               dc2, dop, drd, gx, gy, gz, acc4, accr, accg);
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    if (want_pose) write_pose_partial(acc, s_pose, pose_partials, tile);
}

// Per-pixel list replay: every lane walks the ids its pixel added, recorded
// by the forward, from the last to the first, loading each record one step
// ahead.  No filtering and no block barriers in the walk; tiles with a block
// flagged in blk_ovf (a pixel exceeded the list capacity) are left to
// k_composite_bwd.
// Views = true compiles the source-view gradient path (mode VT_GRAD_VIEWS)
// into k_composite_bwd_list_views; the tracking and mapping paths launch
// k_composite_bwd_list, which does not carry it.
template <bool Views>
__device__ __forceinline__ void bwd_list_body(
    const SecTable &Tab, const Camera &cam, const float4 *geo, const float4 *app,
    const uint32_t *pix_nadd, const float *pix_T, const uint2 *plist, int plist_cap,
    const uint32_t *blk_ovf, const float *g_rgb, const float *g_depth, const float *g_sil,
    int mode, double *pose_partials, float4 *acc4, float *accr, float4 *accg, const Status *st,
    double (*s_pose)[12]) {
    if (st->flags) return;
    const int tile = blockIdx.x;
    if (tile_flagged(blk_ovf, tile)) return;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px = tx * kTile + (warp & 1) * 8 + (lane & 7);
    const int py = ty * kTile + (warp >> 1) * 4 + (lane >> 3);
    const bool inside = px < cam.W && py < cam.H;
    const bool want_attr = (mode & VT_GRAD_ATTR) != 0, want_pose = (mode & VT_GRAD_POSE) != 0;
    const bool want_views = Views && (mode & VT_GRAD_VIEWS) != 0;
    const size_t HW = (size_t)cam.W * cam.H;
    const size_t p = inside ? (size_t)py * cam.W + px : 0;
    int n = inside ? (int)pix_nadd[p] : 0;
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
    if (gC0 == 0.f && gC1 == 0.f && gC2 == 0.f && gD == 0.f && gS == 0.f) n = 0;
    BwdPixel P;
    bwd_pixel_init(P, inside ? pix_T[p] : 1.f, gC0, gC1, gC2, gD, gS, px, py, cam);
    PoseAcc acc;
#pragma unroll
    for (int i = 0; i < 12; ++i) acc.a[i] = 0.f;
    const uint2 *mylist = plist + p * (size_t)plist_cap;
    // Two-stage prefetch: the list entry two steps ahead and the records one
    // step ahead are in flight while the current Gaussian is processed.
    uint2 e_n = make_uint2(0u, 0u), e_nn = e_n;
    float4 g0n = make_float4(0.f, 0.f, 0.f, 0.f), g1n = g0n, an = g0n;
    if (n > 0) {
        e_n = mylist[n - 1];
        g0n = geo[2 * (size_t)e_n.x];
        g1n = geo[2 * (size_t)e_n.x + 1];
        an = app[e_n.x];
    }
    if (n > 1) e_nn = mylist[n - 2];
    for (int k = n - 1; k >= 0; --k) {
        const uint32_t g = e_n.x;
        const float Ti = __uint_as_float(e_n.y);
        const float4 g0 = g0n, g1 = g1n, a = an;
        if (k > 0) {   // records of the next (nearer) Gaussian
            e_n = e_nn;
            g0n = geo[2 * (size_t)e_n.x];
            g1n = geo[2 * (size_t)e_n.x + 1];
            an = app[e_n.x];
        }
        if (k > 1) e_nn = mylist[k - 2];
        float du, dv;
        const float t = pair_t_at(px, py, g0, g1, du, dv);
        const float G = exp2_approx(t);
        const float ah = __fmul_rn(g1.w, G);
        float dc0, dc1, dc2, dop, drd, gx, gy, gz;
        bwd_pair(P, g0, g1, a, t, du, dv, G, ah, cam, want_pose, acc, dc0, dc1, dc2, dop, drd,
                 want_views, gx, gy, gz, Ti);
        if (want_attr || want_views)
            add_pair_grads(Tab, g, want_attr, want_views, dc0, dc1, dc2, dop, drd, gx, gy, gz,
                           acc4, accr, accg);
    }
    if (want_pose) write_pose_partial(acc, s_pose, pose_partials, tile);
}

__global__ void __launch_bounds__(kBlockPix, 3) k_composite_bwd_list(
    SecTable Tab, Camera cam, const float4 *geo, const float4 *app, const uint32_t *pix_nadd,
    const float *pix_T, const uint2 *plist, int plist_cap, const uint32_t *blk_ovf,
    const float *g_rgb, const float *g_depth, const float *g_sil, int mode,
    double *pose_partials, float4 *acc4, float *accr, float4 *accg, const Status *st) {
    __shared__ double s_pose[kBlockPix / 32][12];
    bwd_list_body<false>(Tab, cam, geo, app, pix_nadd, pix_T, plist, plist_cap, blk_ovf, g_rgb,
                         g_depth, g_sil, mode, pose_partials, acc4, accr, accg, st, s_pose);
}

__global__ void __launch_bounds__(kBlockPix, 3) k_composite_bwd_list_views(
    SecTable Tab, Camera cam, const float4 *geo, const float4 *app, const uint32_t *pix_nadd,
    const float *pix_T, const uint2 *plist, int plist_cap, const uint32_t *blk_ovf,
    const float *g_rgb, const float *g_depth, const float *g_sil, int mode,
    double *pose_partials, float4 *acc4, float *accr, float4 *accg, const Status *st) {
    __shared__ double s_pose[kBlockPix / 32][12];
    bwd_list_body<true>(Tab, cam, geo, app, pix_nadd, pix_T, plist, plist_cap, blk_ovf, g_rgb,
                        g_depth, g_sil, mode, pose_partials, acc4, accr, accg, st, s_pose);
}

// Source-view pose gradients (head-frame bundle adjustment, Sec. 3.4).  The
// Gaussians of one view are a contiguous range of their section (ids are in
// (view, pixel) order).  k_view_grads: kViewChunks blocks per (section, view)
// each sum g X_c^T and g over an equal share of the range (per thread in
// FP32, across the block in FP64, fixed order), with g = dL/dx of the centre
// in the target frame and X_c = D ((u - cx)/fx, (v - cy)/fy, 1), and write
// per-Gaussian depth gradients dL/dD = (R g) . (R_k X_c / D) on the way;
// k_view_finalize: one thread per view sums the chunk partials in order and
// forms
//   dL/dR_k = R A,  dL/dt_k = R s,  dL/drho_k = R_k^T R s,
//   dL/dphi_k = sum X_c x (R_k^T R g)   (from B = R_k^T R A),
// accumulated (+=) into the section's outputs.
__device__ __forceinline__ bool view_of_block(const SecTable &Tab, int b, int &s, int &k) {
    for (s = 0; s < Tab.n; ++s) {
        if (b < Tab.s[s].n_views) {
            k = b;
            return true;
        }
        b -= Tab.s[s].n_views;
    }
    return false;
}

__global__ void __launch_bounds__(256) k_view_grads(SecTable Tab, const float4 *accg,
                                                    const double *pose_copy, double *partials) {
    __shared__ double red[12][kBlockPix / 32];
    __shared__ int64_t range[2];
    const int vb = blockIdx.x / kViewChunks, chunk = blockIdx.x % kViewChunks;
    int s, k;
    if (!view_of_block(Tab, vb, s, k)) return;
    const SecDesc &S = Tab.s[s];
    double *out = partials + (size_t)blockIdx.x * 12;
    if (!S.d_view_twist && !S.d_view_mat && !S.d_depth) return;
    const uint32_t plane = (uint32_t)S.W * (uint32_t)S.H;
    if (threadIdx.x < 2) {   // first index with src >= (k + threadIdx.x) * plane
        const uint64_t key = (uint64_t)(k + threadIdx.x) * plane;
        int64_t lo = 0, hi = S.n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((uint64_t)S.src[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        range[threadIdx.x] = lo;
    }
    __syncthreads();
    const int64_t len = range[1] - range[0];
    const int64_t c0 = range[0] + len * chunk / kViewChunks;
    const int64_t c1 = range[0] + len * (chunk + 1) / kViewChunks;
    const double *R = pose_copy, *Rk = S.poses + 12 * k;
    float Mf[9];   // R_k^T R (for the depth gradient), FP32
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c)
            Mf[3 * a + c] = (float)(Rk[a] * R[c] + Rk[3 + a] * R[3 + c] + Rk[6 + a] * R[6 + c]);
    const float ifx = 1.f / S.fx, ify = 1.f / S.fy;
    float acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = 0.f;
    for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
        const float4 g = accg[S.gbase + i];
        if (g.x == 0.f && g.y == 0.f && g.z == 0.f) continue;
        const uint32_t src = S.src[i], pix = src - (uint32_t)k * plane;
        const uint32_t v = pix / (uint32_t)S.W, u = pix - v * (uint32_t)S.W;
        const float D = S.depth[src];
        const float ray[3] = {((float)u - S.cx) * ifx, ((float)v - S.cy) * ify, 1.f};
        const float X[3] = {D * ray[0], D * ray[1], D};
        const float gv[3] = {g.x, g.y, g.z};
        if (S.d_depth) {   // dL/dD = (R g) . (R_k ray) = ray . (R_k^T R g)
            float dd = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                dd += ray[a] * (Mf[3 * a] * gv[0] + Mf[3 * a + 1] * gv[1] + Mf[3 * a + 2] * gv[2]);
            S.d_depth[i] += dd;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[3 * a + c] = fmaf(gv[a], X[c], acc[3 * a + c]);
            acc[9 + a] += gv[a];
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        const double v = warp_sum_d((double)acc[i]);
        if (lane == 0) red[i][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        double t = 0.0;
        for (int w = 0; w < kBlockPix / 32; ++w) t += red[threadIdx.x][w];
        out[threadIdx.x] = t;
    }
}

__global__ void k_view_finalize(SecTable Tab, const double *pose_copy, const double *partials,
                                int n_views) {
    const int vb = blockIdx.x * blockDim.x + threadIdx.x;
    if (vb >= n_views) return;
    int s, k;
    if (!view_of_block(Tab, vb, s, k)) return;
    const SecDesc &S = Tab.s[s];
    if (!S.d_view_twist && !S.d_view_mat) return;
    double A[9] = {0}, sv[3] = {0};
    for (int c = 0; c < kViewChunks; ++c) {
        const double *p = partials + ((size_t)vb * kViewChunks + c) * 12;
        for (int i = 0; i < 9; ++i) A[i] += p[i];
        for (int i = 0; i < 3; ++i) sv[i] += p[9 + i];
    }
    const double *R = pose_copy, *Rk = S.poses + 12 * k;
    double Am[9], sm[3];
    for (int a = 0; a < 3; ++a) {
        for (int c = 0; c < 3; ++c)
            Am[3 * a + c] = R[3 * a] * A[c] + R[3 * a + 1] * A[3 + c] + R[3 * a + 2] * A[6 + c];
        sm[a] = R[3 * a] * sv[0] + R[3 * a + 1] * sv[1] + R[3 * a + 2] * sv[2];
    }
    if (S.d_view_mat) {
        double *o = S.d_view_mat + 12 * k;
        for (int i = 0; i < 9; ++i) o[i] += Am[i];
        for (int a = 0; a < 3; ++a) o[9 + a] += sm[a];
    }
    if (S.d_view_twist) {
        double B[9], rho[3];
        for (int c = 0; c < 3; ++c) {
            for (int e = 0; e < 3; ++e)
                B[3 * c + e] = Rk[c] * Am[e] + Rk[3 + c] * Am[3 + e] + Rk[6 + c] * Am[6 + e];
            rho[c] = Rk[c] * sm[0] + Rk[3 + c] * sm[1] + Rk[6 + c] * sm[2];
        }
        double *o = S.d_view_twist + 6 * k;
        for (int c = 0; c < 3; ++c) o[c] += rho[c];
        o[3] += B[2 * 3 + 1] - B[1 * 3 + 2];
        o[4] += B[0 * 3 + 2] - B[2 * 3 + 0];
        o[5] += B[1 * 3 + 0] - B[0 * 3 + 1];
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
