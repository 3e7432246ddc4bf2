// Projection, tile binning and per-tile depth sort: the forward steps before
// compositing.  sm_103a; no tensor cores (nothing here is a contraction).
#include "vt_common.cuh"

namespace vt {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// k_setup: one block per source view.  Twelve threads form in FP64 the
// composite transform of the view into the target camera, M = R^T R_k and
// m = R^T (t_k - t), one entry each, in the fixed operation order that
// defines the depth key (each product and sum rounded on its own), then the
// projection rows U = fx M0 + cx M2, V = fy M1 + cy M2, Z = M2 and offsets as
// float-float (FP64 is a narrow pipe: the twelve chains run side by side).
// The block then fills the view's float-float tables, column u:
// (U0, V0, Z0) * a_u and row v: (U1, V1, Z1) * b_v + (U2, V2, Z2), with
// a_u = (u - cx_k)/fx_k, b_v = (v - cy_k)/fy_k, so that the projected centre's
// numerators are D * (A[u] + B[v]) + (mu, mv, mz).
// View k of section S into camera (cam, pose12): X, its table rows tb (W + H
// rows) and, if pose_copy != NULL, a copy of the pose for the backward.
__device__ __forceinline__ void setup_view(const SecDesc &S, int k, const Camera &cam,
                                           const double *pose12, ViewXf &X, TabRow *tb,
                                           double *pose_copy) {
    __shared__ ff rows[9];  // U0 U1 U2 V0 V1 V2 Z0 Z1 Z2
    __shared__ double sM[12];
    const int i = threadIdx.x;
    if (i < 12) {
        const double *R = pose12, *t = pose12 + 9;
        const double *Rk = S.poses + 12 * k, *tk = Rk + 9;
        double acc;
        if (i < 9) {   // M[a][b] = sum_c R[c][a] Rk[c][b]
            const int a = i / 3, b = i % 3;
            acc = __dmul_rn(R[0 * 3 + a], Rk[0 * 3 + b]);
            acc = __dadd_rn(acc, __dmul_rn(R[1 * 3 + a], Rk[1 * 3 + b]));
            acc = __dadd_rn(acc, __dmul_rn(R[2 * 3 + a], Rk[2 * 3 + b]));
        } else {       // m[a] = sum_c R[c][a] (tk[c] - t[c])
            const int a = i - 9;
            acc = __dmul_rn(R[0 * 3 + a], __dsub_rn(tk[0], t[0]));
            acc = __dadd_rn(acc, __dmul_rn(R[1 * 3 + a], __dsub_rn(tk[1], t[1])));
            acc = __dadd_rn(acc, __dmul_rn(R[2 * 3 + a], __dsub_rn(tk[2], t[2])));
        }
        sM[i] = acc;
        X.Mf[i] = __double2float_rn(acc);
        if (pose_copy) pose_copy[i] = pose12[i];
    }
    __syncthreads();
    if (i < 12) {
        const double *M = sM, *m = sM + 9;
        const double fx = cam.fx, fy = cam.fy, cx = cam.cx, cy = cam.cy;
        if (i < 9) {   // rows[r * 3 + b]: r = 0 U, 1 V, 2 Z
            const int r = i / 3, b = i % 3;
            const double v = r == 0 ? fx * M[0 * 3 + b] + cx * M[2 * 3 + b]
                                    : (r == 1 ? fy * M[1 * 3 + b] + cy * M[2 * 3 + b] : M[2 * 3 + b]);
            rows[i] = ff_from_double(v);
        } else {
            const int r = i - 9;
            const double v = r == 0 ? fx * m[0] + cx * m[2] : (r == 1 ? fy * m[1] + cy * m[2] : m[2]);
            const ff o = ff_from_double(v);
            (r == 0 ? X.mu : (r == 1 ? X.mv : X.mz)) = make_float2(o.hi, o.lo);
            if (r == 0) X.pad[0] = X.pad[1] = 0.f;
        }
    }
    __syncthreads();
    const int W = S.W, H = S.H;
    for (int i = threadIdx.x; i < W + H; i += blockDim.x) {
        TabRow out;
        if (i < W) {
            ff a = ff_div(ff_two_sum((float)i, -S.cx), ff{S.fx, 0.f});
            ff pu = ff_mul(rows[0], a), pv = ff_mul(rows[3], a), pz = ff_mul(rows[6], a);
            out.a = make_float2(pu.hi, pu.lo);
            out.b = make_float2(pv.hi, pv.lo);
            out.c = make_float2(pz.hi, pz.lo);
            out.kf = __fdiv_rn(__fsub_rn((float)i, S.cx), S.fx);
        } else {
            ff b = ff_div(ff_two_sum((float)(i - W), -S.cy), ff{S.fy, 0.f});
            ff pu = ff_add(ff_mul(rows[1], b), rows[2]);
            ff pv = ff_add(ff_mul(rows[4], b), rows[5]);
            ff pz = ff_add(ff_mul(rows[7], b), rows[8]);
            out.a = make_float2(pu.hi, pu.lo);
            out.b = make_float2(pv.hi, pv.lo);
            out.c = make_float2(pz.hi, pz.lo);
            out.kf = __fdiv_rn(__fsub_rn((float)(i - W), S.cy), S.fy);
        }
        out.pad = 0.f;
        tb[i] = out;
    }
    __syncthreads();   // rows / sM are reused by the block's next view
}

__global__ void __launch_bounds__(256) k_setup(SecTable T, Camera cam, const double *pose12,
                                               ViewXf *views, TabRow *tab, double *pose_copy) {
    const int gv = blockIdx.x;
    int s = 0;
    for (int j = 1; j < T.n; ++j)
        if (gv >= T.s[j].view_base) s = j;
    const SecDesc &S = T.s[s];
    const int k = gv - S.view_base;
    setup_view(S, k, cam, pose12, views[gv], tab + S.tab_base + (int64_t)k * (S.W + S.H),
               gv == 0 ? pose_copy : nullptr);
}

// Batched form: one block per (item, view) in a grid-stride loop; item i's
// pose is copied to pose_copy[12 i].  The grid also zeroes the tile counts
// of k_preprocess (tile_count[0, n_tiles]).
__global__ void __launch_bounds__(256) kb_setup(const BatchTable *Bp, ViewXf *views, TabRow *tab,
                                                double *pose_copy, uint32_t *tile_count) {
    const BatchTable &B = *Bp;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= B.n_tiles;
         t += (int64_t)gridDim.x * blockDim.x)
        tile_count[t] = 0u;
    for (int gv = blockIdx.x; gv < B.n_views; gv += gridDim.x) {
        const int it = item_of_view(B, gv);
        const BatchItem &I = B.it[it];
        const SecDesc &S = B.sec[I.sec];
        const int k = gv - I.vbase;
        setup_view(S, k, I.cam, I.pose, views[gv], tab + I.tab_base + (int64_t)k * (S.W + S.H),
                   k == 0 ? pose_copy + 12 * it : nullptr);
    }
}

// ---------------------------------------------------------------------------
// Warp-aggregated visit of the tiles that each lane's pixel box (b0 = u0 |
// v0 << 16, b1 = u1 | v1 << 16, inclusive) overlaps: lanes that hit the same
// tile in the same step share one atomic.  fn(tile, peers, rank, tx, ty) is
// called by every active lane; the lowest lane of each peer group is the
// leader.
template <class Fn>
__device__ __forceinline__ void for_each_tile(uint32_t b0, uint32_t b1, uint32_t nt, int tiles_x,
                                              Fn &&fn) {
    const int lane = threadIdx.x & 31;
    const unsigned maxnt = __reduce_max_sync(kFull, nt);
    const uint32_t tx0 = (b0 & 0xffffu) / kTile, ty0 = (b0 >> 16) / kTile;
    const uint32_t w = (b1 & 0xffffu) / kTile - tx0 + 1;
    for (unsigned j = 0; j < maxnt; ++j) {
        const bool act = j < nt;
        const unsigned am = __ballot_sync(kFull, act);
        if (act) {
            const uint32_t jy = j / w, jx = j - jy * w;
            const uint32_t t = (ty0 + jy) * (uint32_t)tiles_x + tx0 + jx;
            const unsigned peers = __match_any_sync(am, t);
            const int rank = __popc(peers & ((1u << lane) - 1u));
            fn(t, peers, rank, tx0 + jx, ty0 + jy);
        }
    }
}

// The 8x4 blocks of tile (tx, ty) (block w at ((w & 1) * 8, (w >> 1) * 4))
// that the pixel box overlaps, bit w.  The box holds every pixel that can
// pass t >= t_min (k_preprocess), so the mask is conservative.
__device__ __forceinline__ uint32_t box_block_mask(uint32_t b0, uint32_t b1, uint32_t tx,
                                                   uint32_t ty) {
    const int u0 = (int)(b0 & 0xffffu) - (int)(tx * kTile), u1 = (int)(b1 & 0xffffu) - (int)(tx * kTile);
    const int v0 = (int)(b0 >> 16) - (int)(ty * kTile), v1 = (int)(b1 >> 16) - (int)(ty * kTile);
    const uint32_t cols = (u0 <= 7 && u1 >= 0 ? 1u : 0u) | (u0 <= 15 && u1 >= 8 ? 2u : 0u);
    uint32_t m = 0u;
#pragma unroll
    for (int r = 0; r < 4; ++r)
        if (v0 <= 4 * r + 3 && v1 >= 4 * r) m |= cols << (2 * r);
    return m;
}

// ---------------------------------------------------------------------------
// Footprint of an ellipsoid (the anisotropic variant): with its scale s and
// normalised quaternion q, the view -> target rotation M (FP32 composite of
// the render) and the Jacobian of the projection at the centre,
//   J = [[fx/z, 0, -(u_c - cx)/z], [0, fy/z, -(v_c - cy)/z]],
// T = J M R(q) diag(s) (2 x 3) and Sigma_2D = T T^T + 0.3 I (sums of squares
// on the diagonal, no cancellation there).  The determinant takes the
// product Sigma_01^2 with its rounding error (two FMAs), so the conic
// Q = Sigma_2D^-1 keeps a few ulp where the ellipse is thin.  Returns the
// record (a', b', c', o) = (kTScale Q00, 2 kTScale Q01, kTScale Q11, o) and
// the half extents sqrt(qlim Sigma_ii) of the ellipse q <= qlim, widened.
__device__ __forceinline__ bool ellipse_footprint(const SecDesc &S, int64_t li, const float *Mf,
                                                  float ucr, float vcr, float z,
                                                  const Camera &cam, float o, float qlim,
                                                  float4 &g1, float &ex, float &ey) {
    const float s0 = ld_attr(S.scale, S.prec, 3 * li), s1 = ld_attr(S.scale, S.prec, 3 * li + 1),
                s2 = ld_attr(S.scale, S.prec, 3 * li + 2);
    float qw = ld_attr(S.rot, S.prec, 4 * li), qx = ld_attr(S.rot, S.prec, 4 * li + 1),
          qy = ld_attr(S.rot, S.prec, 4 * li + 2), qz = ld_attr(S.rot, S.prec, 4 * li + 3);
    const float qn2 = qw * qw + qx * qx + qy * qy + qz * qz;
    if (!(s0 > 0.f && s1 > 0.f && s2 > 0.f && isfinite(s0 + s1 + s2) && qn2 > 0.f &&
          isfinite(qn2)))
        return false;
    const float iq = rsqrtf(qn2);
    qw *= iq;
    qx *= iq;
    qy *= iq;
    qz *= iq;
    const float Rq[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz),
                         2.f * (qx * qz + qw * qy),       2.f * (qx * qy + qw * qz),
                         1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                         2.f * (qx * qz - qw * qy),       2.f * (qy * qz + qw * qx),
                         1.f - 2.f * (qx * qx + qy * qy)};
    const float iz = 1.f / z;
    const float j00 = cam.fx * iz, j02 = -ucr * iz, j11 = cam.fy * iz, j12 = -vcr * iz;
    float B0[3], B1[3];   // J M
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        B0[c] = j00 * Mf[c] + j02 * Mf[6 + c];
        B1[c] = j11 * Mf[3 + c] + j12 * Mf[6 + c];
    }
    const float sc[3] = {s0, s1, s2};
    float T0[3], T1[3];   // J M R(q) diag(s)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        T0[k] = (B0[0] * Rq[k] + B0[1] * Rq[3 + k] + B0[2] * Rq[6 + k]) * sc[k];
        T1[k] = (B1[0] * Rq[k] + B1[1] * Rq[3 + k] + B1[2] * Rq[6 + k]) * sc[k];
    }
    const float S00 = T0[0] * T0[0] + T0[1] * T0[1] + T0[2] * T0[2] + kLowPass;
    const float S11 = T1[0] * T1[0] + T1[1] * T1[1] + T1[2] * T1[2] + kLowPass;
    const float S01 = T0[0] * T1[0] + T0[1] * T1[1] + T0[2] * T1[2];
    const float w = S01 * S01;
    const float det = __fmaf_rn(S00, S11, -w) - __fmaf_rn(S01, S01, -w);
    if (!(det > 0.f) || !isfinite(det)) return false;
    const float idet = 1.f / det;
    const float Q00 = S11 * idet, Q01 = -S01 * idet, Q11 = S00 * idet;
    g1 = make_float4(Q00 * kTScale, 2.f * Q01 * kTScale, Q11 * kTScale, o);
    ex = sqrtf(qlim * S00) * 1.001f + 1e-2f;
    ey = sqrtf(qlim * S11) * 1.001f + 1e-2f;
    return isfinite(g1.x) && isfinite(g1.y) && isfinite(g1.z);
}

// ---------------------------------------------------------------------------
// k_preprocess: one thread per Gaussian.  Gathers its depth pixel, computes
// the FP32 depth key (fixed operation order, identical to the definition),
// culls invalid depth, z_key < 0.1 and opacity < 1/255, projects the centre
// in float-float, derives the footprint coefficients kx = (z / (fx r))^2,
// ky = (z / (fy r))^2 (q = du^2 kx + dv^2 ky in pixels) and the conservative
// pixel box of the disc q <= min(9, 2 ln(255 o)), and counts its tiles.
// The records keep kx, ky scaled to the base-2 exponent t = -q log2(e)/2
// (see pair_t) and 1/r for the backward; info keeps the pixel box, the depth
// key and the tile count.  Ellipsoids (Aniso) keep the conic instead (see
// ellipse_footprint).
// Gaussian li of section S (workspace slot gid; its views at view_base, its
// table rows at tab_base): records, info and the pixel box r0, r1 with its
// tile count nt (0 when culled).
template <bool Aniso>
__device__ __forceinline__ void preprocess_gauss(const SecDesc &S, int64_t li, int64_t gid,
                                                 int32_t view_base, int64_t tab_base,
                                                 const Camera &cam, const ViewXf *views,
                                                 const TabRow *tab, float4 *geo, float4 *app,
                                                 uint4 *info, uint32_t &r0, uint32_t &r1,
                                                 uint32_t &nt) {
    uint32_t zbits = 0;
    {
        const uint32_t src = S.src[li];
        const uint32_t plane = (uint32_t)S.W * (uint32_t)S.H;
        const uint32_t k = src / plane;
        const uint32_t pix = src - k * plane;
        const uint32_t v = pix / (uint32_t)S.W;
        const uint32_t u = pix - v * (uint32_t)S.W;
        const bool in_range = k < (uint32_t)S.n_views;   // src beyond the views: no Gaussian
        const float D = in_range ? S.depth[src] : 0.f;
        const float o = ld_attr(S.opacity, S.prec, li);
        const float r = Aniso ? 1.f : ld_attr(S.radius, S.prec, li);
        bool ok = in_range && isfinite(D) && D > 0.f && o >= kAlphaMin && r > 0.f && isfinite(r);
        const ViewXf &X = views[view_base + (ok ? k : 0)];
        const TabRow *tb = tab + tab_base + (int64_t)(ok ? k : 0) * (S.W + S.H);
        TabRow A, B;
        float zkey = 0.f;
        if (ok) {
            A = tb[u];
            B = tb[S.W + v];
            // depth key: a = (u - cx)/fx, b = (v - cy)/fy (FP32 divisions of the
            // view tables), X = D a, Y = D b, z = ((M20 X + M21 Y) + M22 D) + m2,
            // every step rounded to FP32.
            const float Xc = __fmul_rn(D, A.kf), Yc = __fmul_rn(D, B.kf);
            float z = __fmul_rn(X.Mf[6], Xc);
            z = __fadd_rn(z, __fmul_rn(X.Mf[7], Yc));
            z = __fadd_rn(z, __fmul_rn(X.Mf[8], D));
            zkey = __fadd_rn(z, X.Mf[11]);
            ok = zkey >= kZNear;
        }
        if (ok) {
            const ff hu = ff_add(ff_from(A.a), ff_from(B.a));
            const ff hv = ff_add(ff_from(A.b), ff_from(B.b));
            const ff hz = ff_add(ff_from(A.c), ff_from(B.c));
            const ff nu = ff_add(ff_mul_f(hu, D), ff_from(X.mu));
            const ff nv = ff_add(ff_mul_f(hv, D), ff_from(X.mv));
            const ff nz = ff_add(ff_mul_f(hz, D), ff_from(X.mz));
            const ff uc = ff_div(nu, nz), vc = ff_div(nv, nz);
            const float z = nz.hi;
            float qlim = kQMax;
            const float qo = 2.f * __logf(255.f * o);   // box bound only (slack below)
            if (qo < qlim) qlim = qo;
            qlim = qlim * 1.0001f + 1e-4f;
            float ex, ey;
            float4 g1;
            if constexpr (!Aniso) {
                const float tx = __fdiv_rn(z, __fmul_rn(cam.fx, r));
                const float ty = __fdiv_rn(z, __fmul_rn(cam.fy, r));
                const float kx = __fmul_rn(tx, tx), ky = __fmul_rn(ty, ty);
                ex = sqrtf(__fdividef(qlim, kx)) + 1e-3f;   // box bound only (slack)
                ey = sqrtf(__fdividef(qlim, ky)) + 1e-3f;
                ok = kx > 0.f && ky > 0.f && isfinite(kx) && isfinite(ky);
                g1 = make_float4(__fmul_rn(kx, kTScale), __fmul_rn(ky, kTScale), __frcp_rn(r), o);
            } else {
                ok = ellipse_footprint(S, li, X.Mf, __fadd_rn(__fsub_rn(uc.hi, cam.cx), uc.lo),
                                       __fadd_rn(__fsub_rn(vc.hi, cam.cy), vc.lo), z, cam, o,
                                       qlim, g1, ex, ey);
            }
            ok = ok && z > 0.f && fabsf(uc.hi) < 16777216.f && fabsf(vc.hi) < 16777216.f;
            if (ok) {
                const float u0 = fmaxf(ceilf(uc.hi - ex), 0.f);
                const float u1 = fminf(floorf(uc.hi + ex), (float)(cam.W - 1));
                const float v0 = fmaxf(ceilf(vc.hi - ey), 0.f);
                const float v1 = fminf(floorf(vc.hi + ey), (float)(cam.H - 1));
                ok = u0 <= u1 && v0 <= v1;
                if (ok) {
                    const uint32_t tx0 = (uint32_t)u0 / kTile, tx1 = (uint32_t)u1 / kTile;
                    const uint32_t ty0 = (uint32_t)v0 / kTile, ty1 = (uint32_t)v1 / kTile;
                    r0 = (uint32_t)u0 | ((uint32_t)v0 << 16);
                    r1 = (uint32_t)u1 | ((uint32_t)v1 << 16);
                    nt = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
                    zbits = __float_as_uint(zkey);
                    const int iu = __float2int_rn(uc.hi), iv = __float2int_rn(vc.hi);
                    const float fu = __fadd_rn(__fsub_rn(uc.hi, (float)iu), uc.lo);
                    const float fv = __fadd_rn(__fsub_rn(vc.hi, (float)iv), vc.lo);
                    geo[2 * gid] = make_float4(__int_as_float(iu), fu, __int_as_float(iv), fv);
                    geo[2 * gid + 1] = g1;
                    const float c0 = ld_attr(S.colour, S.prec, 3 * li + 0);
                    const float c1 = ld_attr(S.colour, S.prec, 3 * li + 1);
                    const float c2 = ld_attr(S.colour, S.prec, 3 * li + 2);
                    app[gid] = make_float4(c0, c1, c2, z);
                }
            }
        }
        info[gid] = make_uint4(r0, r1, zbits, nt);
    }
}

template <bool Aniso>
__device__ __forceinline__ void preprocess_body(const SecTable &T, const Camera &cam,
                                                const ViewXf *views, const TabRow *tab,
                                                float4 *geo, float4 *app, uint4 *info,
                                                uint32_t *tile_count) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t r0 = 0, r1 = 0, nt = 0;
    if (gid < T.n_total) {
        const SecDesc &S = T.s[find_section(T, gid)];
        preprocess_gauss<Aniso>(S, gid - S.gbase, gid, S.view_base, S.tab_base, cam, views, tab,
                                geo, app, info, r0, r1, nt);
    }
    for_each_tile(r0, r1, nt, cam.tiles_x,
                  [&](uint32_t t, unsigned peers, int rank, uint32_t, uint32_t) {
                      if (rank == 0) atomicAdd(&tile_count[t], (uint32_t)__popc(peers));
                  });
}

__global__ void __launch_bounds__(256) k_preprocess(SecTable T, Camera cam, const ViewXf *views,
                                                    const TabRow *tab, float4 *geo, float4 *app,
                                                    uint4 *info, uint32_t *tile_count) {
    preprocess_body<false>(T, cam, views, tab, geo, app, info, tile_count);
}

__global__ void __launch_bounds__(256) k_preprocess_aniso(SecTable T, Camera cam,
                                                          const ViewXf *views, const TabRow *tab,
                                                          float4 *geo, float4 *app, uint4 *info,
                                                          uint32_t *tile_count) {
    preprocess_body<true>(T, cam, views, tab, geo, app, info, tile_count);
}

// Batched form (spheres): blocks of 256 Gaussian slots in a grid-stride loop;
// a block lies inside one item (item ranges start at multiples of 256), and
// the slots past an item's end get empty info.
__global__ void __launch_bounds__(256) kb_preprocess(const BatchTable *Bp, const ViewXf *views,
                                                     const TabRow *tab, float4 *geo, float4 *app,
                                                     uint4 *info, uint32_t *tile_count) {
    const BatchTable &B = *Bp;
    ItemCursor cur;
    const auto gstart = [&](int i) { return B.it[i].gbase; };
    for (int64_t g0 = (int64_t)blockIdx.x * 256; g0 < B.n_gauss; g0 += (int64_t)gridDim.x * 256) {
        const BatchItem &I = B.it[cur.at(B, gstart, g0)];
        const int64_t gid = g0 + threadIdx.x, li = gid - I.gbase;
        uint32_t r0 = 0, r1 = 0, nt = 0;
        if (li < I.n)
            preprocess_gauss<false>(B.sec[I.sec], li, gid, I.vbase, I.tab_base, I.cam, views, tab,
                                    geo, app, info, r0, r1, nt);
        else
            info[gid] = make_uint4(0u, 0u, 0u, 0u);
        uint32_t *tc = tile_count + I.tbase;
        for_each_tile(r0, r1, nt, I.cam.tiles_x,
                      [&](uint32_t t, unsigned peers, int rank, uint32_t, uint32_t) {
                          if (rank == 0) atomicAdd(&tc[t], (uint32_t)__popc(peers));
                      });
    }
}

// ---------------------------------------------------------------------------
// k_scan_tiles: one block; exclusive prefix sum of the per-tile counts into
// tile offsets (tile_off[n_tiles] = instance total) and insertion cursors.
// Flags a capacity shortage instead of letting later kernels overrun.
// Also lists, in tile order, the tiles whose lists are longer than
// kSortLongMin (long_tiles[0, st->n_long)): the long-list launches take their
// tiles from there instead of visiting every tile.
__device__ __forceinline__ void scan_tiles_body(const uint32_t *tile_count, int n_tiles,
                                                uint32_t *tile_off, uint32_t *tile_cursor,
                                                Status *st, unsigned long long cap,
                                                uint32_t *long_tiles) {
    __shared__ unsigned long long warp_sums[32];
    __shared__ unsigned long long carry;
    __shared__ uint32_t long_warp[32], long_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        carry = 0;
        long_carry = 0;
    }
    __syncthreads();
    for (int base = 0; base < n_tiles; base += 1024) {
        const int i = base + tid;
        const unsigned long long c = i < n_tiles ? tile_count[i] : 0ull;
        unsigned long long x = c;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = warp_sums[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(kFull, w, o);
                if (lane >= o) w += y;
            }
            warp_sums[lane] = w;
        }
        __syncthreads();
        const unsigned long long excl = carry + (warp ? warp_sums[warp - 1] : 0ull) + x - c;
        if (i < n_tiles) {
            tile_off[i] = (uint32_t)excl;
            tile_cursor[i] = (uint32_t)excl;
        }
        const bool is_long = i < n_tiles && c > (unsigned long long)kSortLongMin;
        const unsigned lb = __ballot_sync(kFull, is_long);
        if (lane == 0) long_warp[warp] = __popc(lb);
        __syncthreads();
        if (is_long) {
            uint32_t pos = long_carry + __popc(lb & ((1u << lane) - 1u));
            for (int w = 0; w < warp; ++w) pos += long_warp[w];
            long_tiles[pos] = (uint32_t)i;
        }
        __syncthreads();
        if (tid == 1023) carry = excl + c;
        if (tid == 0) {
            uint32_t tot = 0;
            for (int w = 0; w < 32; ++w) tot += long_warp[w];
            long_carry += tot;
        }
        __syncthreads();
    }
    if (tid == 0) {
        tile_off[n_tiles] = (uint32_t)carry;
        st->n_instances = carry;
        st->n_overflow_tiles = 0;
        st->sort_next[0] = st->sort_next[1] = 0u;
        st->n_long = long_carry;
        st->flags = carry > cap || carry >= 0xffffffffull ? kFlagCapacity : 0;
    }
}

__global__ void __launch_bounds__(1024) k_scan_tiles(const uint32_t *tile_count, int n_tiles,
                                                     uint32_t *tile_off, uint32_t *tile_cursor,
                                                     Status *st, unsigned long long cap,
                                                     uint32_t *long_tiles) {
    scan_tiles_body(tile_count, n_tiles, tile_off, tile_cursor, st, cap, long_tiles);
}

__global__ void __launch_bounds__(1024) kb_scan_tiles(const BatchTable *Bp,
                                                      const uint32_t *tile_count,
                                                      uint32_t *tile_off, uint32_t *tile_cursor,
                                                      Status *st, unsigned long long cap,
                                                      uint32_t *long_tiles) {
    scan_tiles_body(tile_count, Bp->n_tiles, tile_off, tile_cursor, st, cap, long_tiles);
}

// ---------------------------------------------------------------------------
// k_emit: one thread per Gaussian; appends (zkey << 32 | gid) to the bucket of
// every tile of its pixel box (the same tiles counted in k_preprocess), and
// the entry's block mask (box_block_mask) at the same position of bmask_u.
__device__ __forceinline__ void emit_gauss(const uint4 &in, int64_t gid, int tiles_x,
                                           uint32_t *tile_cursor, unsigned long long *bucket,
                                           uint8_t *bmask_u) {
    const unsigned long long key = ((unsigned long long)in.z << 32) | (unsigned long long)gid;
    const int lane = threadIdx.x & 31;
    for_each_tile(in.x, in.y, in.w, tiles_x,
                  [&](uint32_t t, unsigned peers, int rank, uint32_t tx, uint32_t ty) {
                      const int leader = __ffs(peers) - 1;
                      uint32_t base = 0;
                      if (lane == leader) base = atomicAdd(&tile_cursor[t], (uint32_t)__popc(peers));
                      base = __shfl_sync(peers, base, leader);
                      bucket[base + rank] = key;
                      bmask_u[base + rank] = (uint8_t)box_block_mask(in.x, in.y, tx, ty);
                  });
}

__global__ void __launch_bounds__(256) k_emit(int64_t n, const uint4 *info, Camera cam,
                                              uint32_t *tile_cursor, unsigned long long *bucket,
                                              uint8_t *bmask_u, const Status *st) {
    if (st->flags) return;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint4 in = make_uint4(0, 0, 0, 0);
    if (gid < n) in = info[gid];
    emit_gauss(in, gid, cam.tiles_x, tile_cursor, bucket, bmask_u);
}

// Batched form: blocks of 256 Gaussian slots (one item each) in a
// grid-stride loop; the item's tiles start at tile_cursor + tbase.
__global__ void __launch_bounds__(256) kb_emit(const BatchTable *Bp, const uint4 *info,
                                               uint32_t *tile_cursor, unsigned long long *bucket,
                                               uint8_t *bmask_u, const Status *st) {
    if (st->flags) return;
    const BatchTable &B = *Bp;
    ItemCursor cur;
    const auto gstart = [&](int i) { return B.it[i].gbase; };
    for (int64_t g0 = (int64_t)blockIdx.x * 256; g0 < B.n_gauss; g0 += (int64_t)gridDim.x * 256) {
        const BatchItem &I = B.it[cur.at(B, gstart, g0)];
        const int64_t gid = g0 + threadIdx.x;
        emit_gauss(info[gid], gid, I.cam.tiles_x, tile_cursor + I.tbase, bucket, bmask_u);
    }
}

// ---------------------------------------------------------------------------
// Per-tile stable LSD radix sort (one block of 512 threads per tile).
//
// Keys are 64-bit.  Pass A sorts by the depth key only: (zkey - zmin) sits in
// the high word and only its significant bits are sorted.  If two entries
// then share a depth key, pass B re-sorts by (zrel << bits_g | gid - gmin),
// which orders ties by Gaussian id.  A launch handles the tiles whose list
// length lies in (lo, hi]; lists of up to smem_n entries are sorted in shared
// memory, longer ones in place in the tile's own range of the bucket and its
// twin buffer.  Next to each sorted id goes the entry's 8-bit block mask
// (tile_block_mask): which 8x4 pixel blocks of the tile it can reach.

constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;

// Lanes of the warp holding the same nbits-bit digit as this lane (valid lanes
// only): one ballot per digit bit, cheaper than a general match instruction.
__device__ __forceinline__ unsigned digit_peers(unsigned d, int nbits, bool valid) {
    unsigned m = __ballot_sync(kFull, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        if (b < nbits) {
            const bool bit = (d >> b) & 1u;
            const unsigned bb = __ballot_sync(kFull, bit);
            m &= bit ? bb : ~bb;
        }
    }
    return m;
}

// One stable LSD pass on bits [shift, shift + nbits) of the keys in[0, n)
// into out.  Each warp histograms its contiguous chunk in groups of 32 (peer
// lanes holding the same digit found with one ballot per digit bit), the
// block scans the per-warp histograms in (digit, warp) order, and each warp
// scatters its chunk.  With G > 0 and chunks of at most G groups, every
// lane keeps its digit, its rank among its peers and their count in
// registers between the two phases instead of ranking twice.
template <int G>
__device__ __forceinline__ void radix_pass(const unsigned long long *in, unsigned long long *out,
                                           int n, int shift, int nbits, uint32_t *hist) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned dmask = (1u << nbits) - 1u;
    const int per = (n + kSortWarps - 1) / kSortWarps;
    const int lo = min(n, warp * per), hi = min(n, lo + per);
    const unsigned lt = (1u << lane) - 1u;
    const bool cache = G > 0 && per <= G * 32;
    uint32_t pk[G > 0 ? G : 1];
    for (int i = tid; i < kSortWarps * 256; i += kSortThreads) hist[i] = 0;
    __syncthreads();
    uint32_t *h = hist + warp * 256;
    if (cache) {
#pragma unroll
        for (int gi = 0; gi < (G > 0 ? G : 1); ++gi) {
            if (lo + gi * 32 >= hi) break;
            const int i = lo + gi * 32 + lane;
            const bool valid = i < hi;
            const unsigned d = valid ? (unsigned)(in[i] >> shift) & dmask : 0u;
            const unsigned peers = digit_peers(d, nbits, valid);
            const unsigned rank = __popc(peers & lt), cnt = __popc(peers);
            pk[gi] = d | (rank << 8) | (cnt << 13);
            if (valid && rank == 0) h[d] += cnt;
            __syncwarp();
        }
    } else {
        // without the register cache (the long lists, read from global
        // memory in the largest class) the keys of the next two groups are
        // in flight while a group is ranked
        constexpr bool ahead = G == 0;
        unsigned long long k1 = ahead && lo + lane < hi ? in[lo + lane] : 0ull;
        unsigned long long k2 = ahead && lo + 32 + lane < hi ? in[lo + 32 + lane] : 0ull;
        for (int i0 = lo; i0 < hi; i0 += 32) {
            const int i = i0 + lane;
            const bool valid = i < hi;
            unsigned long long k = 0ull;
            if (ahead) {
                k = k1;
                k1 = k2;
                k2 = i + 64 < hi ? in[i + 64] : 0ull;
            } else if (valid) {
                k = in[i];
            }
            const unsigned d = valid ? (unsigned)(k >> shift) & dmask : 0u;
            const unsigned peers = digit_peers(d, nbits, valid);
            if (valid && lane == __ffs(peers) - 1) h[d] += __popc(peers);
            __syncwarp();
        }
    }
    __syncthreads();
    // exclusive scan in (digit, warp) order
    __shared__ uint32_t dsum[256];
    if (tid < 256) {
        uint32_t run = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = hist[w * 256 + tid];
            hist[w * 256 + tid] = run;
            run += c;
        }
        dsum[tid] = run;
    }
    __syncthreads();
    if (tid < 32) {
        uint32_t v[8], tot = 0;
        for (int j = 0; j < 8; ++j) {
            v[j] = dsum[tid * 8 + j];
            tot += v[j];
        }
        uint32_t x = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, x, o);
            if (tid >= o) x += y;
        }
        uint32_t run = x - tot;
        for (int j = 0; j < 8; ++j) {
            dsum[tid * 8 + j] = run;
            run += v[j];
        }
    }
    __syncthreads();
    if (tid < 256)
        for (int w = 0; w < kSortWarps; ++w) hist[w * 256 + tid] += dsum[tid];
    __syncthreads();
    if (cache) {
#pragma unroll
        for (int gi = 0; gi < (G > 0 ? G : 1); ++gi) {
            if (lo + gi * 32 >= hi) break;
            const int i = lo + gi * 32 + lane;
            const bool valid = i < hi;
            const unsigned d = pk[gi] & 0xFFu, rank = (pk[gi] >> 8) & 31u, cnt = pk[gi] >> 13;
            if (valid) out[h[d] + rank] = in[i];
            __syncwarp();
            if (valid && rank == 0) h[d] += cnt;
            __syncwarp();
        }
    } else {
        constexpr bool ahead = G == 0;
        unsigned long long k1 = ahead && lo + lane < hi ? in[lo + lane] : 0ull;
        unsigned long long k2 = ahead && lo + 32 + lane < hi ? in[lo + 32 + lane] : 0ull;
        for (int i0 = lo; i0 < hi; i0 += 32) {
            const int i = i0 + lane;
            const bool valid = i < hi;
            unsigned long long key = 0ull;
            if (ahead) {
                key = k1;
                k1 = k2;
                k2 = i + 64 < hi ? in[i + 64] : 0ull;
            } else if (valid) {
                key = in[i];
            }
            const unsigned d = valid ? (unsigned)(key >> shift) & dmask : 0u;
            const unsigned peers = digit_peers(d, nbits, valid);
            if (valid) {
                const uint32_t pos = h[d] + __popc(peers & lt);
                out[pos] = key;
            }
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) h[d] += __popc(peers);
            __syncwarp();
        }
    }
    __syncthreads();
}

__device__ __forceinline__ unsigned bits_of(uint32_t span) { return span ? 32 - __clz(span) : 0; }

// Writes the sorted ids of a tile and their block masks, the masks computed
// from the records (used where the sort could not carry them): id_of(i)
// gives entry i.  Without records (geo NULL: ellipse records, which the
// sphere test does not read) every block is marked.
struct SortOut {
    uint32_t *__restrict__ sorted;
    uint8_t *__restrict__ bmask;
    const float4 *__restrict__ geo;
    Camera cam;
    uint32_t start;
    int tx, ty;
    template <class F>
    __device__ __forceinline__ void put_all(int n, int tid, F id_of) const {
        for (int i = tid; i < n; i += kSortThreads) {
            const uint32_t g = id_of(i);
            sorted[start + i] = g;
            bmask[start + i] = geo ? (uint8_t)tile_block_mask(__ldg(geo + 2 * (size_t)g),
                                                              __ldg(geo + 2 * (size_t)g + 1), tx,
                                                              ty, cam)
                                   : (uint8_t)0xFFu;
        }
    }
};

// Sorts one tile's list [start, start + n) (2 <= n) with the whole block
// (G: register-cached radix ranks for chunks of up to G groups per warp).
// Lists sorted in shared memory carry (block mask << 24 | position in the
// bucket) in the low word, so the masks written by k_emit travel with the
// entries and the ids are read back from the bucket (which stays intact);
// lists sorted in place carry the id and their masks are recomputed.
template <int G>
__device__ __forceinline__ void sort_tile(unsigned long long *bucket, unsigned long long *alt,
                                          const uint8_t *bmask_u, const SortOut &out,
                                          Status *st, uint32_t start, int n, int smem_n,
                                          unsigned long long *sm, uint32_t (*red)[kSortWarps],
                                          int tid, int lane, int warp) {
    const bool big = n > smem_n;
    // lists sorted in global memory need only the histograms in shared memory
    uint32_t *hist = reinterpret_cast<uint32_t *>(big ? sm : sm + 2 * smem_n);
    unsigned long long *A = big ? bucket + start : sm;
    unsigned long long *B = big ? alt + start : sm + smem_n;
    if (big && tid == 0) atomicAdd(&st->n_overflow_tiles, 1ull);
    const unsigned long long *orig = bucket + start;
    // id of an entry from its low word
    auto id_of = [&](uint32_t lw) { return big ? lw : (uint32_t)orig[lw & 0xffffffu]; };
    uint32_t zmin = 0xffffffffu, zmax = 0, gmin = 0xffffffffu, gmax = 0;
    for (int i = tid; i < n; i += kSortThreads) {
        const unsigned long long k = bucket[start + i];
        const uint32_t z = (uint32_t)(k >> 32), g = (uint32_t)k;
        zmin = min(zmin, z);
        zmax = max(zmax, z);
        gmin = min(gmin, g);
        gmax = max(gmax, g);
    }
    zmin = __reduce_min_sync(kFull, zmin);
    zmax = __reduce_max_sync(kFull, zmax);
    gmin = __reduce_min_sync(kFull, gmin);
    gmax = __reduce_max_sync(kFull, gmax);
    if (lane == 0) {
        red[0][warp] = zmin;
        red[1][warp] = zmax;
        red[2][warp] = gmin;
        red[3][warp] = gmax;
    }
    __syncthreads();
    zmin = red[0][0];
    zmax = red[1][0];
    gmin = red[2][0];
    gmax = red[3][0];
    for (int w = 1; w < kSortWarps; ++w) {
        zmin = min(zmin, red[0][w]);
        zmax = max(zmax, red[1][w]);
        gmin = min(gmin, red[2][w]);
        gmax = max(gmax, red[3][w]);
    }
    const unsigned bz = bits_of(zmax - zmin), bg = bits_of(gmax - gmin);
    // pass A: depth key relative to the tile minimum in the high word
    for (int i = tid; i < n; i += kSortThreads) {
        const unsigned long long k = orig[i];
        const uint32_t lw = big ? (uint32_t)k : ((uint32_t)bmask_u[start + i] << 24) | (uint32_t)i;
        A[i] = ((unsigned long long)((uint32_t)(k >> 32) - zmin) << 32) | lw;
    }
    __syncthreads();
    unsigned long long *cur = A, *oth = B;
    for (unsigned b = 0; b < bz; b += 8) {
        radix_pass<G>(cur, oth, n, 32 + b, min(8u, bz - b), hist);
        unsigned long long *tmp = cur;
        cur = oth;
        oth = tmp;
    }
    // Runs of equal depth keys (a few per tile: ~2700 FP32 keys over a depth
    // range of some 2^22 values collide) are ordered by id in place, each by
    // the thread at its start; only a run longer than kMaxRun (e.g. a
    // fronto-parallel wall seen from its own view) needs pass B.  Threads
    // only move the low words inside their own run, so the depth keys other
    // threads read stay fixed.
    constexpr int kMaxRun = 32;
    int long_run = 0;
    for (int i = tid; i < n; i += kSortThreads) {
        const uint32_t zi = (uint32_t)(cur[i] >> 32);
        const bool first = i == 0 || (uint32_t)(cur[i - 1] >> 32) != zi;
        if (!first || i + 1 >= n || (uint32_t)(cur[i + 1] >> 32) != zi) continue;
        int e = i + 1;
        while (e < n && e - i <= kMaxRun && (uint32_t)(cur[e] >> 32) == zi) ++e;
        if (e - i > kMaxRun) {
            long_run = 1;
            continue;
        }
        for (int a = i + 1; a < e; ++a) {   // insertion sort by id
            const unsigned long long k = cur[a];
            const uint32_t gk = id_of((uint32_t)k);
            int b = a - 1;
            while (b >= i && id_of((uint32_t)cur[b]) > gk) {
                cur[b + 1] = cur[b];
                --b;
            }
            cur[b + 1] = k;
        }
    }
    long_run = __syncthreads_or(long_run);
    if (!long_run) {
        if (big) {
            out.put_all(n, tid, [&](int i) { return (uint32_t)cur[i]; });
        } else {
            for (int i = tid; i < n; i += kSortThreads) {
                const uint32_t lw = (uint32_t)cur[i];
                out.sorted[start + i] = id_of(lw);
                out.bmask[start + i] = (uint8_t)(lw >> 24);
            }
        }
        return;
    }
    // pass B: (zrel, gid - gmin) packed into bz + bg <= 64 bits
    for (int i = tid; i < n; i += kSortThreads) {
        const unsigned long long k = cur[i];
        const unsigned long long zr = k >> 32, gr = id_of((uint32_t)k) - gmin;
        cur[i] = (bg == 64 ? 0ull : (zr << bg)) | gr;
    }
    __syncthreads();
    const unsigned tot = bz + bg;
    for (unsigned b = 0; b < tot; b += 8) {
        radix_pass<G>(cur, oth, n, b, min(8u, tot - b), hist);
        unsigned long long *tmp = cur;
        cur = oth;
        oth = tmp;
    }
    const unsigned long long gm = bg >= 64 ? ~0ull : ((1ull << bg) - 1ull);
    out.put_all(n, tid, [&](int i) { return gmin + (uint32_t)(cur[i] & gm); });
}

template <int G>
// With B != NULL (batched launches) the tiles are those of all work items
// (B->n_tiles), each with its item's camera and tile coordinates.
__device__ __forceinline__ void sort_tiles_body(const uint32_t *tile_off, int n_tiles,
                                                unsigned long long *bucket,
                                                unsigned long long *alt, const uint8_t *bmask_u,
                                                uint32_t *sorted, uint8_t *bmask,
                                                const float4 *geo, const Camera &cam, Status *st,
                                                int smem_n, int lo, int hi,
                                                const BatchTable *B = nullptr,
                                                uint32_t *wctr = nullptr,
                                                const uint32_t *long_tiles = nullptr) {
    extern __shared__ unsigned long long sm[];
    __shared__ uint32_t red[4][kSortWarps];
    __shared__ int s_next;
    if (st->flags) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (B) n_tiles = B->n_tiles;
    ItemCursor cur;
    // A launch may have fewer blocks than tiles: blocks stride over the tiles,
    // or, in the long-list launches, take the next of the tiles the tile scan
    // listed from a work counter (the long lists vary in length by 5x: a
    // fixed stride leaves the block with the longest share running alone at
    // the end).
    auto next = [&](int j) {
        if (!wctr) return j + (int)gridDim.x;
        __syncthreads();   // every thread has read the previous s_next
        if (tid == 0) s_next = (int)atomicAdd(wctr, 1u);
        __syncthreads();
        return s_next;
    };
    const int n_iter = wctr ? (int)st->n_long : n_tiles;
    for (int j = wctr ? next(0) : (int)blockIdx.x; j < n_iter; j = next(j)) {
        const int t = wctr ? (int)long_tiles[j] : j;
        const uint32_t start = tile_off[t];
        const int n = (int)(tile_off[t + 1] - start);
        if (n <= lo || n > hi) continue;   // another launch sorts this size class
        const BatchItem *I =
            B ? &B->it[cur.at(*B, [&](int i) { return (int64_t)B->it[i].tbase; }, t)] : nullptr;
        const Camera &c = I ? I->cam : cam;
        const int lt = I ? t - I->tbase : t;
        const SortOut out{sorted, bmask, geo, c, start, lt % c.tiles_x, lt / c.tiles_x};
        if (n == 1) {
            if (tid == 0) {
                sorted[start] = (uint32_t)bucket[start];
                bmask[start] = bmask_u[start];
            }
            continue;
        }
        sort_tile<G>(bucket, alt, bmask_u, out, st, start, n, smem_n, sm, red, tid, lane, warp);
        __syncthreads();   // shared memory is reused by the next tile
    }
}

// One kernel per list-length class, each caching the radix ranks of up to
// (class limit / 16 warps) entries per warp, with registers capped for two
// blocks of 512 threads per SM; the long lists (one block per SM) and the
// lists sorted in global memory (two blocks per SM, shared memory for the
// histograms only) rank twice.
// CTR: the work counter of the launch (-1: blocks stride over the tiles).
#define VT_SORT_KERNEL(name, G, MIN_BLOCKS, CTR)                                                 \
    __global__ void __launch_bounds__(kSortThreads, MIN_BLOCKS) name(                            \
        const uint32_t *tile_off, int n_tiles, unsigned long long *bucket,                       \
        unsigned long long *alt, const uint8_t *bmask_u, uint32_t *sorted, uint8_t *bmask,       \
        const float4 *geo, Camera cam, Status *st, int smem_n, int lo, int hi,                   \
        const uint32_t *long_tiles) {                                                            \
        sort_tiles_body<G>(tile_off, n_tiles, bucket, alt, bmask_u, sorted, bmask, geo, cam, st, \
                           smem_n, lo, hi, nullptr,                                              \
                           CTR < 0 ? nullptr : &st->sort_next[CTR < 0 ? 0 : CTR], long_tiles);   \
    }
VT_SORT_KERNEL(k_sort_tiles, 3, 2, -1)
VT_SORT_KERNEL(k_sort_tiles_mid, 7, 2, -1)
VT_SORT_KERNEL(k_sort_tiles_large, 12, 2, -1)
VT_SORT_KERNEL(k_sort_tiles_long, 0, 1, 0)
VT_SORT_KERNEL(k_sort_tiles_xl, 0, 2, 1)
#undef VT_SORT_KERNEL

// Batched forms: the same classes over the tiles of every work item.
#define VT_SORT_KERNEL_B(name, G, MIN_BLOCKS, CTR)                                               \
    __global__ void __launch_bounds__(kSortThreads, MIN_BLOCKS) name(                            \
        const BatchTable *B, const uint32_t *tile_off, unsigned long long *bucket,               \
        unsigned long long *alt, const uint8_t *bmask_u, uint32_t *sorted, uint8_t *bmask,       \
        const float4 *geo, Status *st, int smem_n, int lo, int hi,                               \
        const uint32_t *long_tiles) {                                                            \
        sort_tiles_body<G>(tile_off, 0, bucket, alt, bmask_u, sorted, bmask, geo, B->it[0].cam,  \
                           st, smem_n, lo, hi, B,                                                \
                           CTR < 0 ? nullptr : &st->sort_next[CTR < 0 ? 0 : CTR], long_tiles);   \
    }
VT_SORT_KERNEL_B(kb_sort_tiles, 3, 2, -1)
VT_SORT_KERNEL_B(kb_sort_tiles_mid, 7, 2, -1)
VT_SORT_KERNEL_B(kb_sort_tiles_large, 12, 2, -1)
VT_SORT_KERNEL_B(kb_sort_tiles_long, 0, 1, 0)
VT_SORT_KERNEL_B(kb_sort_tiles_xl, 0, 2, 1)
#undef VT_SORT_KERNEL_B

}  // namespace vt
