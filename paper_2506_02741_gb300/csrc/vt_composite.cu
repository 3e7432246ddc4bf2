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

// The same for an ellipse record (a', b', c'): row by row the pixels with
// a' du^2 + b' dv du + c' dv^2 >= t_min lie in the interval of du around
// b' dv / (2 |a'|) of half-width sqrt((b' dv)^2 + 4 |a'| (c' dv^2 - t_min))
// / (2 |a'|).  The threshold is loosened by 1e-3 relative and the interval
// widened by 1e-3 px plus 1e-4 of its centre and half-width.
__device__ __forceinline__ uint32_t pixel_mask_aniso(float du0, float dv0, float a, float b,
                                                     float c, float tmin, int lxmax, int lymax) {
    const float tl = tmin * 1.001f - 1e-5f;
    const float na = -a;                          // > 0
    const float h2 = 0.5f * rcp_approx(na);       // 1 / (2 |a'|)
    uint32_t m = 0u;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float dv = dv0 + (float)r;
        const float bd = b * dv;
        const float disc = bd * bd + 4.f * na * (c * dv * dv - tl);
        if (r <= lymax && disc >= 0.f) {
            const float ctr = bd * h2;
            const float hw0 = sqrt_approx(disc) * h2;
            const float hw = hw0 * 1.0001f + 1e-3f + 1e-4f * (fabsf(ctr) + hw0);
            const int lo = max(0, (int)ceilf(ctr - hw - du0));
            const int hi = min(lxmax, (int)floorf(ctr + hw - du0));
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
// Aniso = true composites ellipsoid records (a', b', c', o): their pixel
// sets come from pixel_mask_aniso and the pair exponent from pair_t_aniso.
constexpr int kQueue = 256;   // ring of list indices per warp (>= 31 + 128)

template <bool Aniso>
__device__ __forceinline__ void fwd_body(
    const Camera &cam, int tile, const uint32_t *tile_off, const uint32_t *sorted,
    const uint8_t *bmask, const float4 *geo, const float4 *app, float *rgb, float *depth,
    float *sil, uint32_t *pix_last, uint32_t *pix_nadd, float *pix_T, uint2 *plist, int plist_cap,
    uint32_t *blk_ovf, const Status *st) {
    // two staging halves of 32 entries per warp (see the walk below)
    __shared__ float4 s_f[kWarps][64], s_k[kWarps][64], s_c[kWarps][64];
    __shared__ uint32_t s_gid[kWarps][64], s_idx[kWarps][64];
    __shared__ uint32_t s_q[kWarps][kQueue];
    __shared__ float s_b[Aniso ? kWarps : 1][64];   // b' of the ellipse records
    if (st->flags) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lx = lane & 7, ly = lane >> 3;
    const float lxf = (float)lx, lyf = (float)ly;
    float4 (&fs)[64] = s_f[warp];
    float4 (&ks)[64] = s_k[warp];
    float4 (&cs)[64] = s_c[warp];
    uint32_t (&ids)[64] = s_gid[warp];
    uint32_t (&lidx)[64] = s_idx[warp];
    float (&bs)[64] = s_b[Aniso ? warp : 0];
    uint32_t (&q)[kQueue] = s_q[warp];
    const size_t HW = (size_t)cam.W * cam.H;

    const int item = tile * kWarps + warp;
    const int sub = warp;
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
    int lastj = -1;   // staging slot of the last Gaussian added in this walk
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
    // Each lane walks its own candidates: lanes work on different Gaussians
    // at once.  The walk of a batch is lagged by one: while any lane still
    // has candidates of the previous batch (cand_old, half ho), every lane
    // takes its next candidate from there, or, once its own are done, from
    // the current batch (cand_new, half hn), so lanes with few candidates
    // run ahead instead of idling until the busiest pixel of the batch is
    // through.  Per lane the order stays the list order.
    uint32_t cand_old = 0u;
    int ho = 1;
    // next candidate of this lane in walk order (previous batch first)
    auto pick = [&](uint32_t &cand_new, int hn, int &j) {
        const bool fo = cand_old != 0u;
        const uint32_t src = fo ? cand_old : cand_new;
        if (!src) return false;
        j = (fo ? ho : hn) * 32 + __ffs(src) - 1;
        if (fo)
            cand_old &= cand_old - 1u;
        else
            cand_new &= cand_new - 1u;
        return true;
    };
    auto exponent = [&](int j, float4 &k) {
        const float4 f = fs[j];
        k = ks[j];
        const float du = __fsub_rn(__fadd_rn(f.x, lxf), f.z);
        const float dv = __fsub_rn(__fadd_rn(f.y, lyf), f.w);
        return Aniso ? pair_t_aniso(du, dv, k.x, bs[j], k.y) : pair_t(du, dv, k.x, k.y);
    };
    // composite candidate j (exponent t >= t_min, G = 2^t); false once the
    // pixel terminates
    auto add = [&](int j, float G, const float4 &k, uint32_t &cand_new) {
        const float al = fminf(__fmul_rn(k.w, G), kAlphaClamp);
        const float Tn = __fmaf_rn(-al, T, T);   // T (1 - alpha), one rounding
        if (Tn < kTMin) {
            done = true;
            cand_old = 0u;
            cand_new = 0u;
            return false;
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
        lastj = j;   // its list index is read once the walk is through
        ++nadd;
        return true;
    };
    // two candidates per step: their exponents and 2^t are independent and
    // overlap; the second is composited after the first, unless the first
    // terminated the pixel
    auto walk = [&](uint32_t &cand_new, int hn) {
        while (__any_sync(kFullMask, cand_old != 0u)) {
            int ja = 0, jb = 0;
            if (!pick(cand_new, hn, ja)) continue;
            const bool two = pick(cand_new, hn, jb);
            float4 ka, kb;
            const float ta = exponent(ja, ka);
            const float tb = two ? exponent(jb, kb) : 0.f;
            const float Ga = exp2_approx(ta), Gb = exp2_approx(tb);
            if (ta >= ka.z && !add(ja, Ga, ka, cand_new)) continue;
            if (two && tb >= kb.z) add(jb, Gb, kb, cand_new);
        }
        if (lastj >= 0) {   // both staging halves are intact until the next batch
            last = lidx[lastj] + 1u;
            lastj = -1;
        }
    };
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
        uint32_t pm = 0u;
        if (lane < cnt)
            pm = Aniso ? pixel_mask_aniso(ku - g0.y, kv - g0.w, g1.x, g1.y, g1.z, tmin, lxmaxi,
                                          lymaxi)
                       : pixel_mask(ku - g0.y, kv - g0.w, g1.x, g1.y, tmin, lxmaxi, lymaxi);
        if (!__any_sync(kFullMask, pm != 0u)) continue;
        // stage the batch in the half that the previous batch does not hold
        const int hn = ho ^ 1, sl = hn * 32 + lane;
        __syncwarp();
        fs[sl] = make_float4(ku, kv, g0.y, g0.w);
        ks[sl] = make_float4(g1.x, Aniso ? g1.z : g1.y, tmin, g1.w);
        if (Aniso) bs[sl] = g1.y;
        cs[sl] = a;
        ids[sl] = gid;
        lidx[sl] = idx;
        // this pixel's candidates of the batch, in list order (bit j = entry j)
        uint32_t cand_new = transpose32(pm, lane);
        __syncwarp();
        if (done) cand_new = 0u;
        walk(cand_new, hn);
        cand_old = cand_new;
        ho = hn;
    }
    uint32_t none = 0u;
    walk(none, ho ^ 1);   // the last batch's remaining candidates
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

__global__ void __launch_bounds__(kBlockPix) k_composite_fwd(
    Camera cam, const uint32_t *tile_off, const uint32_t *sorted, const uint8_t *bmask,
    const float4 *geo, const float4 *app, float *rgb, float *depth, float *sil,
    uint32_t *pix_last, uint32_t *pix_nadd, float *pix_T, uint2 *plist, int plist_cap,
    uint32_t *blk_ovf, const Status *st) {
    fwd_body<false>(cam, blockIdx.x, tile_off, sorted, bmask, geo, app, rgb, depth, sil, pix_last,
                    pix_nadd, pix_T, plist, plist_cap, blk_ovf, st);
}

__global__ void __launch_bounds__(kBlockPix) k_composite_fwd_aniso(
    Camera cam, const uint32_t *tile_off, const uint32_t *sorted, const uint8_t *bmask,
    const float4 *geo, const float4 *app, float *rgb, float *depth, float *sil,
    uint32_t *pix_last, uint32_t *pix_nadd, float *pix_T, uint2 *plist, int plist_cap,
    uint32_t *blk_ovf, const Status *st) {
    fwd_body<true>(cam, blockIdx.x, tile_off, sorted, bmask, geo, app, rgb, depth, sil, pix_last,
                   pix_nadd, pix_T, plist, plist_cap, blk_ovf, st);
}

// Next tile of a persistent batched stage: thread 0 takes it from the work
// counter, the block reads it after a barrier.
__device__ __forceinline__ int next_tile(uint32_t *ctr) {
    __shared__ int s_next;
    __syncthreads();   // every thread has read the previous value
    if (threadIdx.x == 0) s_next = (int)atomicAdd(ctr, 1u);
    __syncthreads();
    return s_next;
}

// Batched forward: the tiles of every work item, taken one at a time from a
// work counter by a persistent grid; each item's images are its own image
// planes (rgb, depth, silhouette) and its per-pixel state starts at pbase.
__global__ void __launch_bounds__(kBlockPix, 3) kb_composite_fwd(
    const BatchTable *Bp, uint32_t *ctr, const uint32_t *tile_off, const uint32_t *sorted,
    const uint8_t *bmask, const float4 *geo, const float4 *app, uint32_t *pix_last,
    uint32_t *pix_nadd, float *pix_T, uint2 *plist, int plist_cap, uint32_t *blk_ovf,
    const Status *st) {
    const BatchTable &B = *Bp;
    ItemCursor cur;
    const auto tstart = [&](int i) { return (int64_t)B.it[i].tbase; };
    for (int t = next_tile(ctr); t < B.n_tiles; t = next_tile(ctr)) {
        const BatchItem &I = B.it[cur.at(B, tstart, t)];
        const int64_t P = (int64_t)I.cam.W * I.cam.H;
        fwd_body<false>(I.cam, t - I.tbase, tile_off + I.tbase, sorted, bmask, geo, app, I.image,
                        I.image + 3 * P, I.image + 4 * P, pix_last + I.pbase, pix_nadd + I.pbase,
                        pix_T + I.pbase, plist ? plist + I.pbase * (int64_t)plist_cap : nullptr,
                        plist_cap, blk_ovf + (int64_t)I.tbase * kWarps, st);
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
// the warp in float-float and over the block in FP64, and written as one
// partial per tile.


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

// Warp sum of FP32 values in float-float (TwoSum-based additions, error
// ~2^-47 of the sum of magnitudes): FP64 arithmetic is a narrow pipe on this
// part, FP32 is not.  Every lane gets the same sum; to_double() widens it.
__device__ __forceinline__ ff warp_sum_ff(float v) {
    ff a{v, 0.f};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        a = ff_add(a, ff{__shfl_xor_sync(kFullMask, a.hi, o), __shfl_xor_sync(kFullMask, a.lo, o)});
    return a;
}

__device__ __forceinline__ double to_double(ff a) { return (double)a.hi + (double)a.lo; }

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

// The footprint-independent part of a back-to-front step: the Gaussian's
// alpha, the transmittance in front of it (the forward's, or recovered by
// division), its weight w and dL/dalpha from the pixel's running sums;
// bwd_advance then moves the sums past it.
struct BwdStep {
    float om, Ti, w, dal;
};

__device__ __forceinline__ BwdStep bwd_step(BwdPixel &P, const float4 &a, float ah,
                                            float Ti_fwd) {
    BwdStep S;
    const float al = fminf(ah, kAlphaClamp);
    S.om = 1.f - al;
    // (the division only where no forward transmittance was recorded)
    if (Ti_fwd >= 0.f)
        S.Ti = Ti_fwd;
    else
        S.Ti = P.T / S.om;
    S.w = al * S.Ti;
    const float z = a.w;
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
    S.dal = __fdividef(num, S.om);   // om in [0.01, 1]: within 2 ulp
    return S;
}

__device__ __forceinline__ void bwd_advance(BwdPixel &P, const float4 &a, const BwdStep &S) {
    const float e0 = a.x - P.cr0, e1 = a.y - P.cr1, e2 = a.z - P.cr2, ez = a.w - P.zr;
    P.A0 = __fmaf_rn(S.w, e0, P.A0);
    P.A1 = __fmaf_rn(S.w, e1, P.A1);
    P.A2 = __fmaf_rn(S.w, e2, P.A2);
    P.Bd = __fmaf_rn(S.w, ez, P.Bd);
    P.Sb += S.w;
    P.T = S.Ti;
}

// One added Gaussian of the pixel, visited back to front (g0, g1: footprint
// record with 1/r in g1.z, a: colour and depth z, t: exponent of pair_t,
// G = 2^t, ah = o G).  Returns its colour / opacity / radius gradient terms
// and adds its pose terms to acc.  Ti_fwd >= 0 is the forward's transmittance in front
// of this Gaussian (recorded in the per-pixel list); otherwise it is
// recovered by division, which accumulates the rounding of every Gaussian
// behind.  Twist = true accumulates only what the twist gradient needs:
// acc.a[0..2] = sum (z gy - y gz, x gz - z gx, y gx - x gy) (the
// antisymmetric part of sum x g^T) and acc.a[3..5] = sum g.
template <bool Twist = false>
__device__ __forceinline__ void bwd_pair(BwdPixel &P, const float4 &g0, const float4 &g1,
                                         const float4 &a, float t, float du, float dv, float G,
                                         float ah, const Camera &cam, bool want_pose, PoseAcc &acc,
                                         float &dc0, float &dc1, float &dc2, float &dop,
                                         float &drd, bool want_geo, float &gxo, float &gyo,
                                         float &gzo, float Ti_fwd = -1.f) {
    const float ifx = 1.f / cam.fx, ify = 1.f / cam.fy;
    const BwdStep S = bwd_step(P, a, ah, Ti_fwd);
    const float w = S.w, dal = S.dal;
    const float z = a.w, q = t * kQFromT;
    const float ir = g1.z, ir2 = ir * ir;
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
        if constexpr (Twist) {
            acc.a[0] = __fmaf_rn(-X[1], gz, __fmaf_rn(X[2], gy, acc.a[0]));
            acc.a[1] = __fmaf_rn(-X[2], gx, __fmaf_rn(X[0], gz, acc.a[1]));
            acc.a[2] = __fmaf_rn(-X[0], gy, __fmaf_rn(X[1], gx, acc.a[2]));
            acc.a[3] += gx;
            acc.a[4] += gy;
            acc.a[5] += gz;
        } else {
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
    }
    bwd_advance(P, a, S);
}

// The same step for an ellipse record g1 = (a', b', c', o): with
// dL/dt = dL/dalpha ahat ln 2 below the clamp, the pair adds
//   dL/d(a', b', c') = dL/dt (du^2, du dv, dv^2),
//   dL/du_c = -dL/dt (2 a' du + b' dv),  dL/dv_c = -dL/dt (b' du + 2 c' dv),
// and the direct depth term gD w; the per-Gaussian pass (k_aniso_chain)
// turns their sums into scale, quaternion and pose gradients.
__device__ __forceinline__ void bwd_pair_aniso(BwdPixel &P, const float4 &g1, const float4 &a,
                                               float du, float dv, float G, float ah,
                                               float &dc0, float &dc1, float &dc2, float &dop,
                                               float4 &dgq, float2 &dm, float Ti_fwd) {
    const BwdStep S = bwd_step(P, a, ah, Ti_fwd);
    dc0 = P.gC0 * S.w;
    dc1 = P.gC1 * S.w;
    dc2 = P.gC2 * S.w;
    float dt = 0.f;
    dop = 0.f;
    if (ah < kAlphaClamp) {
        dop = S.dal * G;
        dt = S.dal * ah * kLn2;
    }
    const float tu = dt * du, tv = dt * dv;
    dgq = make_float4(tu * du, tu * dv, tv * dv, P.gD * S.w);
    dm = make_float2(-(2.f * g1.x * tu + g1.y * tv), -(g1.y * tu + 2.f * g1.z * tv));
    bwd_advance(P, a, S);
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

// Ellipsoids: (colour, opacity) as above when the section wants them; the
// conic / depth terms and the centre terms when the pose gradient or the
// section's scale / quaternion gradients are wanted.
__device__ __forceinline__ void add_pair_grads_aniso(const SecTable &Tab, int64_t g, bool want_attr,
                                                     bool want_pose, float dc0, float dc1,
                                                     float dc2, float dop, const float4 &dgq,
                                                     const float2 &dm, float4 *acc4,
                                                     float4 *accg, float2 *accm) {
    const SecDesc &S = Tab.s[find_section(Tab, g)];
    if (want_attr && (S.d_colour || S.d_opacity))
        atomicAdd(acc4 + g, make_float4(dc0, dc1, dc2, dop));
    if (want_pose || (want_attr && (S.d_scale || S.d_rot))) {
        atomicAdd(accg + g, dgq);
        atomicAdd(accm + g, dm);
    }
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

// Block sum of the per-lane pose terms (warps in float-float, the block's
// eight warp sums in FP64, fixed order), written as the tile's partial.
__device__ __forceinline__ void write_pose_partial(const PoseAcc &acc, double (*s_pose)[12],
                                                   double *pose_partials, int tile) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        const ff v = warp_sum_ff(acc.a[i]);
        if (lane == 0) s_pose[warp][i] = to_double(v);
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        double v = 0.0;
        for (int w = 0; w < kBlockPix / 32; ++w) v += s_pose[w][threadIdx.x];
        pose_partials[(size_t)tile * 12 + threadIdx.x] = v;
    }
}

// The same for the twist-only terms (bwd_pair<true>), written in the slots
// of the full partial that the twist is formed from (k_pose_finalize:
// dL/dphi = (A21 - A12, A02 - A20, A10 - A01), dL/drho = -s): A21, A02, A10
// hold the three sums, the other A slots zero, so tiles summed by the full
// terms (the tile replay) and by these add up in the same slots.
__device__ __forceinline__ void write_twist_partial(const PoseAcc &acc, double (*s_pose)[12],
                                                    double *pose_partials, int tile) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const ff v = warp_sum_ff(acc.a[i]);
        if (lane == 0) s_pose[warp][i] = to_double(v);
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        // slot -> twist sum: A02 <- 1, A10 <- 2, A21 <- 0, s <- 3..5
        const int src = threadIdx.x == 2 ? 1 : threadIdx.x == 3 ? 2 : threadIdx.x == 7 ? 0
                      : threadIdx.x >= 9 ? threadIdx.x - 6 : -1;
        double v = 0.0;
        if (src >= 0)
            for (int w = 0; w < kBlockPix / 32; ++w) v += s_pose[w][src];
        pose_partials[(size_t)tile * 12 + threadIdx.x] = v;
    }
}

// One ellipse entry of a replay batch for the whole warp (every lane one
// pixel): the lanes whose pixel added it take their step, and the warp's
// sums go to the per-Gaussian accumulators from lane 0.
__device__ __forceinline__ void replay_pair_aniso(const SecTable &Tab, BwdPixel &P,
                                                  const float4 &g0, const float4 &g1,
                                                  const float4 &a, float tmin, uint32_t gid,
                                                  bool before_last, int px, int py, int lane,
                                                  bool want_attr, bool want_pose, float4 *acc4,
                                                  float4 *accg, float2 *accm) {
    float dc0 = 0.f, dc1 = 0.f, dc2 = 0.f, dop = 0.f;
    float4 dgq = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 dm = make_float2(0.f, 0.f);
    bool contrib = false;
    if (before_last) {
        float du, dv;
        const float t = pair_t_at_aniso(px, py, g0, g1, du, dv);
        if (t >= tmin) {
            const float G = exp2_approx(t);
            contrib = true;
            bwd_pair_aniso(P, g1, a, du, dv, G, __fmul_rn(g1.w, G), dc0, dc1, dc2, dop, dgq, dm,
                           -1.f);
        }
    }
    if (!__any_sync(kFullMask, contrib)) return;
    dc0 = warp_sum(dc0);
    dc1 = warp_sum(dc1);
    dc2 = warp_sum(dc2);
    dop = warp_sum(dop);
    dgq = make_float4(warp_sum(dgq.x), warp_sum(dgq.y), warp_sum(dgq.z), warp_sum(dgq.w));
    dm = make_float2(warp_sum(dm.x), warp_sum(dm.y));
    if (lane == 0)
        add_pair_grads_aniso(Tab, gid, want_attr, want_pose, dc0, dc1, dc2, dop, dgq, dm, acc4,
                             accg, accm);
}

// Tile replay: the block walks its tile's list from the largest list end of
// its pixels back to the front in shared-memory batches; each warp visits the
// Gaussians whose disc touches its 8x4 block.  Used when no per-pixel lists
// were kept (memory budget) and for tiles whose lists overflowed (tile_mask:
// only tiles with tile_mask[t] != 0; NULL = all tiles).
// Aniso = true replays ellipsoid records (k_composite_bwd_aniso): every
// entry of the batch is visited (no block filter for the rotated conic), the
// warp sums each Gaussian's terms and adds them per Gaussian.
template <bool Aniso>
__device__ __forceinline__ void replay_body(
    const SecTable &Tab, const Camera &cam, const uint32_t *tile_off, const uint32_t *sorted,
    const float4 *geo, const float4 *app, const uint32_t *pix_last, const float *pix_T,
    const float *g_rgb, const float *g_depth, const float *g_sil, int mode,
    double *pose_partials, const uint32_t *tile_mask, float4 *acc4, float *accr, float4 *accg,
    float2 *accm, const Status *st, int tile) {
    __shared__ float4 s_g0[kBatch], s_g1[kBatch], s_a[kBatch];
    __shared__ float s_tmin[kBatch];
    __shared__ uint32_t s_gid[kBatch];
    __shared__ double s_pose[kBlockPix / 32][12];
    __shared__ uint32_t s_last;
    if (st->flags) return;
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
                        rel = Aniso || block_touches((float)(bx0 - __float_as_int(h0.x)) - h0.y,
                                                     (float)(by0 - __float_as_int(h0.z)) - h0.w,
                                                     h1.x, h1.y, s_tmin[jj], lxmax, lymax);
                    }
                    unsigned mask = __ballot_sync(kFullMask, rel);
                    while (mask) {
                        const int bit = 31 - __clz(mask);
                        mask &= ~(1u << bit);
                        const int j = j0 + bit;
                        if constexpr (Aniso) {
                            replay_pair_aniso(Tab, P, s_g0[j], s_g1[j], s_a[j], s_tmin[j],
                                              s_gid[j], (uint32_t)(b0 + j) < my_last, px, py,
                                              lane, want_attr, want_pose, acc4, accg, accm);
                            continue;
                        }
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
    if (want_pose && !Aniso) write_pose_partial(acc, s_pose, pose_partials, tile);
}

__global__ void __launch_bounds__(kBlockPix) k_composite_bwd(
    SecTable Tab, Camera cam, const uint32_t *tile_off, const uint32_t *sorted, const float4 *geo,
    const float4 *app, const uint32_t *pix_last, const float *pix_T,
    const float *g_rgb, const float *g_depth, const float *g_sil, int mode,
    double *pose_partials, const uint32_t *tile_mask, float4 *acc4, float *accr, float4 *accg,
    const Status *st) {
    replay_body<false>(Tab, cam, tile_off, sorted, geo, app, pix_last, pix_T, g_rgb, g_depth,
                       g_sil, mode, pose_partials, tile_mask, acc4, accr, accg, nullptr, st,
                       blockIdx.x);
}

__global__ void __launch_bounds__(kBlockPix) k_composite_bwd_aniso(
    SecTable Tab, Camera cam, const uint32_t *tile_off, const uint32_t *sorted, const float4 *geo,
    const float4 *app, const uint32_t *pix_last, const float *pix_T, const float *g_rgb,
    const float *g_depth, const float *g_sil, int mode, const uint32_t *tile_mask, float4 *acc4,
    float4 *accg, float2 *accm, const Status *st) {
    replay_body<true>(Tab, cam, tile_off, sorted, geo, app, pix_last, pix_T, g_rgb, g_depth,
                      g_sil, mode, nullptr, tile_mask, acc4, nullptr, accg, accm, st, blockIdx.x);
}

// Per-pixel list replay: every lane walks the ids its pixel added, recorded
// by the forward, from the last to the first, loading each record one step
// ahead.  No filtering and no block barriers in the walk; tiles with a block
// flagged in blk_ovf (a pixel exceeded the list capacity) are left to
// k_composite_bwd.
// Views = true compiles the source-view gradient path (mode VT_GRAD_VIEWS)
// into k_composite_bwd_list_views; the tracking and mapping paths launch
// k_composite_bwd_list, which does not carry it.  Aniso = true walks
// ellipsoid records (k_composite_bwd_list_aniso): per-Gaussian accumulation
// instead of per-lane pose sums.  PoseOnly = true (k_composite_bwd_list_pose)
// leaves out the per-Gaussian terms, which tracking does not use.
template <bool Views, bool Aniso, bool PoseOnly = false, bool Twist = false>
__device__ __forceinline__ void bwd_list_body(
    const SecTable &Tab, const Camera &cam, const float4 *geo, const float4 *app,
    const uint32_t *pix_nadd, const float *pix_T, const uint2 *plist, int plist_cap,
    const uint32_t *blk_ovf, const float *g_rgb, const float *g_depth, const float *g_sil,
    int mode, double *pose_partials, float4 *acc4, float *accr, float4 *accg, float2 *accm,
    const Status *st, double (*s_pose)[12], int tile) {
    if (st->flags) return;
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
        const float t = Aniso ? pair_t_at_aniso(px, py, g0, g1, du, dv)
                              : pair_t_at(px, py, g0, g1, du, dv);
        const float G = exp2_approx(t);
        const float ah = __fmul_rn(g1.w, G);
        if constexpr (Aniso) {
            float dc0, dc1, dc2, dop;
            float4 dgq;
            float2 dm;
            bwd_pair_aniso(P, g1, a, du, dv, G, ah, dc0, dc1, dc2, dop, dgq, dm, Ti);
            add_pair_grads_aniso(Tab, g, want_attr, want_pose, dc0, dc1, dc2, dop, dgq, dm, acc4,
                                 accg, accm);
        } else {
            float dc0, dc1, dc2, dop, drd, gx, gy, gz;
            bwd_pair<Twist>(P, g0, g1, a, t, du, dv, G, ah, cam, want_pose, acc, dc0, dc1, dc2,
                            dop, drd, want_views, gx, gy, gz, Ti);
            if (!PoseOnly && (want_attr || want_views))
                add_pair_grads(Tab, g, want_attr, want_views, dc0, dc1, dc2, dop, drd, gx, gy, gz,
                               acc4, accr, accg);
        }
    }
    if (want_pose && !Aniso) {
        if constexpr (Twist)
            write_twist_partial(acc, s_pose, pose_partials, tile);
        else
            write_pose_partial(acc, s_pose, pose_partials, tile);
    }
}

__global__ void __launch_bounds__(kBlockPix, 3) k_composite_bwd_list(
    SecTable Tab, Camera cam, const float4 *geo, const float4 *app, const uint32_t *pix_nadd,
    const float *pix_T, const uint2 *plist, int plist_cap, const uint32_t *blk_ovf,
    const float *g_rgb, const float *g_depth, const float *g_sil, int mode,
    double *pose_partials, float4 *acc4, float *accr, float4 *accg, const Status *st) {
    __shared__ double s_pose[kBlockPix / 32][12];
    bwd_list_body<false, false>(Tab, cam, geo, app, pix_nadd, pix_T, plist, plist_cap, blk_ovf,
                                g_rgb, g_depth, g_sil, mode, pose_partials, acc4, accr, accg,
                                nullptr, st, s_pose, blockIdx.x);
}

__global__ void __launch_bounds__(kBlockPix, 3) k_composite_bwd_list_pose(
    SecTable Tab, Camera cam, const float4 *geo, const float4 *app, const uint32_t *pix_nadd,
    const float *pix_T, const uint2 *plist, int plist_cap, const uint32_t *blk_ovf,
    const float *g_rgb, const float *g_depth, const float *g_sil, int mode,
    double *pose_partials, float4 *acc4, float *accr, float4 *accg, const Status *st) {
    __shared__ double s_pose[kBlockPix / 32][12];
    bwd_list_body<false, false, true, true>(Tab, cam, geo, app, pix_nadd, pix_T, plist,
                                            plist_cap, blk_ovf, g_rgb, g_depth, g_sil,
                                            VT_GRAD_POSE, pose_partials, acc4, accr, accg,
                                            nullptr, st, s_pose, blockIdx.x);
}

// The pose-only list backward with the matrix gradient too (all twelve sums
// of x g^T and g), for callers that ask for dL/d[R|t].
__global__ void __launch_bounds__(kBlockPix, 3) k_composite_bwd_list_posemat(
    SecTable Tab, Camera cam, const float4 *geo, const float4 *app, const uint32_t *pix_nadd,
    const float *pix_T, const uint2 *plist, int plist_cap, const uint32_t *blk_ovf,
    const float *g_rgb, const float *g_depth, const float *g_sil, int mode,
    double *pose_partials, float4 *acc4, float *accr, float4 *accg, const Status *st) {
    __shared__ double s_pose[kBlockPix / 32][12];
    bwd_list_body<false, false, true>(Tab, cam, geo, app, pix_nadd, pix_T, plist, plist_cap,
                                      blk_ovf, g_rgb, g_depth, g_sil, VT_GRAD_POSE, pose_partials,
                                      acc4, accr, accg, nullptr, st, s_pose, blockIdx.x);
}

__global__ void __launch_bounds__(kBlockPix, 3) k_composite_bwd_list_aniso(
    SecTable Tab, Camera cam, const float4 *geo, const float4 *app, const uint32_t *pix_nadd,
    const float *pix_T, const uint2 *plist, int plist_cap, const uint32_t *blk_ovf,
    const float *g_rgb, const float *g_depth, const float *g_sil, int mode,
    double *pose_partials, float4 *acc4, float *accr, float4 *accg, float2 *accm,
    const Status *st) {
    bwd_list_body<false, true>(Tab, cam, geo, app, pix_nadd, pix_T, plist, plist_cap, blk_ovf,
                               g_rgb, g_depth, g_sil, mode, pose_partials, acc4, accr, accg, accm,
                               st, nullptr, blockIdx.x);
}

__global__ void __launch_bounds__(kBlockPix, 3) k_composite_bwd_list_views(
    SecTable Tab, Camera cam, const float4 *geo, const float4 *app, const uint32_t *pix_nadd,
    const float *pix_T, const uint2 *plist, int plist_cap, const uint32_t *blk_ovf,
    const float *g_rgb, const float *g_depth, const float *g_sil, int mode,
    double *pose_partials, float4 *acc4, float *accr, float4 *accg, const Status *st) {
    __shared__ double s_pose[kBlockPix / 32][12];
    bwd_list_body<true, false>(Tab, cam, geo, app, pix_nadd, pix_T, plist, plist_cap, blk_ovf,
                               g_rgb, g_depth, g_sil, mode, pose_partials, acc4, accr, accg,
                               nullptr, st, s_pose, blockIdx.x);
}

// Ellipsoids, one thread per Gaussian (grid-stride; one FP64 pose partial
// per block).  From the accumulated dL/d(a', b', c'), the direct depth term
// and dL/d(u_c, v_c):
//   M_Q = kTScale [[da', db'], [db', dc']]       (t = kTScale d^T Q d),
//   G2 = dL/dSigma_2D = -Q M_Q Q,  Gc = dL/dSigma_c = J^T G2 J,
//   dL/dJ = 2 G2 J Sigma_c,
//   g = dL/dx through (u_c, v_c), J(x) and the depth output;
// the pose terms A = x g^T + 2 Sigma_c Gc and s = g (k_pose_finalize forms
// the twist and the matrix from them: R^T Sigma_w R = Sigma_c gives dL/dR =
// R Sigma_c (Gc + Gc^T) for the covariance), and with the section's
// scale / quaternion gradients Gk = M^T Gc M, dL/ds_i = 2 s_i (R^T Gk R)_ii,
// dL/dR(q) = 2 Gk R(q) diag(s^2), chained through the normalisation of q.
// FP32 per Gaussian; the pose sums in float-float across the warp and FP64
// across the block.
__global__ void __launch_bounds__(256) k_aniso_chain(SecTable Tab, Camera cam,
                                                     const ViewXf *views, const float4 *geo,
                                                     const float4 *app, const float4 *accg,
                                                     const float2 *accm, int want_pose,
                                                     int want_attr, double *pose_partials) {
    __shared__ double red[12][8];
    float acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Tab.n_total;
         i += stride) {
        const float4 dg = accg[i];
        const float2 dm = accm[i];
        if (dg.x == 0.f && dg.y == 0.f && dg.z == 0.f && dg.w == 0.f && dm.x == 0.f &&
            dm.y == 0.f)
            continue;
        const SecDesc &S = Tab.s[find_section(Tab, i)];
        const int64_t li = i - S.gbase;
        const float4 g0 = geo[2 * i], g1 = geo[2 * i + 1];
        const float z = app[i].w, iz = 1.f / z;
        const float ucr = ((float)__float_as_int(g0.x) - cam.cx) + g0.y;
        const float vcr = ((float)__float_as_int(g0.z) - cam.cy) + g0.w;
        const float J0[3] = {cam.fx * iz, 0.f, -ucr * iz}, J1[3] = {0.f, cam.fy * iz, -vcr * iz};
        // G2 = -Q M_Q Q
        const float ik = 1.f / kTScale;
        const float Q00 = g1.x * ik, Q01 = 0.5f * g1.y * ik, Q11 = g1.z * ik;
        const float m00 = kTScale * dg.x, m01 = kTScale * dg.y, m11 = kTScale * dg.z;
        const float a00 = Q00 * m00 + Q01 * m01, a01 = Q00 * m01 + Q01 * m11;
        const float a10 = Q01 * m00 + Q11 * m01, a11 = Q01 * m01 + Q11 * m11;
        const float G00 = -(a00 * Q00 + a01 * Q01), G01 = -(a00 * Q01 + a01 * Q11);
        const float G11 = -(a10 * Q01 + a11 * Q11);
        // P = G2 J (2 x 3), Gc = J^T P
        float P0[3], P1[3], Gc[9];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            P0[c] = G00 * J0[c] + G01 * J1[c];
            P1[c] = G01 * J0[c] + G11 * J1[c];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) Gc[3 * a + b] = J0[a] * P0[b] + J1[a] * P1[b];
        // Sigma_c = U U^T, U = M R(q) diag(s)
        const uint32_t plane = (uint32_t)S.W * (uint32_t)S.H;
        const float *Mf = views[S.view_base + S.src[li] / plane].Mf;
        const float sc[3] = {ld_attr(S.scale, S.prec, 3 * li), ld_attr(S.scale, S.prec, 3 * li + 1),
                             ld_attr(S.scale, S.prec, 3 * li + 2)};
        float qv[4] = {ld_attr(S.rot, S.prec, 4 * li), ld_attr(S.rot, S.prec, 4 * li + 1),
                       ld_attr(S.rot, S.prec, 4 * li + 2), ld_attr(S.rot, S.prec, 4 * li + 3)};
        const float qn = sqrtf(qv[0] * qv[0] + qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3]);
        const float iq = 1.f / qn;
        const float w = qv[0] * iq, x = qv[1] * iq, y = qv[2] * iq, zq = qv[3] * iq;
        const float Rq[9] = {1.f - 2.f * (y * y + zq * zq), 2.f * (x * y - w * zq),
                             2.f * (x * zq + w * y),        2.f * (x * y + w * zq),
                             1.f - 2.f * (x * x + zq * zq), 2.f * (y * zq - w * x),
                             2.f * (x * zq - w * y),        2.f * (y * zq + w * x),
                             1.f - 2.f * (x * x + y * y)};
        float U[9], Sc[9];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                U[3 * a + k] = (Mf[3 * a] * Rq[k] + Mf[3 * a + 1] * Rq[3 + k] +
                                Mf[3 * a + 2] * Rq[6 + k]) * sc[k];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                Sc[3 * a + b] = U[3 * a] * U[3 * b] + U[3 * a + 1] * U[3 * b + 1] +
                                U[3 * a + 2] * U[3 * b + 2];
        // dL/dJ = 2 P Sigma_c, only the entries of J that vary
        float GJ0[3], GJ1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            GJ0[c] = 2.f * (P0[0] * Sc[c] + P0[1] * Sc[3 + c] + P0[2] * Sc[6 + c]);
            GJ1[c] = 2.f * (P1[0] * Sc[c] + P1[1] * Sc[3 + c] + P1[2] * Sc[6 + c]);
        }
        float g[3];
        g[0] = dm.x * J0[0] - GJ0[2] * J0[0] * iz;
        g[1] = dm.y * J1[1] - GJ1[2] * J1[1] * iz;
        g[2] = -(dm.x * ucr + dm.y * vcr) * iz -
               iz * (GJ0[0] * J0[0] + GJ1[1] * J1[1] + 2.f * (GJ0[2] * J0[2] + GJ1[2] * J1[2])) +
               dg.w;
        if (want_pose) {
            const float X[3] = {ucr * z / cam.fx, vcr * z / cam.fy, z};
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b)
                    acc[3 * a + b] += X[a] * g[b] + 2.f * (Sc[3 * a] * Gc[b] +
                                                           Sc[3 * a + 1] * Gc[3 + b] +
                                                           Sc[3 * a + 2] * Gc[6 + b]);
#pragma unroll
            for (int b = 0; b < 3; ++b) acc[9 + b] += g[b];
        }
        if (want_attr && (S.d_scale || S.d_rot)) {
            float Gk[9], RG[9], V[3];   // M^T Gc M, Gk R(q), diag(R^T Gk R)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float T_[3];
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    T_[d] = Gc[3 * a] * Mf[d] + Gc[3 * a + 1] * Mf[3 + d] + Gc[3 * a + 2] * Mf[6 + d];
#pragma unroll
                for (int d = 0; d < 3; ++d) RG[3 * a + d] = T_[d];   // (Gc M)[a][d]
            }
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    Gk[3 * b + d] = Mf[b] * RG[d] + Mf[3 + b] * RG[3 + d] + Mf[6 + b] * RG[6 + d];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    RG[3 * a + k] = Gk[3 * a] * Rq[k] + Gk[3 * a + 1] * Rq[3 + k] +
                                    Gk[3 * a + 2] * Rq[6 + k];
#pragma unroll
            for (int k = 0; k < 3; ++k)
                V[k] = Rq[k] * RG[k] + Rq[3 + k] * RG[3 + k] + Rq[6 + k] * RG[6 + k];
            if (S.d_scale) {
#pragma unroll
                for (int k = 0; k < 3; ++k) S.d_scale[3 * li + k] += 2.f * sc[k] * V[k];
            }
            if (S.d_rot) {
                float gR[9];   // 2 Gk R(q) diag(s^2)
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int k = 0; k < 3; ++k) gR[3 * a + k] = 2.f * RG[3 * a + k] * sc[k] * sc[k];
                const float dw = 2.f * (-zq * gR[1] + y * gR[2] + zq * gR[3] - x * gR[5] -
                                        y * gR[6] + x * gR[7]);
                const float dx = 2.f * (y * gR[1] + zq * gR[2] + y * gR[3] - 2.f * x * gR[4] -
                                        w * gR[5] + zq * gR[6] + w * gR[7] - 2.f * x * gR[8]);
                const float dy = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] +
                                        zq * gR[5] - w * gR[6] + zq * gR[7] - 2.f * y * gR[8]);
                const float dz = 2.f * (-2.f * zq * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] -
                                        2.f * zq * gR[4] + y * gR[5] + x * gR[6] + y * gR[7]);
                const float proj = dw * w + dx * x + dy * y + dz * zq;
                S.d_rot[4 * li + 0] += (dw - w * proj) * iq;
                S.d_rot[4 * li + 1] += (dx - x * proj) * iq;
                S.d_rot[4 * li + 2] += (dy - y * proj) * iq;
                S.d_rot[4 * li + 3] += (dz - zq * proj) * iq;
            }
        }
    }
    if (!want_pose) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const ff v = warp_sum_ff(acc[k]);
        if (lane == 0) red[k][warp] = to_double(v);
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[threadIdx.x][w];
        pose_partials[(size_t)blockIdx.x * 12 + threadIdx.x] = t;
    }
}

// Source-view pose gradients (head-frame bundle adjustment, Sec. 3.4).  The
// Gaussians of one view are a contiguous range of their section (ids are in
// (view, pixel) order).  k_view_grads: kViewChunks blocks per (section, view)
// each sum g X_c^T and g over an equal share of the range (per thread in
// FP32, across the warp in float-float and the block in FP64, fixed order), with g = dL/dx of the centre
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
        const ff v = warp_sum_ff(acc[i]);
        if (lane == 0) red[i][warp] = to_double(v);
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

// ---------------------------------------------------------------------------
// Batched pose backward of the tracking items.  The per-Gaussian terms are
// not formed (pose only), so the section table the bodies take is an empty
// one.
__device__ SecTable g_no_sections;

// Per-pixel list walks: tiles of tracking items taken from a work counter;
// each item's upstream gradient is its planes of `grads` (4 x P from 4 pbase:
// rgb, depth), its pose terms go to pose_partials[12 t] per tile t.  Tiles
// whose lists overflowed are left to kb_composite_bwd_pose.
__global__ void __launch_bounds__(kBlockPix, 3) kb_composite_bwd_list_pose(
    const BatchTable *Bp, uint32_t *ctr, const float4 *geo, const float4 *app,
    const uint32_t *pix_nadd, const float *pix_T, const uint2 *plist, int plist_cap,
    const uint32_t *blk_ovf, const float *grads, double *pose_partials, const Status *st) {
    __shared__ double s_pose[kBlockPix / 32][12];
    const BatchTable &B = *Bp;
    ItemCursor cur;
    const auto tstart = [&](int i) { return (int64_t)B.it[i].tbase; };
    for (int t = next_tile(ctr); t < B.n_tiles; t = next_tile(ctr)) {
        const BatchItem &I = B.it[cur.at(B, tstart, t)];
        if (!I.track) continue;
        const int64_t P = (int64_t)I.cam.W * I.cam.H;
        const float *g = grads + 4 * I.pbase;
        bwd_list_body<false, false, true>(
            g_no_sections, I.cam, geo, app, pix_nadd + I.pbase, pix_T + I.pbase,
            plist + I.pbase * (int64_t)plist_cap, plist_cap, blk_ovf + (int64_t)I.tbase * kWarps,
            g, g + 3 * P, nullptr, VT_GRAD_POSE, pose_partials + 12 * (int64_t)I.tbase, nullptr,
            nullptr, nullptr, nullptr, st, s_pose, t - I.tbase);
    }
}

// Tile replay of the tracking items' tiles whose per-pixel lists overflowed
// (blk_ovf; all of them when the batch keeps no lists).
__global__ void __launch_bounds__(kBlockPix) kb_composite_bwd_pose(
    const BatchTable *Bp, const uint32_t *tile_off, const uint32_t *sorted, const float4 *geo,
    const float4 *app, const uint32_t *pix_last, const float *pix_T, const uint32_t *blk_ovf,
    const float *grads, double *pose_partials, const Status *st) {
    const BatchTable &B = *Bp;
    ItemCursor cur;
    const auto tstart = [&](int i) { return (int64_t)B.it[i].tbase; };
    for (int t = blockIdx.x; t < B.n_tiles; t += gridDim.x) {
        const BatchItem &I = B.it[cur.at(B, tstart, t)];
        if (!I.track) continue;
        if (!tile_flagged(blk_ovf + (int64_t)I.tbase * kWarps, t - I.tbase)) continue;
        const int64_t P = (int64_t)I.cam.W * I.cam.H;
        const float *g = grads + 4 * I.pbase;
        replay_body<false>(g_no_sections, I.cam, tile_off + I.tbase, sorted, geo, app,
                           pix_last + I.pbase, pix_T + I.pbase, g, g + 3 * P, nullptr,
                           VT_GRAD_POSE, pose_partials + 12 * (int64_t)I.tbase,
                           blk_ovf + (int64_t)I.tbase * kWarps, nullptr, nullptr, nullptr,
                           nullptr, st, t - I.tbase);
        __syncthreads();   // shared staging is reused by the next tile
    }
}

// Fixed-order FP64 sum of the per-tile partials, then
//   twist: dL/drho = -s,  dL/dphi = (A21 - A12, A02 - A20, A10 - A01)
//   matrix: dL/dR = R A,  dL/dt = -R s          (A_ab = sum x_a g_b)
// accumulated (+=) into the outputs.
// With overwrite the outputs are set instead of accumulated.  384 threads.
__device__ __forceinline__ void pose_finalize_body(const double *partials, int n_parts,
                                                   const double *pose_copy, double *d_twist,
                                                   double *d_mat, bool overwrite) {
    __shared__ double tot[12];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double v = 0.0;
    for (int i = lane; i < n_parts; i += 32) v += partials[(size_t)i * 12 + warp];
    v = warp_sum_d(v);
    if (lane == 0) tot[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double *A = tot, *s = tot + 9, *R = pose_copy;
        if (overwrite) {
            for (int i = 0; i < 6; ++i) d_twist[i] = 0.0;
            for (int i = 0; i < 12; ++i) d_mat[i] = 0.0;
        }
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


__global__ void __launch_bounds__(384) k_pose_finalize(const double *partials, int n_parts,
                                                       const double *pose_copy, double *d_twist,
                                                       double *d_mat) {
    pose_finalize_body(partials, n_parts, pose_copy, d_twist, d_mat, false);
}

// Results of the batch's tracking items, one block of 384 per item in a
// grid-stride loop: result[0] = Eq. 1 loss (the fixed-order sums of the
// item's masked-L1 block partials l1_part[2 b], b from pbase / 256),
// result[1..6] = dL/dtwist, result[7..18] = dL/dR and dL/dt (fixed-order FP64
// sums of the item's tile partials), overwritten.
__global__ void __launch_bounds__(384) kb_finalize(const BatchTable *Bp, const double *l1_part,
                                                   const double *pose_partials,
                                                   const double *pose_copy) {
    __shared__ double s[2][12];
    const BatchTable &B = *Bp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int it = blockIdx.x; it < B.n_items; it += gridDim.x) {
        const BatchItem &I = B.it[it];
        if (!I.track) continue;
        const int64_t P = (int64_t)I.cam.W * I.cam.H;
        const int64_t b0 = I.pbase / 256, nb = (P + 255) / 256;
        double a = 0.0, b = 0.0;
        for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) {
            a += l1_part[2 * (b0 + i)];
            b += l1_part[2 * (b0 + i) + 1];
        }
        a = warp_sum_d(a);
        b = warp_sum_d(b);
        if (lane == 0) {
            s[0][warp] = a;
            s[1][warp] = b;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double A = 0.0, Bs = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                A += s[0][w];
                Bs += s[1][w];
            }
            const double wc = B.w_rgb / (3.0 * (double)P), wd = B.w_depth / (double)P;
            I.result[0] = __dadd_rn(__dmul_rn(wc, A), __dmul_rn(wd, Bs));
        }
        pose_finalize_body(pose_partials + 12 * (int64_t)I.tbase, I.cam.tiles_x * I.cam.tiles_y,
                           pose_copy + 12 * it, I.result + 1, I.result + 7, true);
        __syncthreads();
    }
}

}  // namespace vt
