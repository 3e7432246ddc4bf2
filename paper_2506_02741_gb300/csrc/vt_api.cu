// C ABI of the vtsplat library: argument checks, the render context and its
// workspace, kernel launches, back-projection and section initialisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdarg>
#include <cstring>
#include <string>
#include <vector>

#include "vt_common.cuh"

using namespace vt;

namespace {

thread_local std::string g_err;

vt_status fail(vt_status s, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
vt_status fail(vt_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

vt_status cuda_fail(cudaError_t e, const char *what) {
    return fail(VT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define VT_CUDA(call, what)                         \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Tile lists are sorted in shared memory by size class, each class by a
// launch whose blocks hold just enough shared memory for its longest list, so
// that short lists run several blocks per SM (4, 3 and 2 of 228 KB):
// (1536, 3584] on the caller's stream, (3584, kSortSmemN] and then
// (0, 1536] on a second auxiliary stream (in the batched launches all three
// on the caller's stream);
// the few longer ones (up to kSortSmemBig in shared memory, one block per
// SM; beyond that in global memory, two blocks per SM with shared memory for
// the histograms only) by launches on an auxiliary stream that overlap the
// others.
constexpr int kSortClassS = 1536, kSortClassM = 3584;
constexpr size_t sort_smem_bytes(int n) { return 2 * (size_t)n * 8 + 16 * 256 * 4; }
// Upper bound of the third class; lists up to kSortSmemBig sort in shared
// memory with one block per SM, longer ones in global memory.
constexpr int kSortSmemN = 6000;
constexpr size_t kSortSmemBytes = 2 * kSortSmemN * sizeof(unsigned long long) + 16 * 256 * 4;
constexpr int kSortSmemBig = 13312;
static_assert(kSortSmemN == kSortLongMin, "the tile scan lists the long-list launches' tiles");
static_assert(kSortSmemBig < (1 << 24), "shared-memory sorts carry 24-bit bucket positions");
constexpr size_t kSortSmemBigBytes =
    2 * kSortSmemBig * sizeof(unsigned long long) + 16 * 256 * 4;
constexpr size_t kSortHistBytes = 16 * 256 * 4;

enum KernelId {
    K_SETUP, K_PREPROCESS, K_SCAN, K_EMIT, K_SORT, K_FWD, K_BWD, K_POSE, K_BACKPROJECT,
    K_SECTION_INIT, K_COUNT, K_BWD_LIST, K_SORT_BIG, K_SCATTER, K_L1, K_L1_SUM, K_POSE_ADAM,
    K_ADAM_COUNT, K_ATTR_ADAM, K_SORT_M, K_SORT_L, K_SSIM_FWD, K_SSIM_BWD, K_SSIM_SUM,
    K_VIEW_GRADS, K_PRE_AN, K_FWD_AN, K_BWD_LIST_AN, K_BWD_AN, K_CHAIN, K_SHAPE_ADAM,
    K_SORT_XL, K_VIEW_FIN, K_BWD_LIST_POSE, K_BWD_LIST_VIEWS, KB_SETUP, KB_PREPROCESS, KB_SCAN,
    KB_EMIT, KB_SORT, KB_SORT_M, KB_SORT_L, KB_SORT_LONG, KB_SORT_XL, KB_FWD, KB_L1, KB_BWD_LIST,
    KB_BWD, KB_FINALIZE, K_ADAM_INIT, K_BWD_LIST_POSEMAT, K_NUM
};
const char *kKernelNames[K_NUM] = {"k_setup",         "k_preprocess",    "k_scan_tiles",
                                   "k_emit",          "k_sort_tiles",    "k_composite_fwd",
                                   "k_composite_bwd", "k_pose_finalize", "k_backproject",
                                   "k_section_init",  "k_count_valid",   "k_composite_bwd_list",
                                   "k_sort_tiles_long", "k_attr_scatter", "k_masked_l1",
                                   "k_sum_partials",  "k_pose_adam",     "k_adam_step_count",
                                   "k_attr_adam",     "k_sort_tiles_mid", "k_sort_tiles_large",
                                   "k_ssim_fwd",      "k_ssim_bwd",       "k_ssim_sum",
                                   "k_view_grads",    "k_preprocess_aniso",
                                   "k_composite_fwd_aniso", "k_composite_bwd_list_aniso",
                                   "k_composite_bwd_aniso", "k_aniso_chain", "k_shape_adam",
                                   "k_sort_tiles_xl", "k_view_finalize",
                                   "k_composite_bwd_list_pose", "k_composite_bwd_list_views",
                                   "kb_setup", "kb_preprocess", "kb_scan_tiles", "kb_emit",
                                   "kb_sort_tiles", "kb_sort_tiles_mid", "kb_sort_tiles_large",
                                   "kb_sort_tiles_long", "kb_sort_tiles_xl", "kb_composite_fwd",
                                   "kb_masked_l1", "kb_composite_bwd_list_pose",
                                   "kb_composite_bwd_pose", "kb_finalize", "k_adam_init",
                                   "k_composite_bwd_list_posemat"};
constexpr int kDefaultListCap = 256;  // per-pixel ids kept for the backward

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

bool finite_pos(float x) { return std::isfinite(x) && x > 0.f; }
bool finite(float x) { return std::isfinite(x); }

}  // namespace

// Lets other translation units of the library report an error message for
// vt_last_error (not exported).
__attribute__((visibility("hidden"))) vt_status vt_internal_fail(vt_status s, const char *msg) {
    g_err = msg;
    return s;
}

struct vt_ctx {
    int device = 0;
    // capacities
    int64_t cap_g = 0, cap_i = 0, cap_p = 0, cap_t = 0, cap_v = 0, cap_tab = 0;
    int64_t reserved_i = 0;
    void *arena = nullptr;
    size_t arena_bytes = 0;
    float4 *geo = nullptr, *app = nullptr;
    uint4 *info = nullptr;
    uint32_t *tile_count = nullptr, *tile_off = nullptr, *tile_cursor = nullptr;
    uint32_t *long_tiles = nullptr;   // tiles of the long-list sorts (listed by the tile scan)
    unsigned long long *bucket = nullptr, *alt = nullptr;
    uint32_t *sorted = nullptr;
    uint8_t *bmask = nullptr;         // per sorted entry: 8x4 blocks of the tile it reaches
    uint8_t *bmask_u = nullptr;       // the same per bucket entry, before the sort
    uint32_t *pix_last = nullptr, *pix_nadd = nullptr;
    float *pix_T = nullptr;
    Status *status = nullptr;
    ViewXf *views = nullptr;
    TabRow *tab = nullptr;
    double *pose_partials = nullptr, *pose_copy = nullptr;
    uint32_t *blk_ovf = nullptr;      // list overflow flag per 8x4 pixel block
    cudaStream_t aux = nullptr;       // auxiliary stream of the long-list sort
    cudaStream_t aux2 = nullptr;      // second one: the large and the shortest class
    int n_sm = 1;                     // SMs of the device
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
    double *loss_part = nullptr;      // masked-L1 block partials (separate allocation)
    int64_t loss_cap = 0;             // blocks they hold
    double *view_part = nullptr;      // per-view chunk partials of the view gradients
    size_t view_part_bytes = 0;
    void *ssim_buf = nullptr;         // SSIM maps (15 floats per pixel) + block partials
    int64_t ssim_cap = 0;             // pixels it holds
    float4 *acc4 = nullptr;       // attribute-gradient accumulators (colour, opacity)
    float *accr = nullptr;        // and radius, per Gaussian
    float4 *accg = nullptr;       // dL/dx of each centre (source-view gradients); for
                                  // ellipsoids dL/d(a', b', c') and the direct depth term
    float2 *accm = nullptr;       // ellipsoids: dL/d(u_c, v_c) per Gaussian
    // per-pixel lists of added Gaussians (separate allocation)
    int list_cap = kDefaultListCap;
    uint2 *plist = nullptr;       // (id, transmittance in front) per added Gaussian
    size_t plist_bytes = 0;
    size_t budget = (size_t)-1;
    bool used_lists = false;
    // last render
    bool has_render = false;
    bool aniso = false;           // the last render's sections are ellipsoids
    SecTable table{};
    Camera cam{};
    int n_tiles = 0;
    cudaStream_t stream = nullptr;
    // instrumentation
    int64_t launches = 0;
    bool timing = false;
    struct Pending {
        int kernel;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    int64_t t_launches[K_NUM] = {0};
    double t_ms[K_NUM] = {0};
    // batched launches (vt_batch_*): the arena above sized for the batch
    // totals, plus the work-item table (device copy and pinned staging), the
    // image gradients (4 floats per pixel), masked-L1 block partials and the
    // items' pose copies
    bool batch = false;           // reserved for batches
    bool batch_set = false;       // a table is staged
    bool batch_lists = false;     // per-pixel lists kept for the batch backward
    int64_t bcap_g = 0, bcap_p = 0, bcap_t = 0, bcap_i = 0, bcap_v = 0, bcap_tab = 0;
    BatchTable *btab = nullptr, *btab_host = nullptr;
    void *barena = nullptr;
    float *bgrads = nullptr;
    double *bl1 = nullptr, *bpose = nullptr;
    cudaEvent_t bev_upload = nullptr;
    bool bev_pending = false;
};

namespace {

cudaEvent_t get_event(vt_ctx *c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket one launch with events when timing is on.
struct LaunchScope {
    vt_ctx *c;
    int k;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    LaunchScope(vt_ctx *c_, int k_, cudaStream_t s_) : c(c_), k(k_), s(s_) {
        if (c->timing) {
            a = get_event(c);
            cudaEventRecord(a, s);
        }
        c->launches++;
    }
    ~LaunchScope() {
        if (c->timing) {
            cudaEvent_t b = get_event(c);
            cudaEventRecord(b, s);
            c->pending.push_back({k, a, b});
        }
    }
};

void free_arena(vt_ctx *c, cudaStream_t s) {
    if (c->arena) cudaFreeAsync(c->arena, s);
    c->arena = nullptr;
    c->arena_bytes = 0;
}

size_t arena_bytes_for(int64_t g, int64_t i, int64_t p, int64_t t, int64_t v, int64_t tab) {
    size_t b = 0;
    b += align_up(sizeof(float4) * 2 * g);               // geo
    b += align_up(sizeof(float4) * g);                   // app
    b += align_up(sizeof(uint4) * g);                    // info
    b += 4 * align_up(sizeof(uint32_t) * (t + 1));       // tile count/off/cursor, long tiles
    b += 2 * align_up(sizeof(unsigned long long) * i);   // bucket, alt
    b += align_up(sizeof(uint32_t) * i);                 // sorted
    b += 2 * align_up(i);                                // block masks (bucket, sorted)
    b += 3 * align_up(sizeof(uint32_t) * p);             // last, nadd, T
    b += align_up(sizeof(Status));
    b += align_up(sizeof(ViewXf) * v);
    b += align_up(sizeof(TabRow) * tab);
    b += align_up(sizeof(double) * 12 * t);              // pose partials
    b += align_up(sizeof(double) * 12);                  // pose copy
    b += align_up(sizeof(uint32_t) * 8 * t);             // block overflow flags
    b += align_up(sizeof(float4) * g) + align_up(sizeof(float) * g);   // gradient accumulators
    b += align_up(sizeof(float4) * g);                   // centre gradients
    b += align_up(sizeof(float2) * g);                   // ellipse centre terms
    return b;
}

vt_status ensure(vt_ctx *c, int64_t g, int64_t i, int64_t p, int64_t t, int64_t v, int64_t tab,
                 cudaStream_t s) {
    if (g <= c->cap_g && i <= c->cap_i && p <= c->cap_p && t <= c->cap_t && v <= c->cap_v &&
        tab <= c->cap_tab && c->arena)
        return VT_OK;
    g = std::max(g, c->cap_g);
    i = std::max(i, c->cap_i);
    p = std::max(p, c->cap_p);
    t = std::max(t, c->cap_t);
    v = std::max(v, c->cap_v);
    tab = std::max(tab, c->cap_tab);
    const size_t bytes = arena_bytes_for(g, i, p, t, v, tab);
    free_arena(c, s);
    void *a = nullptr;
    cudaError_t e = cudaMallocAsync(&a, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->cap_g = c->cap_i = c->cap_p = c->cap_t = c->cap_v = c->cap_tab = 0;
        c->has_render = false;
        return fail(VT_ERR_OOM, "workspace allocation of %zu bytes failed: %s", bytes,
                    cudaGetErrorString(e));
    }
    c->arena = a;
    c->arena_bytes = bytes;
    char *q = static_cast<char *>(a);
    auto take = [&](size_t n) {
        char *r = q;
        q += align_up(n);
        return r;
    };
    c->geo = reinterpret_cast<float4 *>(take(sizeof(float4) * 2 * g));
    c->app = reinterpret_cast<float4 *>(take(sizeof(float4) * g));
    c->info = reinterpret_cast<uint4 *>(take(sizeof(uint4) * g));
    c->tile_count = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * (t + 1)));
    c->tile_off = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * (t + 1)));
    c->tile_cursor = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * (t + 1)));
    c->long_tiles = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * (t + 1)));
    c->bucket = reinterpret_cast<unsigned long long *>(take(sizeof(unsigned long long) * i));
    c->alt = reinterpret_cast<unsigned long long *>(take(sizeof(unsigned long long) * i));
    c->sorted = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * i));
    c->bmask = reinterpret_cast<uint8_t *>(take(i));
    c->bmask_u = reinterpret_cast<uint8_t *>(take(i));
    c->pix_last = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * p));
    c->pix_nadd = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * p));
    c->pix_T = reinterpret_cast<float *>(take(sizeof(float) * p));
    c->status = reinterpret_cast<Status *>(take(sizeof(Status)));
    c->views = reinterpret_cast<ViewXf *>(take(sizeof(ViewXf) * v));
    c->tab = reinterpret_cast<TabRow *>(take(sizeof(TabRow) * tab));
    c->pose_partials = reinterpret_cast<double *>(take(sizeof(double) * 12 * t));
    c->pose_copy = reinterpret_cast<double *>(take(sizeof(double) * 12));
    c->blk_ovf = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t) * 8 * t));
    c->acc4 = reinterpret_cast<float4 *>(take(sizeof(float4) * g));
    c->accr = reinterpret_cast<float *>(take(sizeof(float) * g));
    c->accg = reinterpret_cast<float4 *>(take(sizeof(float4) * g));
    c->accm = reinterpret_cast<float2 *>(take(sizeof(float2) * g));
    c->cap_g = g;
    c->cap_i = i;
    c->cap_p = p;
    c->cap_t = t;
    c->cap_v = v;
    c->cap_tab = tab;
    c->has_render = false;
    VT_CUDA(cudaMemsetAsync(c->status, 0, sizeof(Status), s), "status init");
    return VT_OK;
}

// Scratch of the masked-L1 loss: two doubles per block of 256 pixels.  Grows
// on the stream; refuses to grow while the stream is being captured.
vt_status ensure_loss(vt_ctx *c, int64_t blocks, cudaStream_t s) {
    if (blocks <= c->loss_cap) return VT_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    VT_CUDA(cudaStreamIsCapturing(s, &cs), "capture query");
    if (cs != cudaStreamCaptureStatusNone)
        return fail(VT_ERR_STATE, "vt_masked_l1: scratch must be reserved before graph capture");
    if (c->loss_part) cudaFreeAsync(c->loss_part, s);
    c->loss_part = nullptr;
    c->loss_cap = 0;
    void *p = nullptr;
    const cudaError_t e = cudaMallocAsync(&p, sizeof(double) * 2 * blocks, s);
    if (e != cudaSuccess)
        return fail(VT_ERR_OOM, "loss scratch of %lld blocks: %s", (long long)blocks,
                    cudaGetErrorString(e));
    c->loss_part = static_cast<double *>(p);
    c->loss_cap = blocks;
    return VT_OK;
}

int64_t default_instances(int64_t g) { return 4 * g + 65536; }

vt_status check_intrinsics(const vt_intrinsics &K, const char *who) {
    if (!finite_pos(K.fx) || !finite_pos(K.fy) || !finite(K.cx) || !finite(K.cy))
        return fail(VT_ERR_INVALID_ARG, "%s: intrinsics must be finite with fx, fy > 0", who);
    return VT_OK;
}

vt_status check_image(int32_t W, int32_t H, const char *who) {
    // pixel boxes pack u and v into 16 bits each
    if (W <= 0 || H <= 0 || (int64_t)W * H > (int64_t)1 << 31 || W > 65535 || H > 65535)
        return fail(VT_ERR_INVALID_ARG, "%s: image size %d x %d out of range", who, W, H);
    return VT_OK;
}

bool sort_attr_set = false;

}  // namespace
// The image-size rule of every entry point, for other translation units
// (not exported).
__attribute__((visibility("hidden"))) vt_status vt_internal_check_image(int32_t W, int32_t H,
                                                                       const char *who) {
    return check_image(W, H, who);
}

// ---------------------------------------------------------------------------

extern "C" {

const char *vt_last_error(void) { return g_err.c_str(); }

const char *vt_version(void) { return "vtsplat 0.1 (sm_103a)"; }

vt_status vt_ctx_create(vt_ctx **ctx) {
    if (!ctx) return fail(VT_ERR_INVALID_ARG, "vt_ctx_create: ctx is NULL");
    vt_ctx *c = new (std::nothrow) vt_ctx();
    if (!c) return fail(VT_ERR_OOM, "vt_ctx_create: out of host memory");
    cudaGetDevice(&c->device);
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device) !=
            cudaSuccess ||
        cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->aux2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming) != cudaSuccess) {
        vt_ctx_destroy(c);
        return fail(VT_ERR_CUDA, "vt_ctx_create: cannot create the auxiliary stream");
    }
    *ctx = c;
    return VT_OK;
}

void vt_ctx_destroy(vt_ctx *c) {
    if (!c) return;
    // the teardown touches only this context's streams and memory: let it run
    // while another thread captures a graph in global mode
    cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
    cudaThreadExchangeStreamCaptureMode(&mode);
    free_arena(c, c->stream);
    if (c->plist) cudaFreeAsync(c->plist, c->stream);
    if (c->loss_part) cudaFreeAsync(c->loss_part, c->stream);
    if (c->ssim_buf) cudaFreeAsync(c->ssim_buf, c->stream);
    if (c->view_part) cudaFreeAsync(c->view_part, c->stream);
    if (c->btab) cudaFreeAsync(c->btab, c->stream);
    if (c->barena) cudaFreeAsync(c->barena, c->stream);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->btab_host) cudaFreeHost(c->btab_host);
    if (c->bev_upload) cudaEventDestroy(c->bev_upload);
    for (auto &p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    if (c->aux) {
        cudaStreamSynchronize(c->aux);
        cudaStreamDestroy(c->aux);
    }
    if (c->aux2) {
        cudaStreamSynchronize(c->aux2);
        cudaStreamDestroy(c->aux2);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_join2) cudaEventDestroy(c->ev_join2);
    delete c;
    cudaThreadExchangeStreamCaptureMode(&mode);
}

size_t vt_workspace_bytes(int64_t n_gaussians, int32_t W, int32_t H, int64_t n_instances) {
    if (n_gaussians < 0 || W <= 0 || H <= 0) return 0;
    if (n_instances <= 0) n_instances = default_instances(n_gaussians);
    const int64_t tiles = (int64_t)((W + kTile - 1) / kTile) * ((H + kTile - 1) / kTile);
    return arena_bytes_for(n_gaussians, n_instances, (int64_t)W * H, tiles, 0, 0);
}

vt_status vt_ctx_reserve(vt_ctx *c, int64_t n_gaussians, int32_t W, int32_t H,
                         int64_t n_instances, vt_stream stream) {
    if (!c) return fail(VT_ERR_INVALID_ARG, "vt_ctx_reserve: ctx is NULL");
    if (n_gaussians < 0) return fail(VT_ERR_INVALID_ARG, "vt_ctx_reserve: n_gaussians < 0");
    vt_status st = check_image(W, H, "vt_ctx_reserve");
    if (st) return st;
    if (n_instances <= 0) n_instances = default_instances(n_gaussians);
    c->reserved_i = std::max(c->reserved_i, n_instances);  // later renders keep this capacity
    const int64_t tiles = (int64_t)((W + kTile - 1) / kTile) * ((H + kTile - 1) / kTile);
    c->stream = stream;
    if ((st = ensure_loss(c, ((int64_t)W * H + 255) / 256, stream))) return st;
    return ensure(c, std::max<int64_t>(n_gaussians, 1), n_instances, (int64_t)W * H, tiles,
                  std::max<int64_t>(c->cap_v, 1), std::max<int64_t>(c->cap_tab, 1), stream);
}

vt_status vt_ctx_sync_status(vt_ctx *c, vt_stream stream, int64_t *needed) {
    if (!c) return fail(VT_ERR_INVALID_ARG, "vt_ctx_sync_status: ctx is NULL");
    VT_CUDA(cudaStreamSynchronize(stream), "vt_ctx_sync_status");
    if (!c->status) {
        if (needed) *needed = 0;
        return VT_OK;
    }
    Status h;
    VT_CUDA(cudaMemcpy(&h, c->status, sizeof h, cudaMemcpyDeviceToHost), "status copy");
    if (needed) *needed = (int64_t)h.n_instances;
    if (h.flags & kFlagCapacity)
        return fail(VT_ERR_CAPACITY, "render needed %llu tile instances, workspace holds %lld",
                    h.n_instances, (long long)c->cap_i);
    return VT_OK;
}

vt_status vt_ctx_set_timing(vt_ctx *c, int32_t enable) {
    if (!c) return fail(VT_ERR_INVALID_ARG, "vt_ctx_set_timing: ctx is NULL");
    c->timing = enable != 0;
    return VT_OK;
}

int32_t vt_ctx_timing(vt_ctx *c, vt_stream stream, const char **names, int64_t *launches,
                      double *ms, int32_t n_max, int32_t reset) {
    if (!c) return -VT_ERR_INVALID_ARG;
    cudaStreamSynchronize(stream);
    for (auto &p : c->pending) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
            c->t_ms[p.kernel] += t;
            c->t_launches[p.kernel] += 1;
        }
        c->event_pool.push_back(p.a);
        c->event_pool.push_back(p.b);
    }
    c->pending.clear();
    int32_t n = 0;
    for (int k = 0; k < K_NUM && n < n_max; ++k) {
        if (names) names[n] = kKernelNames[k];
        if (launches) launches[n] = c->t_launches[k];
        if (ms) ms[n] = c->t_ms[k];
        ++n;
    }
    if (reset)
        for (int k = 0; k < K_NUM; ++k) {
            c->t_ms[k] = 0;
            c->t_launches[k] = 0;
        }
    return n;
}

int64_t vt_ctx_launch_count(const vt_ctx *c) { return c ? c->launches : 0; }

vt_status vt_ctx_set_list_capacity(vt_ctx *c, int32_t cap) {
    if (!c) return fail(VT_ERR_INVALID_ARG, "vt_ctx_set_list_capacity: ctx is NULL");
    if (cap < 0 || cap > 65536)
        return fail(VT_ERR_INVALID_ARG, "vt_ctx_set_list_capacity: %d out of [0, 65536]", cap);
    c->list_cap = cap;
    return VT_OK;
}

vt_status vt_ctx_set_workspace_budget(vt_ctx *c, size_t bytes) {
    if (!c) return fail(VT_ERR_INVALID_ARG, "vt_ctx_set_workspace_budget: ctx is NULL");
    c->budget = bytes ? bytes : (size_t)-1;
    return VT_OK;
}

size_t vt_ctx_workspace_bytes(const vt_ctx *c) {
    return c ? c->arena_bytes + c->plist_bytes : 0;
}

int32_t vt_ctx_used_lists(const vt_ctx *c) { return c && c->has_render && c->used_lists; }

vt_status vt_render(vt_ctx *c, const vt_section *secs, int32_t n_secs, const double *pose12,
                    vt_intrinsics K, int32_t W, int32_t H, float *rgb, float *depth,
                    float *silhouette, vt_stream stream) {
    if (!c) return fail(VT_ERR_INVALID_ARG, "vt_render: ctx is NULL");
    if (!pose12) return fail(VT_ERR_INVALID_ARG, "vt_render: pose is NULL");
    if (n_secs < 0 || n_secs > kMaxSecs || (n_secs > 0 && !secs))
        return fail(VT_ERR_INVALID_ARG, "vt_render: n_secs must be in [0, %d]", kMaxSecs);
    vt_status st = check_intrinsics(K, "vt_render");
    if (st) return st;
    if ((st = check_image(W, H, "vt_render"))) return st;
    SecTable T{};
    T.n = n_secs;
    int64_t total = 0, views = 0, tabrows = 0;
    bool aniso = false;
    for (int s = 0; s < n_secs; ++s) {
        const vt_section &S = secs[s];
        if (S.n < 0) return fail(VT_ERR_INVALID_ARG, "vt_render: section %d has n < 0", s);
        if (S.n_views <= 0 || S.W <= 0 || S.H <= 0 ||
            (int64_t)S.n_views * S.W * S.H > (int64_t)0xffffffffll)
            return fail(VT_ERR_INVALID_ARG, "vt_render: section %d views/size out of range", s);
        if (S.prec != VT_F32 && S.prec != VT_F16)
            return fail(VT_ERR_INVALID_ARG, "vt_render: section %d precision %d unknown", s,
                        (int)S.prec);
        if ((st = check_intrinsics(S.K, "vt_render section"))) return st;
        const bool ell = S.scale != nullptr;
        if (s == 0) aniso = ell;
        if (ell != aniso)
            return fail(VT_ERR_INVALID_ARG, "vt_render: sections %d and 0 differ in footprint "
                                            "(ellipsoids and spheres in one render)", s);
        if (S.n > 0 && (!S.poses || !S.depth || !S.src || !S.colour || !S.opacity ||
                        (ell ? !S.rot : !S.radius)))
            return fail(VT_ERR_INVALID_ARG, "vt_render: section %d has a NULL array", s);
        SecDesc &D = T.s[s];
        D.poses = S.poses;
        D.depth = S.depth;
        D.src = S.src;
        D.colour = S.colour;
        D.opacity = S.opacity;
        D.radius = S.radius;
        D.scale = S.scale;
        D.rot = S.rot;
        D.d_colour = D.d_opacity = D.d_radius = nullptr;
        D.d_scale = D.d_rot = nullptr;
        D.gbase = total;
        D.n = S.n;
        D.tab_base = tabrows;
        D.view_base = (int32_t)views;
        D.n_views = S.n_views;
        D.W = S.W;
        D.H = S.H;
        D.prec = (int32_t)S.prec;
        D.fx = S.K.fx;
        D.fy = S.K.fy;
        D.cx = S.K.cx;
        D.cy = S.K.cy;
        total += S.n;
        views += S.n_views;
        tabrows += (int64_t)S.n_views * (S.W + S.H);
    }
    if (total >= (int64_t)0xffffffffll)
        return fail(VT_ERR_INVALID_ARG, "vt_render: %lld Gaussians exceed 2^32 - 1",
                    (long long)total);
    T.n_total = total;
    Camera cam;
    cam.fx = K.fx;
    cam.fy = K.fy;
    cam.cx = K.cx;
    cam.cy = K.cy;
    cam.W = W;
    cam.H = H;
    cam.tiles_x = (W + kTile - 1) / kTile;
    cam.tiles_y = (H + kTile - 1) / kTile;
    const int n_tiles = cam.tiles_x * cam.tiles_y;
    const int64_t want_i = c->reserved_i > 0 ? c->reserved_i : default_instances(total);
    c->stream = stream;
    if ((st = ensure(c, std::max<int64_t>(total, 1), want_i, (int64_t)W * H,
                     n_tiles, std::max<int64_t>(views, 1), std::max<int64_t>(tabrows, 1), stream)))
        return st;
    if (!sort_attr_set) {
        for (auto kern : {k_sort_tiles, k_sort_tiles_mid, k_sort_tiles_large, k_sort_tiles_long})
            VT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSortSmemBigBytes),
                    "sort smem attribute");
        sort_attr_set = true;
    }
    c->has_render = false;
    // Per-pixel lists for the backward, unless they would exceed the budget
    // (then the backward replays the tile lists instead).
    c->used_lists = false;
    if (c->list_cap > 0) {
        const size_t need = sizeof(uint2) * (size_t)c->list_cap * (size_t)W * (size_t)H;
        if (c->arena_bytes + need <= c->budget) {
            if (need > c->plist_bytes) {
                if (c->plist) cudaFreeAsync(c->plist, stream);
                c->plist = nullptr;
                c->plist_bytes = 0;
                void *q = nullptr;
                if (cudaMallocAsync(&q, need, stream) == cudaSuccess) {
                    c->plist = static_cast<uint2 *>(q);
                    c->plist_bytes = need;
                } else {
                    cudaGetLastError();   // fall back to the tile replay
                }
            }
            c->used_lists = c->plist != nullptr;
        }
    }
    VT_CUDA(cudaMemsetAsync(c->tile_count, 0, sizeof(uint32_t) * (n_tiles + 1), stream),
            "tile count reset");
    if (views > 0) {
        LaunchScope ls(c, K_SETUP, stream);
        k_setup<<<(unsigned)views, 256, 0, stream>>>(T, cam, pose12, c->views, c->tab,
                                                    c->pose_copy);
    } else {
        VT_CUDA(cudaMemcpyAsync(c->pose_copy, pose12, 12 * sizeof(double),
                                cudaMemcpyDeviceToDevice, stream),
                "pose copy");
    }
    const unsigned gblocks = (unsigned)((total + 255) / 256);
    if (total > 0) {
        LaunchScope ls(c, aniso ? K_PRE_AN : K_PREPROCESS, stream);
        auto kern = aniso ? k_preprocess_aniso : k_preprocess;
        kern<<<gblocks, 256, 0, stream>>>(T, cam, c->views, c->tab, c->geo, c->app, c->info,
                                          c->tile_count);
    }
    {
        LaunchScope ls(c, K_SCAN, stream);
        k_scan_tiles<<<1, 1024, 0, stream>>>(c->tile_count, n_tiles, c->tile_off, c->tile_cursor,
                                             c->status, (unsigned long long)c->cap_i,
                                             c->long_tiles);
    }
    if (total > 0) {
        LaunchScope ls(c, K_EMIT, stream);
        k_emit<<<gblocks, 256, 0, stream>>>(total, c->info, cam, c->tile_cursor, c->bucket,
                                            c->bmask_u, c->status);
    }
    // fork: the long lists sort on the auxiliary stream (few blocks: they
    // leave most SMs free), the large and then the shortest class on the
    // second one, the middle class on the caller's, all three branches at
    // once and of similar length (works under graph capture too: the fork
    // and join events make them parallel branches)
    VT_CUDA(cudaEventRecord(c->ev_fork, stream), "sort fork");
    VT_CUDA(cudaStreamWaitEvent(c->aux, c->ev_fork, 0), "sort fork");
    VT_CUDA(cudaStreamWaitEvent(c->aux2, c->ev_fork, 0), "sort fork");
    {
        LaunchScope ls(c, K_SORT_BIG, c->aux);
        // one block per SM at most: these lists are few, and the launch must
        // not hold every SM's shared memory while the others run
        k_sort_tiles_long<<<std::min(n_tiles, c->n_sm), 512, kSortSmemBigBytes, c->aux>>>(
            c->tile_off, n_tiles, c->bucket, c->alt, c->bmask_u, c->sorted, c->bmask,
            aniso ? nullptr : c->geo, cam, c->status, kSortSmemBig, kSortSmemN, kSortSmemBig, c->long_tiles);
    }
    {
        LaunchScope ls(c, K_SORT_L, c->aux2);
        k_sort_tiles_large<<<n_tiles, 512, kSortSmemBytes, c->aux2>>>(
            c->tile_off, n_tiles, c->bucket, c->alt, c->bmask_u, c->sorted, c->bmask,
            aniso ? nullptr : c->geo, cam, c->status, kSortSmemN, kSortClassM, kSortSmemN, c->long_tiles);
    }
    {
        LaunchScope ls(c, K_SORT, c->aux2);
        k_sort_tiles<<<n_tiles, 512, sort_smem_bytes(kSortClassS), c->aux2>>>(
            c->tile_off, n_tiles, c->bucket, c->alt, c->bmask_u, c->sorted, c->bmask,
            aniso ? nullptr : c->geo, cam, c->status, kSortClassS, 0, kSortClassS, c->long_tiles);
    }
    VT_CUDA(cudaEventRecord(c->ev_join2, c->aux2), "sort join");
    {
        LaunchScope ls(c, K_SORT_XL, c->aux);
        k_sort_tiles_xl<<<std::min(n_tiles, 2 * c->n_sm), 512, kSortHistBytes, c->aux>>>(
            c->tile_off, n_tiles, c->bucket, c->alt, c->bmask_u, c->sorted, c->bmask,
            aniso ? nullptr : c->geo, cam, c->status, kSortSmemBig, kSortSmemBig, 0x7fffffff, c->long_tiles);
    }
    VT_CUDA(cudaEventRecord(c->ev_join, c->aux), "sort join");
    {
        LaunchScope ls(c, K_SORT_M, stream);
        k_sort_tiles_mid<<<n_tiles, 512, sort_smem_bytes(kSortClassM), stream>>>(
            c->tile_off, n_tiles, c->bucket, c->alt, c->bmask_u, c->sorted, c->bmask,
            aniso ? nullptr : c->geo, cam, c->status, kSortClassM, kSortClassS, kSortClassM, c->long_tiles);
    }
    VT_CUDA(cudaStreamWaitEvent(stream, c->ev_join, 0), "sort join");
    VT_CUDA(cudaStreamWaitEvent(stream, c->ev_join2, 0), "sort join");
    {
        LaunchScope ls(c, aniso ? K_FWD_AN : K_FWD, stream);
        auto kern = aniso ? k_composite_fwd_aniso : k_composite_fwd;
        kern<<<n_tiles, kBlockPix, 0, stream>>>(
            cam, c->tile_off, c->sorted, c->bmask, c->geo, c->app, rgb, depth, silhouette,
            c->pix_last, c->pix_nadd, c->pix_T, c->used_lists ? c->plist : nullptr, c->list_cap,
            c->blk_ovf, c->status);
    }
    VT_CUDA(cudaGetLastError(), "vt_render launch");
    c->aniso = aniso;
    c->table = T;
    c->cam = cam;
    c->n_tiles = n_tiles;
    c->has_render = true;
    return VT_OK;
}

// Backward of an ellipsoid render: per-pair terms accumulated per Gaussian
// by the list (and replay) kernels, colour / opacity scattered as for the
// spheres, then the per-Gaussian chain to scale, quaternion and pose.
static vt_status backward_aniso(vt_ctx *c, SecTable &T, const float *dL_drgb,
                                const float *dL_ddepth, const float *dL_dsil, int32_t mode,
                                const vt_grads *grads, double *d_twist, double *d_mat,
                                cudaStream_t stream) {
    if (mode & VT_GRAD_VIEWS)
        return fail(VT_ERR_INVALID_ARG,
                    "vt_render_backward: source-view gradients are not available for ellipsoids");
    const bool attr = (mode & VT_GRAD_ATTR) != 0, pose = (mode & VT_GRAD_POSE) != 0;
    for (int s = 0; s < T.n; ++s) {
        if (!attr) continue;
        T.s[s].d_colour = grads[s].d_colour;
        T.s[s].d_opacity = grads[s].d_opacity;
        T.s[s].d_radius = nullptr;
        T.s[s].d_scale = grads[s].d_scale;
        T.s[s].d_rot = grads[s].d_rot;
    }
    if (T.n_total > 0) {
        if (attr)
            VT_CUDA(cudaMemsetAsync(c->acc4, 0, sizeof(float4) * T.n_total, stream),
                    "grad acc reset");
        VT_CUDA(cudaMemsetAsync(c->accg, 0, sizeof(float4) * T.n_total, stream), "grad acc reset");
        VT_CUDA(cudaMemsetAsync(c->accm, 0, sizeof(float2) * T.n_total, stream), "grad acc reset");
    }
    if (c->used_lists) {
        LaunchScope ls(c, K_BWD_LIST_AN, stream);
        k_composite_bwd_list_aniso<<<c->n_tiles, kBlockPix, 0, stream>>>(
            T, c->cam, c->geo, c->app, c->pix_nadd, c->pix_T, c->plist, c->list_cap, c->blk_ovf,
            dL_drgb, dL_ddepth, dL_dsil, mode, c->pose_partials, c->acc4, c->accr, c->accg,
            c->accm, c->status);
    }
    {   // tiles without complete per-pixel lists (all of them when none were kept)
        LaunchScope ls(c, K_BWD_AN, stream);
        k_composite_bwd_aniso<<<c->n_tiles, kBlockPix, 0, stream>>>(
            T, c->cam, c->tile_off, c->sorted, c->geo, c->app, c->pix_last, c->pix_T, dL_drgb,
            dL_ddepth, dL_dsil, mode, c->blk_ovf, c->acc4, c->accg, c->accm, c->status);
    }
    if (attr && T.n_total > 0) {
        LaunchScope ls(c, K_SCATTER, stream);
        k_attr_scatter<<<(unsigned)((T.n_total + 255) / 256), 256, 0, stream>>>(T, c->acc4,
                                                                               c->accr);
    }
    const int chain_blocks =
        (int)std::max<int64_t>(1, std::min<int64_t>((T.n_total + 255) / 256, c->n_tiles));
    {
        LaunchScope ls(c, K_CHAIN, stream);
        k_aniso_chain<<<chain_blocks, 256, 0, stream>>>(T, c->cam, c->views, c->geo, c->app,
                                                       c->accg, c->accm, (int)pose, (int)attr,
                                                       c->pose_partials);
    }
    if (pose) {
        LaunchScope ls(c, K_POSE, stream);
        k_pose_finalize<<<1, 384, 0, stream>>>(c->pose_partials, chain_blocks, c->pose_copy,
                                               d_twist, d_mat);
    }
    VT_CUDA(cudaGetLastError(), "vt_render_backward launch");
    return VT_OK;
}

vt_status vt_render_backward(vt_ctx *c, const float *dL_drgb, const float *dL_ddepth,
                             const float *dL_dsil, int32_t mode, const vt_grads *grads,
                             double *d_twist, double *d_mat, vt_stream stream) {
    if (!c) return fail(VT_ERR_INVALID_ARG, "vt_render_backward: ctx is NULL");
    if (!c->has_render) return fail(VT_ERR_STATE, "vt_render_backward: no render on this context");
    if (mode & ~(VT_GRAD_ATTR | VT_GRAD_POSE | VT_GRAD_VIEWS))
        return fail(VT_ERR_INVALID_ARG, "vt_render_backward: unknown mode bits 0x%x", mode);
    if ((mode & (VT_GRAD_ATTR | VT_GRAD_VIEWS)) && !grads && c->table.n > 0)
        return fail(VT_ERR_INVALID_ARG, "vt_render_backward: ATTR / VIEWS mode needs grads");
    if ((mode & VT_GRAD_POSE) && !d_twist && !d_mat)
        return fail(VT_ERR_INVALID_ARG, "vt_render_backward: POSE mode needs d_twist or d_mat");
    if (!mode) return VT_OK;
    SecTable T = c->table;
    if (c->aniso)
        return backward_aniso(c, T, dL_drgb, dL_ddepth, dL_dsil, mode, grads, d_twist, d_mat,
                              stream);
    for (int s = 0; s < T.n; ++s) {
        if (mode & VT_GRAD_ATTR) {
            T.s[s].d_colour = grads[s].d_colour;
            T.s[s].d_opacity = grads[s].d_opacity;
            T.s[s].d_radius = grads[s].d_radius;
        }
        if (mode & VT_GRAD_VIEWS) {
            T.s[s].d_view_twist = grads[s].d_view_twist;
            T.s[s].d_view_mat = grads[s].d_view_mat;
            T.s[s].d_depth = grads[s].d_depth;
        }
    }
    const bool views = (mode & VT_GRAD_VIEWS) != 0;
    if (views && T.n_total > 0)
        VT_CUDA(cudaMemsetAsync(c->accg, 0, sizeof(float4) * T.n_total, stream), "grad acc reset");
    const bool attr = (mode & VT_GRAD_ATTR) != 0;
    if (attr && T.n_total > 0) {
        VT_CUDA(cudaMemsetAsync(c->acc4, 0, sizeof(float4) * T.n_total, stream), "grad acc reset");
        VT_CUDA(cudaMemsetAsync(c->accr, 0, sizeof(float) * T.n_total, stream), "grad acc reset");
    }
    if (c->used_lists) {
        // the pose alone: without a matrix gradient to return, the twist's six
        // sums replace the twelve of x g^T and g
        const bool posemat = d_mat != nullptr;
        LaunchScope ls(c, views ? K_BWD_LIST_VIEWS
                                : (attr ? K_BWD_LIST
                                        : (posemat ? K_BWD_LIST_POSEMAT : K_BWD_LIST_POSE)),
                       stream);
        auto kern = views ? k_composite_bwd_list_views
                          : (attr ? k_composite_bwd_list
                                  : (posemat ? k_composite_bwd_list_posemat
                                             : k_composite_bwd_list_pose));
        kern<<<c->n_tiles, kBlockPix, 0, stream>>>(
            T, c->cam, c->geo, c->app, c->pix_nadd, c->pix_T, c->plist, c->list_cap, c->blk_ovf,
            dL_drgb, dL_ddepth, dL_dsil, mode, c->pose_partials, c->acc4, c->accr, c->accg,
            c->status);
    }
    {   // tiles without complete per-pixel lists (all of them when none were kept)
        LaunchScope ls(c, K_BWD, stream);
        k_composite_bwd<<<c->n_tiles, kBlockPix, 0, stream>>>(
            T, c->cam, c->tile_off, c->sorted, c->geo, c->app, c->pix_last, c->pix_T, dL_drgb,
            dL_ddepth, dL_dsil, mode, c->pose_partials, c->blk_ovf, c->acc4, c->accr, c->accg,
            c->status);
    }
    if (attr && T.n_total > 0) {
        LaunchScope ls(c, K_SCATTER, stream);
        k_attr_scatter<<<(unsigned)((T.n_total + 255) / 256), 256, 0, stream>>>(T, c->acc4,
                                                                               c->accr);
    }
    if (views && T.n_total > 0) {
        int n_views = 0;
        for (int s = 0; s < T.n; ++s) n_views += T.s[s].n_views;
        const size_t need = sizeof(double) * 12 * (size_t)n_views * kViewChunks;
        if (need > c->view_part_bytes) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            VT_CUDA(cudaStreamIsCapturing(stream, &cs), "capture query");
            if (cs != cudaStreamCaptureStatusNone)
                return fail(VT_ERR_STATE, "vt_render_backward: view-gradient scratch must be "
                                          "sized by a call before graph capture");
            if (c->view_part) cudaFreeAsync(c->view_part, stream);
            c->view_part = nullptr;
            c->view_part_bytes = 0;
            void *p = nullptr;
            VT_CUDA(cudaMallocAsync(&p, need, stream), "view-gradient scratch");
            c->view_part = static_cast<double *>(p);
            c->view_part_bytes = need;
        }
        {
            LaunchScope ls(c, K_VIEW_GRADS, stream);
            k_view_grads<<<n_views * kViewChunks, kBlockPix, 0, stream>>>(T, c->accg, c->pose_copy,
                                                                          c->view_part);
        }
        LaunchScope ls(c, K_VIEW_FIN, stream);
        k_view_finalize<<<(n_views + 63) / 64, 64, 0, stream>>>(T, c->pose_copy, c->view_part,
                                                              n_views);
    }
    if (mode & VT_GRAD_POSE) {
        LaunchScope ls(c, K_POSE, stream);
        k_pose_finalize<<<1, 384, 0, stream>>>(c->pose_partials, c->n_tiles, c->pose_copy, d_twist,
                                               d_mat);
    }
    VT_CUDA(cudaGetLastError(), "vt_render_backward launch");
    return VT_OK;
}

// Shared checks of the visibility entry points; fills vv.
static vt_status vis_args(const char *who, const float *depth, int32_t W, int32_t H,
                          vt_intrinsics K, const double *pose12, const vt_view *views,
                          int32_t n_views, double rel_tol, const void *out, VisViews &vv) {
    vt_status st = check_image(W, H, who);
    if (st) return st;
    if ((st = check_intrinsics(K, who))) return st;
    if (!depth || !pose12 || !out || !views)
        return fail(VT_ERR_INVALID_ARG, "%s: NULL depth, pose, views or output", who);
    if (n_views < 1 || n_views > VT_MAX_VIS_VIEWS)
        return fail(VT_ERR_INVALID_ARG, "%s: n_views = %d outside [1, %d]", who, n_views,
                    VT_MAX_VIS_VIEWS);
    if (!(std::isfinite(rel_tol) && rel_tol >= 0.0))
        return fail(VT_ERR_INVALID_ARG, "%s: rel_tol must be finite and >= 0", who);
    vv = VisViews{};
    vv.n = n_views;
    for (int k = 0; k < n_views; ++k) {
        const vt_view &V = views[k];
        if ((st = check_image(V.W, V.H, who))) return st;
        if ((st = check_intrinsics(V.K, who))) return st;
        if (!V.depth || !V.pose12)
            return fail(VT_ERR_INVALID_ARG, "%s: view %d has NULL depth or pose", who, k);
        vv.v[k] = VisView{V.depth, V.W, V.H, V.K.fx, V.K.fy, V.K.cx, V.K.cy, V.pose12};
    }
    return VT_OK;
}

vt_status vt_visibility_counts(const float *depth, int32_t W, int32_t H, vt_intrinsics K,
                               const double *pose12, const vt_view *views, int32_t n_views,
                               double rel_tol, uint32_t *counts, uint32_t *n_valid,
                               vt_stream stream) {
    VisViews vv;
    vt_status st = vis_args("vt_visibility_counts", depth, W, H, K, pose12, views, n_views,
                            rel_tol, counts, vv);
    if (st) return st;
    VT_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * n_views, stream), "counts reset");
    if (n_valid) VT_CUDA(cudaMemsetAsync(n_valid, 0, sizeof(uint32_t), stream), "counts reset");
    const int64_t P = (int64_t)W * H;
    k_visibility_counts<<<(unsigned)((P + 255) / 256), 256, 0, stream>>>(
        depth, W, H, K.fx, K.fy, K.cx, K.cy, pose12, vv, rel_tol, counts, n_valid);
    VT_CUDA(cudaGetLastError(), "vt_visibility_counts launch");
    return VT_OK;
}

vt_status vt_visibility(const float *depth, int32_t W, int32_t H, vt_intrinsics K,
                        const double *pose12, const vt_view *views, int32_t n_views,
                        double rel_tol, uint8_t *visible, vt_stream stream) {
    VisViews vv;
    vt_status st = vis_args("vt_visibility", depth, W, H, K, pose12, views, n_views, rel_tol,
                            visible, vv);
    if (st) return st;
    const int64_t P = (int64_t)W * H;
    k_visibility<<<(unsigned)((P + 255) / 256), 256, 0, stream>>>(
        depth, W, H, K.fx, K.fy, K.cx, K.cy, pose12, vv, rel_tol, visible);
    VT_CUDA(cudaGetLastError(), "vt_visibility launch");
    return VT_OK;
}

vt_status vt_masked_l1(vt_ctx *c, int32_t W, int32_t H, const float *rgb, const float *depth,
                       const float *silhouette, const float *obs_rgb, const float *obs_depth,
                       const uint8_t *visible, vt_l1_weights w, float *d_rgb, float *d_depth,
                       double *loss, vt_stream stream) {
    if (!c) return fail(VT_ERR_INVALID_ARG, "vt_masked_l1: ctx is NULL");
    vt_status st = check_image(W, H, "vt_masked_l1");
    if (st) return st;
    if (!rgb || !depth || !obs_rgb || !obs_depth)
        return fail(VT_ERR_INVALID_ARG, "vt_masked_l1: NULL image");
    if (w.sil_min >= 0.f && !silhouette)
        return fail(VT_ERR_INVALID_ARG, "vt_masked_l1: coverage mask needs the silhouette");
    if (!std::isfinite(w.w_rgb) || !std::isfinite(w.w_depth) || std::isnan(w.sil_min))
        return fail(VT_ERR_INVALID_ARG, "vt_masked_l1: weights must be finite");
    const int64_t P = (int64_t)W * H;
    const int64_t nb = (P + 255) / 256;
    if (loss && (st = ensure_loss(c, nb, stream))) return st;
    const double wc = w.w_rgb / (3.0 * (double)P), wd = w.w_depth / (double)P;
    {
        LaunchScope ls(c, K_L1, stream);
        k_masked_l1<<<(unsigned)nb, 256, 0, stream>>>(
            P, rgb, depth, silhouette, obs_rgb, obs_depth, visible, w.sil_min,
            w.rgb_needs_depth ? 1 : 0, (float)wc, (float)wd, d_rgb, d_depth,
            loss ? c->loss_part : nullptr);
    }
    if (loss) {
        LaunchScope ls(c, K_L1_SUM, stream);
        k_sum_partials<<<1, 256, 0, stream>>>(c->loss_part, (int)nb, wc, wd, loss);
    }
    VT_CUDA(cudaGetLastError(), "vt_masked_l1 launch");
    return VT_OK;
}

vt_status vt_ssim(vt_ctx *c, int32_t W, int32_t H, const float *rgb, const float *obs_rgb,
                  double weight, float *d_rgb, double *loss, vt_stream stream) {
    if (!c) return fail(VT_ERR_INVALID_ARG, "vt_ssim: ctx is NULL");
    vt_status st = check_image(W, H, "vt_ssim");
    if (st) return st;
    if (!rgb || !obs_rgb) return fail(VT_ERR_INVALID_ARG, "vt_ssim: NULL image");
    if (!std::isfinite(weight)) return fail(VT_ERR_INVALID_ARG, "vt_ssim: weight must be finite");
    const int64_t P = (int64_t)W * H;
    const dim3 grid((W + kSsimTileW - 1) / kSsimTileW, (H + kSsimTileH - 1) / kSsimTileH);
    const int64_t nb = (int64_t)grid.x * grid.y;
    // 15 map floats per pixel (5 maps x 3 channels), then 2 doubles per block
    const int64_t need = std::max<int64_t>(P, 256 * nb);
    if (need > c->ssim_cap) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        VT_CUDA(cudaStreamIsCapturing(stream, &cs), "capture query");
        if (cs != cudaStreamCaptureStatusNone)
            return fail(VT_ERR_STATE, "vt_ssim: scratch must be sized before graph capture");
        if (c->ssim_buf) cudaFreeAsync(c->ssim_buf, stream);
        c->ssim_buf = nullptr;
        c->ssim_cap = 0;
        const int64_t cap = need;
        void *p = nullptr;
        const size_t bytes =
            align_up(sizeof(float) * 15 * (size_t)cap) + sizeof(double) * 2 * (cap / 256 + 1);
        const cudaError_t e = cudaMallocAsync(&p, bytes, stream);
        if (e != cudaSuccess)
            return fail(VT_ERR_OOM, "SSIM scratch of %zu bytes: %s", bytes, cudaGetErrorString(e));
        c->ssim_buf = p;
        c->ssim_cap = cap;
    }
    float *maps = static_cast<float *>(c->ssim_buf);
    double *part = reinterpret_cast<double *>(static_cast<char *>(c->ssim_buf) +
                                              align_up(sizeof(float) * 15 * (size_t)c->ssim_cap));
    SsimWindow win{};
    double g[11], sum = 0.0;
    for (int k = -5; k <= 5; ++k) sum += (g[k + 5] = std::exp(-(double)(k * k) / 4.5));
    for (int k = 0; k < 11; ++k) win.g[k] = (float)(g[k] / sum);
    const double n = 3.0 * (double)P;
    {
        LaunchScope ls(c, K_SSIM_FWD, stream);
        k_ssim_fwd<<<grid, 256, 0, stream>>>(W, H, rgb, obs_rgb, win, maps, loss ? part : nullptr);
    }
    if (loss) {   // weight (1 - sum SSIM / n) = (weight / n) (count - sum SSIM)
        LaunchScope ls(c, K_SSIM_SUM, stream);
        k_sum_partials<<<1, 256, 0, stream>>>(part, (int)nb, -weight / n, weight / n, loss);
    }
    if (d_rgb) {
        LaunchScope ls(c, K_SSIM_BWD, stream);
        k_ssim_bwd<<<grid, 256, 0, stream>>>(W, H, rgb, obs_rgb, win, maps, (float)(-weight / n),
                                             d_rgb);
    }
    VT_CUDA(cudaGetLastError(), "vt_ssim launch");
    return VT_OK;
}

vt_status vt_pose_adam(vt_ctx *c, double *pose12, double *d_twist, double *state,
                       const double *lr, double beta1, double beta2, double eps,
                       vt_stream stream) {
    if (!pose12 || !d_twist || !state || !lr)
        return fail(VT_ERR_INVALID_ARG, "vt_pose_adam: NULL pose, gradient, state or rates");
    PoseAdamParams prm{};
    for (int i = 0; i < 6; ++i) {
        if (!std::isfinite(lr[i]) || lr[i] < 0.0)
            return fail(VT_ERR_INVALID_ARG, "vt_pose_adam: learning rates must be finite, >= 0");
        prm.lr[i] = lr[i];
    }
    if (!(beta1 >= 0.0 && beta1 < 1.0 && beta2 >= 0.0 && beta2 < 1.0 && eps >= 0.0 &&
          std::isfinite(eps)))
        return fail(VT_ERR_INVALID_ARG, "vt_pose_adam: need 0 <= beta < 1 and finite eps >= 0");
    prm.beta1 = beta1;
    prm.beta2 = beta2;
    prm.eps = eps;
    if (c) {
        LaunchScope ls(c, K_POSE_ADAM, stream);
        k_pose_adam<<<1, 32, 0, stream>>>(pose12, d_twist, state, prm);
    } else {
        k_pose_adam<<<1, 32, 0, stream>>>(pose12, d_twist, state, prm);   // one warp
    }
    VT_CUDA(cudaGetLastError(), "vt_pose_adam launch");
    return VT_OK;
}

vt_status vt_adam_init(vt_ctx *c, int64_t n, vt_precision prec, const void *colour,
                       const void *opacity, const void *radius, const void *scale,
                       const void *rot, float *theta, float *m, float *v, double *step,
                       vt_stream stream) {
    if (n < 0) return fail(VT_ERR_INVALID_ARG, "vt_adam_init: n < 0");
    if (prec != VT_F32 && prec != VT_F16)
        return fail(VT_ERR_INVALID_ARG, "vt_adam_init: unknown precision %d", (int)prec);
    if (!step) return fail(VT_ERR_INVALID_ARG, "vt_adam_init: NULL step");
    if (n > 0 && (!theta || !m || !v ||
                  (scale ? !rot : (!colour || !opacity || !radius))))
        return fail(VT_ERR_INVALID_ARG, "vt_adam_init: NULL array");
    VT_CUDA(cudaMemsetAsync(step, 0, 3 * sizeof(double), stream), "vt_adam_init step");
    if (n > 0) {
        const unsigned nb = (unsigned)((n + 255) / 256);
        auto go = [&]() {
            k_adam_init<<<nb, 256, 0, stream>>>(n, (int)prec, colour, opacity, radius, scale,
                                                rot, theta, m, v);
        };
        if (c) {
            LaunchScope ls(c, K_ADAM_INIT, stream);
            go();
        } else {
            go();
        }
    }
    VT_CUDA(cudaGetLastError(), "vt_adam_init launch");
    return VT_OK;
}

vt_status vt_attr_adam(vt_ctx *c, int64_t n, float *theta, float *m, float *v, double *step,
                       float *d_colour, float *d_opacity, float *d_radius, vt_precision prec,
                       void *colour, void *opacity, void *radius, vt_adam_params p,
                       vt_stream stream) {
    if (n < 0) return fail(VT_ERR_INVALID_ARG, "vt_attr_adam: n < 0");
    if (prec != VT_F32 && prec != VT_F16)
        return fail(VT_ERR_INVALID_ARG, "vt_attr_adam: unknown precision %d", (int)prec);
    if (!step) return fail(VT_ERR_INVALID_ARG, "vt_attr_adam: NULL step");
    if (n > 0 && (!theta || !m || !v || !d_colour || !d_opacity || !d_radius || !colour ||
                  !opacity || !radius))
        return fail(VT_ERR_INVALID_ARG, "vt_attr_adam: NULL array");
    AttrAdamParams prm{};
    for (int k = 0; k < 5; ++k) {
        if (!std::isfinite(p.lr[k]) || p.lr[k] < 0.f)
            return fail(VT_ERR_INVALID_ARG, "vt_attr_adam: learning rates must be finite, >= 0");
        prm.lr[k] = p.lr[k];
    }
    if (!(p.beta1 >= 0.f && p.beta1 < 1.f && p.beta2 >= 0.f && p.beta2 < 1.f && p.eps >= 0.f &&
          std::isfinite(p.eps)))
        return fail(VT_ERR_INVALID_ARG, "vt_attr_adam: need 0 <= beta < 1 and finite eps >= 0");
    prm.beta1 = p.beta1;
    prm.beta2 = p.beta2;
    prm.eps = p.eps;
    auto launch = [&]() {
        k_adam_step_count<<<1, 32, 0, stream>>>(step, (double)p.beta1, (double)p.beta2);
    };
    if (c) {
        LaunchScope ls(c, K_ADAM_COUNT, stream);
        launch();
    } else {
        launch();
    }
    if (n > 0) {
        const unsigned nb = (unsigned)((n + 255) / 256);
        auto upd = [&]() {
            k_attr_adam<<<nb, 256, 0, stream>>>(n, theta, m, v, step, d_colour, d_opacity,
                                                d_radius, (int)prec, colour, opacity, radius,
                                                prm);
        };
        if (c) {
            LaunchScope ls(c, K_ATTR_ADAM, stream);
            upd();
        } else {
            upd();
        }
    }
    VT_CUDA(cudaGetLastError(), "vt_attr_adam launch");
    return VT_OK;
}

vt_status vt_shape_adam(vt_ctx *c, int64_t n, float *theta, float *m, float *v, double *step,
                        float *d_scale, float *d_rot, vt_precision prec, void *scale, void *rot,
                        vt_shape_adam_params p, vt_stream stream) {
    if (n < 0) return fail(VT_ERR_INVALID_ARG, "vt_shape_adam: n < 0");
    if (prec != VT_F32 && prec != VT_F16)
        return fail(VT_ERR_INVALID_ARG, "vt_shape_adam: unknown precision %d", (int)prec);
    if (!step) return fail(VT_ERR_INVALID_ARG, "vt_shape_adam: NULL step");
    if (n > 0 && (!theta || !m || !v || !d_scale || !d_rot || !scale || !rot))
        return fail(VT_ERR_INVALID_ARG, "vt_shape_adam: NULL array");
    if (!(std::isfinite(p.lr_scale) && p.lr_scale >= 0.f && std::isfinite(p.lr_rot) &&
          p.lr_rot >= 0.f))
        return fail(VT_ERR_INVALID_ARG, "vt_shape_adam: learning rates must be finite, >= 0");
    if (!(p.beta1 >= 0.f && p.beta1 < 1.f && p.beta2 >= 0.f && p.beta2 < 1.f && p.eps >= 0.f &&
          std::isfinite(p.eps)))
        return fail(VT_ERR_INVALID_ARG, "vt_shape_adam: need 0 <= beta < 1 and finite eps >= 0");
    const ShapeAdamParams prm{p.lr_scale, p.lr_rot, p.beta1, p.beta2, p.eps};
    auto count = [&]() {
        k_adam_step_count<<<1, 32, 0, stream>>>(step, (double)p.beta1, (double)p.beta2);
    };
    if (c) {
        LaunchScope ls(c, K_ADAM_COUNT, stream);
        count();
    } else {
        count();
    }
    if (n > 0) {
        const unsigned nb = (unsigned)((n + 255) / 256);
        auto upd = [&]() {
            k_shape_adam<<<nb, 256, 0, stream>>>(n, theta, m, v, step, d_scale, d_rot, (int)prec,
                                                 scale, rot, prm);
        };
        if (c) {
            LaunchScope ls(c, K_SHAPE_ADAM, stream);
            upd();
        } else {
            upd();
        }
    }
    VT_CUDA(cudaGetLastError(), "vt_shape_adam launch");
    return VT_OK;
}

// Ordered compaction scratch: per-block counts and offsets, stream-ordered
// allocation released on the same stream after the launches.
static vt_status compaction_scratch(int64_t total, uint32_t **counts, uint32_t **offs,
                                    int64_t *nb, cudaStream_t s) {
    *nb = (total + kInitBlock - 1) / kInitBlock;
    void *p = nullptr;
    const size_t bytes = sizeof(uint32_t) * 2 * (size_t)std::max<int64_t>(*nb, 1);
    cudaError_t e = cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(VT_ERR_OOM, "compaction scratch of %zu bytes: %s", bytes,
                    cudaGetErrorString(e));
    }
    *counts = static_cast<uint32_t *>(p);
    *offs = *counts + std::max<int64_t>(*nb, 1);
    return VT_OK;
}

vt_status vt_backproject(const float *depth, int32_t W, int32_t H, vt_intrinsics K,
                         const double *pose12, float *centres, uint32_t *pix, int64_t cap,
                         int64_t *n_out, vt_stream stream) {
    vt_status st = check_image(W, H, "vt_backproject");
    if (st) return st;
    if ((st = check_intrinsics(K, "vt_backproject"))) return st;
    if (!depth || !pose12 || !n_out || cap < 0 || (cap > 0 && (!centres || !pix)))
        return fail(VT_ERR_INVALID_ARG, "vt_backproject: NULL pointer or negative capacity");
    const int64_t total = (int64_t)W * H;
    uint32_t *counts, *offs;
    int64_t nb;
    if ((st = compaction_scratch(total, &counts, &offs, &nb, stream))) return st;
    k_count_valid<<<(unsigned)nb, kInitBlock, 0, stream>>>(depth, total, counts);
    k_scan_counts<<<1, 1024, 0, stream>>>(counts, nb, offs, reinterpret_cast<long long *>(n_out));
    k_backproject<<<(unsigned)nb, kInitBlock, 0, stream>>>(depth, W, H, K, pose12, offs, centres,
                                                           pix, cap);
    cudaFreeAsync(counts, stream);
    VT_CUDA(cudaGetLastError(), "vt_backproject launch");
    return VT_OK;
}

vt_status vt_section_init(const float *depth, const float *rgb, int32_t n_views, int32_t W,
                          int32_t H, vt_intrinsics K, vt_precision prec, uint32_t *src,
                          void *colour, void *opacity, void *radius, int64_t cap,
                          int64_t *n_out, vt_stream stream) {
    vt_status st = check_image(W, H, "vt_section_init");
    if (st) return st;
    if ((st = check_intrinsics(K, "vt_section_init"))) return st;
    if (n_views <= 0 || (int64_t)n_views * W * H > (int64_t)0xffffffffll)
        return fail(VT_ERR_INVALID_ARG, "vt_section_init: n_views out of range");
    if (prec != VT_F32 && prec != VT_F16)
        return fail(VT_ERR_INVALID_ARG, "vt_section_init: unknown precision");
    if (!depth || !rgb || !n_out || cap < 0 ||
        (cap > 0 && (!src || !colour || !opacity || !radius)))
        return fail(VT_ERR_INVALID_ARG, "vt_section_init: NULL pointer or negative capacity");
    const int64_t plane = (int64_t)W * H, total = plane * n_views;
    uint32_t *counts, *offs;
    int64_t nb;
    if ((st = compaction_scratch(total, &counts, &offs, &nb, stream))) return st;
    k_count_valid<<<(unsigned)nb, kInitBlock, 0, stream>>>(depth, total, counts);
    k_scan_counts<<<1, 1024, 0, stream>>>(counts, nb, offs, reinterpret_cast<long long *>(n_out));
    k_section_init<<<(unsigned)nb, kInitBlock, 0, stream>>>(depth, rgb, nullptr, 0.f, plane,
                                                            total, K.fx, (int)prec, offs, 0u, src,
                                                            colour, opacity, radius, cap);
    cudaFreeAsync(counts, stream);
    VT_CUDA(cudaGetLastError(), "vt_section_init launch");
    return VT_OK;
}

vt_status vt_section_complement(const float *depth, const float *rgb, const float *silhouette,
                                int32_t W, int32_t H, vt_intrinsics K, float sil_max,
                                int32_t view, vt_precision prec, uint32_t *src, void *colour,
                                void *opacity, void *radius, int64_t cap, int64_t *n_out,
                                vt_stream stream) {
    vt_status st = check_image(W, H, "vt_section_complement");
    if (st) return st;
    if ((st = check_intrinsics(K, "vt_section_complement"))) return st;
    if (view < 0 || (int64_t)(view + 1) * W * H > (int64_t)0xffffffffll)
        return fail(VT_ERR_INVALID_ARG, "vt_section_complement: view %d out of range", view);
    if (prec != VT_F32 && prec != VT_F16)
        return fail(VT_ERR_INVALID_ARG, "vt_section_complement: unknown precision");
    if (!std::isfinite(sil_max))
        return fail(VT_ERR_INVALID_ARG, "vt_section_complement: sil_max must be finite");
    if (!depth || !rgb || !silhouette || !n_out || cap < 0 ||
        (cap > 0 && (!src || !colour || !opacity || !radius)))
        return fail(VT_ERR_INVALID_ARG,
                    "vt_section_complement: NULL pointer or negative capacity");
    const int64_t plane = (int64_t)W * H;
    uint32_t *counts, *offs;
    int64_t nb;
    if ((st = compaction_scratch(plane, &counts, &offs, &nb, stream))) return st;
    k_count_yield<<<(unsigned)nb, kInitBlock, 0, stream>>>(depth, plane, silhouette, sil_max,
                                                           counts);
    k_scan_counts<<<1, 1024, 0, stream>>>(counts, nb, offs, reinterpret_cast<long long *>(n_out));
    k_section_init<<<(unsigned)nb, kInitBlock, 0, stream>>>(
        depth, rgb, silhouette, sil_max, plane, plane, K.fx, (int)prec, offs,
        (uint32_t)((int64_t)view * plane), src, colour, opacity, radius, cap);
    cudaFreeAsync(counts, stream);
    VT_CUDA(cudaGetLastError(), "vt_section_complement launch");
    return VT_OK;
}

// ---------------------------------------------------------------------------
// Batched work items.

size_t vt_batch_workspace_bytes(int64_t max_gaussians, int64_t max_pixels, int64_t max_tiles,
                                int64_t max_instances, int64_t max_views,
                                int64_t max_table_rows, int32_t list_cap) {
    if (max_gaussians < 0 || max_pixels < 0 || max_tiles < 0 || max_instances < 0 ||
        max_views < 0 || max_table_rows < 0 || list_cap < 0)
        return 0;
    return arena_bytes_for(max_gaussians, max_instances, max_pixels, max_tiles, max_views,
                           max_table_rows) +
           sizeof(BatchTable) + align_up(sizeof(float) * 4 * max_pixels) +
           align_up(sizeof(double) * 2 * (max_pixels / 256 + 1)) +
           align_up(sizeof(double) * 12 * kMaxItems) +
           sizeof(uint2) * (size_t)list_cap * (size_t)max_pixels;
}

vt_status vt_batch_reserve(vt_ctx *c, int64_t max_gaussians, int64_t max_pixels,
                           int64_t max_tiles, int64_t max_instances, int64_t max_views,
                           int64_t max_table_rows, vt_stream stream) {
    if (!c) return fail(VT_ERR_INVALID_ARG, "vt_batch_reserve: ctx is NULL");
    if (max_gaussians <= 0 || max_pixels <= 0 || max_tiles <= 0 || max_instances <= 0 ||
        max_views <= 0 || max_table_rows <= 0 || max_gaussians >= (int64_t)0xffffffffll ||
        max_instances >= (int64_t)0xffffffffll || max_tiles > (int64_t)0x7fffffff)
        return fail(VT_ERR_INVALID_ARG, "vt_batch_reserve: capacities out of range");
    // every item's Gaussian and pixel ranges start at a multiple of 256
    const int64_t g = max_gaussians + 256 * (int64_t)kMaxItems;
    const int64_t p = max_pixels + 256 * (int64_t)kMaxItems;
    c->stream = stream;
    vt_status st = ensure(c, g, max_instances, p, max_tiles, max_views, max_table_rows, stream);
    if (st) return st;
    if (!c->btab_host) {
        VT_CUDA(cudaMallocHost(&c->btab_host, sizeof(BatchTable)), "batch table staging");
        VT_CUDA(cudaEventCreateWithFlags(&c->bev_upload, cudaEventDisableTiming),
                "batch upload event");
    }
    if (!c->btab) {
        void *q = nullptr;
        VT_CUDA(cudaMallocAsync(&q, sizeof(BatchTable), stream), "batch table");
        c->btab = static_cast<BatchTable *>(q);
    }
    if (c->barena) cudaFreeAsync(c->barena, stream);
    c->barena = nullptr;
    const size_t gb = align_up(sizeof(float) * 4 * p), lb = align_up(sizeof(double) * 2 * (p / 256 + 1));
    const size_t pb = align_up(sizeof(double) * 12 * kMaxItems);
    void *q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, gb + lb + pb, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(VT_ERR_OOM, "vt_batch_reserve: %zu bytes: %s", gb + lb + pb,
                    cudaGetErrorString(e));
    }
    c->barena = q;
    c->bgrads = static_cast<float *>(q);
    c->bl1 = reinterpret_cast<double *>(static_cast<char *>(q) + gb);
    c->bpose = reinterpret_cast<double *>(static_cast<char *>(q) + gb + lb);
    // per-pixel lists for the tracking items' backward, within the budget
    c->batch_lists = false;
    if (c->list_cap > 0) {
        const size_t need = sizeof(uint2) * (size_t)c->list_cap * (size_t)p;
        if (c->arena_bytes + need <= c->budget) {
            if (need > c->plist_bytes) {
                if (c->plist) cudaFreeAsync(c->plist, stream);
                c->plist = nullptr;
                c->plist_bytes = 0;
                void *r = nullptr;
                if (cudaMallocAsync(&r, need, stream) == cudaSuccess) {
                    c->plist = static_cast<uint2 *>(r);
                    c->plist_bytes = need;
                } else {
                    cudaGetLastError();
                }
            }
            c->batch_lists = c->plist != nullptr;
        }
    }
    if (!sort_attr_set) {
        for (auto kern : {k_sort_tiles, k_sort_tiles_mid, k_sort_tiles_large, k_sort_tiles_long})
            VT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSortSmemBigBytes),
                    "sort smem attribute");
        sort_attr_set = true;
    }
    for (auto kern : {kb_sort_tiles, kb_sort_tiles_mid, kb_sort_tiles_large, kb_sort_tiles_long})
        VT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSortSmemBigBytes),
                "batch sort smem attribute");
    c->bcap_g = g;
    c->bcap_p = p;
    c->bcap_t = max_tiles;
    c->bcap_i = max_instances;
    c->bcap_v = max_views;
    c->bcap_tab = max_table_rows;
    c->batch = true;
    c->batch_set = false;
    c->has_render = false;
    return VT_OK;
}

vt_status vt_batch_set(vt_ctx *c, const vt_section *secs, int32_t n_secs,
                       const vt_batch_item *items, int32_t n_items, vt_l1_weights w) {
    if (!c) return fail(VT_ERR_INVALID_ARG, "vt_batch_set: ctx is NULL");
    if (!c->batch) return fail(VT_ERR_STATE, "vt_batch_set: call vt_batch_reserve first");
    if (n_items < 1 || n_items > kMaxItems || !items)
        return fail(VT_ERR_INVALID_ARG, "vt_batch_set: n_items must be in [1, %d]", kMaxItems);
    if (n_secs < 1 || n_secs > kMaxItems || !secs)
        return fail(VT_ERR_INVALID_ARG, "vt_batch_set: n_secs must be in [1, %d]", kMaxItems);
    if (!std::isfinite(w.w_rgb) || !std::isfinite(w.w_depth))
        return fail(VT_ERR_INVALID_ARG, "vt_batch_set: loss weights must be finite");
    vt_status st;
    for (int s = 0; s < n_secs; ++s) {
        const vt_section &S = secs[s];
        if (S.n < 0 || S.n >= (int64_t)0xffffffffll || S.n_views <= 0 || S.W <= 0 || S.H <= 0 ||
            (int64_t)S.n_views * S.W * S.H > (int64_t)0xffffffffll)
            return fail(VT_ERR_INVALID_ARG, "vt_batch_set: section %d sizes out of range", s);
        if (S.prec != VT_F32 && S.prec != VT_F16)
            return fail(VT_ERR_INVALID_ARG, "vt_batch_set: section %d precision unknown", s);
        if (S.scale)
            return fail(VT_ERR_INVALID_ARG, "vt_batch_set: section %d: batches take spheres only",
                        s);
        if ((st = check_intrinsics(S.K, "vt_batch_set section"))) return st;
        if (S.n > 0 && (!S.poses || !S.depth || !S.src || !S.colour || !S.opacity || !S.radius))
            return fail(VT_ERR_INVALID_ARG, "vt_batch_set: section %d has a NULL array", s);
    }
    // wait until the previous eager launch has uploaded the staged table
    if (c->bev_pending) {
        VT_CUDA(cudaEventSynchronize(c->bev_upload), "vt_batch_set: previous upload");
        c->bev_pending = false;
    }
    BatchTable &B = *c->btab_host;
    std::memset(&B, 0, sizeof(BatchTable));
    int64_t g = 0, p = 0, tab = 0;
    int64_t t = 0, v = 0;
    for (int i = 0; i < n_items; ++i) {
        const vt_batch_item &It = items[i];
        if (It.section < 0 || It.section >= n_secs)
            return fail(VT_ERR_INVALID_ARG, "vt_batch_set: item %d names section %d", i,
                        It.section);
        if ((st = check_image(It.W, It.H, "vt_batch_set item"))) return st;
        if ((st = check_intrinsics(It.K, "vt_batch_set item"))) return st;
        if (!It.pose12 || !It.image || (It.track && (!It.obs || !It.result)))
            return fail(VT_ERR_INVALID_ARG, "vt_batch_set: item %d has a NULL pointer", i);
        const vt_section &S = secs[It.section];
        BatchItem &I = B.it[i];
        I.cam.fx = It.K.fx;
        I.cam.fy = It.K.fy;
        I.cam.cx = It.K.cx;
        I.cam.cy = It.K.cy;
        I.cam.W = It.W;
        I.cam.H = It.H;
        I.cam.tiles_x = (It.W + kTile - 1) / kTile;
        I.cam.tiles_y = (It.H + kTile - 1) / kTile;
        I.pose = It.pose12;
        I.image = It.image;
        I.obs = It.obs;
        I.result = It.result;
        I.gbase = g;
        I.n = S.n;
        I.pbase = p;
        I.tab_base = tab;
        I.tbase = (int32_t)t;
        I.vbase = (int32_t)v;
        I.sec = It.section;
        I.track = It.track ? 1 : 0;
        g += (S.n + 255) / 256 * 256;
        p += ((int64_t)It.W * It.H + 255) / 256 * 256;
        t += (int64_t)I.cam.tiles_x * I.cam.tiles_y;
        v += S.n_views;
        tab += (int64_t)S.n_views * (S.W + S.H);
    }
    if (g > c->bcap_g || p > c->bcap_p || t > c->bcap_t || v > c->bcap_v || tab > c->bcap_tab)
        return fail(VT_ERR_CAPACITY,
                    "vt_batch_set: batch needs %lld Gaussian slots, %lld pixels, %lld tiles, "
                    "%lld views, %lld table rows; reserved %lld, %lld, %lld, %lld, %lld",
                    (long long)g, (long long)p, (long long)t, (long long)v, (long long)tab,
                    (long long)c->bcap_g, (long long)c->bcap_p, (long long)c->bcap_t,
                    (long long)c->bcap_v, (long long)c->bcap_tab);
    for (int s = 0; s < n_secs; ++s) {
        const vt_section &S = secs[s];
        SecDesc &D = B.sec[s];
        D.poses = S.poses;
        D.depth = S.depth;
        D.src = S.src;
        D.colour = S.colour;
        D.opacity = S.opacity;
        D.radius = S.radius;
        D.n = S.n;
        D.n_views = S.n_views;
        D.W = S.W;
        D.H = S.H;
        D.prec = (int32_t)S.prec;
        D.fx = S.K.fx;
        D.fy = S.K.fy;
        D.cx = S.K.cx;
        D.cy = S.K.cy;
    }
    B.n_items = n_items;
    B.n_secs = n_secs;
    B.n_tiles = (int32_t)t;
    B.n_views = (int32_t)v;
    B.n_gauss = g;
    B.n_pix = p;
    B.w_rgb = w.w_rgb;
    B.w_depth = w.w_depth;
    B.sil_min = w.sil_min;
    B.rgb_needs_depth = w.rgb_needs_depth ? 1 : 0;
    c->batch_set = true;
    return VT_OK;
}

vt_status vt_batch_launch(vt_ctx *c, vt_stream stream, vt_event obs_ready) {
    if (!c) return fail(VT_ERR_INVALID_ARG, "vt_batch_launch: ctx is NULL");
    if (!c->batch || !c->batch_set)
        return fail(VT_ERR_STATE, "vt_batch_launch: no batch staged (vt_batch_set)");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    VT_CUDA(cudaStreamIsCapturing(stream, &cs), "capture query");
    c->stream = stream;
    c->has_render = false;   // the batch overwrites a single render's state
    const int nsm = c->n_sm;
    BatchTable *B = c->btab;
    // Grids: outside a capture one block per unit of work of the staged
    // batch (the stages then yield SMs block by block, so stream priorities
    // between concurrent batches take effect); inside a capture persistent
    // grids sized by the SM count, which serve any later batch the table
    // describes.
    const BatchTable &H = *c->btab_host;
    const bool exact = cs == cudaStreamCaptureStatusNone;
    auto grid = [&](int64_t units, int per_sm) -> unsigned {
        const int64_t g = exact ? units : (int64_t)per_sm * nsm;
        return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 0x7fffffff));
    };
    const int64_t g_chunks = H.n_gauss / 256, p_chunks = H.n_pix / 256;
    VT_CUDA(cudaMemcpyAsync(B, c->btab_host, sizeof(BatchTable), cudaMemcpyHostToDevice, stream),
            "batch table upload");
    if (cs == cudaStreamCaptureStatusNone) {
        VT_CUDA(cudaEventRecord(c->bev_upload, stream), "batch upload event");
        c->bev_pending = true;
    }
    {
        LaunchScope ls(c, KB_SETUP, stream);
        kb_setup<<<grid(std::max<int64_t>(H.n_views, (H.n_tiles + 256) / 256), 2), 256, 0, stream>>>(B, c->views, c->tab, c->bpose, c->tile_count);
    }
    {
        LaunchScope ls(c, KB_PREPROCESS, stream);
        kb_preprocess<<<grid(g_chunks, 8), 256, 0, stream>>>(B, c->views, c->tab, c->geo, c->app, c->info,
                                                   c->tile_count);
    }
    {
        LaunchScope ls(c, KB_SCAN, stream);
        kb_scan_tiles<<<1, 1024, 0, stream>>>(B, c->tile_count, c->tile_off, c->tile_cursor,
                                              c->status, (unsigned long long)c->bcap_i,
                                              c->long_tiles);
    }
    {
        LaunchScope ls(c, KB_EMIT, stream);
        kb_emit<<<grid(g_chunks, 8), 256, 0, stream>>>(B, c->info, c->tile_cursor, c->bucket, c->bmask_u,
                                             c->status);
    }
    VT_CUDA(cudaEventRecord(c->ev_fork, stream), "sort fork");
    VT_CUDA(cudaStreamWaitEvent(c->aux, c->ev_fork, 0), "sort fork");
    {
        LaunchScope ls(c, KB_SORT_LONG, c->aux);
        kb_sort_tiles_long<<<grid(std::min<int64_t>(H.n_tiles, nsm), 1), 512, kSortSmemBigBytes, c->aux>>>(
            B, c->tile_off, c->bucket, c->alt, c->bmask_u, c->sorted, c->bmask, c->geo, c->status,
            kSortSmemBig, kSortSmemN, kSortSmemBig, c->long_tiles);
    }
    {
        LaunchScope ls(c, KB_SORT_XL, c->aux);
        kb_sort_tiles_xl<<<grid(std::min<int64_t>(H.n_tiles, 2 * nsm), 2), 512, kSortHistBytes, c->aux>>>(
            B, c->tile_off, c->bucket, c->alt, c->bmask_u, c->sorted, c->bmask, c->geo, c->status,
            kSortSmemBig, kSortSmemBig, 0x7fffffff, c->long_tiles);
    }
    VT_CUDA(cudaEventRecord(c->ev_join, c->aux), "sort join");
    {
        LaunchScope ls(c, KB_SORT, stream);
        kb_sort_tiles<<<grid(H.n_tiles, 4), 512, sort_smem_bytes(kSortClassS), stream>>>(
            B, c->tile_off, c->bucket, c->alt, c->bmask_u, c->sorted, c->bmask, c->geo, c->status,
            kSortClassS, 0, kSortClassS, c->long_tiles);
    }
    {
        LaunchScope ls(c, KB_SORT_M, stream);
        kb_sort_tiles_mid<<<grid(H.n_tiles, 3), 512, sort_smem_bytes(kSortClassM), stream>>>(
            B, c->tile_off, c->bucket, c->alt, c->bmask_u, c->sorted, c->bmask, c->geo, c->status,
            kSortClassM, kSortClassS, kSortClassM, c->long_tiles);
    }
    {
        LaunchScope ls(c, KB_SORT_L, stream);
        kb_sort_tiles_large<<<grid(H.n_tiles, 2), 512, kSortSmemBytes, stream>>>(
            B, c->tile_off, c->bucket, c->alt, c->bmask_u, c->sorted, c->bmask, c->geo, c->status,
            kSortSmemN, kSortClassM, kSortSmemN, c->long_tiles);
    }
    VT_CUDA(cudaStreamWaitEvent(stream, c->ev_join, 0), "sort join");
    const int cap = c->batch_lists ? c->list_cap : 0;
    {
        LaunchScope ls(c, KB_FWD, stream);
        kb_composite_fwd<<<grid(H.n_tiles, 6), kBlockPix, 0, stream>>>(
            B, &B->ctr[0], c->tile_off, c->sorted, c->bmask, c->geo, c->app, c->pix_last,
            c->pix_nadd, c->pix_T, c->batch_lists ? c->plist : nullptr, cap, c->blk_ovf,
            c->status);
    }
    if (obs_ready)   // the observations arrive while the render stages run
        VT_CUDA(cudaStreamWaitEvent(stream, reinterpret_cast<cudaEvent_t>(obs_ready), 0),
                "vt_batch_launch: observation event");
    {
        LaunchScope ls(c, KB_L1, stream);
        kb_masked_l1<<<grid(p_chunks, 8), 256, 0, stream>>>(B, c->bgrads, c->bl1);
    }
    if (c->batch_lists) {
        LaunchScope ls(c, KB_BWD_LIST, stream);
        kb_composite_bwd_list_pose<<<grid(H.n_tiles, 3), kBlockPix, 0, stream>>>(
            B, &B->ctr[1], c->geo, c->app, c->pix_nadd, c->pix_T, c->plist, cap, c->blk_ovf,
            c->bgrads, c->pose_partials, c->status);
    }
    {
        LaunchScope ls(c, KB_BWD, stream);
        kb_composite_bwd_pose<<<grid(H.n_tiles, 2), kBlockPix, 0, stream>>>(
            B, c->tile_off, c->sorted, c->geo, c->app, c->pix_last, c->pix_T, c->blk_ovf,
            c->bgrads, c->pose_partials, c->status);
    }
    {
        LaunchScope ls(c, KB_FINALIZE, stream);
        kb_finalize<<<exact ? (unsigned)H.n_items : (unsigned)kMaxItems, 384, 0, stream>>>(B, c->bl1, c->pose_partials, c->bpose);
    }
    VT_CUDA(cudaGetLastError(), "vt_batch_launch");
    return VT_OK;
}

int64_t vt_ctx_debug_copy(vt_ctx *c, int32_t what, void *dst, int64_t capacity,
                          vt_stream stream) {
    if (!c || !dst || capacity < 0) return -VT_ERR_INVALID_ARG;
    if (!c->has_render) return -VT_ERR_STATE;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return -VT_ERR_CUDA;
    Status h;
    if (cudaMemcpy(&h, c->status, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
        return -VT_ERR_CUDA;
    const int64_t P = (int64_t)c->cam.W * c->cam.H;
    const void *src = nullptr;
    int64_t bytes = 0;
    std::vector<uint4> tmp;
    switch (what) {
        case 0: {
            const int64_t n = c->table.n_total;
            bytes = n * 4;
            if (bytes > capacity) return -VT_ERR_INVALID_ARG;
            tmp.resize(n);
            if (n && cudaMemcpy(tmp.data(), c->info, n * sizeof(uint4), cudaMemcpyDeviceToHost) !=
                         cudaSuccess)
                return -VT_ERR_CUDA;
            uint32_t *o = static_cast<uint32_t *>(dst);
            for (int64_t i = 0; i < n; ++i) o[i] = tmp[i].z;
            return bytes;
        }
        case 1: src = c->tile_off; bytes = 4 * (int64_t)(c->n_tiles + 1); break;
        case 2: src = c->sorted; bytes = 4 * std::min<int64_t>(h.n_instances, c->cap_i); break;
        case 3: src = c->pix_last; bytes = 4 * P; break;
        case 4: src = c->pix_nadd; bytes = 4 * P; break;
        case 5: src = c->pix_T; bytes = 4 * P; break;
        default: return -VT_ERR_INVALID_ARG;
    }
    if (bytes > capacity) return -VT_ERR_INVALID_ARG;
    if (bytes && cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        return -VT_ERR_CUDA;
    return bytes;
}

vt_status vt_ctx_debug_pixel_lists(vt_ctx *c, int32_t x0, int32_t y0, int32_t w, int32_t h,
                                   int32_t cap, uint32_t *ids, float *T_front, uint32_t *counts,
                                   int32_t *kept, vt_stream stream) {
    if (!c || !counts || cap < 0 || (cap > 0 && !ids))
        return fail(VT_ERR_INVALID_ARG, "vt_ctx_debug_pixel_lists: bad arguments");
    if (!c->has_render) return fail(VT_ERR_STATE, "vt_ctx_debug_pixel_lists: no render");
    if (x0 < 0 || y0 < 0 || w < 0 || h < 0 || x0 + w > c->cam.W || y0 + h > c->cam.H)
        return fail(VT_ERR_INVALID_ARG, "vt_ctx_debug_pixel_lists: rectangle outside the image");
    if (!c->used_lists)
        return fail(VT_ERR_STATE, "vt_ctx_debug_pixel_lists: the last render kept no lists");
    VT_CUDA(cudaStreamSynchronize(stream), "vt_ctx_debug_pixel_lists");
    const int64_t lc = c->list_cap;
    if (kept) *kept = (int32_t)lc;
    std::vector<uint2> row((size_t)w * (size_t)lc);
    for (int32_t y = 0; y < h; ++y) {
        const int64_t p0 = (int64_t)(y0 + y) * c->cam.W + x0;
        VT_CUDA(cudaMemcpy(counts + (size_t)y * w, c->pix_nadd + p0, sizeof(uint32_t) * w,
                           cudaMemcpyDeviceToHost),
                "pixel list counts");
        if (w == 0 || lc == 0) continue;
        VT_CUDA(cudaMemcpy(row.data(), c->plist + p0 * lc, sizeof(uint2) * row.size(),
                           cudaMemcpyDeviceToHost),
                "pixel lists");
        for (int32_t x = 0; x < w; ++x) {
            const int64_t n = std::min<int64_t>({(int64_t)counts[(size_t)y * w + x], lc, cap});
            for (int64_t j = 0; j < n; ++j) {
                const size_t o = ((size_t)y * w + x) * (size_t)cap + (size_t)j;
                const uint2 e = row[(size_t)x * lc + j];
                ids[o] = e.x;
                if (T_front) std::memcpy(&T_front[o], &e.y, sizeof(float));
            }
        }
    }
    return VT_OK;
}

}  // extern "C"
