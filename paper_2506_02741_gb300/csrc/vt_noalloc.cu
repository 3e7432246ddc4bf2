// Allocation-free back-projection.
//
// vt_backproject needs two small scratch arrays (per-block counts and their
// prefix sums) and obtains them with a stream-ordered cudaMallocAsync.  Some
// callers cannot have the library allocate: code that runs while a CUDA
// graph is being captured without a memory pool, programs that must not
// touch the CUDA allocator after start-up (real-time loops, hosts that hand
// every byte of device memory to their own pool), or embedders whose
// allocator policy forbids foreign allocations.  vt_backproject_noalloc
// computes the same result with its scratch in a fixed array of device memory
// that is part of the loaded library.
#include <cuda_runtime.h>

#include <mutex>

#include "vt_common.cuh"

vt_status vt_internal_fail(vt_status s, const char *msg);
vt_status vt_internal_check_image(int32_t W, int32_t H, const char *who);

namespace {

// Largest depth map the allocation-free path accepts: 2^24 pixels (e.g.
// 4096 x 4096), i.e. 65536 blocks of 256 pixels.  The scratch holds one count
// and one offset per block: 512 KiB, held by every GPU that loads the library
// until the process exits.
constexpr int64_t kNoAllocMaxPixels = int64_t(1) << 24;
constexpr int64_t kNoAllocMaxBlocks = kNoAllocMaxPixels / vt::kInitBlock;

// Host code may not use this name as a device address (on the host it is a
// stand-in object); the device address is looked up per device below.
static __device__ __align__(256) uint32_t g_backproject_scratch[2 * kNoAllocMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  It is looked
// up (cudaGetSymbolAddress, with the device current) on every call made while
// `stream` is not being captured, so that a device reset, after which the
// module and its array may be loaded at another address, is followed; calls
// made during a stream capture use the address cached by the last such
// lookup on this device and fail if there was none.
vt_status scratch_on_current_device(cudaStream_t stream, uint32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return vt_internal_fail(VT_ERR_CUDA, "vt_backproject_noalloc: cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices)
        return vt_internal_fail(VT_ERR_INVALID_ARG, "vt_backproject_noalloc: device index too large");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return vt_internal_fail(VT_ERR_CUDA, "vt_backproject_noalloc: cudaStreamIsCapturing failed");
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_backproject_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return vt_internal_fail(VT_ERR_CUDA,
                                    "vt_backproject_noalloc: cudaGetSymbolAddress of the scratch "
                                    "array failed");
        }
        g_scratch_ptr[dev] = static_cast<uint32_t *>(p);
    } else if (!g_scratch_ptr[dev]) {
        return vt_internal_fail(VT_ERR_STATE,
                                "vt_backproject_noalloc: the first call on a device must come "
                                "before any stream capture");
    }
    *out = g_scratch_ptr[dev];
    return VT_OK;
}

}  // namespace

extern "C" vt_status vt_backproject_noalloc(const float *depth, int32_t W, int32_t H,
                                            vt_intrinsics K, const double *pose12,
                                            float *centres, uint32_t *pix, int64_t cap,
                                            int64_t *n_out, vt_stream stream) {
    vt_status st = vt_internal_check_image(W, H, "vt_backproject_noalloc");
    if (st != VT_OK) return st;
    const int64_t total = (int64_t)W * H;
    if (total > kNoAllocMaxPixels)
        return vt_internal_fail(VT_ERR_INVALID_ARG,
                                "vt_backproject_noalloc: depth map larger than the 2^24-pixel "
                                "limit of the fixed scratch; use vt_backproject");
    if (!(K.fx > 0.f) || !(K.fy > 0.f) || !isfinite(K.fx) || !isfinite(K.fy) ||
        !isfinite(K.cx) || !isfinite(K.cy))
        return vt_internal_fail(VT_ERR_INVALID_ARG,
                                "vt_backproject_noalloc: intrinsics must be finite with fx, fy > 0");
    if (!depth || !pose12 || !n_out || cap < 0 || (cap > 0 && (!centres || !pix)))
        return vt_internal_fail(VT_ERR_INVALID_ARG,
                                "vt_backproject_noalloc: NULL pointer or negative capacity");
    uint32_t *scratch = nullptr;
    st = scratch_on_current_device(stream, &scratch);
    if (st != VT_OK) return st;
    const int64_t nb = (total + vt::kInitBlock - 1) / vt::kInitBlock;
    uint32_t *counts = scratch, *offs = scratch + kNoAllocMaxBlocks;
    // every count and offset used below is written before it is read, so the
    // array needs no clearing between calls
    vt::k_count_valid<<<(unsigned)nb, vt::kInitBlock, 0, stream>>>(depth, total, counts);
    vt::k_scan_counts<<<1, 1024, 0, stream>>>(counts, nb, offs, reinterpret_cast<long long *>(n_out));
    vt::k_backproject<<<(unsigned)nb, vt::kInitBlock, 0, stream>>>(depth, W, H, K, pose12, offs,
                                                                   centres, pix, cap);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return vt_internal_fail(VT_ERR_CUDA, "vt_backproject_noalloc: kernel launch failed");
    return VT_OK;
}
