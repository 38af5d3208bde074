// noalloc.cu -- gbssim_ssim_map_static: SSIM map + MSSIM for callers that
// cannot allocate device memory.
//
// Some callers have no way to provide the workspace gbssim_ssim_map asks for:
// a per-frame filter running inside a host application that owns the GPU
// allocator and hands plugins only their input and output buffers, or a
// latency-critical pipeline that forbids cudaMalloc after start-up (the call
// can block and synchronise the device).  This entry point needs no
// workspace: its scratch (the per-tile partial sums that the deterministic
// pooling adds up) lives in the file-scope device array below, which every
// GPU that loads the library holds until the process exits.
//
// Set-up: the array's name is only a host-side stand-in in host code, so the
// first call on each device (with that device current) asks the runtime for
// the array's device address (cudaGetSymbolAddress) and caches it.  Make that
// first call on a device before any stream capture.  A lookup that fails (for
// example one made while a capture is open) is not cached: the next call
// tries again.
//
// Sharing: every call uses the same array and it keeps the previous call's
// contents.  Nothing needs clearing: each call writes every slot it later
// reads.  Calls whose GPU work overlaps (other streams, other threads) race
// on the array; serialise them.
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace {

// 65536 (sum Q, sum cs) slots = 1 MiB per device.
constexpr size_t kScratchSlots = size_t(GBSSIM_STATIC_SCRATCH_BYTES) / sizeof(double2);
static __device__ __align__(256) double2 g_scratch[kScratchSlots];

constexpr int kMaxDevices = 64;
struct DeviceScratch {
    std::mutex m;
    std::atomic<void *> ptr{nullptr};
};
DeviceScratch g_devices[kMaxDevices];

int scratch_address(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GBSSIM_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return GBSSIM_ERR_UNSUPPORTED;
    DeviceScratch &d = g_devices[dev];
    void *q = d.ptr.load(std::memory_order_acquire);
    if (!q) {
        std::lock_guard<std::mutex> lock(d.m);
        q = d.ptr.load(std::memory_order_relaxed);
        if (!q) {
            if (cudaGetSymbolAddress(&q, g_scratch) != cudaSuccess || !q) {
                cudaGetLastError();  // leave no error behind for later launch checks
                return GBSSIM_ERR_CUDA;
            }
            d.ptr.store(q, std::memory_order_release);
        }
    }
    *out = q;
    return GBSSIM_OK;
}

}  // namespace

extern "C" int gbssim_ssim_map_static(const gbssim_plane *x, const gbssim_plane *y,
                                      const gbssim_params *p, float *map_out, int64_t map_ld,
                                      int64_t map_image_stride, double *mean_out, void *stream) {
    // Argument errors first, exactly as gbssim_ssim_map reports them: without
    // a workspace it checks every other argument and then stops with
    // GBSSIM_ERR_WORKSPACE before enqueueing anything.
    int rc = gbssim_ssim_map(x, y, p, map_out, map_ld, map_image_stride, mean_out, nullptr, 0, stream);
    if (rc != GBSSIM_ERR_WORKSPACE) return rc;
    size_t need = 0;
    rc = gbssim_workspace_size(x, p, GBSSIM_OP_SSIM, &need);
    if (rc != GBSSIM_OK) return rc;
    if (need > sizeof(g_scratch)) return GBSSIM_ERR_TOO_LARGE;
    void *ws = nullptr;
    rc = scratch_address(&ws);
    if (rc != GBSSIM_OK) return rc;
    return gbssim_ssim_map(x, y, p, map_out, map_ld, map_image_stride, mean_out, ws, sizeof(g_scratch),
                           stream);
}
