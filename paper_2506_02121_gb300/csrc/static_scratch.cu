// Allocation-free distance map: cc_distance_map_static.
//
// Some callers cannot allocate device memory when they need a distance map: a plugin
// running inside a host application whose device memory is owned by the host's own
// allocator, a process whose device-memory budget is already fully reserved, or a
// latency-critical loop that must never enter the allocator.  They cannot supply the
// caller-owned scratch that cc_distance_map requires.  This entry point runs the same
// kernels with their scratch in a fixed array of this library's device memory instead.
//
// The array is a file-scope static __device__ buffer of CC_DISTANCE_MAP_STATIC_MAX_PIXELS
// * 8 + 512 bytes (8 MiB + 512 B).  Every GPU that loads the library holds it until the
// process exits.  Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it.  That first call should therefore come before any stream
// capture on that device.
//
// All calls share the one array and it keeps the last call's contents.  The kernels write
// every scratch entry before reading it, so nothing needs clearing between calls.  Calls
// whose work overlaps on the GPU (other streams, other threads) race on the array: order
// them on one stream or serialise them.
#include <mutex>

#include "cc_internal.h"

static __device__ __align__(256) unsigned char
    cc_static_distance_scratch[(size_t)CC_DISTANCE_MAP_STATIC_MAX_PIXELS * 8 + 512];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch[kMaxDevices] = {};

// Device address of the static scratch on the current device (looked up once per device).
int static_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ccg::api_error(CC_ECUDA, "cc_distance_map_static: cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return ccg::api_error(CC_EINVAL, "cc_distance_map_static: device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, cc_static_distance_scratch);
        if (e != cudaSuccess || !p)
            return ccg::api_error(CC_ECUDA, "cc_distance_map_static: cudaGetSymbolAddress of the static scratch failed");
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return CC_OK;
}

}  // namespace

extern "C" int cc_distance_map_static(const int32_t* ncc, int32_t W, int32_t H, double pixel, double* d_out,
                                      cc_stream_t stream) {
    if (!ncc || !d_out) return ccg::api_error(CC_EINVAL, "cc_distance_map_static: NULL buffer");
    if (W < 1 || H < 1) return ccg::api_error(CC_EINVAL, "cc_distance_map_static: W, H must be >= 1");
    if ((int64_t)W * H > (int64_t)CC_DISTANCE_MAP_STATIC_MAX_PIXELS)
        return ccg::api_error(CC_EINVAL,
                              "cc_distance_map_static: W * H exceeds the static scratch limit of "
                              "CC_DISTANCE_MAP_STATIC_MAX_PIXELS (1048576) pixels; use cc_distance_map");
    if (!(pixel > 0) || !(pixel < 1e308)) return ccg::api_error(CC_EINVAL, "cc_distance_map_static: pixel must be finite and > 0");
    void* ws = nullptr;
    if (int r = static_scratch(&ws)) return r;
    cudaError_t e = ccg::launch_distance_map(ncc, W, H, pixel, d_out, ws, (cudaStream_t)stream);
    if (e != cudaSuccess) return ccg::api_error(CC_ECUDA, cudaGetErrorString(e));
    return CC_OK;
}
