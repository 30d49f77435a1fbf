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
// call in each CUDA context looks the address up with cudaGetSymbolAddress (with that
// context's device current) and caches it under the context's ID.  That first call should
// therefore come before any stream capture on that device.  The address is tied to the
// context: after a reset of the device's primary context (cudaDeviceReset) the next call
// runs in a new context and looks the address up again.
//
// All calls share the one array and it keeps the last call's contents.  The kernels write
// every scratch entry before reading it, so nothing needs clearing between calls.  Calls
// whose work overlaps on the GPU (other streams, other threads) race on the array: order
// them on one stream or serialise them.
#include <cmath>

#include <cuda.h>

#include "cc_internal.h"
#include "symbol_cache.h"

static __device__ __align__(256) unsigned char
    cc_static_distance_scratch[(size_t)CC_DISTANCE_MAP_STATIC_MAX_PIXELS * 8 + 512];

namespace {

ccg::SymbolAddressCache<64> g_cache;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// ID of the current CUDA context (the runtime makes the device's primary context current
// first).  The driver calls come through the runtime's entry-point table, so the library
// does not link the driver library directly.
int current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)p;
    });
    if (!get_current || !get_id)
        return ccg::api_error(CC_ECUDA, "cc_distance_map_static: the driver's context queries are unavailable");
    // cudaFree(0) makes the runtime bind (or create) the current device's primary context
    cudaError_t e = cudaFree(nullptr);
    if (e != cudaSuccess) return ccg::api_error(CC_ECUDA, "cc_distance_map_static: no CUDA context");
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, id) != CUDA_SUCCESS)
        return ccg::api_error(CC_ECUDA, "cc_distance_map_static: cannot identify the current CUDA context");
    return CC_OK;
}

// Device address of the static scratch in the current context (looked up once per context).
int static_scratch(void** out) {
    unsigned long long ctx = 0;
    if (int r = current_context_id(&ctx)) return r;
    return g_cache.get(
        ctx,
        [](void** addr) -> int {
            cudaError_t e = cudaGetSymbolAddress(addr, cc_static_distance_scratch);
            if (e != cudaSuccess || !*addr)
                return ccg::api_error(CC_ECUDA, "cc_distance_map_static: cudaGetSymbolAddress of the static scratch failed");
            return CC_OK;
        },
        out);
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
    if (!(pixel > 0) || !std::isfinite(pixel))
        return ccg::api_error(CC_EINVAL, "cc_distance_map_static: pixel must be finite and > 0");
    // the scratch address belongs to the current device: the stream must run there too
    int dev = 0, sdev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaStreamGetDevice((cudaStream_t)stream, &sdev) != cudaSuccess)
        return ccg::api_error(CC_ECUDA, "cc_distance_map_static: cannot query the device of the stream");
    if (sdev != dev)
        return ccg::api_error(CC_EINVAL, "cc_distance_map_static: the stream belongs to another device than the "
                                         "current one; make the stream's device current");
    void* ws = nullptr;
    if (int r = static_scratch(&ws)) return r;
    cudaError_t e = ccg::launch_distance_map(ncc, W, H, pixel, d_out, ws, (cudaStream_t)stream);
    if (e != cudaSuccess) return ccg::api_error(CC_ECUDA, cudaGetErrorString(e));
    return CC_OK;
}
