// dc_decolorize_tonemap_global_noalloc: the global tone-mapping call for callers
// that cannot allocate device memory themselves.
//
// Some callers have no way to call cudaMalloc or to own a device buffer: code
// running inside a framework whose allocator is not reachable, plugins handed only
// input and output pointers, or programs that must not allocate after start-up.
// This entry point needs no workspace argument: its scratch is a fixed array in
// the library's own device memory (every GPU that loads the library holds it until
// the process exits).  The caller still passes the input and output images.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "../../include/decolor.h"
#include "dc_internal.h"

namespace {

// Scratch of the global pass: a 256-byte header plus about 1.1 KiB of counters per
// image, so 64 KiB covers a batch of a few dozen images.
constexpr size_t kScratchBytes = DC_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// In host code this name is only a stand-in for the device array; its device
// address comes from cudaGetSymbolAddress below.
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::atomic<void*> g_scratch_addr[kMaxDevices];

// Device address of the scratch array on the current device (looked up once per
// device, with that device current).
int scratch_address(void** out, void* stream)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DC_ERR_CUDA;
    void* p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (p == nullptr) {
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return DC_ERR_CUDA;
        // zeroed once and registered: the calls keep their control block clean
        if (dc_workspace_prepare(p, kScratchBytes, stream) != DC_OK) return DC_ERR_CUDA;
        g_scratch_addr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return DC_OK;
}

}  // namespace

extern "C" DC_API int dc_decolorize_tonemap_global_noalloc(const dc_image_in* in, const dc_image_out* out,
                                                           int32_t n, const dc_decolor_params* params,
                                                           const dc_global_params* gparams,
                                                           dc_global_stats* stats, void* stream)
{
    const size_t need = dc::workspace_min_bytes(DC_OP_GLOBAL, in, n, nullptr);  // no optional plane
    if (need == 0) return DC_ERR_INVALID_ARG;
    if (need > kScratchBytes) return DC_ERR_WORKSPACE;  // batch too large for the fixed scratch
    void* ws = nullptr;
    const int rc = scratch_address(&ws, stream);
    if (rc != DC_OK) return rc;
    // the call clears the counters it uses before its first pass
    return dc_decolorize_tonemap_global(in, out, n, params, gparams, stats, ws, kScratchBytes, stream);
}
