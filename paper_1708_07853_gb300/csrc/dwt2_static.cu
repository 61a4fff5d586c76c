// dwt2_static.cu -- dwt2_forward_static: the forward transform for callers that cannot allocate
// device memory.
//
// Some callers have no way to allocate: code running where cudaMalloc is forbidden or unsafe
// (inside a real-time loop with a no-allocation rule, a plugin whose host owns all device memory
// and hands over only the input and output buffers, or code that must not touch the allocator
// because it would synchronise the device).  The regular entry point asks them for a workspace
// (the intermediate LL planes of the level recursion and a status word).  This entry point
// instead uses a fixed-size scratch array that lives in the library itself, so the caller passes
// only the image and the coefficient buffer.
//
// The scratch array is a file-scope __device__ variable: every GPU on which this code is loaded
// holds its kStaticScratchBytes until the process exits.  All calls share it and it keeps the
// contents of the previous call; calls whose execution overlaps on the GPU (different streams,
// or different host threads) race on it and must be ordered by the caller.
#include <cstdio>

#include "../../include/dwt2.h"
#include "dwt2_internal.h"

#define DWT2_EXPORT extern "C" __attribute__((visibility("default")))

namespace dwt2 {
void set_last_error(const char* msg);
}

namespace {

constexpr size_t kStaticScratchBytes = size_t(24) << 20;  // DWT2_STATIC_SCRATCH_BYTES

static_assert(kStaticScratchBytes == DWT2_STATIC_SCRATCH_BYTES, "header and library disagree");

// The scratch itself.  In host code `g_scratch` is only a stand-in symbol, not a device address;
// the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

// Device address of g_scratch in the current device's current context.  Looked up on every call
// (a host-side lookup): a cached address would go stale after cudaDeviceReset, or belong to
// another context when the caller switches contexts, and the kernels would then write through
// it.  The first lookup in a context loads the library's device code there.
int scratch_address(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
        dwt2::set_last_error(e != cudaSuccess ? cudaGetErrorString(e)
                                              : "cudaGetSymbolAddress returned null");
        return DWT2_ECUDA;
    }
    *out = p;
    return DWT2_OK;
}

}  // namespace

DWT2_EXPORT int dwt2_forward_static(const void* img, int64_t img_pitch_bytes, int H, int W,
                                    int img_dtype, void* coeffs, int wavelet, int levels,
                                    int band_dtype, void* stream) {
    const size_t need = dwt2_workspace_bytes(H, W, levels, wavelet, band_dtype);
    if (need == 0) return DWT2_EINVAL;  // invalid size / level count / types
    if (need > kStaticScratchBytes) {
        char msg[192];
        std::snprintf(msg, sizeof(msg),
                      "dwt2_forward_static: %dx%d with %d levels needs %zu bytes of scratch; the "
                      "built-in scratch holds %zu bytes (use dwt2_forward with a workspace)",
                      H, W, levels, need, kStaticScratchBytes);
        dwt2::set_last_error(msg);
        return DWT2_ENOMEM;
    }
    void* ws = nullptr;
    const int rc = scratch_address(&ws);
    if (rc) return rc;
    // Every argument is checked before anything is queued on the stream; then the status word is
    // cleared (the LL planes are fully written before they are read).
    return dwt2::forward_into_scratch(img, img_pitch_bytes, H, W, img_dtype, coeffs, ws,
                                      kStaticScratchBytes, wavelet, levels, band_dtype,
                                      static_cast<cudaStream_t>(stream));
}
