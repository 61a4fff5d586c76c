// dwt2_selftest.cu -- exercises the bounded device waits every kernel of the library relies on:
// an mbarrier phase that no thread completes (the stage ring's wait) and a completion counter
// that no CTA increments (the persistent kernels' dependency wait).  Each wait gives up after its
// time limit, records DWT2_ETIMEOUT in the workspace status word and returns; nothing faults or
// traps, and the context stays usable.  The paper has no counterpart: this is failure detection
// for the library itself.
#include "../../include/dwt2.h"
#include "dwt2_internal.h"

#define DWT2_EXPORT extern "C" __attribute__((visibility("default")))

namespace dwt2 {
void set_last_error(const char* msg);

namespace {

constexpr int kCounterOffset = 128;  // bytes into the workspace header (zeroed by its init)

__global__ void k_wait_selftest(int which, int* status, const int* counter) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (which == 0) {
        // phase 0 of a fresh barrier with one expected arrival and none made
        mbar_wait(&bar, 0, &abort_flag, status);
    } else if (threadIdx.x == 0) {
        // a counter the host zeroed and nothing increments
        wait_count(counter, 1, &abort_flag, status);
    }
}

}  // namespace
}  // namespace dwt2

using namespace dwt2;

DWT2_EXPORT int dwt2_selftest_wait_timeout(int which, void* workspace, size_t ws_bytes,
                                           void* stream) {
    if (which < 0 || which > 1 || !workspace || ws_bytes < 256 ||
        reinterpret_cast<uintptr_t>(workspace) % 16 != 0)
        return DWT2_EINVAL;
    char* ws = static_cast<char*>(workspace);
    k_wait_selftest<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(
        which, reinterpret_cast<int*>(ws), reinterpret_cast<const int*>(ws + kCounterOffset));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return DWT2_ECUDA;
    }
    return DWT2_OK;
}
