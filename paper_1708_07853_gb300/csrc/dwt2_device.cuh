// dwt2_device.cuh -- device primitives: mbarrier / TMA (cp.async.bulk.tensor) wrappers with
// time-bounded waits, warp neighbour exchange, element conversions and vector memory access.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dwt2 {

constexpr unsigned kFull = 0xffffffffu;
// A pipeline wait that has not completed after this many nanoseconds gives up, records
// DWT2_ETIMEOUT and lets the kernel wind down (no wait in this library can spin forever).
constexpr unsigned long long kWaitTimeoutNs = 2000000000ull;
constexpr int kStatusTimeout = 5;  // DWT2_ETIMEOUT

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Makes the initialised barriers visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// One bounded wait on a phase: the thread may be suspended in hardware until the phase
// completes or kSuspendNs elapses (so a waiting warp does not spin on issue slots).
constexpr uint32_t kSuspendNs = 1000000;

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// Waits for the phase of the given parity to complete.  Returns false if the CTA-wide abort
// flag is raised or the wait exceeds kWaitTimeoutNs (then it raises the flag itself and records
// the timeout in *status).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          int* status) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer_ns() - t0 > kWaitTimeoutNs) {
            *abort_flag = 1;
            if (status) atomicExch(status, kStatusTimeout);
            return false;
        }
    }
}

// 2-D tiled TMA load of one box into shared memory, completing on an mbarrier (transaction
// bytes).  x must be a multiple of 16 bytes / element size (the caller guarantees it).
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// 3-D variant: (x, y, z) with z the image of a batch.
__device__ __forceinline__ void tma_load_3d(void* smem_dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// The same with an L2 eviction priority (a createpolicy operand) for the loaded lines.
__device__ __forceinline__ void tma_load_3d_hint(void* smem_dst, const CUtensorMap* map,
                                                 uint64_t* bar, int x, int y, int z,
                                                 uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        ".L2::cache_hint [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar)),
        "l"(policy)
        : "memory");
}

// L2 eviction policies (createpolicy, the whole access range).  A level whose LL output the next
// level reads stores it evict_last, so that it stays in L2 while the level streams its input and
// detail bands through; the next level reads it back with evict_normal, which returns the lines
// to the normal priority once they are used.
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_normal() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Bulk (non-tensor) copy of `bytes` bytes from global to shared memory, completing on an
// mbarrier (transaction bytes).  Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* smem_dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(smem_dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes),
        "r"(smem_u32(bar))
        : "memory");
}

// cp.async of one 4-byte element into shared memory; valid == false writes zero and reads
// nothing.  Goes through L1 (.ca), so it is only used on planes that no CTA of the running kernel
// writes.
__device__ __forceinline__ void cp_async_4(void* smem_dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(smem_dst)),
                 "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}

// cp.async of one 16-byte chunk (both addresses 16-byte aligned), through L2 only.
__device__ __forceinline__ void cp_async_16(void* smem_dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(src)
                 : "memory");
}

// The barrier's current phase also waits for every cp.async this thread has issued so far
// (pending count +1 now, -1 when they have landed).
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Programmatic dependent launch: wait until the grid this one depends on (the previous level)
// has completed and its memory is visible; then let the next grid start its own prologue.  Both
// are no-ops for a grid launched without the programmatic-serialization attribute.
__device__ __forceinline__ void grid_dependency_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void allow_dependent_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ------------------------------------------------------------------ whole-sample reflection
// Index i of the whole-sample symmetric extension of a length-n signal (period 2n - 2, mirrored
// about samples 0 and n - 1); n == 1 maps everything to 0.
__host__ __device__ __forceinline__ int refl(int i, int n) {
    if (n <= 1) return 0;
    const int p = 2 * n - 2;
    i %= p;
    if (i < 0) i += p;
    return i >= n ? p - i : i;
}

// ------------------------------------------------------------------------- conversions
template <typename T> struct Compute { using type = float; };
template <> struct Compute<int32_t> { using type = int32_t; };

__device__ __forceinline__ float to_c(float v) { return v; }
__device__ __forceinline__ int32_t to_c(int32_t v) { return v; }
__device__ __forceinline__ float to_c(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_c(__half v) { return __half2float(v); }

template <typename T> __device__ __forceinline__ T from_c(float v);
template <> __device__ __forceinline__ float from_c<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_c<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half from_c<__half>(float v) { return __float2half_rn(v); }
template <typename T> __device__ __forceinline__ T from_c(int32_t v);
template <> __device__ __forceinline__ int32_t from_c<int32_t>(int32_t v) { return v; }

template <typename T> __device__ __forceinline__ T zero_of() { return T(0); }
template <> __device__ __forceinline__ __nv_bfloat16 zero_of<__nv_bfloat16>() {
    return __float2bfloat16_rn(0.f);
}
template <> __device__ __forceinline__ __half zero_of<__half>() { return __float2half_rn(0.f); }

// Global load that bypasses L1 (.cg): for planes another SM may have written during this kernel.
template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
    return __ldcg(p);
}

// --------------------------------------------------------------- vector shared / global access
// Four consecutive elements (16 B for 32-bit types, 8 B for 16-bit types); p is aligned to that.
template <typename T, typename C>
__device__ __forceinline__ void ld4(const T* p, C (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        const uint4 u = *reinterpret_cast<const uint4*>(p);
        const T* t = reinterpret_cast<const T*>(&u);
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = to_c(t[k]);
    } else {
        const uint2 u = *reinterpret_cast<const uint2*>(p);
        const T* t = reinterpret_cast<const T*>(&u);
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = to_c(t[k]);
    }
}

// Two consecutive elements (8 B or 4 B), aligned.
template <typename T, typename C>
__device__ __forceinline__ void ld2(const T* p, C (&v)[2]) {
    if constexpr (sizeof(T) == 4) {
        const uint2 u = *reinterpret_cast<const uint2*>(p);
        const T* t = reinterpret_cast<const T*>(&u);
        v[0] = to_c(t[0]);
        v[1] = to_c(t[1]);
    } else {
        const uint32_t u = *reinterpret_cast<const uint32_t*>(p);
        const T* t = reinterpret_cast<const T*>(&u);
        v[0] = to_c(t[0]);
        v[1] = to_c(t[1]);
    }
}

template <typename T, typename C>
__device__ __forceinline__ void st2(T* p, C v0, C v1) {
    if constexpr (sizeof(T) == 4) {
        T t[2] = {from_c<T>(v0), from_c<T>(v1)};
        *reinterpret_cast<uint2*>(p) = *reinterpret_cast<const uint2*>(t);
    } else {
        T t[2] = {from_c<T>(v0), from_c<T>(v1)};
        *reinterpret_cast<uint32_t*>(p) = *reinterpret_cast<const uint32_t*>(t);
    }
}

template <typename T, typename C>
__device__ __forceinline__ void st4(T* p, C v0, C v1, C v2, C v3) {
    T t[4] = {from_c<T>(v0), from_c<T>(v1), from_c<T>(v2), from_c<T>(v3)};
    if constexpr (sizeof(T) == 4)
        *reinterpret_cast<uint4*>(p) = *reinterpret_cast<const uint4*>(t);
    else
        *reinterpret_cast<uint2*>(p) = *reinterpret_cast<const uint2*>(t);
}

// Vector stores to global memory with an L2 eviction policy (from createpolicy).
template <typename T, typename C>
__device__ __forceinline__ void st2_hint(T* p, C v0, C v1, uint64_t pol) {
    T t[2] = {from_c<T>(v0), from_c<T>(v1)};
    if constexpr (sizeof(T) == 4) {
        const uint2 u = *reinterpret_cast<const uint2*>(t);
        asm volatile("st.global.L2::cache_hint.v2.b32 [%0], {%1, %2}, %3;" ::"l"(p), "r"(u.x),
                     "r"(u.y), "l"(pol));
    } else {
        const uint32_t u = *reinterpret_cast<const uint32_t*>(t);
        asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"(u), "l"(pol));
    }
}
template <typename T, typename C>
__device__ __forceinline__ void st4_hint(T* p, C v0, C v1, C v2, C v3, uint64_t pol) {
    T t[4] = {from_c<T>(v0), from_c<T>(v1), from_c<T>(v2), from_c<T>(v3)};
    if constexpr (sizeof(T) == 4) {
        const uint4 u = *reinterpret_cast<const uint4*>(t);
        asm volatile("st.global.L2::cache_hint.v4.b32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p),
                     "r"(u.x), "r"(u.y), "r"(u.z), "r"(u.w), "l"(pol));
    } else {
        const uint2 u = *reinterpret_cast<const uint2*>(t);
        asm volatile("st.global.L2::cache_hint.v2.b32 [%0], {%1, %2}, %3;" ::"l"(p), "r"(u.x),
                     "r"(u.y), "l"(pol));
    }
}

// ------------------------------------------------------------------ warp neighbour exchange
// Each lane owns N adjacent quads (q = 0 .. N-1).  right_of gives the value of quad m + 1 for
// every quad of the lane, left_of the value of quad m - 1; the one value that crosses into the
// next / previous lane moves by warp shuffle.  Lanes 0 and 31 are halo lanes whose out-of-warp
// neighbour values are never used for a stored result.
template <typename C, int N>
__device__ __forceinline__ void right_of(const C (&v)[N], C (&r)[N]) {
#pragma unroll
    for (int q = 0; q + 1 < N; ++q) r[q] = v[q + 1];
    r[N - 1] = __shfl_down_sync(kFull, v[0], 1);
}
template <typename C, int N>
__device__ __forceinline__ void left_of(const C (&v)[N], C (&l)[N]) {
#pragma unroll
    for (int q = N - 1; q > 0; --q) l[q] = v[q - 1];
    l[0] = __shfl_up_sync(kFull, v[N - 1], 1);
}

// N consecutive elements (N = 2, 4, 8) from aligned shared memory.
template <int N, typename T, typename C>
__device__ __forceinline__ void ldN(const T* p, C (&v)[N]) {
    if constexpr (N == 2) {
        ld2(p, v);
    } else if constexpr (N == 4) {
        ld4(p, v);
    } else {
        C a[4], b[4];
        ld4(p, a);
        ld4(p + 4, b);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = a[k];
            v[4 + k] = b[k];
        }
    }
}

// N consecutive elements (N = 2, 4, 8) to aligned global memory.
template <int N, typename T, typename C>
__device__ __forceinline__ void stN(T* p, const C (&v)[N]) {
    if constexpr (N == 2) {
        st2(p, v[0], v[1]);
    } else if constexpr (N == 4) {
        st4(p, v[0], v[1], v[2], v[3]);
    } else {
        st4(p, v[0], v[1], v[2], v[3]);
        st4(p + 4, v[4], v[5], v[6], v[7]);
    }
}

}  // namespace dwt2
