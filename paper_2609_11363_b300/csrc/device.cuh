// Device-side helpers shared by the kernels: status codes, bounded waits and
// acquire/release flags.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sinv {

// must match sinv_status in include/sinv.h
enum : int32_t { ST_OK = 0, ST_SINGULAR = 3, ST_TIMEOUT = 6, ST_UNSUPPORTED = 7, ST_INTERNAL = 100 };

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int32_t ld_volatile(const int32_t* p) { return *(const volatile int32_t*)p; }

// Record the first error of a call (later errors are dropped).
__device__ __forceinline__ void set_status(int32_t* status, int32_t code) { atomicCAS(status, 0, code); }

// Spin until *flag == want, with a poll limit.  Returns false (and records
// ST_TIMEOUT) when the limit ran out, or when another warp already recorded an
// error (so that every waiter leaves once one of them gave up).
__device__ __forceinline__ bool wait_flag(const uint32_t* flag, uint32_t want, int32_t* status, int64_t limit) {
    int64_t it = 0;
    while (ld_acquire(flag) != want) {
        if ((it & 63) == 63 && ld_volatile(status) != ST_OK) return false;
        if (++it > limit) {
            set_status(status, ST_TIMEOUT);
            return false;
        }
        if (it > 16) __nanosleep(32);
    }
    return true;
}

}  // namespace sinv
