// Device-side helpers shared by the kernels: status codes, bounded waits and
// acquire/release flags.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sinv {

// must match sinv_status in include/sinv.h
enum : int32_t { ST_OK = 0, ST_SINGULAR = 3, ST_TIMEOUT = 6, ST_UNSUPPORTED = 7, ST_INTERNAL = 100, ST_BOUNDS = 101 };

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int32_t ld_volatile(const int32_t* p) { return *(const volatile int32_t*)p; }

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Record the first error of a call (later errors are dropped).
__device__ __forceinline__ void set_status(int32_t* status, int32_t code) { atomicCAS(status, 0, code); }

// Bounds checks of the checked build (-DSINV_CHECKED): an index read from the plan
// or the maps that falls outside its array records ST_BOUNDS in the status word
// and the access is skipped (nothing traps).  The regular build compiles them out.
#ifdef SINV_CHECKED
__device__ __forceinline__ bool in_range(int32_t* status, int64_t idx, int64_t lo, int64_t hi) {
    if (idx >= lo && idx < hi) return true;
    set_status(status, ST_BOUNDS);
    return false;
}
#else
__device__ __forceinline__ bool in_range(int32_t*, int64_t, int64_t, int64_t) { return true; }
#endif

// Spin until *flag == want, with a poll limit.  Returns false (and records
// ST_TIMEOUT) when the limit ran out, or when another warp already recorded an
// error (so that every waiter leaves once one of them gave up).  The spin polls
// with relaxed loads; one acquire load of the flag, once it is seen set, orders
// the caller's later reads after the producer's release.
__device__ __forceinline__ bool wait_flag(const uint32_t* flag, uint32_t want, int32_t* status, int64_t limit) {
    int64_t it = 0;
    if (ld_acquire(flag) == want) return true;
    while (ld_relaxed(flag) != want || ld_acquire(flag) != want) {
        if ((it & 63) == 63 && ld_volatile(status) != ST_OK) return false;
        if (++it > limit) {
            set_status(status, ST_TIMEOUT);
            return false;
        }
        if (it > 16) __nanosleep(32);
    }
    return true;
}

// Device-wide clock in nanoseconds (for the per-supernode timeline).
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Timeline of one SelInv call (null when not recorded): per supernode J, first[J] is
// the earliest start of any of its work items (atomic min over parts, initialised to
// all ones), and last[3J + k] the latest (atomic max, initialised to 0) of: k = 0 its
// dependencies had published, k = 1 its contraction was done, k = 2 it published.
struct Timeline {
    unsigned long long* first;
    unsigned long long* last;
};
__device__ __forceinline__ void tl_start(const Timeline& tl, int J) {
    if (tl.first) atomicMin(tl.first + J, (unsigned long long)gtimer());
}
__device__ __forceinline__ void tl_mark(const Timeline& tl, int J, int k) {
    if (tl.last) atomicMax(tl.last + 3 * (int64_t)J + k, (unsigned long long)gtimer());
}

}  // namespace sinv
