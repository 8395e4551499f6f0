// Open-addressing hash tables of row indices (linear probing), shared by the
// NInv kernels.  A table is `mask + 1` int32 keys initialised to -1; a slot
// index doubles as the index of any per-row value kept beside the keys.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sinv {

__device__ __forceinline__ uint32_t hash_row(int32_t r, uint32_t mask) {
    return ((uint32_t)r * 2654435761u) & mask;
}

// insert r (if absent) and return its slot
__device__ __forceinline__ uint32_t table_insert(int32_t* keys, uint32_t mask, int32_t r) {
    uint32_t h = hash_row(r, mask);
    for (;;) {
        int32_t old = atomicCAS(keys + h, -1, r);
        if (old == -1 || old == r) return h;
        h = (h + 1) & mask;
    }
}

// slot of r, or -1 when r is not in the table
__device__ __forceinline__ int32_t table_find(const int32_t* keys, uint32_t mask, int32_t r) {
    uint32_t h = hash_row(r, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        int32_t k = keys[h];
        if (k == r) return (int32_t)h;
        if (k == -1) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

// smallest power-of-two table (minus one) with load <= 1/2 for `entries` keys
__host__ __device__ __forceinline__ uint32_t table_mask(int64_t entries) {
    uint32_t s = 16;
    while ((int64_t)s < 2 * entries) s <<= 1;
    return s - 1;
}

}  // namespace sinv
