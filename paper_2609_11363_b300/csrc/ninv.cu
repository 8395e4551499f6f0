// NInv (Section 2.2): truncated Neumann series of L^{-1}, eq. (2.6), and the
// product (L^inv)^T D^{-1} L^inv of eq. (2.8), evaluated on S only.
//
// With L = I - E, W = sum_{t=0}^{m} E^t is built by m Horner steps
//     W_t = I + E W_{t-1}      (column form: W_t[:, j] = e_j + sum_{k in struct(j)} E_kj W_{t-1}[:, k])
// on the fixed pattern P_W of the truncated series.  P_W is stored by columns
// with every column's rows grouped by the first power that reaches them, so
// the nonzeros of W_{t-1}[:, k] are exactly the prefix "groups 0..t-1" of
// column k and no step touches a structural zero.
//
// Horner step: one CTA owns one column j.  Its rows go into a shared-memory
// hash table (row -> slot).  Warp v handles the columns k of struct(j) with
// k = v mod 4 and accumulates E_kj W_{t-1}[r, k] into its own copy of the
// column (the lanes of one instruction touch distinct rows, so no atomic is
// needed); the copies are summed at the end.
//
// Product on S: N_ij = sum_r W_ri (D^{-1} W)_rj for (i, j) in S_lo.  One CTA
// owns column j: it tabulates y = (D^{-1} W)[:, j] (the 2x2 blocks of D^{-1}
// couple a row with its partner, which may add rows outside column j's
// pattern), then one warp per entry (i, j) streams column i of W and sums
// W_ri y_r over the rows found in the table.
//
// Columns too long for shared memory use the same code on a per-CTA slice of
// global scratch, with atomic accumulation.
#include <algorithm>

#include "device.cuh"
#include "kernels.h"

namespace sinv {

namespace {

constexpr int kWarpsH = 4;                    // warps per CTA, Horner step
constexpr int kThreadsH = kWarpsH * 32;
constexpr int kSlotsH = 4096;                 // hash slots in shared memory
constexpr int kColH = kSlotsH / 2;            // longest column kept in shared memory
constexpr int kWarpsP = 8;                    // warps per CTA, product
constexpr int kThreadsP = kWarpsP * 32;
constexpr int kSlotsP = 8192;
constexpr int kEntP = kSlotsP / 2;            // table entries (column rows + partner rows)
constexpr int kUnroll = 8;                    // column entries per lane with loads in flight

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

__device__ __forceinline__ int32_t table_find(const int32_t* keys, const int32_t* vals, uint32_t mask, int32_t r) {
    uint32_t h = hash_row(r, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        int32_t k = keys[h];
        if (k == r) return vals[h];
        if (k == -1) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

__host__ __device__ __forceinline__ uint32_t table_mask(int64_t entries) {
    uint32_t s = 16;
    while ((int64_t)s < 2 * entries) s <<= 1;
    return s - 1;
}

template <class T>
__global__ void ninv_init(const int64_t* __restrict__ Wcp, T* __restrict__ W, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        W[Wcp[j]] = T(1);  // group 0 of column j is row j
}

// D^{-1} per row: dr[r] = (D^{-1})_rr, dp[r] = (D^{-1})_{r, partner}, part[r] = partner or -1.
__global__ void ninv_dinv(int64_t n, const int32_t* __restrict__ dpos, const int8_t* __restrict__ pstart,
                          const double* __restrict__ Dval, double* __restrict__ dr, double* __restrict__ dp,
                          int32_t* __restrict__ part, int32_t* status) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const bool first = pstart[r] != 0;
        const bool two = first ? (r + 1 < n && pstart[r + 1] == 0) : true;
        const double* d = Dval + dpos[r];
        if (!two) {
            if (d[0] == 0.0) set_status(status, ST_SINGULAR);
            dr[r] = 1.0 / d[0];
            dp[r] = 0.0;
            part[r] = -1;
        } else {
            double det = d[0] * d[2] - d[1] * d[1];
            if (det == 0.0) set_status(status, ST_SINGULAR);
            dr[r] = (first ? d[2] : d[0]) / det;
            dp[r] = -d[1] / det;
            part[r] = (int32_t)(first ? r + 1 : r - 1);
        }
    }
}

template <class T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }

struct Scratch {
    int32_t* keys;   // per CTA: slots int32 keys, slots int32 vals, slots int32 extra rows
    void* acc;       // per CTA: accumulators / y values
    int64_t slots;   // slots per CTA (0 when every column fits shared memory)
};

template <class T>
__global__ void __launch_bounds__(kThreadsH) ninv_horner(NinvArgs a, int t, const T* __restrict__ Wp, T* __restrict__ Wn,
                                                         int32_t* ticket, Scratch gs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t* skeys = reinterpret_cast<int32_t*>(smem_raw);
    int32_t* svals = skeys + kSlotsH;
    T* sacc = reinterpret_cast<T*>(svals + kSlotsH);  // kWarpsH copies of kColH
    __shared__ int32_t s_j;
    const int G = a.m + 2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_j = atomicAdd(ticket, 1);
        __syncthreads();
        const int64_t j = s_j;
        __syncthreads();
        if (j >= a.n) break;
        const int64_t base = a.Wcp[j];
        const int32_t nj = a.grp[j * G + t + 1];  // rows of groups 0..t
        const bool small = nj <= kColH;
        const uint32_t mask = small ? (uint32_t)(kSlotsH - 1) : table_mask(nj);
        int32_t* keys = small ? skeys : gs.keys + (int64_t)blockIdx.x * 3 * gs.slots;
        int32_t* vals = small ? svals : keys + gs.slots;
        T* gacc = reinterpret_cast<T*>(gs.acc) + (int64_t)blockIdx.x * gs.slots;
        for (uint32_t s = threadIdx.x; s <= mask; s += kThreadsH) keys[s] = -1;
        if (small) {
            for (int32_t e = threadIdx.x; e < kWarpsH * nj; e += kThreadsH) sacc[(e / nj) * kColH + e % nj] = T(0);
        } else {
            for (int32_t e = threadIdx.x; e < nj; e += kThreadsH) gacc[e] = T(0);
        }
        __syncthreads();
        for (int32_t e = threadIdx.x; e < nj; e += kThreadsH) vals[table_insert(keys, mask, a.Wr[base + e])] = e;
        __syncthreads();
        T* acc = small ? sacc + wid * kColH : gacc;
        // sum_k E_kj W_{t-1}[:, k]: warp wid takes k = wid, wid+4, ...; lanes over column k's groups 0..t-1
        for (int64_t q = a.Lcp[j] + wid; q < a.Lcp[j + 1]; q += kWarpsH) {
            const int32_t k = a.Lri[q];
            const T ekj = T(-a.Lval[a.Lcsr[q]]);
            const int64_t kb = a.Wcp[k];
            const int32_t nk = a.grp[(int64_t)k * G + t];
            // kUnroll entries per lane in flight; all rows of one column are distinct, so the
            // lanes of a batch never touch the same slot
            for (int32_t e0 = 0; e0 < nk; e0 += 32 * kUnroll) {
                int32_t r[kUnroll];
                T v[kUnroll];
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const int32_t e = e0 + u * 32 + lane;
                    r[u] = e < nk ? a.Wr[kb + e] : -1;
                    v[u] = e < nk ? Wp[kb + e] : T(0);
                }
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    if (r[u] < 0) continue;
                    const int32_t idx = table_find(keys, vals, mask, r[u]);
                    if (idx >= 0) {
                        if (small) acc[idx] = fma_t<T>(ekj, v[u], acc[idx]);
                        else atomicAdd(acc + idx, ekj * v[u]);
                    } else {
                        set_status(a.status, ST_INTERNAL);  // row outside the pattern: never expected
                    }
                }
                __syncwarp();
            }
        }
        __syncthreads();
        for (int32_t e = threadIdx.x; e < nj; e += kThreadsH) {
            T s = e == 0 ? T(1) : T(0);
            if (small) {
#pragma unroll
                for (int v = 0; v < kWarpsH; ++v) s += sacc[v * kColH + e];
            } else {
                s += gacc[e];
            }
            Wn[base + e] = s;
        }
        __syncthreads();
    }
}

template <class T>
__global__ void __launch_bounds__(kThreadsP) ninv_product(NinvArgs a, const T* __restrict__ W, const double* __restrict__ dr,
                                                          const double* __restrict__ dp, const int32_t* __restrict__ part,
                                                          double* __restrict__ N, int32_t* ticket, Scratch gs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t* skeys = reinterpret_cast<int32_t*>(smem_raw);
    int32_t* svals = skeys + kSlotsP;
    T* syv = reinterpret_cast<T*>(svals + kSlotsP);          // kEntP y values
    __shared__ int32_t s_j, s_extra;
    __shared__ int32_t s_xrow[kEntP / 2];                      // rows of the extra (partner) entries
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) {
            s_j = atomicAdd(ticket, 1);
            s_extra = 0;
        }
        __syncthreads();
        const int64_t j = s_j;
        __syncthreads();
        if (j >= a.n) break;
        const int64_t base = a.Wcp[j];
        const int32_t nj = (int32_t)(a.Wcp[j + 1] - base);
        const bool small = 2 * nj <= kEntP;
        const uint32_t mask = small ? (uint32_t)(kSlotsP - 1) : table_mask(2 * (int64_t)nj);
        int32_t* keys = small ? skeys : gs.keys + (int64_t)blockIdx.x * 3 * gs.slots;
        int32_t* vals = small ? svals : keys + gs.slots;
        T* yv = small ? syv : reinterpret_cast<T*>(gs.acc) + (int64_t)blockIdx.x * gs.slots;
        int32_t* xrow = small ? s_xrow : vals + gs.slots;
        for (uint32_t s = threadIdx.x; s <= mask; s += kThreadsP) keys[s] = -1;
        __syncthreads();
        for (int32_t e = threadIdx.x; e < nj; e += kThreadsP) vals[table_insert(keys, mask, a.Wr[base + e])] = e;
        __syncthreads();
        // partner rows of 2x2 blocks that are not in column j: y is nonzero there too
        for (int32_t e = threadIdx.x; e < nj; e += kThreadsP) {
            const int32_t p = part[a.Wr[base + e]];
            if (p >= 0 && table_find(keys, vals, mask, p) < 0) {
                int32_t x = atomicAdd(&s_extra, 1);
                xrow[x] = p;
                vals[table_insert(keys, mask, p)] = nj + x;
            }
        }
        __syncthreads();
        const int32_t ntot = nj + s_extra;
        for (int32_t e = threadIdx.x; e < ntot; e += kThreadsP) {
            const int32_t r = e < nj ? a.Wr[base + e] : xrow[e - nj];
            double y = e < nj ? dr[r] * (double)W[base + e] : 0.0;
            const int32_t p = part[r];
            if (p >= 0) {
                const int32_t x = table_find(keys, vals, mask, p);
                if (x >= 0 && x < nj) y += dp[r] * (double)W[base + x];
            }
            yv[e] = T(y);
        }
        __syncthreads();
        // entries of S_lo in column j: the diagonal, the 2x2 partner row, struct(j)
        const bool two_first = a.pstart[j] != 0 && j + 1 < a.n && a.pstart[j + 1] == 0;
        const int64_t q0 = a.Lcp[j], q1 = a.Lcp[j + 1];
        const int64_t cnt = (q1 - q0) + 1 + (two_first ? 1 : 0);
        for (int64_t e = wid; e < cnt; e += kWarpsP) {
            int64_t i, spos;
            if (e == 0) {
                i = j;
                spos = a.Srp[j + 1] - 1;          // (j, j): last entry of row j
            } else if (two_first && e == 1) {
                i = j + 1;
                spos = a.Srp[j + 2] - 2;          // (j+1, j): before the diagonal of row j+1
            } else {
                const int64_t q = q0 + e - 1 - (two_first ? 1 : 0);
                i = a.Lri[q];
                // row i of S_lo starts with row i of L, so L(i, j) keeps its offset in the row
                spos = a.Srp[i] + ((int64_t)a.Lcsr[q] - a.Lrp[i]);
            }
            const int64_t ib = a.Wcp[i], ie = a.Wcp[i + 1];
            T s = T(0);
            for (int64_t f0 = ib; f0 < ie; f0 += 32 * kUnroll) {
                int32_t r[kUnroll];
                T wv[kUnroll];
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const int64_t f = f0 + u * 32 + lane;
                    r[u] = f < ie ? a.Wr[f] : -1;
                    wv[u] = f < ie ? W[f] : T(0);
                }
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    if (r[u] < 0) continue;
                    const int32_t x = table_find(keys, vals, mask, r[u]);
                    if (x >= 0) s = fma_t<T>(wv[u], yv[x], s);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) N[spos] = (double)s;
        }
        __syncthreads();
    }
}

template <class T>
constexpr size_t horner_smem() { return kSlotsH * 2 * sizeof(int32_t) + (size_t)kWarpsH * kColH * sizeof(T); }
template <class T>
constexpr size_t product_smem() { return kSlotsP * 2 * sizeof(int32_t) + (size_t)kEntP * sizeof(T); }

int64_t global_slots(const NinvArgs& a) {
    // the longest column may hold up to 2 max_col table entries (partner rows)
    if (a.max_col <= kColH && 2 * a.max_col <= kEntP) return 0;
    return (int64_t)table_mask(2 * a.max_col) + 1;
}

}  // namespace

cudaError_t ninv_configure() {
    cudaError_t e;
    e = cudaFuncSetAttribute(ninv_horner<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)horner_smem<double>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ninv_horner<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)horner_smem<float>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ninv_product<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)product_smem<double>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(ninv_product<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)product_smem<float>());
}

static int ninv_grid(const NinvArgs& a) { return a.num_sms * 2; }

size_t ninv_work_bytes(const NinvArgs& a, int prec) {
    size_t ts = prec == 0 ? sizeof(double) : sizeof(float);
    size_t b = 2 * ((size_t)a.nnzW * ts + 256);                 // ping-pong W
    b += (size_t)a.n * (2 * sizeof(double) + sizeof(int32_t)) + 3 * 256;
    b += sizeof(int32_t) * 64 + 256;                            // tickets
    int64_t slots = global_slots(a);
    if (slots) b += (size_t)ninv_grid(a) * slots * (3 * sizeof(int32_t) + sizeof(double)) + 2 * 256;
    return b + 4096;
}

template <class T>
static cudaError_t ninv_run(const NinvArgs& a, void* work, double* N_out, cudaStream_t st) {
    char* p = reinterpret_cast<char*>(work);
    auto take = [&](size_t bytes) {
        char* r = p;
        p += (bytes + 255) & ~(size_t)255;
        return r;
    };
    T* W0 = reinterpret_cast<T*>(take((size_t)a.nnzW * sizeof(T)));
    T* W1 = reinterpret_cast<T*>(take((size_t)a.nnzW * sizeof(T)));
    double* dr = reinterpret_cast<double*>(take((size_t)a.n * sizeof(double)));
    double* dp = reinterpret_cast<double*>(take((size_t)a.n * sizeof(double)));
    int32_t* part = reinterpret_cast<int32_t*>(take((size_t)a.n * sizeof(int32_t)));
    int32_t* tickets = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * 64));
    const int grid = ninv_grid(a);
    Scratch gs{nullptr, nullptr, global_slots(a)};
    if (gs.slots) {
        gs.keys = reinterpret_cast<int32_t*>(take((size_t)grid * gs.slots * 3 * sizeof(int32_t)));
        gs.acc = take((size_t)grid * gs.slots * sizeof(double));
    }
    cudaError_t e = cudaMemsetAsync(tickets, 0, sizeof(int32_t) * 64, st);
    if (e != cudaSuccess) return e;
    ninv_dinv<<<a.num_sms * 4, 256, 0, st>>>(a.n, a.dpos, a.pstart, a.Dval, dr, dp, part, a.status);
    ninv_init<T><<<a.num_sms * 4, 256, 0, st>>>(a.Wcp, W0, a.n);
    T* cur = W0;
    T* nxt = W1;
    for (int t = 1; t <= a.m; ++t) {
        ninv_horner<T><<<grid, kThreadsH, horner_smem<T>(), st>>>(a, t, cur, nxt, tickets + t, gs);
        std::swap(cur, nxt);
    }
    ninv_product<T><<<grid, kThreadsP, product_smem<T>(), st>>>(a, cur, dr, dp, part, N_out, tickets + 63, gs);
    return cudaGetLastError();
}

cudaError_t ninv_launch(const NinvArgs& a, int prec, void* work, double* N_out, cudaStream_t st) {
    if (a.n == 0) return cudaSuccess;
    if (a.m > 60) return cudaErrorInvalidValue;
    if (prec == 0) return ninv_run<double>(a, work, N_out, st);
    return ninv_run<float>(a, work, N_out, st);
}

}  // namespace sinv
