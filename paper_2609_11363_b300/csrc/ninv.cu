// NInv (Section 2.2): truncated Neumann series of L^{-1}, eq. (2.6), and the
// product (L^inv)^T D^{-1} L^inv of eq. (2.8), evaluated on S only.
//
// With L = I - E, W = sum_{t=0}^{m} E^t is built by m Horner steps
//     W_t = I + E W_{t-1}      (column form: W_t[:, j] = e_j + sum_{k in struct(j)} E_kj W_{t-1}[:, k])
// on the fixed pattern P_W of the truncated series.  P_W is stored by columns
// with every column's rows grouped by the first power that reaches them, so
// the nonzeros of W_{t-1}[:, k] are exactly the prefix "groups 0..t-1" of
// column k and no step touches a structural zero.  One CTA owns one column:
// the column's rows go into a shared-memory hash table (row -> slot), the
// products E_kj W_{t-1}[r, k] are accumulated into the slot of r.
//
// Product on S: N_ij = sum_r W_ri (D^{-1} W)_rj for (i, j) in S_lo.  A CTA
// owns column j: it hashes column j of W, then one warp per entry (i, j)
// streams column i of W (rows >= i, all useful) and reads W_rj and
// W_{partner(r), j} from the table; the 2x2 blocks of D^{-1} couple r with
// its partner.
#include <algorithm>

#include "device.cuh"
#include "kernels.h"

namespace sinv {

namespace {

constexpr int kThreads = 256;
constexpr int kWarpsN = kThreads / 32;
constexpr int kSmemSlots = 8192;   // hash slots held in shared memory (cols up to 4096 rows)

__device__ __forceinline__ uint32_t hash_row(int32_t r, uint32_t mask) {
    return ((uint32_t)r * 2654435761u) & mask;
}

__device__ __forceinline__ void table_insert(int32_t* keys, int32_t* vals, uint32_t mask, int32_t r, int32_t v) {
    uint32_t h = hash_row(r, mask);
    for (;;) {
        int32_t old = atomicCAS(keys + h, -1, r);
        if (old == -1 || old == r) {
            vals[h] = v;
            return;
        }
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

__device__ __forceinline__ uint32_t table_mask(int64_t entries) {
    uint32_t s = 16;
    while ((int64_t)s < 2 * entries) s <<= 1;
    return s - 1;
}

struct Table {
    int32_t* keys;
    int32_t* vals;
    uint32_t mask;
};

// shared-memory table when it fits, else this CTA's slice of the global scratch
__device__ __forceinline__ Table get_table(int64_t entries, int32_t* skeys, int32_t* svals, int32_t* gscratch,
                                           int64_t gslots) {
    Table t;
    t.mask = table_mask(entries);
    if ((int64_t)t.mask + 1 <= kSmemSlots) {
        t.keys = skeys;
        t.vals = svals;
    } else {
        t.keys = gscratch + (int64_t)blockIdx.x * 2 * gslots;
        t.vals = t.keys + gslots;
    }
    return t;
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
__global__ void __launch_bounds__(kThreads) ninv_horner(NinvArgs a, int t, const T* __restrict__ Wp, T* __restrict__ Wn,
                                                        int32_t* ticket, int32_t* gscratch, int64_t gslots,
                                                        T* gacc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t* skeys = reinterpret_cast<int32_t*>(smem_raw);
    int32_t* svals = skeys + kSmemSlots;
    T* sacc = reinterpret_cast<T*>(svals + kSmemSlots);
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
        Table tb = get_table(nj, skeys, svals, gscratch, gslots);
        T* acc = ((int64_t)tb.mask + 1 <= kSmemSlots) ? sacc : gacc + (int64_t)blockIdx.x * gslots;
        for (uint32_t s = threadIdx.x; s <= tb.mask; s += kThreads) tb.keys[s] = -1;
        for (int32_t e = threadIdx.x; e < nj; e += kThreads) acc[e] = T(0);
        __syncthreads();
        for (int32_t e = threadIdx.x; e < nj; e += kThreads) table_insert(tb.keys, tb.vals, tb.mask, a.Wr[base + e], e);
        __syncthreads();
        // sum_k E_kj W_{t-1}[:, k]; warp per k, lanes over column k's groups 0..t-1
        for (int64_t q = a.Lcp[j] + wid; q < a.Lcp[j + 1]; q += kWarpsN) {
            const int32_t k = a.Lri[q];
            const T ekj = T(-a.Lval[a.Lcsr[q]]);
            const int64_t kb = a.Wcp[k];
            const int32_t nk = a.grp[(int64_t)k * G + t];
            for (int32_t e = lane; e < nk; e += 32) {
                int32_t r = a.Wr[kb + e];
                T v = ekj * Wp[kb + e];
                int32_t idx = table_find(tb.keys, tb.vals, tb.mask, r);
                if (idx >= 0) atomicAdd(acc + idx, v);
                else set_status(a.status, ST_INTERNAL);  // row outside the pattern: never expected
            }
        }
        __syncthreads();
        for (int32_t e = threadIdx.x; e < nj; e += kThreads) Wn[base + e] = acc[e] + (e == 0 ? T(1) : T(0));
        __syncthreads();
    }
}

template <class T>
__global__ void __launch_bounds__(kThreads) ninv_product(NinvArgs a, const T* __restrict__ W, const double* __restrict__ dr,
                                                         const double* __restrict__ dp, const int32_t* __restrict__ part,
                                                         double* __restrict__ N, int32_t* ticket, int32_t* gscratch,
                                                         int64_t gslots) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t* skeys = reinterpret_cast<int32_t*>(smem_raw);
    int32_t* svals = skeys + kSmemSlots;
    __shared__ int32_t s_j;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_j = atomicAdd(ticket, 1);
        __syncthreads();
        const int64_t j = s_j;
        __syncthreads();
        if (j >= a.n) break;
        const int64_t base = a.Wcp[j];
        const int32_t nj = (int32_t)(a.Wcp[j + 1] - base);
        Table tb = get_table(nj, skeys, svals, gscratch, gslots);
        for (uint32_t s = threadIdx.x; s <= tb.mask; s += kThreads) tb.keys[s] = -1;
        __syncthreads();
        for (int32_t e = threadIdx.x; e < nj; e += kThreads) table_insert(tb.keys, tb.vals, tb.mask, a.Wr[base + e], e);
        __syncthreads();
        // entries of S_lo in column j: the diagonal, the 2x2 partner row, struct(j)
        const bool two_first = a.pstart[j] != 0 && j + 1 < a.n && a.pstart[j + 1] == 0;
        const int64_t q0 = a.Lcp[j], q1 = a.Lcp[j + 1];
        const int64_t cnt = (q1 - q0) + 1 + (two_first ? 1 : 0);
        for (int64_t e = wid; e < cnt; e += kWarpsN) {
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
            double s = 0.0;
            for (int64_t f = ib + lane; f < ie; f += 32) {
                const int32_t r = a.Wr[f];
                const double wri = (double)W[f];
                int32_t x = table_find(tb.keys, tb.vals, tb.mask, r);
                double y = x >= 0 ? dr[r] * (double)W[base + x] : 0.0;
                const int32_t pr = part[r];
                if (pr >= 0) {
                    int32_t xp = table_find(tb.keys, tb.vals, tb.mask, pr);
                    if (xp >= 0) y += dp[r] * (double)W[base + xp];
                }
                s += wri * y;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) N[spos] = s;
        }
        __syncthreads();
    }
}

template <class T>
constexpr size_t horner_smem() { return kSmemSlots * 2 * sizeof(int32_t) + kSmemSlots * sizeof(T); }
constexpr size_t product_smem() { return kSmemSlots * 2 * sizeof(int32_t); }

}  // namespace

cudaError_t ninv_configure() {
    cudaError_t e;
    e = cudaFuncSetAttribute(ninv_horner<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)horner_smem<double>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ninv_horner<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)horner_smem<float>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ninv_product<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)product_smem());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(ninv_product<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)product_smem());
}

size_t ninv_work_bytes(const NinvArgs& a, int prec) {
    size_t ts = prec == 0 ? sizeof(double) : sizeof(float);
    size_t b = 2 * (size_t)a.nnzW * ts;            // ping-pong W
    b += (size_t)a.n * (2 * sizeof(double) + sizeof(int32_t)) + 256;
    b += 2 * sizeof(int32_t) * 64;                 // tickets
    int64_t slots = 16;
    while (slots < 2 * a.max_col) slots <<= 1;
    if (slots > kSmemSlots) {
        size_t ctas = (size_t)a.num_sms * 2;
        b += ctas * (size_t)slots * (2 * sizeof(int32_t) + ts) + 1024;
    }
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
    int64_t slots = 16;
    while (slots < 2 * a.max_col) slots <<= 1;
    int32_t* gscratch = nullptr;
    T* gacc = nullptr;
    const int grid = a.num_sms * 2;
    if (slots > kSmemSlots) {
        gscratch = reinterpret_cast<int32_t*>(take((size_t)grid * slots * 2 * sizeof(int32_t)));
        gacc = reinterpret_cast<T*>(take((size_t)grid * slots * sizeof(T)));
    } else {
        slots = 0;
    }
    cudaError_t e = cudaMemsetAsync(tickets, 0, sizeof(int32_t) * 64, st);
    if (e != cudaSuccess) return e;
    ninv_dinv<<<a.num_sms * 4, 256, 0, st>>>(a.n, a.dpos, a.pstart, a.Dval, dr, dp, part, a.status);
    ninv_init<T><<<a.num_sms * 4, 256, 0, st>>>(a.Wcp, W0, a.n);
    T* cur = W0;
    T* nxt = W1;
    for (int t = 1; t <= a.m; ++t) {
        ninv_horner<T><<<grid, kThreads, horner_smem<T>(), st>>>(a, t, cur, nxt, tickets + t, gscratch, slots, gacc);
        std::swap(cur, nxt);
    }
    ninv_product<T><<<grid, kThreads, product_smem(), st>>>(a, cur, dr, dp, part, N_out, tickets + 63, gscratch, slots);
    return cudaGetLastError();
}

cudaError_t ninv_launch(const NinvArgs& a, int prec, void* work, double* N_out, cudaStream_t st) {
    if (a.n == 0) return cudaSuccess;
    if (a.m > 60) return cudaErrorInvalidValue;
    if (prec == 0) return ninv_run<double>(a, work, N_out, st);
    return ninv_run<float>(a, work, N_out, st);
}

}  // namespace sinv
