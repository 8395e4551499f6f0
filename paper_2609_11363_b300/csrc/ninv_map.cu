// NInv in map form (Section 2.2, Eqs. (6) and (8)): the arithmetic of the hash
// form in ninv.cu, with every hash search replaced by a position resolved once
// per pattern and m.
//
// Horner step W_t[:, j] = e_j + sum_{k in struct(j)} E_kj W_{t-1}[:, k].  One CTA
// owns column j and accumulates it in shared memory, indexed by the local
// position of a row in column j.  For every entry E_kj (an entry q of L) the map
// hmap[moff[q] + e] holds the position in column j of the e-th row of column k;
// column k's rows of powers <= t - 1 are a prefix of it, so step t streams the
// prefix of the map beside the prefix of W_{t-1}[:, k] (both coalesced) and adds
// E_kj W_{t-1}[r, k] at the mapped position with a shared-memory atomic.
//
// Product on S: N_ij = sum_r W_ri y_r with y = (D^{-1} W)[:, j].  One CTA owns
// column j and tabulates y in shared memory: positions [0, |col j|) are the rows
// of column j, then one extra position for every partner row (2x2 block of D)
// that is not in column j.  For every entry (i, j) of S_lo the map
// pmap[poff[e] + f] holds the table position of the f-th row of column i (or
// 0xFFFF when y is zero there); a warp streams column i with its map and sums
// W_ri y_r.  ypart holds, for the rows of 2x2 blocks, the table position of the
// partner row inside their own column's table.
//
// The FP64 Horner step (hm_step_fx) sums in exact 64-bit fixed point with integer
// shared atomics (bit-reproducible; one FP64 multiply per product).
//
// Pair form (SINV_FP32X2): the same fixed-point Horner steps also write W as pairs
// hi + lo of floats where a product follows, and the product on S (pp_product)
// runs in double-float arithmetic on the FP32 pipes, with y formed in pairs (one
// writer per position): no FP64 operation is left in the product.  (A Horner step
// with double-float products in the same fixed point was slower: its integer
// rounding of two parts per product outweighed the FP64 multiply it saves.)
//
// The maps are built on the GPU from the same shared-memory tables as the hash
// form.  A column with its extra partner rows must fit a table: columns up to
// kIdxEnt rows run several CTAs per SM, longer ones (up to kIdxEntLong) run in a
// second launch with the large tables, one CTA per SM.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "device.cuh"
#include "hash.cuh"
#include "kernels.h"
#include "plan.h"

namespace sinv {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kSlotsShort = 8192;     // hash slots of a short column's table (kIdxEnt rows at most)
constexpr int kSlotsLong = 32768;     // ... of a long column's table (kIdxEntLong rows at most)
constexpr int kUnrollM = 8;
constexpr int32_t kRowMask = 0x7FFFFFFF;
constexpr int32_t kTwoFlag = (int32_t)0x80000000u;
constexpr uint16_t kNone = 0xFFFF;

// The columns a launch handles: a list (short columns or long columns, see
// NinvMaps), taken one per CTA from a ticket counter.  Returns -1 when done.
struct ColumnList {
    const int32_t* cols;
    int64_t count;
};

__device__ __forceinline__ int64_t take_column(int32_t* ticket, int32_t* s_j, ColumnList cl) {
    if (threadIdx.x == 0) *s_j = atomicAdd(ticket, 1);
    __syncthreads();
    const int64_t t = *s_j;
    __syncthreads();
    return t < cl.count ? (int64_t)cl.cols[t] : -1;
}

template <int kSlots>
struct TableSmem {
    int32_t keys[kSlots];
    uint16_t loc[kSlots];
};

// rows of column j -> local position
template <int kSlots>
__device__ __forceinline__ void column_table(const NinvArgs& a, int64_t base, int32_t nj, TableSmem<kSlots>& t) {
    for (int s = threadIdx.x; s < kSlots; s += kThreads) t.keys[s] = -1;
    __syncthreads();
    for (int32_t e = threadIdx.x; e < nj; e += kThreads)
        t.loc[table_insert(t.keys, kSlots - 1, a.Wr[base + e] & kRowMask)] = (uint16_t)e;
    __syncthreads();
}

template <int kSlots>
__device__ __forceinline__ uint16_t lookup(const TableSmem<kSlots>& t, int32_t r) {
    const int32_t h = table_find(t.keys, kSlots - 1, r);
    return h < 0 ? kNone : t.loc[h];
}

// Horner maps: hmap[moff[q] + e] = position in column j of row e of column k (e over
// the powers 0..m-1 of column k), for every entry q = (k, j) of E.
template <int kSlots>
__global__ void __launch_bounds__(kThreads) hmap_build(NinvArgs a, NinvMaps x, ColumnList cl, int32_t* ticket) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TableSmem<kSlots>& tb = *reinterpret_cast<TableSmem<kSlots>*>(smem_raw);
    __shared__ int32_t s_j;
    const int G = a.m + 2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        const int64_t j = take_column(ticket, &s_j, cl);
        if (j < 0) break;
        const int64_t base = a.Wcp[j];
        column_table(a, base, (int32_t)(a.Wcp[j + 1] - base), tb);
        for (int64_t q = a.Lcp[j] + wid; q < a.Lcp[j + 1]; q += kWarps) {
            const int32_t k = a.Lri[q];
            const int64_t kb = a.Wcp[k];
            const int32_t nk = a.grp[(int64_t)k * G + a.m];
            uint16_t* mp = x.hmap + x.moff[q];
            for (int32_t e = lane; e < nk; e += 32) {
                const uint16_t p = lookup(tb, a.Wr[kb + e] & kRowMask);
                if (p == kNone) set_status(a.status, ST_INTERNAL);
                mp[e] = p;
            }
        }
        __syncthreads();
    }
}

// y tables and product maps.
template <int kSlots>
__global__ void __launch_bounds__(kThreads) pmap_build(NinvArgs a, NinvMaps x, const int32_t* __restrict__ part,
                                                       ColumnList cl, int32_t* ticket, unsigned long long* hits) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TableSmem<kSlots>& tb = *reinterpret_cast<TableSmem<kSlots>*>(smem_raw);
    __shared__ int32_t s_j, s_extra;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long nhit = 0;
    for (;;) {
        const int64_t j = take_column(ticket, &s_j, cl);
        if (j < 0) break;
        const int64_t base = a.Wcp[j];
        const int32_t nj = (int32_t)(a.Wcp[j + 1] - base);
        if (threadIdx.x == 0) s_extra = 0;
        column_table(a, base, nj, tb);
        // partner rows: in the column, or an extra position (each row has one partner,
        // so every extra row is inserted by a single thread)
        for (int32_t e = threadIdx.x; e < nj; e += kThreads) {
            const int32_t rf = a.Wr[base + e];
            uint16_t pp = kNone;
            if (rf & kTwoFlag) {
                const int32_t p = part[rf & kRowMask];
                const int32_t h = table_find(tb.keys, kSlots - 1, p);
                if (h >= 0) {
                    pp = tb.loc[h];
                } else {
                    const int32_t slot = (int32_t)table_insert(tb.keys, kSlots - 1, p);
                    pp = (uint16_t)(nj + atomicAdd(&s_extra, 1));
                    tb.loc[slot] = pp;
                }
            }
            x.ypart[base + e] = pp;
        }
        __syncthreads();
        if (threadIdx.x == 0) x.ynx[j] = s_extra;
        const bool two_first = a.pstart[j] != 0 && j + 1 < a.n && a.pstart[j + 1] == 0;
        const int64_t q0 = a.Lcp[j];
        const int64_t cnt = (a.Lcp[j + 1] - q0) + 1 + (two_first ? 1 : 0);
        for (int64_t e = wid; e < cnt; e += kWarps) {
            int64_t i, spos;
            if (e == 0) {
                i = j;
                spos = a.Srp[j + 1] - 1;
            } else if (two_first && e == 1) {
                i = j + 1;
                spos = a.Srp[j + 2] - 2;
            } else {
                const int64_t q = q0 + e - 1 - (two_first ? 1 : 0);
                i = a.Lri[q];
                spos = a.Srp[i] + ((int64_t)a.Lcsr[q] - a.Lrp[i]);
            }
            const int64_t ib = a.Wcp[i];
            const int32_t ni = (int32_t)(a.Wcp[i + 1] - ib);
            uint16_t* mp = x.pmap + x.poff[spos];
            for (int32_t f = lane; f < ni; f += 32) {
                const uint16_t p = lookup(tb, a.Wr[ib + f] & kRowMask);
                mp[f] = p;
                nhit += p != kNone ? 1 : 0;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nhit += __shfl_xor_sync(0xffffffffu, nhit, o);
    if (lane == 0 && nhit) atomicAdd(hits, nhit);
}

__global__ void mmap_partner(int64_t n, const int8_t* __restrict__ pstart, int32_t* __restrict__ part) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const bool first = pstart[r] != 0;
        const bool two = first ? (r + 1 < n && pstart[r + 1] == 0) : true;
        part[r] = two ? (int32_t)(first ? r + 1 : r - 1) : -1;
    }
}

// ---- numeric kernels ----

// Streams the entries [0, count) of a column beside its map, 32 lanes wide with
// kUnrollM chunks of loads in flight.  In the last, partial block a chunk that is
// empty for the whole warp is skipped by a warp-uniform test, so no instruction of
// apply runs for it (on the FP64 pipe an idle lane costs as much as a busy one).
// load(e, p, v) reads entry e; apply(p, v) uses it when p != kNone.
// The same with every block predicated instead (no uniform branches): faster where the
// apply step is a cheap FP32 operation.
template <class V, class Load, class Apply>
__device__ __forceinline__ void stream_column_pred(int32_t count, int lane, Load load, Apply apply) {
    for (int32_t e0 = 0; e0 < count; e0 += 32 * kUnrollM) {
        uint16_t p[kUnrollM];
        V v[kUnrollM];
#pragma unroll
        for (int u = 0; u < kUnrollM; ++u) {
            const int32_t e = e0 + u * 32 + lane;
            p[u] = kNone;
            if (e < count) load(e, p[u], v[u]);
        }
#pragma unroll
        for (int u = 0; u < kUnrollM; ++u)
            if (p[u] != kNone) apply(p[u], v[u]);
    }
}

template <class V, class Load, class Apply>
__device__ __forceinline__ void stream_column(int32_t count, int lane, Load load, Apply apply) {
    int32_t e0 = 0;
    for (; e0 + 32 * kUnrollM <= count; e0 += 32 * kUnrollM) {
        uint16_t p[kUnrollM];
        V v[kUnrollM];
#pragma unroll
        for (int u = 0; u < kUnrollM; ++u) load(e0 + u * 32 + lane, p[u], v[u]);
#pragma unroll
        for (int u = 0; u < kUnrollM; ++u)
            if (p[u] != kNone) apply(p[u], v[u]);
    }
    if (e0 < count) {
        uint16_t p[kUnrollM];
        V v[kUnrollM];
#pragma unroll
        for (int u = 0; u < kUnrollM; ++u) {
            const int32_t e = e0 + u * 32 + lane;
            p[u] = kNone;
            if (e0 + u * 32 < count && e < count) load(e, p[u], v[u]);
        }
#pragma unroll
        for (int u = 0; u < kUnrollM; ++u) {
            if (e0 + u * 32 >= count) break;  // warp-uniform
            if (p[u] != kNone) apply(p[u], v[u]);
        }
    }
}


// ---- the product in pairs of floats (FP64-class accuracy on the FP32 pipes) ----
//
// A value x is carried as hi + lo with hi = fl32(x) and lo = fl32(x - hi).  The
// product of two pairs keeps hi_a hi_b exactly (its rounding error comes from a
// fused multiply-add) and adds both cross terms hi_a lo_b + lo_a hi_b; the sum
// runs as (s, c): s takes the high parts with an error-free two-sum and c
// collects every error term and low part in FP32 (its own rounding stays at the
// 2^-48 level relative to the terms).  These are the error-free transformations
// of double-word arithmetic: Knuth's two-sum and the product error obtained with
// a fused multiply-add (Dekker's exact product).  The intrinsics keep the
// compiler from contracting the two-sum.

__device__ __forceinline__ float2 split_pair(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ void pair_mac(float2 a, float2 b, float& s, float& c) {
    const float ph = __fmul_rn(a.x, b.x);
    float pl = __fmaf_rn(a.x, b.x, -ph);
    pl = __fmaf_rn(a.x, b.y, pl);
    pl = __fmaf_rn(a.y, b.x, pl);
    const float t = __fadd_rn(s, ph);
    const float v = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, v)), __fsub_rn(ph, v));
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, pl));
}

__device__ __forceinline__ void pair_add(float& s, float& c, float s2, float c2) {
    const float t = __fadd_rn(s, s2);
    const float v = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, v)), __fsub_rn(s2, v));
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, c2));
}

template <class T>
__device__ __forceinline__ T fma_m(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_m<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_m<float>(float a, float b, float c) { return fmaf(a, b, c); }

template <class T>
__global__ void __launch_bounds__(kThreads) hm_step(NinvArgs a, NinvMaps x, ColumnList cl, int t,
                                                    const T* __restrict__ Wp, T* __restrict__ Wn, int32_t* ticket) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* acc = reinterpret_cast<T*>(smem_raw);
    __shared__ int32_t s_j;
    const int G = a.m + 2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        const int64_t j = take_column(ticket, &s_j, cl);
        if (j < 0) break;
        const int64_t base = a.Wcp[j];
        const int32_t nt = a.grp[j * G + t + 1];  // rows of powers 0..t
        for (int32_t e = threadIdx.x; e < nt; e += kThreads) acc[e] = T(0);
        __syncthreads();
        for (int64_t q = a.Lcp[j] + wid; q < a.Lcp[j + 1]; q += kWarps) {
            const int32_t k = a.Lri[q];
            const T ekj = T(-a.Lval[a.Lcsr[q]]);
            const T* __restrict__ wk = Wp + a.Wcp[k];
            const uint16_t* __restrict__ mp = x.hmap + x.moff[q];
            const int32_t nk = a.grp[(int64_t)k * G + t];  // rows of powers 0..t-1
            stream_column<T>(
                nk, lane,
                [&](int32_t e, uint16_t& p, T& v) {
                    p = mp[e];
                    v = wk[e];
                },
                [&](uint16_t p, const T& v) {
                    if (in_range(a.status, p, 0, nt)) atomicAdd(acc + p, ekj * v);
                });
        }
        __syncthreads();
        for (int32_t e = threadIdx.x; e < nt; e += kThreads) {
            const T v = acc[e] + (e == 0 ? T(1) : T(0));
            Wn[base + e] = (e != 0 && fabs((double)v) < a.delta) ? T(0) : v;  // drop below the tolerance
        }
        __syncthreads();
    }
}

// FP64 Horner step with exact integer accumulation.  Column j of W_t is bounded a
// priori, |W_t[r, j]| <= B = 1 + sum_k |E_kj| max_r |W_{t-1}[r, k]| (every partial
// sum too), so on the grid 2^-s with s = 50 - ceil(log2 B) every product and every
// partial sum stays below 2^50 in grid units.  One fused multiply-add with the
// constant 1.5 * 2^52 rounds E_kj 2^s W[r, k] to the nearest grid point (a single
// rounding of the exact product) and leaves that integer in the low bits of the
// result; the integers are summed with 64-bit integer shared-memory atomics: an
// order-independent (bit-reproducible) sum, absolute error below
// (|struct(j)| + 1) 2^-(s+1) <= 2^-50 B per entry, and one FP64 operation per
// product.  The step also records max_r |W_t[r, j]| for the next step's bound.
__device__ __forceinline__ double scale_pow2(double v, int s) {
    // v * 2^-s for a normal v whose result stays normal, by the exponent field
    return v == 0.0 ? 0.0 : __longlong_as_double(__double_as_longlong(v) - ((long long)s << 52));
}

constexpr double kRoundMagic = 6755399441055744.0;  // 1.5 * 2^52: its ulp is 1

__global__ void __launch_bounds__(kThreads) hm_step_fx(NinvArgs a, NinvMaps x, ColumnList cl, int t,
                                                       const double* __restrict__ Wp,
                                                       double* __restrict__ Wn, float2* __restrict__ Wx,
                                                       const double* __restrict__ Mp, double* __restrict__ Mn,
                                                       int32_t* ticket) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem_raw);
    __shared__ int32_t s_j, s_s;
    __shared__ unsigned long long s_max;
    const int G = a.m + 2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        const int64_t j = take_column(ticket, &s_j, cl);
        if (j < 0) break;
        const int64_t base = a.Wcp[j];
        const int32_t nt = a.grp[j * G + t + 1];
        const int64_t q0 = a.Lcp[j], q1 = a.Lcp[j + 1];
        if (wid == 0) {
            double b = 0.0;
            for (int64_t q = q0 + lane; q < q1; q += 32) b += fabs(a.Lval[a.Lcsr[q]]) * Mp[a.Lri[q]];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
            if (lane == 0) {
                int ex;
                frexp(1.0 + b, &ex);  // 1 + b < 2^ex
                int sc = 50 - ex;
                if (sc < 0 || !(b < 1e300)) {  // W too large for the fixed-point range
                    set_status(a.status, ST_UNSUPPORTED);
                    sc = 0;
                }
                s_s = sc;
                s_max = 0ull;
            }
        }
        __syncthreads();
        const int sc = s_s;
        for (int32_t e = threadIdx.x; e < nt; e += kThreads) acc[e] = e == 0 ? (1ull << sc) : 0ull;
        __syncthreads();
        for (int64_t q = q0 + wid; q < q1; q += kWarps) {
            const int32_t k = a.Lri[q];
            const double ekj = -a.Lval[a.Lcsr[q]] * ldexp(1.0, sc);  // E_kj 2^s (exact)
            const long long magic = __double_as_longlong(kRoundMagic);
            const double* __restrict__ wk = Wp + a.Wcp[k];
            const uint16_t* __restrict__ mp = x.hmap + x.moff[q];
            const int32_t nk = a.grp[(int64_t)k * G + t];
            stream_column<double>(
                nk, lane,
                [&](int32_t e, uint16_t& p, double& v) {
                    p = mp[e];
                    v = wk[e];
                },
                [&](uint16_t p, const double& v) {
                    const long long q = __double_as_longlong(fma(ekj, v, kRoundMagic)) - magic;
                    if (in_range(a.status, p, 0, nt)) atomicAdd(acc + p, (unsigned long long)q);
                });
        }
        __syncthreads();
        unsigned long long mx = 0ull;
        for (int32_t e = threadIdx.x; e < nt; e += kThreads) {
            const long long iv = (long long)acc[e];
            const unsigned long long av = (unsigned long long)(iv < 0 ? -iv : iv);
            mx = av > mx ? av : mx;
            double v = scale_pow2(__ll2double_rn(iv), sc);
            if (e != 0 && fabs(v) < a.delta) v = 0.0;  // drop below the tolerance
            Wn[base + e] = v;
            if (Wx) Wx[base + e] = split_pair(v);  // for a product in pairs of floats
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, mx, o);
            mx = other > mx ? other : mx;
        }
        if (lane == 0) atomicMax(&s_max, mx);
        __syncthreads();
        if (threadIdx.x == 0) Mn[j] = scale_pow2(__ull2double_ru(s_max), sc);
        __syncthreads();
    }
}

__global__ void fx_init(double* __restrict__ M, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        M[j] = 1.0;  // W_0 = I
}

template <class T>
__global__ void __launch_bounds__(kThreads) pm_product(NinvArgs a, NinvMaps x, ColumnList cl, int tlim,
                                                       const T* __restrict__ W,
                                                       const double* __restrict__ dr, const double* __restrict__ dp,
                                                       double* __restrict__ N, int32_t* ticket) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* y = reinterpret_cast<T*>(smem_raw);
    __shared__ int32_t s_j;
    const int G = a.m + 2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        const int64_t j = take_column(ticket, &s_j, cl);
        if (j < 0) break;
        const int64_t base = a.Wcp[j];
        const int32_t ny = (int32_t)(a.Wcp[j + 1] - base) + x.ynx[j];
        const int32_t nt = a.grp[j * G + tlim + 1];
        for (int32_t e = threadIdx.x; e < ny; e += kThreads) y[e] = T(0);
        __syncthreads();
        // y = D^{-1} W[:, j] on the rows of powers <= tlim: two terms at most per position,
        // so the atomics give the same sum in any order
        for (int32_t e = threadIdx.x; e < nt; e += kThreads) {
            const int32_t rf = a.Wr[base + e];
            const int32_t r = rf & kRowMask;
            const double w = (double)W[base + e];
            atomicAdd(y + e, T(dr[r] * w));
            if ((rf & kTwoFlag) && in_range(a.status, x.ypart[base + e], 0, ny))
                atomicAdd(y + x.ypart[base + e], T(dp[r] * w));
        }
        __syncthreads();
        const bool two_first = a.pstart[j] != 0 && j + 1 < a.n && a.pstart[j + 1] == 0;
        const int64_t q0 = a.Lcp[j];
        const int64_t cnt = (a.Lcp[j + 1] - q0) + 1 + (two_first ? 1 : 0);
        for (int64_t e = wid; e < cnt; e += kWarps) {
            int64_t i, spos;
            if (e == 0) {
                i = j;
                spos = a.Srp[j + 1] - 1;
            } else if (two_first && e == 1) {
                i = j + 1;
                spos = a.Srp[j + 2] - 2;
            } else {
                const int64_t q = q0 + e - 1 - (two_first ? 1 : 0);
                i = a.Lri[q];
                spos = a.Srp[i] + ((int64_t)a.Lcsr[q] - a.Lrp[i]);
            }
            const T* __restrict__ wi = W + a.Wcp[i];
            const uint16_t* __restrict__ mp = x.pmap + x.poff[spos];
            const int32_t ni = a.grp[i * G + tlim + 1];
            T s = T(0);
            auto load = [&](int32_t e, uint16_t& p, T& v) {
                p = mp[e];
                v = wi[e];
            };
            auto apply = [&](uint16_t p, const T& v) {
                if (in_range(a.status, p, 0, ny)) s = fma_m<T>(v, y[p], s);
            };
            if constexpr (std::is_same<T, float>::value) stream_column_pred<T>(ni, lane, load, apply);
            else stream_column<T>(ni, lane, load, apply);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0 && in_range(a.status, spos, 0, a.nnzS)) N[spos] = (double)s;
        }
        __syncthreads();
    }
}

constexpr double kPairMax = 0x1p100;  // magnitude the pairs carry at full accuracy

// D^{-1} per row as pairs (inputs outside the range the pairs carry are reported)
__global__ void pair_prep(int64_t n, int32_t* status, const double* __restrict__ dr, const double* __restrict__ dp,
                          float2* __restrict__ drx, float2* __restrict__ dpx) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        if (!(fabs(dr[r]) < kPairMax) || !(fabs(dp[r]) < kPairMax)) set_status(status, ST_UNSUPPORTED);
        drx[r] = split_pair(dr[r]);
        dpx[r] = split_pair(dp[r]);
    }
}

// (s, c) -> normalised pair (hi, lo)
__device__ __forceinline__ float2 pair_norm(float s, float c) {
    const float h = __fadd_rn(s, c);
    return make_float2(h, __fsub_rn(c, __fsub_rn(h, s)));
}

// Product on S in pairs: y = D^{-1} W[:, j] formed in pairs with one writer per
// position, then the streamed sums of hp_step's arithmetic.
__global__ void __launch_bounds__(kThreads) pp_product(NinvArgs a, NinvMaps x, ColumnList cl, int tlim,
                                                       const float2* __restrict__ W, const float2* __restrict__ drx,
                                                       const float2* __restrict__ dpx, double* __restrict__ N,
                                                       int32_t* ticket) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* y = reinterpret_cast<float2*>(smem_raw);
    __shared__ int32_t s_j;
    const int G = a.m + 2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        const int64_t j = take_column(ticket, &s_j, cl);
        if (j < 0) break;
        const int64_t base = a.Wcp[j];
        const int32_t ny = (int32_t)(a.Wcp[j + 1] - base) + x.ynx[j];
        const int32_t nt = a.grp[j * G + tlim + 1];
        for (int32_t e = threadIdx.x; e < ny; e += kThreads) y[e] = make_float2(0.f, 0.f);
        __syncthreads();
        // y_r = dr_r W_rj + dp_r W_pj for the rows r of powers <= tlim (p the partner of r).
        // A partner p outside that prefix (a later row of the column, or an extra
        // position) has W_pj = 0, so y_p = dp W_rj has the single writer r.
        for (int32_t e = threadIdx.x; e < nt; e += kThreads) {
            const int32_t rf = a.Wr[base + e];
            const int32_t r = rf & kRowMask;
            const float2 w = W[base + e];
            float s = 0.f, c = 0.f;
            pair_mac(drx[r], w, s, c);
            if (rf & kTwoFlag) {
                const int32_t pp = x.ypart[base + e];
                if (pp < nt) {
                    pair_mac(dpx[r], W[base + pp], s, c);
                } else {
                    float s2 = 0.f, c2 = 0.f;
                    pair_mac(dpx[r], w, s2, c2);
                    y[pp] = pair_norm(s2, c2);
                }
            }
            y[e] = pair_norm(s, c);
        }
        __syncthreads();
        const bool two_first = a.pstart[j] != 0 && j + 1 < a.n && a.pstart[j + 1] == 0;
        const int64_t q0 = a.Lcp[j];
        const int64_t cnt = (a.Lcp[j + 1] - q0) + 1 + (two_first ? 1 : 0);
        for (int64_t e = wid; e < cnt; e += kWarps) {
            int64_t i, spos;
            if (e == 0) {
                i = j;
                spos = a.Srp[j + 1] - 1;
            } else if (two_first && e == 1) {
                i = j + 1;
                spos = a.Srp[j + 2] - 2;
            } else {
                const int64_t q = q0 + e - 1 - (two_first ? 1 : 0);
                i = a.Lri[q];
                spos = a.Srp[i] + ((int64_t)a.Lcsr[q] - a.Lrp[i]);
            }
            const float2* __restrict__ wi = W + a.Wcp[i];
            const uint16_t* __restrict__ mp = x.pmap + x.poff[spos];
            const int32_t ni = a.grp[i * G + tlim + 1];
            float s = 0.f, c = 0.f;
            stream_column<float2>(
                ni, lane,
                [&](int32_t e, uint16_t& p, float2& v) {
                    p = mp[e];
                    v = wi[e];
                },
                [&](uint16_t p, const float2& v) { pair_mac(v, y[p], s, c); });
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                pair_add(s, c, __shfl_xor_sync(0xffffffffu, s, o), __shfl_xor_sync(0xffffffffu, c, o));
            if (lane == 0) N[spos] = (double)s + (double)c;
        }
        __syncthreads();
    }
}

__global__ void hp_init(const int64_t* __restrict__ Wcp, float2* __restrict__ W, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        W[Wcp[j]] = make_float2(1.f, 0.f);
}

template <class T>
__global__ void hm_init(const int64_t* __restrict__ Wcp, T* __restrict__ W, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        W[Wcp[j]] = T(1);
}

template <int kSlots>
constexpr size_t table_smem() { return sizeof(TableSmem<kSlots>); }
// accumulator / y table of a column: short columns, or long ones (one CTA per SM)
template <class T>
constexpr size_t acc_smem(bool lng) { return (size_t)(lng ? kIdxEntLong : kIdxEnt) * sizeof(T); }

// Runs f(list, long?, grid, ticket offset) over the short columns, then the long ones.
template <class F>
void for_lists(const NinvMaps& x, int num_sms, F f) {
    f(ColumnList{x.cols, x.n_short}, false, num_sms * 4, 0);
    if (x.n_long) f(ColumnList{x.cols + x.n_short, x.n_long}, true, num_sms, 64);
}

constexpr int kTickets = 128;  // per launch site: [0, 64) short columns, [64, 128) long columns

template <class T>
cudaError_t map_run(const NinvArgs& a, const NinvMaps& x, void* work, double* N_out, double* N_stack,
                    cudaStream_t st) {
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
    int32_t* tickets = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * kTickets));
    double* M0 = reinterpret_cast<double*>(take((size_t)a.n * sizeof(double)));  // column bounds (FP64)
    double* M1 = reinterpret_cast<double*>(take((size_t)a.n * sizeof(double)));
    cudaError_t e = cudaMemsetAsync(tickets, 0, sizeof(int32_t) * kTickets, st);
    if (e != cudaSuccess) return e;
    trace_begin("ninv_dinv", st);
    ninv_dinv_launch(a, dr, dp, part, st);
    trace_end(st);
    trace_begin("ninv_init", st);
    hm_init<T><<<a.num_sms * 4, 256, 0, st>>>(a.Wcp, W0, a.n);
    if constexpr (std::is_same<T, double>::value) fx_init<<<a.num_sms * 4, 256, 0, st>>>(M0, a.n);
    trace_end(st);
    T* cur = W0;
    T* nxt = W1;
    auto product = [&](int t, double* out, int tk) {
        trace_begin("ninv_map_product", st);
        for_lists(x, a.num_sms, [&](ColumnList cl, bool lng, int grid, int off) {
            pm_product<T><<<grid, kThreads, acc_smem<T>(lng), st>>>(a, x, cl, t, cur, dr, dp, out,
                                                                    tickets + off + tk);
        });
        trace_end(st);
    };
    if (N_stack) product(0, N_stack, 62 - a.m);
    for (int t = 1; t <= a.m; ++t) {
        trace_begin("ninv_map_horner", st);
        for_lists(x, a.num_sms, [&](ColumnList cl, bool lng, int grid, int off) {
            if constexpr (std::is_same<T, double>::value)
                hm_step_fx<<<grid, kThreads, acc_smem<double>(lng), st>>>(a, x, cl, t, cur, nxt, nullptr, M0, M1,
                                                                          tickets + off + t);
            else
                hm_step<T><<<grid, kThreads, acc_smem<T>(lng), st>>>(a, x, cl, t, cur, nxt, tickets + off + t);
        });
        trace_end(st);
        std::swap(cur, nxt);
        std::swap(M0, M1);
        if (N_stack && t < a.m) product(t, N_stack + (int64_t)t * a.nnzS, 62 - a.m + t);
    }
    product(a.m, N_stack ? N_stack + (int64_t)a.m * a.nnzS : N_out, 63);
    return cudaGetLastError();
}

// Pair form: the FP64 fixed-point Horner steps also write W as pairs of floats
// where a product follows; the product on S runs in double-float arithmetic.
cudaError_t pair_run(const NinvArgs& a, const NinvMaps& x, void* work, double* N_out, double* N_stack,
                     cudaStream_t st) {
    char* p = reinterpret_cast<char*>(work);
    auto take = [&](size_t bytes) {
        char* r = p;
        p += (bytes + 255) & ~(size_t)255;
        return r;
    };
    double* W0 = reinterpret_cast<double*>(take((size_t)a.nnzW * sizeof(double)));
    double* W1 = reinterpret_cast<double*>(take((size_t)a.nnzW * sizeof(double)));
    double* dr = reinterpret_cast<double*>(take((size_t)a.n * sizeof(double)));
    double* dp = reinterpret_cast<double*>(take((size_t)a.n * sizeof(double)));
    int32_t* part = reinterpret_cast<int32_t*>(take((size_t)a.n * sizeof(int32_t)));
    int32_t* tickets = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * kTickets));
    float2* Wx = reinterpret_cast<float2*>(take((size_t)a.nnzW * sizeof(float2)));
    float2* drx = reinterpret_cast<float2*>(take((size_t)a.n * sizeof(float2)));
    float2* dpx = reinterpret_cast<float2*>(take((size_t)a.n * sizeof(float2)));
    double* M0 = reinterpret_cast<double*>(take((size_t)a.n * sizeof(double)));
    double* M1 = reinterpret_cast<double*>(take((size_t)a.n * sizeof(double)));
    cudaError_t e = cudaMemsetAsync(tickets, 0, sizeof(int32_t) * kTickets, st);
    if (e != cudaSuccess) return e;
    trace_begin("ninv_dinv", st);
    ninv_dinv_launch(a, dr, dp, part, st);
    trace_end(st);
    trace_begin("ninv_pair_prep", st);
    pair_prep<<<a.num_sms * 4, 256, 0, st>>>(a.n, a.status, dr, dp, drx, dpx);
    trace_end(st);
    trace_begin("ninv_init", st);
    hm_init<double><<<a.num_sms * 4, 256, 0, st>>>(a.Wcp, W0, a.n);
    hp_init<<<a.num_sms * 4, 256, 0, st>>>(a.Wcp, Wx, a.n);
    fx_init<<<a.num_sms * 4, 256, 0, st>>>(M0, a.n);
    trace_end(st);
    double* cur = W0;
    double* nxt = W1;
    auto product = [&](int t, double* out, int tk) {
        trace_begin("ninv_pair_product", st);
        for_lists(x, a.num_sms, [&](ColumnList cl, bool lng, int grid, int off) {
            pp_product<<<grid, kThreads, acc_smem<double>(lng), st>>>(a, x, cl, t, Wx, drx, dpx, out,
                                                                      tickets + off + tk);
        });
        trace_end(st);
    };
    if (N_stack) product(0, N_stack, 62 - a.m);
    for (int t = 1; t <= a.m; ++t) {
        const bool pairs = t == a.m || N_stack != nullptr;
        trace_begin("ninv_map_horner", st);
        for_lists(x, a.num_sms, [&](ColumnList cl, bool lng, int grid, int off) {
            hm_step_fx<<<grid, kThreads, acc_smem<double>(lng), st>>>(a, x, cl, t, cur, nxt, pairs ? Wx : nullptr,
                                                                      M0, M1, tickets + off + t);
        });
        trace_end(st);
        std::swap(cur, nxt);
        std::swap(M0, M1);
        if (N_stack && t < a.m) product(t, N_stack + (int64_t)t * a.nnzS, 62 - a.m + t);
    }
    product(a.m, N_stack ? N_stack + (int64_t)a.m * a.nnzS : N_out, 63);
    return cudaGetLastError();
}

}  // namespace

size_t ninv_map_work_bytes(const NinvArgs& a, int prec) {
    const size_t ts = prec == 1 ? sizeof(float) : sizeof(double);  // a pair of floats is 8 bytes too
    const size_t pairs = prec == 2 ? ((size_t)a.nnzW + 2 * (size_t)a.n) * sizeof(float2) + 3 * 256 : 0;
    const size_t bounds = 2 * ((size_t)a.n * sizeof(double) + 256);
    return 2 * ((size_t)a.nnzW * ts + 256) + (size_t)a.n * (2 * sizeof(double) + sizeof(int32_t)) + 3 * 256 +
           sizeof(int32_t) * kTickets + 256 + pairs + bounds + 4096;
}

cudaError_t ninv_map_launch(const NinvArgs& a, const NinvMaps& x, int prec, void* work, double* N_out,
                            cudaStream_t st, double* N_stack) {
    if (a.n == 0) return cudaSuccess;
    if (prec == 1) return map_run<float>(a, x, work, N_out, N_stack, st);
    if (prec == 2) return pair_run(a, x, work, N_out, N_stack, st);
    return map_run<double>(a, x, work, N_out, N_stack, st);
}

void ninv_maps_free(NinvMaps& x) {
    void* ptrs[] = {x.moff, x.hmap, x.poff, x.pmap, x.ypart, x.ynx, x.cols};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    x = NinvMaps();
}

cudaError_t ninv_maps_configure() {
    struct {
        const void* f;
        size_t bytes;
    } ks[] = {
        {(const void*)hmap_build<kSlotsShort>, table_smem<kSlotsShort>()},
        {(const void*)pmap_build<kSlotsShort>, table_smem<kSlotsShort>()},
        {(const void*)hmap_build<kSlotsLong>, table_smem<kSlotsLong>()},
        {(const void*)pmap_build<kSlotsLong>, table_smem<kSlotsLong>()},
        {(const void*)hm_step_fx, acc_smem<double>(true)},
        {(const void*)hm_step<float>, acc_smem<float>(true)},
        {(const void*)pm_product<double>, acc_smem<double>(true)},
        {(const void*)pm_product<float>, acc_smem<float>(true)},
        {(const void*)pp_product, acc_smem<double>(true)},
    };
    for (const auto& k : ks) {
        const cudaError_t e = cudaFuncSetAttribute(k.f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

std::string ninv_maps_build(const NinvArgs& a, const HostPlan& P, const NinvPlan& Wp, int64_t budget,
                            NinvMaps& x, cudaStream_t st, cudaError_t& err) {
    err = cudaSuccess;
    ninv_maps_free(x);
    const int64_t n = a.n;
    const int G = a.m + 2;
    // every column with its partner rows must fit a table: |col j| + 2x2 rows <= kIdxEnt
    // (short columns), else <= kIdxEntLong (long columns, one CTA per SM)
    std::vector<int32_t> cols_short, cols_long;
    for (int64_t j = 0; j < n; ++j) {
        int64_t c = 0;
        for (int64_t e = Wp.Wcp[j]; e < Wp.Wcp[j + 1]; ++e) c += (Wp.Wr[e] & kTwoFlag) ? 1 : 0;
        const int64_t need = Wp.Wcp[j + 1] - Wp.Wcp[j] + c;
        if (need > kIdxEntLong) return "a column of the series pattern exceeds the map tables";
        (need > kIdxEnt ? cols_long : cols_short).push_back((int32_t)j);
    }
    std::vector<int64_t> moff(P.nnzL + 1, 0), poff(P.nnzS + 1, 0);
    for (int64_t q = 0; q < P.nnzL; ++q) moff[q + 1] = moff[q] + Wp.grp[(int64_t)P.Lri[q] * G + a.m];
    for (int64_t i = 0; i < n; ++i) {
        const int64_t len = Wp.Wcp[i + 1] - Wp.Wcp[i];
        for (int64_t q = P.Srp[i]; q < P.Srp[i + 1]; ++q) poff[q + 1] = len;
    }
    for (int64_t q = 0; q < P.nnzS; ++q) poff[q + 1] += poff[q];
    const int64_t bytes = (P.nnzL + 1) * 8 + moff[P.nnzL] * 2 + (P.nnzS + 1) * 8 + poff[P.nnzS] * 2 +
                          a.nnzW * 2 + n * 8;
    if (budget > 0 && bytes > budget) return "maps exceed the memory budget";
    auto alloc = [&](void** ptr, size_t b) { return cudaMalloc(ptr, std::max<size_t>(b, 16)); };
    int32_t* part = nullptr;
    int32_t* tk = nullptr;  // 16 column tickets, then the hit counter
    auto fail = [&](cudaError_t e, const char* what) {
        err = e;
        if (part) cudaFree(part);
        if (tk) cudaFree(tk);
        ninv_maps_free(x);
        return std::string(what) + ": " + cudaGetErrorString(e);
    };
    cudaError_t e;
    if ((e = alloc((void**)&x.moff, moff.size() * 8)) != cudaSuccess ||
        (e = alloc((void**)&x.hmap, moff[P.nnzL] * 2)) != cudaSuccess ||
        (e = alloc((void**)&x.poff, poff.size() * 8)) != cudaSuccess ||
        (e = alloc((void**)&x.pmap, poff[P.nnzS] * 2)) != cudaSuccess ||
        (e = alloc((void**)&x.ypart, a.nnzW * 2)) != cudaSuccess ||
        (e = alloc((void**)&x.ynx, n * 4)) != cudaSuccess || (e = alloc((void**)&x.cols, n * 4)) != cudaSuccess ||
        (e = alloc((void**)&part, n * 4)) != cudaSuccess || (e = alloc((void**)&tk, 128)) != cudaSuccess)
        return fail(e, "map alloc");
    x.n_short = (int64_t)cols_short.size();
    x.n_long = (int64_t)cols_long.size();
    cols_short.insert(cols_short.end(), cols_long.begin(), cols_long.end());
    if ((e = cudaMemcpyAsync(x.moff, moff.data(), moff.size() * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(x.poff, poff.data(), poff.size() * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(x.cols, cols_short.data(), n * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(tk, 0, 128, st)) != cudaSuccess)
        return fail(e, "map upload");
    const ColumnList cs{x.cols, x.n_short}, cl{x.cols + x.n_short, x.n_long};
    unsigned long long* dhits = reinterpret_cast<unsigned long long*>(tk + 16);
    mmap_partner<<<a.num_sms * 4, 256, 0, st>>>(n, a.pstart, part);
    if (a.m > 0) {
        hmap_build<kSlotsShort><<<a.num_sms * 2, kThreads, table_smem<kSlotsShort>(), st>>>(a, x, cs, tk);
        if (x.n_long) hmap_build<kSlotsLong><<<a.num_sms, kThreads, table_smem<kSlotsLong>(), st>>>(a, x, cl, tk + 1);
    }
    pmap_build<kSlotsShort><<<a.num_sms * 2, kThreads, table_smem<kSlotsShort>(), st>>>(a, x, part, cs, tk + 2, dhits);
    if (x.n_long)
        pmap_build<kSlotsLong><<<a.num_sms, kThreads, table_smem<kSlotsLong>(), st>>>(a, x, part, cl, tk + 3, dhits);
    unsigned long long nh = 0;
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(&nh, dhits, sizeof(nh), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(e, "map build");
    x.hits = (int64_t)nh;
    cudaFree(part);
    cudaFree(tk);
    x.m = a.m;
    x.nmap_h = moff[P.nnzL];
    x.nmap_p = poff[P.nnzS];
    x.bytes = bytes;
    x.ready = true;
    return std::string();
}

}  // namespace sinv
