// NInv in gather form (Section 2.2, Eqs. (6) and (8)).  The same arithmetic as
// the hash form in ninv.cu, with the sparse-sparse structure resolved once per
// pattern and m, so that a numeric call is a stream of gathers and fused
// multiply-adds with no searching.
//
// Horner step W_t[r, j] = [r == j] + sum_{k in struct(j)} E_kj W_{t-1}[r, k].
// Every target entry (r, j) of P_W has a list of sources, one per column k of
// struct(j) whose truncated column W_{t-1}[:, k] holds row r.  A source is the
// 32-bit word  slot << 24 | offset : slot = position of k in struct(j) (E_kj and
// the start of column k are staged per column), offset = position of r in
// column k.  A target's sources are ordered by the first power g that reaches r
// from k, then by slot, so step t uses the prefix with g <= t - 1 and every sum
// runs in a fixed order.  Targets are laid out by columns in slices of 32 (one
// per lane); inside a column's group of first power they are sorted by their
// source count, so the lanes of a slice run nearly the same number of terms.
// Slice s keeps its words lane-interleaved: word i of lane l at sb[s] + 32 i + l.
//
// Product N_ij = sum_r W_ri (D^{-1} W)_rj for (i, j) in S_lo: every entry of S_lo
// has the list of rows it meets, as words  pos_i | pos_j << 16 | partner << 31.
// A plain word is a row r in both columns (term (D^{-1})_rr W_ri W_rj, with
// V = diag(D^{-1}) W written by the last Horner step); a partner word is a row r
// of column i in a 2x2 block whose partner p is in column j (term
// (D^{-1})_rp W_ri W_pj).  A warp reduces one entry, lanes over its words.
//
// The index is built on the GPU (count, layout, fill) and needs the columns of
// P_W to fit a shared-memory table (max column <= kIdxEnt) and |struct(j)| <= 255.
#include <algorithm>
#include <vector>

#include "device.cuh"
#include "hash.cuh"
#include "kernels.h"
#include "plan.h"

namespace sinv {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kIdxSlots = 8192;               // hash slots of the build kernels
constexpr int kUnrollG = 4;                   // words per lane in flight (numeric kernels)
constexpr int32_t kRowMask = 0x7FFFFFFF;
constexpr int32_t kTwoFlag = (int32_t)0x80000000u;
constexpr uint16_t kPad = 0xFFFF;             // lane of a slice without a target
constexpr uint32_t kOffMask = 0xFFFFFFu;

__device__ __forceinline__ int64_t take_column(int32_t* ticket, int32_t* s_j) {
    if (threadIdx.x == 0) *s_j = atomicAdd(ticket, 1);
    __syncthreads();
    const int64_t j = *s_j;
    __syncthreads();
    return j;
}

// Table of the rows of column j (all groups): row -> local position.
__device__ __forceinline__ void build_table(const NinvArgs& a, int64_t base, int32_t nj, int32_t* keys,
                                            int16_t* loc) {
    for (int s = threadIdx.x; s < kIdxSlots; s += kThreads) keys[s] = -1;
    __syncthreads();
    for (int32_t e = threadIdx.x; e < nj; e += kThreads) {
        const uint32_t h = table_insert(keys, kIdxSlots - 1, a.Wr[base + e] & kRowMask);
        loc[h] = (int16_t)e;
    }
    __syncthreads();
}

struct BuildSmem {
    int32_t keys[kIdxSlots];
    int16_t loc[kIdxSlots];
    int32_t cnt[kIdxEnt];     // per target: sources of the current power (count), fill position (fill)
    int16_t inv[kIdxEnt];     // per target: its place in the column's slice order (fill)
};

// Pass 1: per target and power g < m, the number of sources in group g of their column k.
__global__ void __launch_bounds__(kThreads) hidx_count(NinvArgs a, int32_t* ticket, uint8_t* cntg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BuildSmem& sm = *reinterpret_cast<BuildSmem*>(smem_raw);
    __shared__ int32_t s_j;
    const int G = a.m + 2;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        const int64_t j = take_column(ticket, &s_j);
        if (j >= a.n) break;
        const int64_t base = a.Wcp[j];
        const int32_t nj = (int32_t)(a.Wcp[j + 1] - base);
        build_table(a, base, nj, sm.keys, sm.loc);
        const int64_t q0 = a.Lcp[j];
        const int32_t ns = (int32_t)(a.Lcp[j + 1] - q0);
        for (int g = 0; g < a.m; ++g) {
            for (int32_t e = threadIdx.x; e < nj; e += kThreads) sm.cnt[e] = 0;
            __syncthreads();
            for (int32_t s = wid; s < ns; s += kWarps) {
                const int32_t k = a.Lri[q0 + s];
                const int64_t kb = a.Wcp[k];
                const int32_t e1 = a.grp[(int64_t)k * G + g + 1];
                for (int32_t e = a.grp[(int64_t)k * G + g] + lane; e < e1; e += 32) {
                    const int32_t h = table_find(sm.keys, kIdxSlots - 1, a.Wr[kb + e] & kRowMask);
                    if (h >= 0) atomicAdd(&sm.cnt[sm.loc[h]], 1);
                    else set_status(a.status, ST_INTERNAL);
                }
            }
            __syncthreads();
            for (int32_t e = threadIdx.x; e < nj; e += kThreads) cntg[(base + e) * a.m + g] = (uint8_t)sm.cnt[e];
            __syncthreads();
        }
    }
}

// Pass 2: slice order of every column (targets sorted by source count inside each
// group of first power), per-step counts in slice order, width of every slice.
__global__ void __launch_bounds__(kThreads) hidx_layout(NinvArgs a, NinvIndex x, const uint8_t* __restrict__ cntg,
                                                        int32_t* ticket, int32_t* width) {
    __shared__ int32_t hist[256];
    __shared__ int32_t s_j;
    const int G = a.m + 2;
    const int lane = threadIdx.x & 31;
    const int64_t NL = x.nslices * 32;
    for (;;) {
        const int64_t j = take_column(ticket, &s_j);
        if (j >= a.n) break;
        const int64_t base = a.Wcp[j];
        const int32_t nj = (int32_t)(a.Wcp[j + 1] - base);
        const int64_t l0 = x.cs[j] * 32;                  // first slice lane of the column
        const int32_t nl = (int32_t)((x.cs[j + 1] - x.cs[j]) * 32);
        auto total = [&](int32_t e) {
            int c = 0;
            for (int g = 0; g < a.m; ++g) c += cntg[(base + e) * a.m + g];
            return c;
        };
        for (int gp = 0; gp <= a.m; ++gp) {
            const int32_t b0 = a.grp[j * G + gp], b1 = a.grp[j * G + gp + 1];
            if (b0 == b1) continue;
            for (int c = threadIdx.x; c < 256; c += kThreads) hist[c] = 0;
            __syncthreads();
            for (int32_t e = b0 + threadIdx.x; e < b1; e += kThreads) atomicAdd(&hist[total(e)], 1);
            __syncthreads();
            if (threadIdx.x == 0) {  // start of every count, largest count first
                int32_t run = 0;
                for (int c = 255; c >= 0; --c) {
                    const int32_t h = hist[c];
                    hist[c] = run;
                    run += h;
                }
            }
            __syncthreads();
            for (int32_t e = b0 + threadIdx.x; e < b1; e += kThreads)
                x.tloc[l0 + b0 + atomicAdd(&hist[total(e)], 1)] = (uint16_t)e;
            __syncthreads();
        }
        for (int32_t p = nj + threadIdx.x; p < nl; p += kThreads) x.tloc[l0 + p] = kPad;
        __syncthreads();
        // nl is a multiple of 32 and kThreads of 32: warp w holds whole slices
        for (int32_t p0 = threadIdx.x - lane; p0 < nl; p0 += kThreads) {
            const int32_t p = p0 + lane;
            const uint16_t tl = x.tloc[l0 + p];
            int c = 0;
            for (int t = 1; t <= a.m; ++t) {
                if (tl != kPad) c += cntg[(base + tl) * a.m + (t - 1)];
                x.scnt[(int64_t)(t - 1) * NL + l0 + p] = (uint8_t)c;
            }
            const int wmax = __reduce_max_sync(0xffffffffu, (unsigned)c);
            if (lane == 0) width[x.cs[j] + p0 / 32] = wmax;
        }
        __syncthreads();
    }
}

// Pass 3: the source words, by power, then slot (one writer per target and slot).
__global__ void __launch_bounds__(kThreads) hidx_fill(NinvArgs a, NinvIndex x, int32_t* ticket) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BuildSmem& sm = *reinterpret_cast<BuildSmem*>(smem_raw);
    __shared__ int32_t s_j;
    const int G = a.m + 2;
    for (;;) {
        const int64_t j = take_column(ticket, &s_j);
        if (j >= a.n) break;
        const int64_t base = a.Wcp[j];
        const int32_t nj = (int32_t)(a.Wcp[j + 1] - base);
        build_table(a, base, nj, sm.keys, sm.loc);
        const int64_t l0 = x.cs[j] * 32;
        for (int32_t p = threadIdx.x; p < nj; p += kThreads) {
            sm.inv[x.tloc[l0 + p]] = (int16_t)p;
            sm.cnt[p] = 0;
        }
        __syncthreads();
        const int64_t q0 = a.Lcp[j];
        const int32_t ns = (int32_t)(a.Lcp[j + 1] - q0);
        for (int g = 0; g < a.m; ++g) {
            for (int32_t s = 0; s < ns; ++s) {
                const int32_t k = a.Lri[q0 + s];
                const int64_t kb = a.Wcp[k];
                const int32_t e1 = a.grp[(int64_t)k * G + g + 1];
                for (int32_t e = a.grp[(int64_t)k * G + g] + threadIdx.x; e < e1; e += kThreads) {
                    const int32_t h = table_find(sm.keys, kIdxSlots - 1, a.Wr[kb + e] & kRowMask);
                    if (h < 0) {
                        set_status(a.status, ST_INTERNAL);
                        continue;
                    }
                    const int32_t tl = sm.loc[h];
                    const int32_t p = sm.inv[tl];
                    const int32_t i = sm.cnt[tl]++;
                    const int64_t sl = x.cs[j] + p / 32;
                    x.src[x.sb[sl] + (int64_t)i * 32 + (p & 31)] = ((uint32_t)s << 24) | (uint32_t)e;
                }
                __syncthreads();
            }
        }
    }
}

// The S_lo entries of column j: the diagonal, the 2x2 partner row, struct(j).
struct ColumnEntries {
    int64_t q0, cnt;
    bool two_first;
    __device__ ColumnEntries(const NinvArgs& a, int64_t j) {
        two_first = a.pstart[j] != 0 && j + 1 < a.n && a.pstart[j + 1] == 0;
        q0 = a.Lcp[j];
        cnt = (a.Lcp[j + 1] - q0) + 1 + (two_first ? 1 : 0);
    }
    __device__ void get(const NinvArgs& a, int64_t j, int64_t e, int64_t& i, int64_t& spos) const {
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
    }
};

// Product index: count (out == nullptr) or write the words of every entry of S_lo.
__global__ void __launch_bounds__(kThreads) pidx_pass(NinvArgs a, NinvIndex x, const int32_t* __restrict__ part,
                                                      int32_t* ticket, int32_t* count, uint32_t* out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BuildSmem& sm = *reinterpret_cast<BuildSmem*>(smem_raw);
    __shared__ int32_t s_j;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (;;) {
        const int64_t j = take_column(ticket, &s_j);
        if (j >= a.n) break;
        const int64_t jb = a.Wcp[j];
        build_table(a, jb, (int32_t)(a.Wcp[j + 1] - jb), sm.keys, sm.loc);
        const ColumnEntries ce(a, j);
        for (int64_t e = wid; e < ce.cnt; e += kWarps) {
            int64_t i, spos;
            ce.get(a, j, e, i, spos);
            const int64_t ib = a.Wcp[i];
            const int32_t ni = (int32_t)(a.Wcp[i + 1] - ib);
            int64_t o = out ? x.hoff[spos] : 0;
            int32_t c = 0;
            for (int32_t f0 = 0; f0 < ni; f0 += 32) {
                const int32_t f = f0 + lane;
                int32_t hm = -1, hp = -1;
                if (f < ni) {
                    const int32_t rf = a.Wr[ib + f];
                    const int32_t r = rf & kRowMask;
                    hm = table_find(sm.keys, kIdxSlots - 1, r);
                    if ((rf & kTwoFlag) && part[r] >= 0) hp = table_find(sm.keys, kIdxSlots - 1, part[r]);
                }
                const uint32_t bm = __ballot_sync(0xffffffffu, hm >= 0);
                const uint32_t bp = __ballot_sync(0xffffffffu, hp >= 0);
                if (out) {
                    if (hm >= 0) out[o + __popc(bm & lt)] = (uint32_t)f | ((uint32_t)sm.loc[hm] << 16);
                    o += __popc(bm);
                    if (hp >= 0) out[o + __popc(bp & lt)] = (uint32_t)f | ((uint32_t)sm.loc[hp] << 16) | 0x80000000u;
                    o += __popc(bp);
                }
                c += __popc(bm) + __popc(bp);
            }
            if (!out && lane == 0) count[spos] = c;
        }
        __syncthreads();
    }
}

// partner row of every row in a 2x2 pivot block, -1 for 1x1 pivots
__global__ void hidx_partner(int64_t n, const int8_t* __restrict__ pstart, int32_t* __restrict__ part) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const bool first = pstart[r] != 0;
        const bool two = first ? (r + 1 < n && pstart[r + 1] == 0) : true;
        part[r] = two ? (int32_t)(first ? r + 1 : r - 1) : -1;
    }
}

// ---- numeric kernels ----

template <class T>
__device__ __forceinline__ T fma_g(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_g<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_g<float>(float a, float b, float c) { return fmaf(a, b, c); }

// One Horner step W_t = I + E W_{t-1} on every target (targets beyond power t get 0).
// A warp owns a column: it stages E_kj and the start of column k per slot, then runs
// the column's slices, one target per lane.  V (optional) receives diag(D^{-1}) W_t.
template <class T>
__global__ void __launch_bounds__(kThreads) hg_step(NinvArgs a, NinvIndex x, int t, const T* __restrict__ Wp,
                                                    T* __restrict__ Wn, T* __restrict__ V,
                                                    const double* __restrict__ dr, int32_t* ticket) {
    __shared__ int64_t s_kb[kWarps][256];
    __shared__ T s_cf[kWarps][256];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint8_t* __restrict__ cnt_t = x.scnt + (int64_t)(t - 1) * x.nslices * 32;
    int64_t* kb = s_kb[wid];
    T* cf = s_cf[wid];
    for (;;) {
        int32_t jj = 0;
        if (lane == 0) jj = atomicAdd(ticket, 1);
        const int64_t j = __shfl_sync(0xffffffffu, jj, 0);
        if (j >= a.n) break;
        const int64_t q0 = a.Lcp[j];
        const int32_t ns = (int32_t)(a.Lcp[j + 1] - q0);
        for (int32_t s = lane; s < ns; s += 32) {
            kb[s] = a.Wcp[a.Lri[q0 + s]];
            cf[s] = T(-a.Lval[a.Lcsr[q0 + s]]);
        }
        __syncwarp();
        const int64_t base = a.Wcp[j];
        for (int64_t sl = x.cs[j]; sl < x.cs[j + 1]; ++sl) {
            const int64_t li = sl * 32 + lane;
            const uint16_t tl = x.tloc[li];
            const int32_t c = cnt_t[li];
            const int32_t iters = (int32_t)__reduce_max_sync(0xffffffffu, (unsigned)c);
            const uint32_t* __restrict__ sp = x.src + x.sb[sl] + lane;
            T acc = tl == 0 ? T(1) : T(0);  // local position 0 is row j (power 0)
            int32_t i = 0;
            for (; i + kUnrollG <= iters; i += kUnrollG) {
                uint32_t w[kUnrollG];
                T v[kUnrollG];
#pragma unroll
                for (int u = 0; u < kUnrollG; ++u) w[u] = i + u < c ? sp[(int64_t)(i + u) * 32] : 0u;
#pragma unroll
                for (int u = 0; u < kUnrollG; ++u) v[u] = i + u < c ? Wp[kb[w[u] >> 24] + (w[u] & kOffMask)] : T(0);
#pragma unroll
                for (int u = 0; u < kUnrollG; ++u)
                    if (i + u < c) acc = fma_g<T>(cf[w[u] >> 24], v[u], acc);
            }
            for (; i < iters; ++i) {
                if (i < c) {
                    const uint32_t w = sp[(int64_t)i * 32];
                    acc = fma_g<T>(cf[w >> 24], Wp[kb[w >> 24] + (w & kOffMask)], acc);
                }
            }
            if (tl != kPad) {
                const int64_t p = base + tl;
                Wn[p] = acc;
                if (V) V[p] = T(dr[a.Wr[p] & kRowMask] * (double)acc);
            }
        }
        __syncwarp();
    }
}

// V = diag(D^{-1}) W on the whole pattern (the product after 0 steps).
template <class T>
__global__ void hg_scale(NinvArgs a, const T* __restrict__ W, const double* __restrict__ dr, T* __restrict__ V) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.nnzW; p += (int64_t)gridDim.x * blockDim.x)
        V[p] = T(dr[a.Wr[p] & kRowMask] * (double)W[p]);
}

// N on S_lo: one warp per entry, lanes over its words.
template <class T>
__global__ void __launch_bounds__(kThreads) pg_product(NinvArgs a, NinvIndex x, const T* __restrict__ W,
                                                       const T* __restrict__ V, const double* __restrict__ dp,
                                                       double* __restrict__ N) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * kWarps;
    for (int64_t sp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); sp < a.nnzS; sp += nw) {
        const int64_t ib = a.Wcp[x.Srow[sp]], jb = a.Wcp[a.Sc[sp]];
        const int64_t h1 = x.hoff[sp + 1];
        T acc = T(0);
        for (int64_t h0 = x.hoff[sp]; h0 < h1; h0 += 32 * kUnrollG) {
            uint32_t w[kUnrollG];
#pragma unroll
            for (int u = 0; u < kUnrollG; ++u) {
                const int64_t h = h0 + u * 32 + lane;
                w[u] = h < h1 ? x.hits[h] : 0xFFFFFFFFu;
            }
#pragma unroll
            for (int u = 0; u < kUnrollG; ++u) {
                if (w[u] == 0xFFFFFFFFu) continue;
                const int64_t pi = ib + (w[u] & 0xFFFFu), pj = jb + ((w[u] >> 16) & 0x7FFFu);
                T vi;
                if (!(w[u] & 0x80000000u)) vi = V[pi];
                else vi = T(dp[a.Wr[pi] & kRowMask] * (double)W[pi]);
                acc = fma_g<T>(vi, W[pj], acc);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) N[sp] = (double)acc;
    }
}

template <class T>
__global__ void hg_init(const int64_t* __restrict__ Wcp, T* __restrict__ W, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        W[Wcp[j]] = T(1);
}

constexpr size_t kBuildSmem = sizeof(BuildSmem);

template <class T>
cudaError_t gather_run(const NinvArgs& a, const NinvIndex& x, void* work, double* N_out, double* N_stack,
                       cudaStream_t st) {
    char* p = reinterpret_cast<char*>(work);
    auto take = [&](size_t bytes) {
        char* r = p;
        p += (bytes + 255) & ~(size_t)255;
        return r;
    };
    T* W0 = reinterpret_cast<T*>(take((size_t)a.nnzW * sizeof(T)));
    T* W1 = reinterpret_cast<T*>(take((size_t)a.nnzW * sizeof(T)));
    T* V = reinterpret_cast<T*>(take((size_t)a.nnzW * sizeof(T)));
    double* dr = reinterpret_cast<double*>(take((size_t)a.n * sizeof(double)));
    double* dp = reinterpret_cast<double*>(take((size_t)a.n * sizeof(double)));
    int32_t* part = reinterpret_cast<int32_t*>(take((size_t)a.n * sizeof(int32_t)));
    int32_t* tickets = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * 64));
    cudaError_t e = cudaMemsetAsync(tickets, 0, sizeof(int32_t) * 64, st);
    if (e != cudaSuccess) return e;
    const bool from_identity = N_stack != nullptr || a.m == 0;  // a product reads W_0 = I in full
    if (from_identity && (e = cudaMemsetAsync(W0, 0, (size_t)a.nnzW * sizeof(T), st)) != cudaSuccess) return e;
    trace_begin("ninv_dinv", st);
    ninv_dinv_launch(a, dr, dp, part, st);
    trace_end(st);
    trace_begin("ninv_init", st);
    hg_init<T><<<a.num_sms * 4, 256, 0, st>>>(a.Wcp, W0, a.n);
    trace_end(st);
    const int grid = a.num_sms * 6;
    auto product = [&](const T* W, double* out) {
        trace_begin("ninv_gather_product", st);
        pg_product<T><<<grid, kThreads, 0, st>>>(a, x, W, V, dp, out);
        trace_end(st);
    };
    T* cur = W0;
    T* nxt = W1;
    if (from_identity) {
        trace_begin("ninv_scale", st);
        hg_scale<T><<<a.num_sms * 8, 256, 0, st>>>(a, W0, dr, V);
        trace_end(st);
        if (N_stack) product(W0, N_stack);
    }
    for (int t = 1; t <= a.m; ++t) {
        const bool need_v = t == a.m || N_stack != nullptr;
        trace_begin("ninv_gather_horner", st);
        hg_step<T><<<grid, kThreads, 0, st>>>(a, x, t, cur, nxt, need_v ? V : nullptr, dr, tickets + t);
        trace_end(st);
        std::swap(cur, nxt);
        if (N_stack && t < a.m) product(cur, N_stack + (int64_t)t * a.nnzS);
    }
    product(cur, N_stack ? N_stack + (int64_t)a.m * a.nnzS : N_out);
    return cudaGetLastError();
}

}  // namespace

size_t ninv_gather_work_bytes(const NinvArgs& a, int prec) {
    const size_t ts = prec == 0 ? sizeof(double) : sizeof(float);
    return 3 * ((size_t)a.nnzW * ts + 256) + (size_t)a.n * (2 * sizeof(double) + sizeof(int32_t)) + 3 * 256 +
           sizeof(int32_t) * 64 + 256 + 4096;
}

cudaError_t ninv_gather_launch(const NinvArgs& a, const NinvIndex& x, int prec, void* work, double* N_out,
                               cudaStream_t st, double* N_stack) {
    if (a.n == 0) return cudaSuccess;
    if (prec == 0) return gather_run<double>(a, x, work, N_out, N_stack, st);
    return gather_run<float>(a, x, work, N_out, N_stack, st);
}

void ninv_index_free(NinvIndex& x) {
    void* ptrs[] = {x.cs, x.sb, x.tloc, x.scnt, x.src, x.Srow, x.hoff, x.hits};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    x = NinvIndex();
}

cudaError_t ninv_index_configure() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(hidx_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBuildSmem)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(hidx_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBuildSmem)) !=
        cudaSuccess)
        return e;
    return cudaFuncSetAttribute(pidx_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBuildSmem);
}

std::string ninv_index_build(const NinvArgs& a, const HostPlan& P, const NinvPlan& Wp, int64_t budget,
                             NinvIndex& x, cudaStream_t st, cudaError_t& err) {
    err = cudaSuccess;
    ninv_index_free(x);
    const int64_t n = a.n;
    if (a.max_col > kIdxEnt) return "a column of the series pattern exceeds the index table";
    for (int64_t j = 0; j < n; ++j)
        if (P.Lcp[j + 1] - P.Lcp[j] > 255) return "a column of L has more than 255 entries";
    std::vector<int64_t> cs(n + 1, 0);
    for (int64_t j = 0; j < n; ++j) cs[j + 1] = cs[j] + (Wp.Wcp[j + 1] - Wp.Wcp[j] + 31) / 32;
    x.m = a.m;
    x.nslices = cs[n];
    const int64_t NL = x.nslices * 32;
    std::vector<void*> temps;
    auto fail = [&](cudaError_t e, const char* what) {
        err = e;
        for (void* t : temps) cudaFree(t);
        ninv_index_free(x);
        return std::string(what) + ": " + cudaGetErrorString(e);
    };
    auto alloc = [&](void** ptr, size_t bytes) { return cudaMalloc(ptr, std::max<size_t>(bytes, 16)); };
    cudaError_t e;
    int64_t held = 0;
    auto hold = [&](int64_t b) {
        held += b;
        return budget <= 0 || held <= budget;
    };
    if (!hold((n + 1) * 8 + (x.nslices + 1) * 8 + NL * 2 + NL * a.m)) {
        ninv_index_free(x);
        return "index exceeds the memory budget";
    }
    if ((e = alloc((void**)&x.cs, (n + 1) * sizeof(int64_t))) != cudaSuccess) return fail(e, "index alloc");
    if ((e = cudaMemcpyAsync(x.cs, cs.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return fail(e, "index upload");
    if ((e = alloc((void**)&x.sb, (x.nslices + 1) * sizeof(int64_t))) != cudaSuccess) return fail(e, "index alloc");
    if ((e = alloc((void**)&x.tloc, NL * sizeof(uint16_t))) != cudaSuccess) return fail(e, "index alloc");
    if ((e = alloc((void**)&x.scnt, NL * (size_t)std::max(a.m, 1))) != cudaSuccess) return fail(e, "index alloc");
    uint8_t* cntg = nullptr;
    int32_t* width = nullptr;
    int32_t* tk = nullptr;
    if ((e = alloc((void**)&cntg, (size_t)a.nnzW * std::max(a.m, 1))) != cudaSuccess) return fail(e, "index alloc");
    temps.push_back(cntg);
    if ((e = alloc((void**)&width, x.nslices * sizeof(int32_t))) != cudaSuccess) return fail(e, "index alloc");
    temps.push_back(width);
    if ((e = alloc((void**)&tk, 8 * sizeof(int32_t))) != cudaSuccess) return fail(e, "index alloc");
    temps.push_back(tk);
    if ((e = cudaMemsetAsync(tk, 0, 8 * sizeof(int32_t), st)) != cudaSuccess) return fail(e, "index memset");
    const int grid = a.num_sms * 2;
    std::vector<int64_t> sb(x.nslices + 1, 0);
    if (a.m > 0) {
        hidx_count<<<grid, kThreads, kBuildSmem, st>>>(a, tk + 0, cntg);
        hidx_layout<<<grid, kThreads, 0, st>>>(a, x, cntg, tk + 1, width);
        std::vector<int32_t> wh(x.nslices);
        if ((e = cudaMemcpyAsync(wh.data(), width, x.nslices * sizeof(int32_t), cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return fail(e, "index layout");
        for (int64_t s = 0; s < x.nslices; ++s) sb[s + 1] = sb[s] + 32 * (int64_t)wh[s];
    } else {
        if ((e = cudaMemsetAsync(x.scnt, 0, 16, st)) != cudaSuccess) return fail(e, "index memset");
    }
    if ((e = cudaMemcpyAsync(x.sb, sb.data(), (x.nslices + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return fail(e, "index upload");
    x.nsrc = sb[x.nslices];
    if (!hold(x.nsrc * 4)) {
        for (void* t : temps) cudaFree(t);
        ninv_index_free(x);
        return "index exceeds the memory budget";
    }
    if ((e = alloc((void**)&x.src, x.nsrc * sizeof(uint32_t))) != cudaSuccess) return fail(e, "index alloc");
    if (a.m > 0) hidx_fill<<<grid, kThreads, kBuildSmem, st>>>(a, x, tk + 2);
    // product words per entry of S_lo
    std::vector<int32_t> srow(a.nnzS);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t q = P.Srp[i]; q < P.Srp[i + 1]; ++q) srow[q] = (int32_t)i;
    if (!hold(a.nnzS * 4 + (a.nnzS + 1) * 8)) {
        for (void* t : temps) cudaFree(t);
        ninv_index_free(x);
        return "index exceeds the memory budget";
    }
    if ((e = alloc((void**)&x.Srow, a.nnzS * sizeof(int32_t))) != cudaSuccess) return fail(e, "index alloc");
    if ((e = cudaMemcpyAsync(x.Srow, srow.data(), a.nnzS * sizeof(int32_t), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return fail(e, "index upload");
    int32_t* hcnt = nullptr;
    int32_t* part = nullptr;
    if ((e = alloc((void**)&hcnt, a.nnzS * sizeof(int32_t))) != cudaSuccess) return fail(e, "index alloc");
    temps.push_back(hcnt);
    if ((e = alloc((void**)&part, (size_t)n * sizeof(int32_t))) != cudaSuccess) return fail(e, "index alloc");
    temps.push_back(part);
    hidx_partner<<<a.num_sms * 4, 256, 0, st>>>(n, a.pstart, part);
    pidx_pass<<<grid, kThreads, kBuildSmem, st>>>(a, x, part, tk + 3, hcnt, nullptr);
    std::vector<int32_t> hc(a.nnzS);
    if ((e = cudaMemcpyAsync(hc.data(), hcnt, a.nnzS * sizeof(int32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(e, "index count");
    std::vector<int64_t> ho(a.nnzS + 1, 0);
    for (int64_t q = 0; q < a.nnzS; ++q) ho[q + 1] = ho[q] + hc[q];
    x.nhits = ho[a.nnzS];
    if (!hold(x.nhits * 4)) {
        for (void* t : temps) cudaFree(t);
        ninv_index_free(x);
        return "index exceeds the memory budget";
    }
    if ((e = alloc((void**)&x.hoff, (a.nnzS + 1) * sizeof(int64_t))) != cudaSuccess) return fail(e, "index alloc");
    if ((e = cudaMemcpyAsync(x.hoff, ho.data(), (a.nnzS + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return fail(e, "index upload");
    if ((e = alloc((void**)&x.hits, x.nhits * sizeof(uint32_t))) != cudaSuccess) return fail(e, "index alloc");
    pidx_pass<<<grid, kThreads, kBuildSmem, st>>>(a, x, part, tk + 4, nullptr, x.hits);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(e, "index build");
    for (void* t : temps) cudaFree(t);
    x.bytes = held;
    x.ready = true;
    return std::string();
}

}  // namespace sinv
