// Supernodal selected inversion on the tensor cores (Section 2.1, Eqs. (4)-(5)):
// the supernodes whose row set C below them is a contiguous range of rows.
//
// For such a supernode J (columns s0 .. s0+w-1, C = [C0, C0+c)) the step of the
// Takahashi recurrence is rewritten around one dense contraction over C:
//     M    = L_JJ^{-1}                         (FP64, w x w)
//     Y    = G~_CC L_CJ                         (c x w: the tensor cores)
//     X    = -Y M                               (stored where (C[i], s0+t) is in S)
//     Z    = L_CJ^T Y                           (w x w, summed over C in FP64)
//     G_JJ = M^T (D_J^{-1} + Z) M              (FP64)
// which is the same step as X = -G~_CC L_CJ L_JJ^{-1} and G_JJ = M^T D^{-1} M -
// (L_CJ M)^T X.  G~_CC reads G on S and zero elsewhere (the restriction of
// Section 2.1): the tier keeps its own symmetric band copy of G (the mirror),
// zero-filled before every call and written wherever the tier writes G, so every
// row of G~_CC is one contiguous run of the mirror.
//
// Precision (split operands): every operand x of Y is cut into x_hi = round(x)
// and x_lo = round(x - x_hi) in the MMA's input type (TF32 or BF16); the tensor
// cores accumulate x_hi y_hi in one FP32 accumulator and the cross terms x_hi
// y_lo + x_lo y_hi in a second (the compensation), and the two are added in FP64.
// The pivot inverses, M, the sum of Z over C and G_JJ are FP64.
//
// Work: one CTA (four warps, row t of a 128-row tile of C = TMEM lane t) per
// (supernode, row tile, part of the contraction over C).  Every part adds its
// share of X = -Y M into the mirror and its share of Z into a block in global
// memory (FP64 atomics); the last part to arrive finishes the supernode (G_JJ)
// and publishes it; the last part of each tile then copies the tile's X into G.  A CTA waits (bounded) until the supernodes
// owning C have published, exactly like the other SelInv kernel, and takes its
// items in level order from a ticket counter.
#include <cuda_bf16.h>

#include "device.cuh"
#include "kernels.h"
#include "plan.h"
#include "tc.cuh"

namespace sinv {

namespace {

constexpr int kThreads = 128;
constexpr int kKC = 32;                   // columns of C per staged chunk
constexpr int kTmemCols = 64;             // hi*hi accumulator at 0, cross terms at 32
constexpr int kW = kTcWMax;               // 32
constexpr int kABytes = kTcRowsTile * kKC * 4;  // one A tile (TF32; BF16 uses half)
constexpr int kBBytes = kW * kKC * 4;           // one B tile

// Everything that does not depend on G is staged before the dependency wait: the B
// tiles (split L_CJ) of all chunks of the part, the L rows and X positions of the
// tile, L_JJ^{-1}, D_J^{-1} and the positions of G_JJ.  After the wait only the rows
// of G~ travel.
struct __align__(128) TcSmem {
    uint8_t a[2][2][kABytes];                   // [stage][hi, lo]
    uint8_t b[kTcMaxChunks][2][kBBytes];        // [chunk of the part][hi, lo]
    float Ls[kTcRowsTile][kW + 1];              // L(R[i], s0 + b) of the tile (FP32)
    int32_t xpos[kTcRowsTile][kW];              // S_lo position of X(R[i], s0 + b), or -1
    double Ljj[kW * kW];                        // L_JJ
    double M[kW * kW];                          // L_JJ^{-1}, row-major (r, b)
    double Dinv[kW * kW];                       // D_J^{-1}
    float Mf[kW * kW];
    int32_t jjs[kW * kW];                       // S_lo positions of (s0 + r, s0 + b), r >= b, or -1
    uint64_t mbar[2];
    uint32_t tmem;
    int32_t item;
    int32_t flag;
};
// the epilogue reuses the A tiles: Y rows of the tile (FP32), then A = D^{-1} + Z and
// B = A M (FP64)
static_assert(kTcRowsTile * (kW + 1) * 4 <= 2 * kABytes, "epilogue scratch");
static_assert(2 * kW * kW * 8 <= kABytes, "epilogue scratch");

// round to TF32 (10 explicit mantissa bits, nearest, ties away) as an FP32 pattern
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// split x into hi + lo in the input type of the MMA
template <int kFmt>
struct Split;
template <>
struct Split<tc::kFmtTF32> {
    static constexpr int kElem = 4;
    static __device__ __forceinline__ void run(double x, float& hi, float& lo) {
        hi = to_tf32((float)x);
        lo = to_tf32((float)(x - (double)hi));
    }
};
template <>
struct Split<tc::kFmtBF16> {
    static constexpr int kElem = 2;
    static __device__ __forceinline__ void run(double x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
        hi = __float2bfloat16((float)x);
        lo = __float2bfloat16((float)(x - (double)__bfloat162float(hi)));
    }
};

// the mirror holds row r from column ((r - band - 64) rounded down to a multiple of
// 4) on: 32-byte aligned groups of four doubles, a margin of 64 columns both ways
__device__ __forceinline__ int64_t mirror_index(const TcArgs& t, int64_t row, int64_t col) {
    const int64_t base = ((row - t.band - 64) >> 2) << 2;
    return (row - t.row0) * t.width + (col - base);
}

// stage the chunk [k0, k0 + 32) (global columns) of rows C0 + i, i in this tile, of
// G~_CC into the stage buffers (the A tiles)
template <int kFmt>
__device__ __forceinline__ void stage_chunk(const TcArgs& t, const SnInfo& I, int C0, int mi, int64_t k0,
                                            uint8_t* ahi, uint8_t* alo) {
    const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
    const int c = I.tc_c;
    constexpr int E = Split<kFmt>::kElem;
    constexpr int kq = kKC * E / 16;            // 16-byte K chunks per row group
    constexpr int per = 16 / E;                 // elements per 16-byte core-matrix row
    constexpr int groups = kKC / per;           // per row
    // 32 rows of this warp x `groups` 16-byte groups = 32 * groups items, 32 per step;
    // the 8 lanes of a quarter warp take the 8 rows of one core matrix.  All loads of
    // the chunk are issued first (one round trip), then split and stored.
    double v[groups][per];
#pragma unroll
    for (int it = 0; it < groups; ++it) {
        const int q = it * 4 + (lane >> 3);          // 0 .. 4 * groups - 1
        const int rg = q & 3, gi = q >> 2;           // row group in the warp's 32 rows, K group
        const int row = g * 32 + rg * 8 + (lane & 7);
        const int i = mi * kTcRowsTile + row;        // local row in C
        const int64_t kb = k0 + gi * per;            // first global column of the group
        if (i < c) {
            const double2* src = reinterpret_cast<const double2*>(t.mirror + mirror_index(t, C0 + i, kb));
#pragma unroll
            for (int e = 0; e < per; e += 2) {
                const double2 d = __ldcg(src + e / 2);
                v[it][e] = d.x;
                v[it][e + 1] = d.y;
            }
        } else {
#pragma unroll
            for (int e = 0; e < per; ++e) v[it][e] = 0.0;
        }
    }
#pragma unroll
    for (int it = 0; it < groups; ++it) {
        const int q = it * 4 + (lane >> 3);
        const int rg = q & 3, gi = q >> 2;
        const int row = g * 32 + rg * 8 + (lane & 7);
        const int64_t kb = k0 + gi * per;
#pragma unroll
        for (int e = 0; e < per; ++e) {
            const int64_t k = kb + e;
            if (k < C0 || k >= (int64_t)C0 + c) v[it][e] = 0.0;
        }
        const uint32_t off = tc::kmajor_offset(row, gi * per, kq, E);
        if constexpr (kFmt == tc::kFmtTF32) {
            float4 h, l;
            Split<kFmt>::run(v[it][0], h.x, l.x);
            Split<kFmt>::run(v[it][1], h.y, l.y);
            Split<kFmt>::run(v[it][2], h.z, l.z);
            Split<kFmt>::run(v[it][3], h.w, l.w);
            *reinterpret_cast<float4*>(ahi + off) = h;
            *reinterpret_cast<float4*>(alo + off) = l;
        } else {
            __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) Split<kFmt>::run(v[it][e], h[e], l[e]);
            *reinterpret_cast<uint4*>(ahi + off) = *reinterpret_cast<const uint4*>(h);
            *reinterpret_cast<uint4*>(alo + off) = *reinterpret_cast<const uint4*>(l);
        }
    }
}

// the B tile of the chunk [k0, k0 + 32): row tt = column s0 + tt of L (tt < N), K = the
// chunk's rows of R; zero outside
template <int kFmt>
__device__ __forceinline__ void stage_b(const SelinvArgs& a, const TcArgs& t, const SnInfo& I, int C0, int64_t k0,
                                        uint8_t* bhi, uint8_t* blo) {
    const int tid = threadIdx.x;
    const int c = I.tc_c, w = I.w;
    constexpr int E = Split<kFmt>::kElem;
    constexpr int kq = kKC * E / 16;
    constexpr int per = 16 / E;
    constexpr int groups = kKC / per;
    const int N = w <= 16 ? 16 : 32;
    for (int u = tid; u < N * groups; u += kThreads) {
        const int tt = u / groups, gi = u % groups;
        int qv[per];
#pragma unroll
        for (int e = 0; e < per; ++e) {
            const int64_t k = k0 + gi * per + e;
            qv[e] = (tt < w && k >= C0 && k < (int64_t)C0 + c) ? t.tcmap[I.tc_map_off + (k - C0) * w + tt] : -1;
        }
        double v[per];
#pragma unroll
        for (int e = 0; e < per; ++e) v[e] = qv[e] >= 0 ? a.Lval[qv[e]] : 0.0;
        const uint32_t off = tc::kmajor_offset(tt, gi * per, kq, E);
        if constexpr (kFmt == tc::kFmtTF32) {
            float4 h, l;
            Split<kFmt>::run(v[0], h.x, l.x);
            Split<kFmt>::run(v[1], h.y, l.y);
            Split<kFmt>::run(v[2], h.z, l.z);
            Split<kFmt>::run(v[3], h.w, l.w);
            *reinterpret_cast<float4*>(bhi + off) = h;
            *reinterpret_cast<float4*>(blo + off) = l;
        } else {
            __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) Split<kFmt>::run(v[e], h[e], l[e]);
            *reinterpret_cast<uint4*>(bhi + off) = *reinterpret_cast<const uint4*>(h);
            *reinterpret_cast<uint4*>(blo + off) = *reinterpret_cast<const uint4*>(l);
        }
    }
}

template <int kFmt>
__device__ __forceinline__ void issue_chunk(const TcSmem& S, int buf, int bidx, uint32_t tmem, int N, bool& first) {
    constexpr int E = Split<kFmt>::kElem;
    constexpr int kq = kKC * E / 16;
    constexpr int ksteps = kKC * E / 32;  // one MMA covers 32 bytes of K
    const uint32_t idesc = tc::instr_desc(kFmt, kTcRowsTile, N);
    const uint32_t ahi = tc::smem_u32(S.a[buf][0]), alo = tc::smem_u32(S.a[buf][1]);
    const uint32_t bhi = tc::smem_u32(S.b[bidx][0]), blo = tc::smem_u32(S.b[bidx][1]);
#pragma unroll
    for (int s = 0; s < ksteps; ++s) {
        const uint32_t o = s * 256;
        const uint64_t dah = tc::smem_desc(ahi + o, 128, kq * 128), dal = tc::smem_desc(alo + o, 128, kq * 128);
        const uint64_t dbh = tc::smem_desc(bhi + o, 128, kq * 128), dbl = tc::smem_desc(blo + o, 128, kq * 128);
        if (kFmt == tc::kFmtTF32) {
            tc::mma_tf32(tmem, dah, dbh, idesc, !first);
            tc::mma_tf32(tmem + 32, dah, dbl, idesc, !first);
            tc::mma_tf32(tmem + 32, dal, dbh, idesc, true);
        } else {
            tc::mma_bf16(tmem, dah, dbh, idesc, !first);
            tc::mma_bf16(tmem + 32, dah, dbl, idesc, !first);
            tc::mma_bf16(tmem + 32, dal, dbh, idesc, true);
        }
        first = false;
    }
}

// Spin until *flag == want with a growing pause between polls (32 ns up to 1 us), at
// most `limit` polls; like wait_flag, but the many CTAs that wait for the next level
// poll the same few flags, so they back off.
__device__ __forceinline__ bool wait_backoff(const uint32_t* flag, uint32_t want, int32_t* status, int64_t limit) {
    uint32_t pause = 32;
    if (ld_acquire(flag) == want) return true;
    for (int64_t it = 0; ld_relaxed(flag) != want || ld_acquire(flag) != want; ++it) {
        if ((it & 15) == 15 && ld_volatile(status) != ST_OK) return false;
        if (it > limit) {
            set_status(status, ST_TIMEOUT);
            return false;
        }
        __nanosleep(pause);
        if (pause < 1024) pause <<= 1;
    }
    return true;
}

// D_J^{-1}(r, b) for local columns r, b of the supernode (blocks of D lie inside it)
__device__ __forceinline__ double dinv_entry(const SelinvArgs& a, int s0, int r, int b) {
    const int cr = s0 + r, cb = s0 + b;
    const bool first = a.pstart[cr] != 0;
    const bool two = first ? (cr + 1 < a.n && a.pstart[cr + 1] == 0) : true;
    const int partner = two ? (first ? cr + 1 : cr - 1) : -1;
    if (cb != cr && cb != partner) return 0.0;
    const double* d = a.Dval + a.dpos[cr];
    if (!two) {
        if (d[0] == 0.0) set_status(a.status, ST_SINGULAR);
        return 1.0 / d[0];
    }
    const double det = d[0] * d[2] - d[1] * d[1];
    if (det == 0.0) set_status(a.status, ST_SINGULAR);
    if (cb != cr) return -d[1] / det;
    return first ? d[2] / det : d[0] / det;
}

template <int kFmt>
__global__ void __launch_bounds__(kThreads) selinv_tc_kernel(SelinvArgs a, TcArgs t, double* __restrict__ G) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        tc::mbar_init(&S.mbar[0], 1);
        tc::mbar_init(&S.mbar[1], 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&S.tmem, kTmemCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = S.tmem;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const uint32_t epoch = *a.epoch;
    uint32_t ph[2] = {0u, 0u};
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            S.item = atomicAdd(t.ticket, 1);
            S.flag = ld_volatile(a.status) != ST_OK;
        }
        __syncthreads();
        if (S.item >= t.nitems || S.flag) break;
        const WorkItem it = t.items[S.item];
        const int J = a.order[it.first];
        const SnInfo I = a.sn[J];
        const int c = I.tc_c, w = I.w, s0 = I.s0;   // c: the range R of rows
        const int ks = I.tc_ks, mi = it.part / ks, kp = it.part % ks;
        const int N = w <= 16 ? 16 : 32;
        const int C0 = c > 0 ? a.Crow[I.crow_off] : 0;
        if (tid == 0) tl_start(a.tl, J);

        // ---- phase A: everything that does not depend on G, before the wait ------------
        const int64_t kbase = ((int64_t)C0 >> 2) << 2;
        const int nch = c > 0 ? (int)((C0 + c - kbase + kKC - 1) / kKC) : 0;
        const int ch0 = nch * kp / ks, ch1 = nch * (kp + 1) / ks;
        if (ch1 - ch0 > kTcMaxChunks) {  // the plan keeps parts within kTcMaxChunks chunks
            if (tid == 0) set_status(a.status, ST_INTERNAL);
            break;
        }
        // L_JJ, D_J^{-1} and the positions of G_JJ
        for (int e = tid; e < w * w; e += kThreads) {
            const int r = e / w, b = e % w;
            const int q = a.JJl[I.ww_off + e];
            S.Ljj[e] = q >= 0 ? a.Lval[q] : 0.0;
            S.Dinv[e] = dinv_entry(a, s0, r, b);
            S.jjs[e] = a.JJs[I.ww_off + e];
        }
        // this thread's row of the tile: L values and the positions X is stored at
        {
            const int i = mi * kTcRowsTile + tid;
            int q[kW];
#pragma unroll
            for (int b = 0; b < kW; ++b) q[b] = (i < c && b < w) ? t.tcmap[I.tc_map_off + (int64_t)i * w + b] : -1;
#pragma unroll
            for (int b = 0; b < kW; ++b) {
                S.Ls[tid][b] = q[b] >= 0 ? (float)a.Lval[q[b]] : 0.f;
                S.xpos[tid][b] = q[b] >= 0 ? a.l2s[q[b]] : -1;
            }
        }
        // the B tiles (split L_CJ) of every chunk of this part
        for (int ch = ch0; ch < ch1; ++ch)
            stage_b<kFmt>(a, t, I, C0, kbase + (int64_t)ch * kKC, S.b[ch - ch0][0], S.b[ch - ch0][1]);
        __syncthreads();
        // M = L_JJ^{-1} (unit lower, FP64; thread b owns column b)
        if (tid < w) {
            const int b = tid;
            double col[kW];
#pragma unroll
            for (int r = 0; r < kW; ++r) {
                double acc = r == b ? 1.0 : 0.0;
                if (r > b && r < w) {
#pragma unroll
                    for (int p = 0; p < kW; ++p)
                        if (p >= b && p < r) acc -= S.Ljj[r * w + p] * col[p];
                }
                col[r] = acc;
            }
#pragma unroll
            for (int r = 0; r < kW; ++r)
                if (r < w) {
                    S.M[r * w + b] = col[r];
                    S.Mf[r * w + b] = (float)col[r];
                }
        }
        // ---- phase B: one warp waits for the distinct supernodes that own C -------------
        bool ok = true;
        if (warp == 0)
            for (int d = tid; d < I.tc_ndep; d += 32)
                if (!wait_backoff(a.done + t.deps[I.tc_dep_off + d], epoch, a.status, a.wait_limit)) {
                    ok = false;
                    break;
                }
        if (__syncthreads_or(!ok)) break;
        if (tid == 0) tl_mark(a.tl, J, 0);

        // ---- phase C: Y = G~_CC L_CJ over this part's chunks of C ------------------------
        bool first = true;
        int pending = 0;   // bit b: a commit on stage b not waited for yet
        for (int ch = ch0; ch < ch1 && ok; ++ch) {
            const int buf = (ch - ch0) & 1;
            if (pending & (1 << buf)) {
                ok = tc::mbar_wait(&S.mbar[buf], ph[buf], a.status, kMlpWaitLimit);
                ph[buf] ^= 1u;
                pending &= ~(1 << buf);
            }
            stage_chunk<kFmt>(t, I, C0, mi, kbase + (int64_t)ch * kKC, S.a[buf][0], S.a[buf][1]);
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                issue_chunk<kFmt>(S, buf, ch - ch0, tmem, N, first);
                tc::commit(&S.mbar[buf]);
            }
            first = false;
            pending |= 1 << buf;
        }
        for (int buf = 0; buf < 2; ++buf)
            if (pending & (1 << buf)) {
                ok = tc::mbar_wait(&S.mbar[buf], ph[buf], a.status, kMlpWaitLimit) && ok;
                ph[buf] ^= 1u;
            }
        tc::fence_after_sync();
        if (__syncthreads_or(!ok)) break;
        if (tid == 0) tl_mark(a.tl, J, 1);

        // ---- epilogue of the part: its shares of X = -Y M and of Z = L_CJ^T Y -------------
        // X is linear in Y, so every part adds -Y_part M into the zero-filled mirror (both
        // triangles) and L_CJ^T Y_part into the Z block with FP64 atomics; the mirror is
        // complete once every part has arrived, and the tile's last part copies its rows
        // into G afterwards.
        const int i = mi * kTcRowsTile + tid;   // local row of R (TMEM lane tid)
        float yf[kW];
#pragma unroll
        for (int b = 0; b < kW; ++b) yf[b] = 0.f;
        if (ch1 > ch0) {
            float hh[16], xx[16];
#pragma unroll
            for (int c0 = 0; c0 < kW; c0 += 16) {
                if (c0 >= N) break;
                tc::ld16(tmem + lane_base + c0, hh);
                tc::ld16(tmem + lane_base + 32 + c0, xx);
                tc::ld_wait();
#pragma unroll
                for (int e = 0; e < 16; ++e) yf[c0 + e] = (float)((double)hh[e] + (double)xx[e]);
            }
        }
        tc::fence_before_sync();
        float* Ys = reinterpret_cast<float*>(S.a[0][0]);                 // [128][kW + 1]
        if (i < c) {
            const int64_t r = C0 + i;
#pragma unroll
            for (int b = 0; b < kW; ++b) {
                if (b >= w) break;
                float s = 0.f;
#pragma unroll
                for (int p = b; p < kW; ++p)
                    if (p < w) s = fmaf(yf[p], S.Mf[p * w + b], s);
                if (S.xpos[tid][b] >= 0 && s != 0.f) {
                    atomicAdd(t.mirror + mirror_index(t, r, s0 + b), (double)-s);
                    atomicAdd(t.mirror + mirror_index(t, s0 + b, r), (double)-s);
                }
                Ys[tid * (kW + 1) + b] = yf[b];
            }
        } else {
            for (int b = 0; b < w; ++b) Ys[tid * (kW + 1) + b] = 0.f;
        }
        __syncthreads();
        {
            const int rows = min(kTcRowsTile, c - mi * kTcRowsTile);
            for (int e = tid; e < w * w; e += kThreads) {
                const int pa = e / w, pb = e % w;
                float z = 0.f;
                for (int r = 0; r < rows; ++r) z = fmaf(S.Ls[r][pa], Ys[r * (kW + 1) + pb], z);
                if (z != 0.f) atomicAdd(t.zacc + I.tc_z_off + e, (double)z);
            }
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const uint32_t nparts = (uint32_t)(I.tc_tiles * ks);
            S.flag = (atomicAdd(a.arrive + J, 1u) == nparts - 1 ? 1 : 0) |
                     (atomicAdd(t.arrive_t + I.tc_t_off + mi, 1u) == (uint32_t)(ks - 1) ? 2 : 0);
        }
        __syncthreads();
        const int flags = S.flag;
        if (flags & 1) {
            __threadfence();

            // ---- the supernode's last part: G_JJ = M^T (D^{-1} + Z) M in FP64 ----------------
            double* A = reinterpret_cast<double*>(S.a[1][0]);   // w x w
            double* B = A + kW * kW;                              // A M
            for (int e = tid; e < w * w; e += kThreads) A[e] = S.Dinv[e] + __ldcg(t.zacc + I.tc_z_off + e);
            __syncthreads();
            for (int e = tid; e < w * w; e += kThreads) {
                const int r = e / w, b = e % w;
                double s = 0.0;
                for (int p = b; p < w; ++p) s += A[r * w + p] * S.M[p * w + b];
                B[e] = s;
            }
            __syncthreads();
            for (int e = tid; e < w * w; e += kThreads) {
                const int r = e / w, b = e % w;
                if (b > r) continue;
                double s = 0.0;
                for (int p = r; p < w; ++p) s += S.M[p * w + r] * B[p * w + b];
                const int sp = S.jjs[r * w + b];
                if (sp >= 0) {
                    G[sp] = s;
                    t.mirror[mirror_index(t, s0 + r, s0 + b)] = s;
                    t.mirror[mirror_index(t, s0 + b, s0 + r)] = s;
                }
            }
            // the barrier orders every thread's writes before the release store
            __syncthreads();
            if (tid == 0) {
                st_release(a.done + J, epoch);
                tl_mark(a.tl, J, 2);
            }
        }  // the supernode's last part
        if (flags & 2) {
            // the tile's last part: its rows of X, now complete in the mirror, into G
            __threadfence();
            if (i < c) {
                const int64_t r = C0 + i;
                for (int b = 0; b < w; ++b) {
                    const int pos = S.xpos[tid][b];
                    if (pos >= 0) G[pos] = __ldcg(t.mirror + mirror_index(t, r, s0 + b));
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

constexpr int kSmem = (int)sizeof(TcSmem);

}  // namespace

cudaError_t selinv_tc_configure() {
    cudaError_t e = cudaFuncSetAttribute(selinv_tc_kernel<tc::kFmtTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(selinv_tc_kernel<tc::kFmtBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
}

cudaError_t selinv_tc_launch(const SelinvArgs& a, const TcArgs& t, int fmt, double* G, cudaStream_t st) {
    if (t.nitems == 0) return cudaSuccess;
    // one CTA per SM (its shared memory); 64 TMEM columns each
    const int grid = std::min(t.nitems, a.num_sms);
    trace_begin(fmt == tc::kFmtTF32 ? "selinv_tc_tf32" : "selinv_tc_bf16", st);
    if (fmt == tc::kFmtTF32)
        selinv_tc_kernel<tc::kFmtTF32><<<grid, kThreads, kSmem, st>>>(a, t, G);
    else
        selinv_tc_kernel<tc::kFmtBF16><<<grid, kThreads, kSmem, st>>>(a, t, G);
    trace_end(st);
    return cudaGetLastError();
}

}  // namespace sinv
