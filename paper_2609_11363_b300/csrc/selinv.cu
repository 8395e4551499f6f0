// Supernodal selected inversion (Section 2.1, eqs. (2.4)-(2.5)) as one
// persistent kernel.
//
// For a supernode J (consecutive pivot blocks [s0, s0+w)) with row set C below
// it, one step of the Takahashi recurrence is
//     Lh   = L_CJ L_JJ^{-1}                         (c x w)
//     X    = -G~_CC Lh                              (G~ = G on S, 0 off S)
//     G_JJ = L_JJ^{-T} D_J^{-1} L_JJ^{-1} - Lh^T X
// and X is stored where (C[i], s0+t) is in S.  The symmetric c x c matrix G~_CC
// is read through a per-supernode list of the pairs (i, k), k < i, whose
// entry is in S (the zeros are never touched), plus the diagonal.
//
// Scheduling: every warp takes the next supernode from a global ticket counter
// in level-major order, waits (bounded) until the supernodes owning its rows C
// have published their results, computes, and publishes with a release store.
// A warp only ever waits for tickets handed out before its own, all held by
// running warps, so the schedule cannot deadlock.
#include <cstdio>

#include "device.cuh"
#include "kernels.h"
#include "plan.h"

namespace sinv {

namespace {

constexpr int kWarps = 8;          // warps per CTA
constexpr int kCW = 512;           // per-warp shared capacity for c*w values
constexpr int kWMax = 16;          // supernode width limit of this kernel

// Arithmetic forms.  Storage type of the working copy of G, the type products
// are formed in, and conversions.
struct F64 {
    using G = double;
    using R = double;
    static __device__ __forceinline__ R ld(const G* p) { return __ldcg(p); }
    static __device__ __forceinline__ void st(G* p, R v) { *p = v; }
    static __device__ __forceinline__ R from_d(double v) { return v; }
    static __device__ __forceinline__ double to_d(R v) { return v; }
};

struct F32 {
    using G = float;
    using R = float;
    static __device__ __forceinline__ R ld(const G* p) { return __ldcg(p); }
    static __device__ __forceinline__ void st(G* p, R v) { *p = v; }
    static __device__ __forceinline__ R from_d(double v) { return (float)v; }
    static __device__ __forceinline__ double to_d(R v) { return (double)v; }
};

struct WarpSmem {
    double lh[kCW];
    double x[kCW];
    double jj[kWMax * kWMax];   // L_JJ, then M = L_JJ^{-1}
    double t[kWMax * kWMax];    // D_J^{-1} M, then Lh^T X
};

template <class Form>
__global__ void __launch_bounds__(kWarps * 32) selinv_persistent(SelinvArgs a, typename Form::G* Gw) {
    using R = typename Form::R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSmem* ws = reinterpret_cast<WarpSmem*>(smem_raw) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const uint32_t epoch = *a.epoch;

    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.ticket, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= a.nsn) break;
        if (ld_volatile(a.status) != ST_OK) break;
        const int J = a.order[t];
        const SnInfo I = a.sn[J];
        const int c = I.c, w = I.w, cw = c * w;
        const int32_t* Crow = a.Crow + I.crow_off;
        const int32_t* Lmap = a.Lmap + I.cw_off;

        // wait until every supernode owning a row of C has published
        bool ok = true;
        for (int i = lane; i < c; i += 32) {
            int s = a.owner[Crow[i]];
            if (!wait_flag(a.done + s, epoch, a.status, a.wait_limit)) ok = false;
        }
        if (__any_sync(0xffffffffu, !ok)) break;
        __syncwarp();
        __threadfence();

        R* lh;
        R* x;
        if (cw <= kCW) {
            lh = reinterpret_cast<R*>(ws->lh);
            x = reinterpret_cast<R*>(ws->x);
        } else {
            lh = reinterpret_cast<R*>(a.scratch + gwarp * 2 * a.max_cw);
            x = lh + a.max_cw;
        }
        // L_CJ and L_JJ
        for (int e = lane; e < cw; e += 32) {
            int q = Lmap[e];
            lh[e] = q >= 0 ? Form::from_d(a.Lval[q]) : R(0);
            x[e] = R(0);
        }
        for (int e = lane; e < w * w; e += 32) {
            int q = a.JJl[I.ww_off + e];
            ws->jj[e] = q >= 0 ? a.Lval[q] : 0.0;
        }
        __syncwarp();
        // Lh = L_CJ L_JJ^{-1}: row by row, columns from the last to the first
        if (w > 1) {
            for (int i = lane; i < c; i += 32) {
                R* row = lh + (int64_t)i * w;
                for (int q = w - 2; q >= 0; --q) {
                    R acc = row[q];
                    for (int p = q + 1; p < w; ++p) acc -= row[p] * Form::from_d(ws->jj[p * w + q]);
                    row[q] = acc;
                }
            }
            __syncwarp();
        }
        // X = -G~_CC Lh : diagonal part (conflict free, lane owns row i) ...
        for (int i = lane; i < c; i += 32) {
            R g = Form::ld(Gw + a.Sdiag[Crow[i]]);
            for (int q = 0; q < w; ++q) x[i * w + q] -= g * lh[i * w + q];
        }
        __syncwarp();
        // ... and the off-diagonal pairs of S, each used for (i, k) and (k, i)
        {
            const uint32_t* hik = a.hit_ik + I.hit_off;
            const int32_t* hpos = a.hit_pos + I.hit_off;
            const int64_t hc = I.hit_cnt;
            if (w == 1) {
                for (int64_t h = lane; h < hc; h += 32) {
                    uint32_t ik = hik[h];
                    int i = ik >> 16, k = ik & 0xffff;
                    R g = Form::ld(Gw + hpos[h]);
                    atomicAdd(x + i, -g * lh[k]);
                    atomicAdd(x + k, -g * lh[i]);
                }
            } else {
                for (int64_t h = lane; h < hc; h += 32) {
                    uint32_t ik = hik[h];
                    int i = ik >> 16, k = ik & 0xffff;
                    R g = Form::ld(Gw + hpos[h]);
                    for (int q = 0; q < w; ++q) {
                        atomicAdd(x + i * w + q, -g * lh[k * w + q]);
                        atomicAdd(x + k * w + q, -g * lh[i * w + q]);
                    }
                }
            }
        }
        __syncwarp();
        // store X on S
        for (int e = lane; e < cw; e += 32) {
            int q = Lmap[e];
            if (q >= 0) Form::st(Gw + a.l2s[q], x[e]);
        }
        // M = L_JJ^{-1} (unit lower), in place in jj; lane b owns column b
        if (w > 1) {
            if (lane < w) {
                const int b = lane;
                // column b of M: M[b][b] = 1, M[r][b] = -sum_{b<=p<r} L[r][p] M[p][b]
                double col[kWMax];
                for (int r = 0; r < w; ++r) col[r] = 0.0;
                col[b] = 1.0;
                for (int r = b + 1; r < w; ++r) {
                    double acc = 0.0;
                    for (int p = b; p < r; ++p) acc -= ws->jj[r * w + p] * col[p];
                    col[r] = acc;
                }
                __syncwarp(__activemask());
                for (int r = 0; r < w; ++r) ws->jj[r * w + b] = col[r];
            }
            __syncwarp();
        } else {
            if (lane == 0) ws->jj[0] = 1.0;
            __syncwarp();
        }
        // T = D_J^{-1} M (FP64 pivot inverses); lane r owns row r
        if (lane < w) {
            const int r = lane;
            const int col = I.s0 + r;
            const bool first = a.pstart[col] != 0;
            const bool two = first ? (col + 1 < a.n && a.pstart[col + 1] == 0) : true;
            const double* d = a.Dval + a.dpos[col];
            double i_rr, i_rs = 0.0;
            int partner = -1;
            if (!two) {
                if (d[0] == 0.0) set_status(a.status, ST_SINGULAR);
                i_rr = 1.0 / d[0];
            } else {
                double det = d[0] * d[2] - d[1] * d[1];
                if (det == 0.0) set_status(a.status, ST_SINGULAR);
                if (first) { i_rr = d[2] / det; partner = r + 1; }
                else { i_rr = d[0] / det; partner = r - 1; }
                i_rs = -d[1] / det;
            }
            for (int b = 0; b < w; ++b) {
                double v = i_rr * ws->jj[r * w + b];
                if (partner >= 0) v += i_rs * ws->jj[partner * w + b];
                ws->t[r * w + b] = v;
            }
        }
        __syncwarp();
        // G_JJ[r][b] = sum_p M[p][r] T[p][b] - sum_i Lh[i][r] X[i][b]   (r >= b)
        for (int r = 0; r < w; ++r) {
            for (int b = 0; b <= r; ++b) {
                double s = 0.0;
                for (int i = lane; i < c; i += 32) s += (double)lh[i * w + r] * (double)x[i * w + b];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) {
                    double m = 0.0;
                    for (int p = 0; p < w; ++p) m += ws->jj[p * w + r] * ws->t[p * w + b];
                    int sp = a.JJs[I.ww_off + r * w + b];
                    if (sp >= 0) Form::st(Gw + sp, Form::from_d(m - s));
                }
            }
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            st_release(a.done + J, epoch);
        }
    }
}

__global__ void prepare_kernel(uint32_t* epoch, int32_t* ticket) {
    uint32_t e = *epoch + 1;
    *epoch = e == 0 ? 1 : e;
    *ticket = 0;
}

template <class Form>
__global__ void widen_to_double(const typename Form::G* __restrict__ src, double* __restrict__ dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = Form::to_d(src[i]);
}

template <class Form>
cudaError_t launch_form(const SelinvArgs& a, typename Form::G* Gw, double* G_out, cudaStream_t st, int grid) {
    size_t smem = sizeof(WarpSmem) * kWarps;
    selinv_persistent<Form><<<grid, kWarps * 32, smem, st>>>(a, Gw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((void*)Gw != (void*)G_out) {
        widen_to_double<Form><<<a.num_sms * 8, 256, 0, st>>>(Gw, G_out, a.nnzS);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

cudaError_t selinv_prepare(uint32_t* epoch, int32_t* ticket, cudaStream_t st) {
    prepare_kernel<<<1, 1, 0, st>>>(epoch, ticket);
    return cudaGetLastError();
}

int selinv_max_width() { return kWMax; }
int selinv_cw_smem() { return kCW; }
int selinv_warps_per_cta() { return kWarps; }

cudaError_t selinv_configure() {
    size_t smem = sizeof(WarpSmem) * kWarps;
    cudaError_t e = cudaFuncSetAttribute(selinv_persistent<F64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(selinv_persistent<F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int selinv_grid(int num_sms) {
    int per_sm = 0;
    size_t smem = sizeof(WarpSmem) * kWarps;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, selinv_persistent<F64>, kWarps * 32, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    return per_sm * num_sms;
}

cudaError_t selinv_launch(const SelinvArgs& a, int prec, void* work, double* G_out, cudaStream_t st, int grid) {
    if (prec == 0) return launch_form<F64>(a, G_out, G_out, st, grid);
    return launch_form<F32>(a, reinterpret_cast<float*>(work), G_out, st, grid);
}

}  // namespace sinv
