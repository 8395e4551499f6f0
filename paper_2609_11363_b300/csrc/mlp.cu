// Learned correction from NInv towards SelInv: a small ReLU MLP (F=16 -> 64 -> 64
// -> 1) evaluated per entry of S, trained on pairs the method produces itself
// (features of the NInv entry, target (SelInv - NInv) / sqrt|N_ii N_jj|).
// The paper has no learned part; this is a proposed addition to the hot path.
//
// Precision: weights are used in BF16 (the FP32 master copy is rounded on
// load), features are stored in BF16, every sum is FP32.  Training is mini-batch
// Adam: one kernel runs forward and backward for 128 entries per CTA and writes
// the CTA's partial gradient (the weight gradients are small dense products
// H1^T dH2 and X^T dH1 formed from shared-memory tiles), a second kernel sums
// the partials, a third applies Adam.
#include <cuda_bf16.h>

#include "device.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace sinv {

namespace {

constexpr int kB = 128;  // entries per CTA (one per thread)

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16(x)); }

struct Weights {
    float W1[kMlpF * kMlpH];
    float b1[kMlpH];
    float W2[kMlpH * kMlpH];
    float b2[kMlpH];
    float W3[kMlpH];
    float b3;
};

// stage the BF16-rounded weights in shared memory
__device__ void load_weights(Weights& w, const float* __restrict__ theta) {
    for (int p = threadIdx.x; p < kMlpF * kMlpH; p += blockDim.x) w.W1[p] = bf(theta[kOffW1 + p]);
    for (int p = threadIdx.x; p < kMlpH * kMlpH; p += blockDim.x) w.W2[p] = bf(theta[kOffW2 + p]);
    for (int p = threadIdx.x; p < kMlpH; p += blockDim.x) {
        w.b1[p] = bf(theta[kOffB1 + p]);
        w.b2[p] = bf(theta[kOffB2 + p]);
        w.W3[p] = bf(theta[kOffW3 + p]);
    }
    if (threadIdx.x == 0) w.b3 = bf(theta[kOffB3]);
}

__device__ __forceinline__ void load_x(const __nv_bfloat16* __restrict__ X, int64_t e, float* x) {
    const uint4* p = reinterpret_cast<const uint4*>(X + e * kMlpF);
    uint4 a = p[0], b = p[1];
    const __nv_bfloat16* ha = reinterpret_cast<const __nv_bfloat16*>(&a);
    const __nv_bfloat16* hb = reinterpret_cast<const __nv_bfloat16*>(&b);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        x[k] = __bfloat162float(ha[k]);
        x[k + 8] = __bfloat162float(hb[k]);
    }
}

// fully unrolled so that h1 / h2 stay in registers
__device__ __forceinline__ float mlp_eval(const Weights& w, const float* x, float* h1, float* h2) {
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) {
        float z = w.b1[j];
#pragma unroll
        for (int k = 0; k < kMlpF; ++k) z = fmaf(x[k], w.W1[k * kMlpH + j], z);
        h1[j] = fmaxf(z, 0.f);
    }
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) {
        float z = w.b2[j];
#pragma unroll
        for (int k = 0; k < kMlpH; ++k) z = fmaf(h1[k], w.W2[k * kMlpH + j], z);
        h2[j] = fmaxf(z, 0.f);
    }
    float o = w.b3;
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) o = fmaf(h2[k], w.W3[k], o);
    return o;
}

// features of every entry of S_lo; one warp per row i
__global__ void features_kernel(int64_t n, const int64_t* __restrict__ Srp, const int32_t* __restrict__ Sc,
                                const int64_t* __restrict__ Lrp, const int64_t* __restrict__ Lcp, int m,
                                const double* __restrict__ Nst, int64_t nnzS, const double* __restrict__ Lval,
                                const double* __restrict__ Dval, const int32_t* __restrict__ dpos,
                                const int8_t* __restrict__ pstart, __nv_bfloat16* __restrict__ X,
                                float* __restrict__ scale) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const double* N = Nst + (int64_t)m * nnzS;
    auto dval = [&](int64_t r) {  // D(r, r)
        const bool first = pstart[r] != 0;
        const bool two = first ? (r + 1 < n && pstart[r + 1] == 0) : true;
        return two ? (first ? Dval[dpos[r]] : Dval[dpos[r] + 2]) : Dval[dpos[r]];
    };
    auto in2 = [&](int64_t r) { return pstart[r] == 0 || (r + 1 < n && pstart[r + 1] == 0); };
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
        const int64_t p0 = Srp[i], p1 = Srp[i + 1];
        const double Nii = N[p1 - 1];
        const double di = dval(i);
        const int64_t nL = Lrp[i + 1] - Lrp[i];
        for (int64_t p = p0 + lane; p < p1; p += 32) {
            const int64_t j = Sc[p];
            const double Njj = N[Srp[j + 1] - 1];
            double s = sqrt(fabs(Nii * Njj));
            if (!(s > 0.0)) s = 1.0;
            float f[kMlpF];
#pragma unroll
            for (int k = 0; k < kMlpF; ++k) f[k] = 0.f;
            f[0] = (float)(N[p] / s);
            for (int t = 1; t <= m && t < kMlpF - 6; ++t)
                f[t] = (float)((Nst[(int64_t)t * nnzS + p] - Nst[(int64_t)(t - 1) * nnzS + p]) / s);
            const int b = (m < kMlpF - 6 ? m : kMlpF - 7) + 1;
            const int64_t o = p - p0;
            const double lij = o < nL ? Lval[Lrp[i] + o] : 0.0;
            const double dj = dval(j);
            f[b] = (float)(lij * sqrt(fabs(dj / di)));
            f[b + 1] = i == j ? 1.f : 0.f;
            f[b + 2] = (in2(i) || in2(j)) ? 1.f : 0.f;
            f[b + 3] = log2f(1.f + (float)(Lcp[i + 1] - Lcp[i])) * 0.125f;
            f[b + 4] = log2f(1.f + (float)(Lcp[j + 1] - Lcp[j])) * 0.125f;
            __align__(16) __nv_bfloat16 hx[kMlpF];
#pragma unroll
            for (int k = 0; k < kMlpF; ++k) hx[k] = __float2bfloat16(f[k]);
            uint4* dst = reinterpret_cast<uint4*>(X + p * kMlpF);
            dst[0] = reinterpret_cast<uint4*>(hx)[0];
            dst[1] = reinterpret_cast<uint4*>(hx)[1];
            scale[p] = (float)s;
        }
    }
}

__global__ void targets_kernel(int64_t count, const double* __restrict__ G, const double* __restrict__ N,
                               const float* __restrict__ scale, float* __restrict__ y) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = (float)((G[e] - N[e]) / (double)scale[e]);
}

struct TrainSmem {
    Weights w;
    float h1[kB][kMlpH + 1];   // h1, later dh1 (padded rows: no bank conflicts on column reads)
    float d2[kB][kMlpH + 1];   // dh2
    float xs[kB][kMlpF + 1];
    float red[kB / 32][kMlpH + 2];
};

// forward + backward of kB entries per CTA; writes the CTA's gradient (and loss sum)
__global__ void __launch_bounds__(kB) fwd_bwd_kernel(const __nv_bfloat16* __restrict__ X, const float* __restrict__ y,
                                                     const int64_t* __restrict__ idx, int64_t count,
                                                     const float* __restrict__ theta, float* __restrict__ partial,
                                                     float* __restrict__ loss_partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
    load_weights(S.w, theta);
    __syncthreads();
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int64_t b = (int64_t)blockIdx.x * kB + t;
    const bool valid = b < count;
    const float invB = 1.f / (float)count;
    float x[kMlpF], h1[kMlpH], h2[kMlpH];
    float dout = 0.f, sq = 0.f;
    if (valid) {
        const int64_t e = idx ? idx[b] : b;
        load_x(X, e, x);
        const float out = mlp_eval(S.w, x, h1, h2);
        const float r = out - y[e];
        sq = r * r;
        dout = 2.f * r * invB;
    } else {
#pragma unroll
        for (int k = 0; k < kMlpF; ++k) x[k] = 0.f;
#pragma unroll
        for (int k = 0; k < kMlpH; ++k) h1[k] = h2[k] = 0.f;
    }
    // dh2 = W3 dout (relu'), dW3 = sum h2 dout, db3 = sum dout
    float* dh2 = h2;  // reuse: h2 is needed only for dW3 and the mask
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) {
        const float g3 = h2[j] * dout;
        float s = g3;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) S.red[wid][j] = s;
        dh2[j] = h2[j] > 0.f ? S.w.W3[j] * dout : 0.f;
    }
    {
        float s = dout, q = sq;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            q += __shfl_xor_sync(0xffffffffu, q, o);
        }
        if (lane == 0) {
            S.red[wid][kMlpH] = s;
            S.red[wid][kMlpH + 1] = q;
        }
    }
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) {
        S.h1[t][k] = h1[k];
        S.d2[t][k] = dh2[k];
    }
#pragma unroll
    for (int k = 0; k < kMlpF; ++k) S.xs[t][k] = x[k];
    __syncthreads();
    float* P = partial + (int64_t)blockIdx.x * kMlpParams;
    // dW3, db3, loss
    if (t < kMlpH) {
        float s = 0.f;
        for (int v = 0; v < kB / 32; ++v) s += S.red[v][t];
        P[kOffW3 + t] = s;
    }
    if (t == 0) {
        float s = 0.f, q = 0.f;
        for (int v = 0; v < kB / 32; ++v) {
            s += S.red[v][kMlpH];
            q += S.red[v][kMlpH + 1];
        }
        P[kOffB3] = s;
        loss_partial[blockIdx.x] = q;
    }
    // dW2[k][j] = sum_t h1[t][k] dh2[t][j]; db2[j] = sum_t dh2[t][j]
    for (int o = t; o < kMlpH * kMlpH; o += kB) {
        const int k = o / kMlpH, j = o % kMlpH;
        float s = 0.f;
#pragma unroll 8
        for (int r = 0; r < kB; ++r) s = fmaf(S.h1[r][k], S.d2[r][j], s);
        P[kOffW2 + o] = s;
    }
    if (t < kMlpH) {
        float s = 0.f;
        for (int r = 0; r < kB; ++r) s += S.d2[r][t];
        P[kOffB2 + t] = s;
    }
    __syncthreads();  // every thread is done reading S.h1 for dW2
    // dh1[k] = sum_j W2[k][j] dh2[j] (relu' of h1): own row, written over h1
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < kMlpH; ++j) s = fmaf(S.w.W2[k * kMlpH + j], dh2[j], s);
        S.h1[t][k] = h1[k] > 0.f ? s : 0.f;
    }
    __syncthreads();
    // dW1[k][j] = sum_t x[t][k] dh1[t][j]; db1[j] = sum_t dh1[t][j]
    for (int o = t; o < kMlpF * kMlpH; o += kB) {
        const int k = o / kMlpH, j = o % kMlpH;
        float s = 0.f;
#pragma unroll 8
        for (int r = 0; r < kB; ++r) s = fmaf(S.xs[r][k], S.h1[r][j], s);
        P[kOffW1 + o] = s;
    }
    if (t < kMlpH) {
        float s = 0.f;
        for (int r = 0; r < kB; ++r) s += S.h1[r][t];
        P[kOffB1 + t] = s;
    }
}

__global__ void reduce_kernel(const float* __restrict__ partial, int nblk, const float* __restrict__ loss_partial,
                              int64_t count, float* __restrict__ grad, float* __restrict__ loss) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kMlpParams; p += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * kMlpParams + p];
        grad[p] = s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
        float q = 0.f;
        for (int b = 0; b < nblk; ++b) q += loss_partial[b];
        *loss = q / (float)count;
    }
}

__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kMlpParams; p += gridDim.x * blockDim.x) {
        const float gp = g[p];
        const float mp = b1 * m[p] + (1.f - b1) * gp;
        const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
        m[p] = mp;
        v[p] = vp;
        theta[p] -= lr * (mp / c1) / (sqrtf(vp / c2) + eps);
    }
}

// ---- inference on the tensor cores ---------------------------------------------------
// A CTA of four warps (thread t owns row t of a tile of 128 entries) loops over
// tiles.  Layer 1 (128 x 16 features times W1, K = 16) and layer 2 (128 x 64 hidden
// times W2, K = 64) are tcgen05 MMAs with BF16 operands in shared memory and FP32
// accumulators in tensor memory (columns 0-63: layer 1, 64-127: layer 2).  The
// epilogues read the accumulators back (tcgen05.ld), add the bias and apply ReLU;
// the first hidden layer is rounded to BF16 as the operand of layer 2, the second
// stays FP32 for the output layer's dot product.
constexpr int kTcRows = 128;
constexpr int kTcCols = 128;   // TMEM columns per CTA
// dynamic shared memory per CTA: sized so that at most four CTAs share an SM,
// whose 512 TMEM columns then hold all four allocations
constexpr int kPredictSmem = 52 * 1024;
constexpr uint32_t kIdescL = tc::instr_desc(tc::kFmtBF16, 128, kMlpH);

struct __align__(128) PredictSmem {
    uint8_t w1t[kMlpH * kMlpF * 2];     // B of layer 1: row j = output unit, K = 16 inputs (2 chunks)
    uint8_t w2t[kMlpH * kMlpH * 2];     // B of layer 2: K = 64 (8 chunks)
    uint8_t xa[kTcRows * kMlpF * 2];    // A of layer 1
    uint8_t ha[kTcRows * kMlpH * 2];    // A of layer 2
    float b1[kMlpH], b2[kMlpH], w3[kMlpH];
    float b3;
    uint32_t tmem;
    uint64_t mbar;
};

__device__ __forceinline__ void st_bf16x8(uint8_t* dst, const float* v) {
    __align__(16) __nv_bfloat16 h[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) h[i] = __float2bfloat16(v[i]);
    *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(h);
}

__global__ void __launch_bounds__(kTcRows) predict_tc_kernel(const __nv_bfloat16* __restrict__ X,
                                                             const float* __restrict__ scale,
                                                             const double* __restrict__ N, int64_t count,
                                                             const float* __restrict__ theta,
                                                             double* __restrict__ out, int32_t* status,
                                                             int64_t wait_limit) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    PredictSmem& S = *reinterpret_cast<PredictSmem*>(smem_raw);
    const int t = threadIdx.x, warp = t >> 5;
    // weights: B operands in the K-major layout (element (j, k) = W[k][j]), BF16
    for (int p = t; p < kMlpH * kMlpF; p += kTcRows) {
        const int j = p / kMlpF, k = p % kMlpF;
        *reinterpret_cast<__nv_bfloat16*>(S.w1t + tc::kmajor_offset(j, k, kMlpF / 8, 2)) =
            __float2bfloat16(theta[kOffW1 + k * kMlpH + j]);
    }
    for (int p = t; p < kMlpH * kMlpH; p += kTcRows) {
        const int j = p / kMlpH, k = p % kMlpH;
        *reinterpret_cast<__nv_bfloat16*>(S.w2t + tc::kmajor_offset(j, k, kMlpH / 8, 2)) =
            __float2bfloat16(theta[kOffW2 + k * kMlpH + j]);
    }
    if (t < kMlpH) {
        S.b1[t] = bf(theta[kOffB1 + t]);
        S.b2[t] = bf(theta[kOffB2 + t]);
        S.w3[t] = bf(theta[kOffW3 + t]);
    }
    if (t == 0) {
        S.b3 = bf(theta[kOffB3]);
        tc::mbar_init(&S.mbar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&S.tmem, kTcCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = S.tmem;
    const uint32_t d1 = tmem, d2 = tmem + kMlpH;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const uint64_t dw1 = tc::smem_desc(tc::smem_u32(S.w1t), 128, (kMlpF / 8) * 128);
    const uint64_t dx = tc::smem_desc(tc::smem_u32(S.xa), 128, (kMlpF / 8) * 128);
    uint32_t phase = 0;
    bool ok = true;
    const int64_t ntiles = (count + kTcRows - 1) / kTcRows;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t e = tile * kTcRows + t;
        const bool valid = e < count;
        // features of row t into the A tile of layer 1
        uint4 xa0 = make_uint4(0, 0, 0, 0), xa1 = xa0;
        if (valid) {
            const uint4* p = reinterpret_cast<const uint4*>(X + e * kMlpF);
            xa0 = __ldcs(p);
            xa1 = __ldcs(p + 1);
        }
        *reinterpret_cast<uint4*>(S.xa + tc::kmajor_offset(t, 0, kMlpF / 8, 2)) = xa0;
        *reinterpret_cast<uint4*>(S.xa + tc::kmajor_offset(t, 8, kMlpF / 8, 2)) = xa1;
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (t == 0) {
            tc::fence_after_sync();
            tc::mma_bf16(d1, dx, dw1, kIdescL, false);
            tc::commit(&S.mbar);
        }
        const double n_e = valid ? __ldcs(N + e) : 0.0;
        const float s_e = valid ? __ldcs(scale + e) : 0.f;
        ok = tc::mbar_wait(&S.mbar, phase, status, wait_limit);
        phase ^= 1u;
        tc::fence_after_sync();
        // layer-1 epilogue: bias, ReLU, BF16 into the A tile of layer 2
#pragma unroll
        for (int c0 = 0; c0 < kMlpH; c0 += 16) {
            float v[16];
            tc::ld16(d1 + lane_base + c0, v);
            tc::ld_wait();
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i] + S.b1[c0 + i], 0.f);
            st_bf16x8(S.ha + tc::kmajor_offset(t, c0, kMlpH / 8, 2), v);
            st_bf16x8(S.ha + tc::kmajor_offset(t, c0 + 8, kMlpH / 8, 2), v + 8);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (t == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int kk = 0; kk < kMlpH / 16; ++kk) {
                const uint64_t da = tc::smem_desc(tc::smem_u32(S.ha) + kk * 256, 128, (kMlpH / 8) * 128);
                const uint64_t db = tc::smem_desc(tc::smem_u32(S.w2t) + kk * 256, 128, (kMlpH / 8) * 128);
                tc::mma_bf16(d2, da, db, kIdescL, kk > 0);
            }
            tc::commit(&S.mbar);
        }
        ok = tc::mbar_wait(&S.mbar, phase, status, wait_limit) && ok;
        phase ^= 1u;
        tc::fence_after_sync();
        // layer-2 epilogue and the output unit
        float o = S.b3;
#pragma unroll
        for (int c0 = 0; c0 < kMlpH; c0 += 16) {
            float v[16];
            tc::ld16(d2 + lane_base + c0, v);
            tc::ld_wait();
#pragma unroll
            for (int i = 0; i < 16; ++i) o = fmaf(fmaxf(v[i] + S.b2[c0 + i], 0.f), S.w3[c0 + i], o);
        }
        if (valid) __stcs(out + e, n_e + (double)s_e * (double)o);
        tc::fence_before_sync();
        // every thread leaves a tile only after the MMAs have finished with its
        // operand tiles and accumulators (the waits above), so they can be reused
        ok = __syncthreads_and(ok) != 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, kTcCols);
}

}  // namespace

cudaError_t mlp_configure() {
    cudaError_t e = cudaFuncSetAttribute(fwd_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem));
    if (e != cudaSuccess) return e;
    static_assert(sizeof(PredictSmem) <= kPredictSmem, "predict shared memory");
    return cudaFuncSetAttribute(predict_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPredictSmem);
}

int mlp_train_blocks(int64_t count) { return (int)((count + kB - 1) / kB); }

cudaError_t mlp_features_launch(int64_t n, const int64_t* Srp, const int32_t* Sc, const int64_t* Lrp,
                                const int64_t* Lcp, int m, const double* Nst, int64_t nnzS, const double* Lval,
                                const double* Dval, const int32_t* dpos, const int8_t* pstart, void* X, float* scale,
                                int num_sms, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    trace_begin("mlp_features", st);
    features_kernel<<<num_sms * 8, 256, 0, st>>>(n, Srp, Sc, Lrp, Lcp, m, Nst, nnzS, Lval, Dval, dpos, pstart,
                                                 reinterpret_cast<__nv_bfloat16*>(X), scale);
    trace_end(st);
    return cudaGetLastError();
}

cudaError_t mlp_targets_launch(int64_t count, const double* G, const double* N, const float* scale, float* y,
                               int num_sms, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    targets_kernel<<<num_sms * 4, 256, 0, st>>>(count, G, N, scale, y);
    return cudaGetLastError();
}

cudaError_t mlp_grad_launch(const void* X, const float* y, const int64_t* idx, int64_t count, const float* theta,
                            float* partial, float* loss_partial, float* grad, float* loss, cudaStream_t st) {
    const int nblk = mlp_train_blocks(count);
    if (nblk == 0) return cudaErrorInvalidValue;
    trace_begin("mlp_fwd_bwd", st);
    fwd_bwd_kernel<<<nblk, kB, sizeof(TrainSmem), st>>>(reinterpret_cast<const __nv_bfloat16*>(X), y, idx, count,
                                                        theta, partial, loss_partial);
    trace_end(st);
    trace_begin("mlp_reduce", st);
    reduce_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(partial, nblk, loss_partial, count, grad, loss);
    trace_end(st);
    return cudaGetLastError();
}

cudaError_t mlp_adam_launch(float* theta, float* m, float* v, const float* g, float lr, int step, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    trace_begin("mlp_adam", st);
    adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(theta, m, v, g, lr, b1, b2, 1e-8f, c1, c2);
    trace_end(st);
    return cudaGetLastError();
}

cudaError_t mlp_predict_launch(const void* X, const float* scale, const double* N, int64_t count, const float* theta,
                               double* out, int32_t* status, int64_t wait_limit, int num_sms, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const int64_t tiles = (count + kTcRows - 1) / kTcRows;
    // four CTAs per SM: their 128 TMEM columns each fill the SM's 512
    const int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms * 4);
    trace_begin("mlp_predict", st);
    predict_tc_kernel<<<grid, kTcRows, kPredictSmem, st>>>(
        reinterpret_cast<const __nv_bfloat16*>(X), scale, N, count, theta, out, status, wait_limit);
    trace_end(st);
    return cudaGetLastError();
}

}  // namespace sinv
