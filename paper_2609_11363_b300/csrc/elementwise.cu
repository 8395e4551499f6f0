// Entry-wise work on S: Mix (Section 2.3) and the low-rank correction applied on
// S as a sampled dense product (Section 2.5, Eq. (9)).
#include <mutex>

#include "device.cuh"
#include "kernels.h"

namespace sinv {

namespace {

// (A_Mix)_ij = G_ij if |G_ij| > eps else N_ij.  Streams 2 x 8 B in, 8 B out per entry.
__global__ void mix_kernel(const double* __restrict__ G, const double* __restrict__ N, double eps,
                           double* __restrict__ M, int64_t nnz) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool vec = ((((uintptr_t)G) | ((uintptr_t)N) | ((uintptr_t)M)) & 15) == 0;
    if (vec) {
        const int64_t n2 = nnz >> 1;
        const double2* G2 = reinterpret_cast<const double2*>(G);
        const double2* N2 = reinterpret_cast<const double2*>(N);
        double2* M2 = reinterpret_cast<double2*>(M);
        for (int64_t i = i0; i < n2; i += stride) {
            double2 g = __ldcs(G2 + i), v = __ldcs(N2 + i), r;
            r.x = fabs(g.x) > eps ? g.x : v.x;
            r.y = fabs(g.y) > eps ? g.y : v.y;
            __stcs(M2 + i, r);
        }
        if (i0 == 0 && (nnz & 1)) {
            int64_t i = nnz - 1;
            M[i] = fabs(G[i]) > eps ? G[i] : N[i];
        }
    } else {
        for (int64_t i = i0; i < nnz; i += stride) M[i] = fabs(G[i]) > eps ? G[i] : N[i];
    }
}

constexpr int kLrWarps = 8;
constexpr int kKMax = kLowrankKMax;

// One warp per row i of S_lo: u = lambda .* V_i staged in shared memory, then
// every entry (i, j) of the row adds u . V_j.  R is the product type.
template <class R>
__global__ void __launch_bounds__(kLrWarps * 32) lowrank_kernel(int64_t n, const int64_t* __restrict__ Srp,
                                                                const int32_t* __restrict__ Sc, int k,
                                                                const R* __restrict__ V, const R* __restrict__ lam,
                                                                double* __restrict__ X) {
    __shared__ R u_s[kLrWarps][kKMax];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    R* u = u_s[wid];
    const int64_t nwarps = (int64_t)gridDim.x * kLrWarps;
    for (int64_t i = (int64_t)blockIdx.x * kLrWarps + wid; i < n; i += nwarps) {
        for (int l = lane; l < k; l += 32) u[l] = lam[l] * V[i * k + l];
        __syncwarp();
        const int64_t e0 = Srp[i], e1 = Srp[i + 1];
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const R* vj = V + (int64_t)Sc[e] * k;
            R s0 = R(0), s1 = R(0), s2 = R(0), s3 = R(0);
            int l = 0;
            for (; l + 4 <= k; l += 4) {
                s0 += u[l] * vj[l];
                s1 += u[l + 1] * vj[l + 1];
                s2 += u[l + 2] * vj[l + 2];
                s3 += u[l + 3] * vj[l + 3];
            }
            for (; l < k; ++l) s0 += u[l] * vj[l];
            X[e] += (double)((s0 + s1) + (s2 + s3));
        }
        __syncwarp();
    }
}

__global__ void to_float(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

__global__ void debug_wait_kernel(uint32_t* flag, int32_t* status, int64_t limit) {
    if (threadIdx.x == 0) wait_flag(flag, 0xFFFFFFFFu, status, limit);
}

}  // namespace

cudaError_t mix_launch(const double* G, const double* N, double eps, double* M, int64_t nnz, int num_sms,
                       cudaStream_t st) {
    if (nnz == 0) return cudaSuccess;
    int64_t blocks = (nnz / 2 + 255) / 256;
    int grid = (int)std::min<int64_t>(std::max<int64_t>(blocks, 1), (int64_t)num_sms * 8);
    trace_begin("mix", st);
    mix_kernel<<<grid, 256, 0, st>>>(G, N, eps, M, nnz);
    trace_end(st);
    return cudaGetLastError();
}

cudaError_t lowrank_launch(int64_t n, const int64_t* Srp, const int32_t* Sc, int k, const double* V,
                           const double* lambda, int prec, void* work, double* X, int num_sms,
                           cudaStream_t st) {
    if (n == 0 || k == 0) return cudaSuccess;
    int64_t blocks = (n + kLrWarps - 1) / kLrWarps;
    int grid = (int)std::min<int64_t>(blocks, (int64_t)num_sms * 16);
    if (prec == 0) {
        trace_begin("lowrank", st);
        lowrank_kernel<double><<<grid, kLrWarps * 32, 0, st>>>(n, Srp, Sc, k, V, lambda, X);
        trace_end(st);
    } else {
        float* Vf = reinterpret_cast<float*>(work);
        float* lf = Vf + n * (int64_t)k;
        trace_begin("lowrank_to_float", st);
        to_float<<<num_sms * 4, 256, 0, st>>>(V, Vf, n * (int64_t)k);
        to_float<<<1, 256, 0, st>>>(lambda, lf, k);
        trace_end(st);
        trace_begin("lowrank", st);
        lowrank_kernel<float><<<grid, kLrWarps * 32, 0, st>>>(n, Srp, Sc, k, Vf, lf, X);
        trace_end(st);
    }
    return cudaGetLastError();
}

// ---- the FP32 low-rank correction without any allocation --------------------------
// Callers that cannot allocate device memory get the FP32 form with its working copy
// of V and lambda in this file-scope array instead of a handle-owned buffer.  Every
// GPU that loads the library keeps these 16 MiB until the process exits.  All calls
// on a device share the array (each call overwrites the part it uses before reading
// it), so calls that overlap on the GPU race with each other.
static __device__ __align__(256) float g_lowrank_scratch[kLowrankStaticFloats];

namespace {
constexpr int kMaxDevices = 256;
std::mutex g_scratch_mu;
float* g_scratch_ptr[kMaxDevices] = {};
}  // namespace

// The array's device address for the current device, looked up once per device (the
// first call on a device does this, so it must come before any stream capture).
static cudaError_t lowrank_static_scratch(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_lowrank_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = reinterpret_cast<float*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

cudaError_t lowrank_noalloc_launch(int64_t n, const int64_t* Srp, const int32_t* Sc, int k, const double* V,
                                   const double* lambda, double* X, cudaStream_t st) {
    if (n == 0 || k == 0) return cudaSuccess;
    if (k < 0 || k > kKMax || n * (int64_t)k + k > kLowrankStaticFloats) return cudaErrorInvalidValue;
    float* Vf = nullptr;
    cudaError_t e = lowrank_static_scratch(&Vf);
    if (e != cudaSuccess) return e;
    int dev = 0, num_sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    float* lf = Vf + n * (int64_t)k;
    const int64_t blocks = (n + kLrWarps - 1) / kLrWarps;
    const int grid = (int)std::min<int64_t>(blocks, (int64_t)num_sms * 16);
    to_float<<<num_sms * 4, 256, 0, st>>>(V, Vf, n * (int64_t)k);
    to_float<<<1, 256, 0, st>>>(lambda, lf, k);
    lowrank_kernel<float><<<grid, kLrWarps * 32, 0, st>>>(n, Srp, Sc, k, Vf, lf, X);
    return cudaGetLastError();
}

cudaError_t debug_wait_launch(uint32_t* flag, int32_t* status, int64_t limit, cudaStream_t st) {
    debug_wait_kernel<<<1, 32, 0, st>>>(flag, status, limit);
    return cudaGetLastError();
}

}  // namespace sinv

// ---- batched runs: per-matrix buffers <-> the batch handle's concatenated layout ----
namespace sinv {
namespace {

// blockIdx.y = matrix of this launch's slice; the pointers travel as a kernel argument,
// so a captured graph replays with the same buffers and no host work
__global__ void batch_copy_kernel(BatchPtrs ptrs, const int64_t* __restrict__ off, int32_t first, int to_cat,
                                  double* __restrict__ cat) {
    const int b = blockIdx.y;
    const int64_t o0 = off[first + b], len = off[first + b + 1] - o0;
    double* mine = const_cast<double*>(ptrs.p[b]);
    if (!mine) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        if (to_cat)
            cat[o0 + e] = __ldg(mine + e);
        else
            mine[e] = cat[o0 + e];
    }
}

}  // namespace

cudaError_t batch_copy_launch(int32_t nmat, const double* const* ptrs, const int64_t* d_off, int to_cat, double* cat,
                              int num_sms, cudaStream_t st) {
    for (int32_t b0 = 0; b0 < nmat; b0 += kBatchPtrs) {
        BatchPtrs bp;
        const int32_t cnt = std::min<int32_t>(kBatchPtrs, nmat - b0);
        for (int32_t b = 0; b < kBatchPtrs; ++b) bp.p[b] = b < cnt ? ptrs[b0 + b] : nullptr;
        dim3 grid((unsigned)std::max(1, 2 * num_sms / std::max(1, (int)std::min(cnt, 64))), (unsigned)cnt);
        batch_copy_kernel<<<grid, 256, 0, st>>>(bp, d_off, b0, to_cat, cat);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sinv
