// Spectral-correction producer (Section 2.5): the kernels of Lanczos with full
// reorthogonalisation on E_inv = A^{-1} - A^inv, where A^{-1} x comes from
// conjugate gradients preconditioned by the ILDL factors,
//   M^{-1} = L^{-T} D^{-1} L^{-1},
// and A^inv x is the approximate inverse on S applied as a symmetric sparse
// matrix.  The iteration itself (scalars, stopping tests) runs on the host in
// api.cu; every vector operation is one of these kernels.  Reductions are two-
// stage with a fixed grid, so every dot product is reproducible.
#include "device.cuh"
#include "kernels.h"

namespace sinv {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int u = 0; u < (int)(blockDim.x >> 5); ++u) s += red[u];
    return s;  // valid in thread 0
}

// y = A x (A in CSR)
__global__ void spmv_csr(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                         const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) s = fma(val[q], x[col[q]], s);
        y[i] = s;
    }
}

// y = X x, X symmetric given on S_lo, read through the columns of S (row i = column i)
__global__ void symv_S(int64_t n, const int64_t* __restrict__ fcp, const int32_t* __restrict__ fri,
                       const int32_t* __restrict__ fpos, const double* __restrict__ X, const double* __restrict__ x,
                       double* __restrict__ y) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t q = fcp[i]; q < fcp[i + 1]; ++q) s = fma(X[fpos[q]], x[fri[q]], s);
        y[i] = s;
    }
}

// one level of L y = b (unit lower): the rows of the level, each reading rows of earlier levels
__global__ void trsv_fwd_level(const int32_t* __restrict__ rows, int count, const int64_t* __restrict__ Lrp,
                               const int32_t* __restrict__ Lcol, const double* __restrict__ Lval,
                               const double* __restrict__ b, double* __restrict__ y) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= count) return;
    const int i = rows[u];
    double s = b[i];
    for (int64_t q = Lrp[i]; q < Lrp[i + 1]; ++q) s = fma(-Lval[q], y[Lcol[q]], s);
    y[i] = s;
}

// one level of L^T x = w: column j reads x at the rows i > j of column j of L
__global__ void trsv_bwd_level(const int32_t* __restrict__ cols, int count, const int64_t* __restrict__ Lcp,
                               const int32_t* __restrict__ Lri, const int32_t* __restrict__ Lcsr,
                               const double* __restrict__ Lval, const double* __restrict__ w,
                               double* __restrict__ x) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= count) return;
    const int j = cols[u];
    double s = w[j];
    for (int64_t q = Lcp[j]; q < Lcp[j + 1]; ++q) s = fma(-Lval[Lcsr[q]], x[Lri[q]], s);
    x[j] = s;
}

// w = D^{-1} y with the per-row diagonal, partner coefficient and partner of D^{-1}
__global__ void dinv_apply(int64_t n, const double* __restrict__ dr, const double* __restrict__ dp,
                           const int32_t* __restrict__ part, const double* __restrict__ y, double* __restrict__ w) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = part[i];
        w[i] = p >= 0 ? fma(dr[i], y[i], dp[i] * y[p]) : dr[i] * y[i];
    }
}

// per-block partial sums of a . b (a fixed grid: the sum is reproducible)
__global__ void dot_partial(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                            double* __restrict__ partial) {
    __shared__ double red[kThreads / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s = fma(a[i], b[i], s);
    s = block_sum(s, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void sum_final(const double* __restrict__ partial, int count, double* __restrict__ out) {
    __shared__ double red[kThreads / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) s += partial[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *out = s;
}

// x += alpha p ; r -= alpha q
__global__ void cg_xr(int64_t n, double alpha, const double* __restrict__ p, const double* __restrict__ q,
                      double* __restrict__ x, double* __restrict__ r) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        r[i] = fma(-alpha, q[i], r[i]);
    }
}

// p = z + beta p
__global__ void cg_p(int64_t n, double beta, const double* __restrict__ z, double* __restrict__ p) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], z[i]);
}

// out = a * x + b * y
__global__ void axpby(int64_t n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                      double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a * x[i] + b * y[i];
}

// c[l] = Q[:, l] . v for l < ncols (one block per column; Q column-major, leading dimension n)
__global__ void qt_v(int64_t n, const double* __restrict__ Q, const double* __restrict__ v, double* __restrict__ c) {
    __shared__ double red[kThreads / 32];
    const double* ql = Q + (int64_t)blockIdx.x * n;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(ql[i], v[i], s);
    s = block_sum(s, red);
    if (threadIdx.x == 0) c[blockIdx.x] = s;
}

// v -= Q[:, :ncols] c
__global__ void v_minus_qc(int64_t n, int ncols, const double* __restrict__ Q, const double* __restrict__ c,
                           double* __restrict__ v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int l = 0; l < ncols; ++l) s = fma(Q[(int64_t)l * n + i], c[l], s);
        v[i] -= s;
    }
}

// Cyclic Jacobi on the dense symmetric m x m matrix T (row-major, overwritten; its
// diagonal ends with the eigenvalues), accumulating the rotations in U (U starts as
// I).  Rotation angles by the classical formula: theta = (t_qq - t_pp) / (2 t_pq),
// tan = sign(theta) / (|theta| + sqrt(theta^2 + 1)).  Sweeps stop once the off-diagonal
// sum of squares is below tol^2 times the total, or after max_sweeps.  Then the k
// eigenvalues of largest modulus go to sel[0..k) (ties: the lower index first).
__global__ void jacobi_eig(int m, double* __restrict__ T, double* __restrict__ U, int max_sweeps, double tol, int k,
                           int32_t* __restrict__ sel, double* __restrict__ lam) {
    __shared__ double cs[2];
    __shared__ double red[kThreads / 32];
    __shared__ int done;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) U[e] = (e / m == e % m) ? 1.0 : 0.0;
    __syncthreads();
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const double t = T[e] * T[e];
            tot += t;
            if (e / m != e % m) off += t;
        }
        off = block_sum(off, red);
        __syncthreads();
        tot = block_sum(tot, red);
        if (threadIdx.x == 0) done = !(off > tol * tol * tot);
        __syncthreads();
        if (done) break;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                if (threadIdx.x == 0) {
                    const double apq = T[p * m + q];
                    double c = 1.0, s = 0.0;
                    if (apq != 0.0) {
                        const double theta = (T[q * m + q] - T[p * m + p]) / (2.0 * apq);
                        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                    }
                    cs[0] = c;
                    cs[1] = s;
                }
                __syncthreads();
                const double c = cs[0], s = cs[1];
                if (s != 0.0) {
                    // T <- J^T T J with J the rotation in the (p, q) plane: columns, then rows
                    for (int r = threadIdx.x; r < m; r += blockDim.x) {
                        const double tp = T[r * m + p], tq = T[r * m + q];
                        T[r * m + p] = c * tp - s * tq;
                        T[r * m + q] = s * tp + c * tq;
                        const double up = U[r * m + p], uq = U[r * m + q];
                        U[r * m + p] = c * up - s * uq;
                        U[r * m + q] = s * up + c * uq;
                    }
                    __syncthreads();
                    for (int r = threadIdx.x; r < m; r += blockDim.x) {
                        const double tp = T[p * m + r], tq = T[q * m + r];
                        T[p * m + r] = c * tp - s * tq;
                        T[q * m + r] = s * tp + c * tq;
                    }
                }
                __syncthreads();
            }
    }
    if (threadIdx.x == 0) {
        for (int l = 0; l < k; ++l) {
            int best = -1;
            for (int i = 0; i < m; ++i) {
                bool used = false;
                for (int u = 0; u < l; ++u) used = used || sel[u] == i;
                if (used) continue;
                if (best < 0 || fabs(T[i * m + i]) > fabs(T[best * m + best])) best = i;
            }
            sel[l] = best;
            lam[l] = T[best * m + best];
        }
    }
}

// V[i, l] = sum_j Q[i, j] U[j, sel[l]] for l < k (V row-major with row stride ldv)
__global__ void ritz_vectors(int64_t n, int m, int k, int ldv, const double* __restrict__ Q,
                             const double* __restrict__ U, const int32_t* __restrict__ sel, double* __restrict__ V) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int l = 0; l < k; ++l) {
            const int cidx = sel[l];
            double s = 0.0;
            for (int j = 0; j < m; ++j) s = fma(Q[(int64_t)j * n + i], U[j * m + cidx], s);
            V[i * ldv + l] = s;
        }
}

int grid_for(int64_t n, int num_sms) {
    const int64_t g = (n + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)num_sms * 8));
}

}  // namespace

int einv_dot_blocks(int num_sms) { return num_sms * 2; }

cudaError_t einv_spmv_A(const EinvArgs& a, const double* x, double* y, cudaStream_t st) {
    spmv_csr<<<grid_for(a.n, a.num_sms), kThreads, 0, st>>>(a.n, a.Arp, a.Acol, a.Aval, x, y);
    return cudaGetLastError();
}

cudaError_t einv_symv_X(const EinvArgs& a, const double* x, double* y, cudaStream_t st) {
    symv_S<<<grid_for(a.n, a.num_sms), kThreads, 0, st>>>(a.n, a.fcp, a.fri, a.fpos, a.X, x, y);
    return cudaGetLastError();
}

cudaError_t einv_precond(const EinvArgs& a, const double* r, double* y, double* w, double* z, cudaStream_t st) {
    for (int l = 0; l < a.nlev_fwd; ++l) {
        const int c = a.fwd_ptr_h[l + 1] - a.fwd_ptr_h[l];
        trsv_fwd_level<<<(c + kThreads - 1) / kThreads, kThreads, 0, st>>>(a.fwd_rows + a.fwd_ptr_h[l], c, a.Lrp,
                                                                            a.Lcol, a.Lval, r, y);
    }
    dinv_apply<<<grid_for(a.n, a.num_sms), kThreads, 0, st>>>(a.n, a.dr, a.dp, a.part, y, w);
    for (int l = 0; l < a.nlev_bwd; ++l) {
        const int c = a.bwd_ptr_h[l + 1] - a.bwd_ptr_h[l];
        trsv_bwd_level<<<(c + kThreads - 1) / kThreads, kThreads, 0, st>>>(a.bwd_cols + a.bwd_ptr_h[l], c, a.Lcp,
                                                                            a.Lri, a.Lcsr, a.Lval, w, z);
    }
    return cudaGetLastError();
}

cudaError_t einv_dot(const EinvArgs& a, const double* x, const double* y, double* partial, double* out,
                     cudaStream_t st) {
    const int nb = einv_dot_blocks(a.num_sms);
    dot_partial<<<nb, kThreads, 0, st>>>(a.n, x, y, partial);
    sum_final<<<1, kThreads, 0, st>>>(partial, nb, out);
    return cudaGetLastError();
}

cudaError_t einv_cg_xr(const EinvArgs& a, double alpha, const double* p, const double* q, double* x, double* r,
                       cudaStream_t st) {
    cg_xr<<<grid_for(a.n, a.num_sms), kThreads, 0, st>>>(a.n, alpha, p, q, x, r);
    return cudaGetLastError();
}

cudaError_t einv_cg_p(const EinvArgs& a, double beta, const double* z, double* p, cudaStream_t st) {
    cg_p<<<grid_for(a.n, a.num_sms), kThreads, 0, st>>>(a.n, beta, z, p);
    return cudaGetLastError();
}

cudaError_t einv_axpby(const EinvArgs& a, double alpha, const double* x, double beta, const double* y, double* out,
                       cudaStream_t st) {
    axpby<<<grid_for(a.n, a.num_sms), kThreads, 0, st>>>(a.n, alpha, x, beta, y, out);
    return cudaGetLastError();
}

cudaError_t einv_reorth(const EinvArgs& a, const double* Q, int ncols, double* c, double* v, cudaStream_t st) {
    qt_v<<<ncols, kThreads, 0, st>>>(a.n, Q, v, c);
    v_minus_qc<<<grid_for(a.n, a.num_sms), kThreads, 0, st>>>(a.n, ncols, Q, c, v);
    return cudaGetLastError();
}

cudaError_t einv_eig(int m, double* T, double* U, int k, int32_t* sel, double* lam, cudaStream_t st) {
    jacobi_eig<<<1, kThreads, 0, st>>>(m, T, U, 60, 1e-15, k, sel, lam);
    return cudaGetLastError();
}

cudaError_t einv_ritz(const EinvArgs& a, int m, int k, int ldv, const double* Q, const double* U,
                      const int32_t* sel, double* V, cudaStream_t st) {
    ritz_vectors<<<grid_for(a.n, a.num_sms), kThreads, 0, st>>>(a.n, m, k, ldv, Q, U, sel, V);
    return cudaGetLastError();
}

}  // namespace sinv
