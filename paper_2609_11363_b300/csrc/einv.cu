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

// ---- persistent triangular solves -----------------------------------------------------
// One launch per solve instead of one per dependency level: a warp takes the next row
// (column) in level order from a ticket, waits (bounded) until every row it reads has
// been published with this call's epoch, computes its value and publishes it with a
// release store.  A row only waits for rows of earlier levels, handed out before its
// own ticket to warps that are running, so the schedule cannot deadlock.

__global__ void trsv_prepare(uint32_t* epoch, int32_t* tickets) {
    uint32_t e = *epoch + 1;
    *epoch = e == 0 ? 1 : e;
    tickets[0] = 0;
    tickets[1] = 0;
}

// y = L^{-1} b (L unit lower, by rows)
__global__ void trsv_fwd_persistent(int64_t n, const int32_t* __restrict__ rows, const int64_t* __restrict__ Lrp,
                                    const int32_t* __restrict__ Lcol, const double* __restrict__ Lval,
                                    const double* __restrict__ b, double* __restrict__ y, uint32_t* flags,
                                    const uint32_t* epoch_p, int32_t* ticket, int32_t* status, int64_t limit) {
    const int lane = threadIdx.x & 31;
    const uint32_t epoch = *epoch_p;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(ticket, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= n) break;
        const int i = rows[t];
        double s = 0.0;
        bool ok = true;
        for (int64_t q = Lrp[i] + lane; q < Lrp[i + 1]; q += 32) {
            const int c = Lcol[q];
            if (!wait_flag(flags + c, epoch, status, limit)) {
                ok = false;
                break;
            }
            s = fma(Lval[q], __ldcg(y + c), s);
        }
        if (!__all_sync(0xffffffffu, ok)) break;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            __stcg(y + i, b[i] - s);
            st_release(flags + i, epoch);
        }
    }
}

// x = L^{-T} w with w = D^{-1} y formed on the fly (D^{-1} by rows: diagonal, partner
// coefficient, partner), L by columns
__global__ void trsv_bwd_persistent(int64_t n, const int32_t* __restrict__ cols, const int64_t* __restrict__ Lcp,
                                    const int32_t* __restrict__ Lri, const int32_t* __restrict__ Lcsr,
                                    const double* __restrict__ Lval, const double* __restrict__ dr,
                                    const double* __restrict__ dp, const int32_t* __restrict__ part,
                                    const double* __restrict__ y, double* __restrict__ x, uint32_t* flags,
                                    const uint32_t* epoch_p, int32_t* ticket, int32_t* status, int64_t limit) {
    const int lane = threadIdx.x & 31;
    const uint32_t epoch = *epoch_p;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(ticket, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= n) break;
        const int j = cols[t];
        double s = 0.0;
        bool ok = true;
        for (int64_t q = Lcp[j] + lane; q < Lcp[j + 1]; q += 32) {
            const int r = Lri[q];
            if (!wait_flag(flags + r, epoch, status, limit)) {
                ok = false;
                break;
            }
            s = fma(Lval[Lcsr[q]], __ldcg(x + r), s);
        }
        if (!__all_sync(0xffffffffu, ok)) break;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const int32_t p = part[j];
            const double wj = p >= 0 ? fma(dr[j], y[j], dp[j] * y[p]) : dr[j] * y[j];
            __stcg(x + j, wj - s);
            st_release(flags + j, epoch);
        }
    }
}

// ---- single-CTA level-synchronous triangular solves ------------------------------------
// For factors whose levels hold few rows (the covariance example: about 12 rows per
// level over 3,289 levels), the hand-off between SMs costs more than the rows: one
// CTA walks the levels with a barrier between them.  A warp takes a row of the level;
// the row's bounds and its entries of L (which do not depend on the solution) for the
// next level are loaded before the barrier, so after it only the solution values are
// read.  Rows beyond 32 entries are read in a loop.
constexpr int kCtaSolve = 1024;

struct RowPre {
    int i;         // row (column), -1 when the warp has none in the level
    int64_t q0, q1;
    int c;         // this lane's first entry: column (row) and value, c = -1 when none
    double v;
};

__device__ __forceinline__ RowPre row_pre_fwd(int t, int t1, const int32_t* rows, const int64_t* Lrp,
                                               const int32_t* Lcol, const double* Lval, int lane) {
    RowPre p;
    p.i = t < t1 ? rows[t] : -1;
    p.q0 = p.i >= 0 ? Lrp[p.i] : 0;
    p.q1 = p.i >= 0 ? Lrp[p.i + 1] : 0;
    p.c = p.q0 + lane < p.q1 ? Lcol[p.q0 + lane] : -1;
    p.v = p.c >= 0 ? Lval[p.q0 + lane] : 0.0;
    return p;
}

__device__ __forceinline__ RowPre row_pre_bwd(int t, int t1, const int32_t* cols, const int64_t* Lcp,
                                               const int32_t* Lri, const int32_t* Lcsr, const double* Lval,
                                               int lane) {
    RowPre p;
    p.i = t < t1 ? cols[t] : -1;
    p.q0 = p.i >= 0 ? Lcp[p.i] : 0;
    p.q1 = p.i >= 0 ? Lcp[p.i + 1] : 0;
    p.c = p.q0 + lane < p.q1 ? Lri[p.q0 + lane] : -1;
    p.v = p.c >= 0 ? Lval[Lcsr[p.q0 + lane]] : 0.0;
    return p;
}

// y = L^{-1} b, levels [0, nlev) of the rows in level order (ptr[l] .. ptr[l+1])
__global__ void __launch_bounds__(kCtaSolve) trsv_fwd_cta(int nlev, const int32_t* __restrict__ ptr,
                                                          const int32_t* __restrict__ rows,
                                                          const int64_t* __restrict__ Lrp,
                                                          const int32_t* __restrict__ Lcol,
                                                          const double* __restrict__ Lval,
                                                          const double* __restrict__ b, double* y) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = kCtaSolve / 32;
    RowPre pre = row_pre_fwd(ptr[0] + wid, ptr[1], rows, Lrp, Lcol, Lval, lane);
    for (int l = 0; l < nlev; ++l) {
        const int t0 = ptr[l], t1 = ptr[l + 1];
        for (int t = t0 + wid; t < t1; t += nw) {
            const RowPre r = t == t0 + wid ? pre : row_pre_fwd(t, t1, rows, Lrp, Lcol, Lval, lane);
            double s = r.c >= 0 ? r.v * y[r.c] : 0.0;
            for (int64_t q = r.q0 + 32 + lane; q < r.q1; q += 32) s = fma(Lval[q], y[Lcol[q]], s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) y[r.i] = b[r.i] - s;
        }
        if (l + 1 < nlev) pre = row_pre_fwd(ptr[l + 1] + wid, ptr[l + 2], rows, Lrp, Lcol, Lval, lane);
        __syncthreads();  // the level's values are visible to the whole CTA
    }
}

// x = L^{-T} w with w = D^{-1} y on the fly, L by columns, levels of the solve with L^T
__global__ void __launch_bounds__(kCtaSolve) trsv_bwd_cta(int nlev, const int32_t* __restrict__ ptr,
                                                          const int32_t* __restrict__ cols,
                                                          const int64_t* __restrict__ Lcp,
                                                          const int32_t* __restrict__ Lri,
                                                          const int32_t* __restrict__ Lcsr,
                                                          const double* __restrict__ Lval,
                                                          const double* __restrict__ dr, const double* __restrict__ dp,
                                                          const int32_t* __restrict__ part,
                                                          const double* __restrict__ y, double* x) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = kCtaSolve / 32;
    RowPre pre = row_pre_bwd(ptr[0] + wid, ptr[1], cols, Lcp, Lri, Lcsr, Lval, lane);
    for (int l = 0; l < nlev; ++l) {
        const int t0 = ptr[l], t1 = ptr[l + 1];
        for (int t = t0 + wid; t < t1; t += nw) {
            const RowPre r = t == t0 + wid ? pre : row_pre_bwd(t, t1, cols, Lcp, Lri, Lcsr, Lval, lane);
            double s = r.c >= 0 ? r.v * x[r.c] : 0.0;
            for (int64_t q = r.q0 + 32 + lane; q < r.q1; q += 32) s = fma(Lval[Lcsr[q]], x[Lri[q]], s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) {
                const int j = r.i;
                const int32_t p = part[j];
                const double wj = p >= 0 ? fma(dr[j], y[j], dp[j] * y[p]) : dr[j] * y[j];
                x[j] = wj - s;
            }
        }
        if (l + 1 < nlev) pre = row_pre_bwd(ptr[l + 1] + wid, ptr[l + 2], cols, Lcp, Lri, Lcsr, Lval, lane);
        __syncthreads();
    }
}

// |D|^{-1} by rows, from D itself: for a 1x1 pivot 1/|d|; for a 2x2 block [a b; b d]
// with eigenpairs (l_k, u_k) (the closed form of a symmetric 2x2), sum_k u_k u_k^T /
// |l_k| -- the inverse of the block's absolute value, so that L |D| L^T is an SPD
// preconditioner.  Written as diagonal, partner coefficient and partner per row, like
// D^{-1} (part = -1 for a 1x1 pivot).
__global__ void absdinv_rows(int64_t n, const int32_t* __restrict__ dpos, const int8_t* __restrict__ pstart,
                             const double* __restrict__ Dval, double* __restrict__ dr, double* __restrict__ dp,
                             int32_t* __restrict__ part, int32_t* status) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const bool first = pstart[r] != 0;
        const bool two = first ? (r + 1 < n && pstart[r + 1] == 0) : true;
        const double* dv = Dval + dpos[r];
        if (!two) {
            if (dv[0] == 0.0) set_status(status, ST_SINGULAR);
            dr[r] = 1.0 / fabs(dv[0]);
            dp[r] = 0.0;
            part[r] = -1;
            continue;
        }
        const double a = dv[0], b = dv[1], d = dv[2];
        const double mean = 0.5 * (a + d), rad = sqrt(0.25 * (a - d) * (a - d) + b * b);
        const double l1 = mean + rad, l2 = mean - rad;
        if (l1 == 0.0 || l2 == 0.0) set_status(status, ST_SINGULAR);
        // unit eigenvector u of l1: (b, l1 - a) or (l1 - d, b), the larger of the two
        double u0 = b, u1 = l1 - a;
        if (fabs(l1 - d) > fabs(l1 - a)) {
            u0 = l1 - d;
            u1 = b;
        }
        const double nu = sqrt(u0 * u0 + u1 * u1);
        if (nu > 0.0) {
            u0 /= nu;
            u1 /= nu;
        } else {  // b = 0 and a = d: any basis
            u0 = 1.0;
            u1 = 0.0;
        }
        // |D|^{-1} = u u^T / |l1| + v v^T / |l2|, v = (-u1, u0)
        const double i1 = 1.0 / fabs(l1), i2 = 1.0 / fabs(l2);
        dr[r] = first ? u0 * u0 * i1 + u1 * u1 * i2 : u1 * u1 * i1 + u0 * u0 * i2;
        dp[r] = u0 * u1 * (i1 - i2);
        part[r] = (int32_t)(first ? r + 1 : r - 1);
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

cudaError_t einv_precond_persistent(const EinvArgs& a, const double* r, double* y, double* z, cudaStream_t st) {
    if (a.cta_solve) {
        trsv_fwd_cta<<<1, kCtaSolve, 0, st>>>(a.nlev_fwd, a.fwd_ptr, a.fwd_rows, a.Lrp, a.Lcol, a.Lval, r, y);
        trsv_bwd_cta<<<1, kCtaSolve, 0, st>>>(a.nlev_bwd, a.bwd_ptr, a.bwd_cols, a.Lcp, a.Lri, a.Lcsr, a.Lval, a.dr,
                                              a.dp, a.part, y, z);
        return cudaGetLastError();
    }
    trsv_prepare<<<1, 1, 0, st>>>(a.tepoch, a.tickets);
    const int grid = a.num_sms * 8;  // 8 warps of 32 per CTA, 8 CTAs per SM
    trsv_fwd_persistent<<<grid, 256, 0, st>>>(a.n, a.fwd_rows, a.Lrp, a.Lcol, a.Lval, r, y, a.fwd_flags, a.tepoch,
                                              a.tickets, a.status, a.wait_limit);
    trsv_bwd_persistent<<<grid, 256, 0, st>>>(a.n, a.bwd_cols, a.Lcp, a.Lri, a.Lcsr, a.Lval, a.dr, a.dp, a.part, y, z,
                                              a.bwd_flags, a.tepoch, a.tickets + 1, a.status, a.wait_limit);
    return cudaGetLastError();
}

cudaError_t einv_absdinv(const EinvArgs& a, const int32_t* dpos, const int8_t* pstart, const double* Dval, double* dr,
                         double* dp, int32_t* part, cudaStream_t st) {
    absdinv_rows<<<grid_for(a.n, a.num_sms), kThreads, 0, st>>>(a.n, dpos, pstart, Dval, dr, dp, part, a.status);
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
