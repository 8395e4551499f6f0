// SPAI refinement on a fixed pattern P (Section 2.4): for every column j,
// Jacobi-preconditioned CG on the normal equations of  min ||A m_j - e_j||_2
// over m_j supported on J_j = {i : (i, j) in P}, started from the current
// values (given on S, zero on the rest of P); then (Y + Y^T) / 2 on P_lo.
// P = S, or S widened by the graph-distance neighbourhoods of A.
//
// One group of threads owns a column for the whole solve.  Its operands live
// in shared memory (a warp per column) or, for columns beyond the warp caps, in
// a CTA's shared memory or a per-CTA global scratch block (a CTA per column).
// The normal matrix B = A_J^T A_J is never formed: B v = A_J^T (A_J v) goes
// through a table y over the rows R = union of struct(A_k), k in J, in two
// passes with no floating-point atomics:
//   y_c = sum over the entries (k, r_c) of the rows k in J of  A_{r_c k} v_k,
//   q_k = sum over the entries (k, r) of row k of  A_rk y_{c(r)}.
// The entries (A_rk, k, c(r)) are staged once per column: a hash insert of r,
// a compaction of the table to ids c, and a counting sort of the entries by c
// give both orders; every CG step reuses them.  A is symmetric, so row k of A
// is read as column k.
#include "device.cuh"
#include "kernels.h"

namespace sinv {

namespace {

constexpr int kWarpsPerCta = 4;
constexpr int kCtaThreads = 128;

// shared-memory footprint of one warp's column (tier W)
struct WarpLayout {
    static constexpr int kE = kSpaiWarpE;  // staged entries
    static constexpr int kJ = kSpaiWarpJ;  // pattern rows of the column
    static constexpr int kH = kSpaiWarpH;  // table slots (>= 2 R for tier-W columns)
    static constexpr size_t kEa = 0;                                        // double[kE]
    static constexpr size_t kPart = kEa + sizeof(double) * kE;              // double[kE] partial sums
    static constexpr size_t kY = kPart + sizeof(double) * kE;               // double[kH]: y, or keys + ids
    static constexpr size_t kVec = kY + sizeof(double) * kH;                // x r p q dinv: double[5 kJ]
    static constexpr size_t kScal = kVec + sizeof(double) * 5 * kJ;         // double[2]
    static constexpr size_t kSoff = kScal + sizeof(double) * 2;             // int32[kH + 1]
    static constexpr size_t kEt = kSoff + sizeof(int32_t) * (kH + 1);       // uint16[kE] row run t
    static constexpr size_t kEs = kEt + sizeof(uint16_t) * kE;              // uint16[kE] table id c
    static constexpr size_t kPerm = kEs + sizeof(uint16_t) * kE;            // uint16[kE] entries by id
    static constexpr size_t kOff = (kPerm + sizeof(uint16_t) * kE + 3) / 4 * 4;  // int32[kJ + 1]
    static constexpr size_t kBytes = (kOff + sizeof(int32_t) * (kJ + 1) + 15) / 16 * 16;
};
static_assert(kSpaiWarpE <= 65536 && kSpaiWarpJ <= 65536 && kSpaiWarpH <= 65536, "16-bit entry indices");

struct WarpGroup {
    __device__ static int size() { return 32; }
    __device__ static int rank() { return threadIdx.x & 31; }
    __device__ static void sync() { __syncwarp(); }
    // butterfly: every lane ends with the same bits (each stage adds the same two values)
    __device__ static double sum(double v, double*) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    }
    __device__ static int scan_excl(int v, int*, int* total) {
        const int lane = threadIdx.x & 31;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        *total = __shfl_sync(0xffffffffu, x, 31);
        return x - v;
    }
    __device__ static int broadcast(int v, int*) { return __shfl_sync(0xffffffffu, v, 0); }
};

struct CtaGroup {
    static constexpr int kW = kCtaThreads / 32;
    __device__ static int size() { return kCtaThreads; }
    __device__ static int rank() { return threadIdx.x; }
    __device__ static void sync() { __syncthreads(); }
    __device__ static int scan_excl(int v, int* tmp, int* total) {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) tmp[w] = x;
        __syncthreads();
        int pre = 0, tot = 0;
#pragma unroll
        for (int u = 0; u < kW; ++u) {
            if (u < w) pre += tmp[u];
            tot += tmp[u];
        }
        __syncthreads();
        *total = tot;
        return pre + x - v;
    }
    __device__ static int broadcast(int v, int* cell) {
        if (threadIdx.x == 0) *cell = v;
        __syncthreads();
        int r = *cell;
        __syncthreads();
        return r;
    }
};

template <class I>
struct ColumnMem {
    double* ea;      // staged A values, in row-run order
    double* part;    // partial sums of the products, at the last entry of each piece
    double* y;       // row table; while staging, int32 keys[h] then int32 ids[h]
    double* x;
    double* r;
    double* p;
    double* q;
    double* dinv;
    int32_t* soff;   // per table id: end of its run in perm (start = end of the previous id)
    I* et;           // per entry: its pattern row t
    I* es;           // per entry: its table id c
    I* perm;         // entries grouped by table id
    int32_t* eoff;   // nj + 1 entry offsets, one run per pattern row
    double* scal;    // 2 scalars the vector warp hands to the group (stop flag, r.z)
    int32_t cap_h;   // table size available (power of two)
};

// One thread's contiguous share [lo, hi) of the staged entries, with the table id and
// the pattern row its first entry belongs to.  Every product walks the same shares, so
// each thread does the same number of multiply-adds (a warp's FP64 instruction costs
// the pipe the same however many of its lanes are active).  A share ends a piece at
// every segment end and at its own end; the piece sums are stored, not added with
// atomics, and one thread per segment adds its pieces up in a fixed order.
struct Share {
    int lo, hi, c, t;
    int chunk;  // odd, so that the lanes' shares start in different shared-memory banks
};

__device__ __forceinline__ uint32_t slot_hash(int32_t r, int shift) {
    return ((uint32_t)r * 2654435761u) >> shift;
}

// largest t in [0, nj) with eoff[t] <= o (rows with no entries have equal offsets)
__device__ __forceinline__ int run_of(const int32_t* eoff, int nj, int o) {
    int lo = 0, hi = nj - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (eoff[mid] <= o) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// in-place exclusive prefix sum of a[0, L) by the group (contiguous chunks per thread);
// returns the total.  Ends with a group barrier.
template <class G>
__device__ int group_scan(int32_t* a, int L, int* tmp) {
    const int tid = G::rank(), gsz = G::size();
    const int chunk = (L + gsz - 1) / gsz;
    const int lo = min(L, tid * chunk), hi = min(L, lo + chunk);
    int local = 0;
    for (int i = lo; i < hi; ++i) local += a[i];
    int total = 0;
    int run = G::scan_excl(local, tmp, &total);
    for (int i = lo; i < hi; ++i) {
        const int v = a[i];
        a[i] = run;
        run += v;
    }
    G::sync();
    return total;
}

// the sum of the pieces of the segment [beg, e): the piece at e - 1, plus one at
// every share end strictly inside (share ends sit at k * chunk - 1)
__device__ __forceinline__ double piece_sum(const double* part, int beg, int e, int chunk) {
    double v = part[e - 1];
    for (int p = (beg + chunk) / chunk * chunk - 1; p < e - 1; p += chunk) v += part[p];
    return v;
}

// q = B v = A_J^T (A_J v) over the staged entries: each thread sums its share in
// table-id order (pieces -> y), then in row order (pieces -> q)
template <class G, class I>
__device__ void apply_normal(const ColumnMem<I>& m, int nj, int R, const Share& sh, const double* v, double* q) {
    const int tid = G::rank(), gsz = G::size();
    if (sh.lo < sh.hi) {
        int c = sh.c, end = m.soff[c];
        double s = 0.0;
        for (int o2 = sh.lo; o2 < sh.hi; ++o2) {
            const int o = m.perm[o2];
            s = fma(m.ea[o], v[m.et[o]], s);
            if (o2 + 1 == end || o2 + 1 == sh.hi) {
                m.part[o2] = s;
                s = 0.0;
                if (o2 + 1 == end && o2 + 1 < sh.hi) end = m.soff[++c];  // every id owns an entry
            }
        }
    }
    G::sync();
    for (int c = tid; c < R; c += gsz) m.y[c] = piece_sum(m.part, c ? m.soff[c - 1] : 0, m.soff[c], sh.chunk);
    G::sync();
    if (sh.lo < sh.hi) {
        int t = sh.t, end = m.eoff[t + 1];
        double s = 0.0;
        for (int o = sh.lo; o < sh.hi; ++o) {
            s = fma(m.ea[o], m.y[m.es[o]], s);
            if (o + 1 == end || o + 1 == sh.hi) {
                m.part[o] = s;
                s = 0.0;
                if (o + 1 == end && o + 1 < sh.hi) {
                    do end = m.eoff[++t + 1];  // rows of A without entries end where they start
                    while (end == o + 1);
                }
            }
        }
    }
    G::sync();
    for (int t = tid; t < nj; t += gsz) {
        const int beg = m.eoff[t], e = m.eoff[t + 1];
        q[t] = beg == e ? 0.0 : piece_sum(m.part, beg, e, sh.chunk);
    }
    G::sync();
}

template <class G, class I>
__device__ void solve_column(const SpaiArgs& a, int j, const ColumnMem<I>& m, int* tmp) {
    const int tid = G::rank(), gsz = G::size();
    const int64_t c0 = a.fcp[j];
    const int nj = (int)(a.fcp[j + 1] - c0);
    const int E = a.fE[j];
    // table: the smallest power of two >= 2R (at least 32), within the space there is
    // (tier W has 2R <= kSpaiWarpH, tier C 2 max R)
    int h = 32;
    while (h < 2 * a.fR[j] && h < m.cap_h) h <<= 1;
    const int shift = 32 - (31 - __clz(h));
    int32_t* keys = reinterpret_cast<int32_t*>(m.y);
    int32_t* ids = keys + h;
    // while staging, p holds per pattern row t: (k, start of row k in A) (nnz(A) < 2^31)
    int2* rowk = reinterpret_cast<int2*>(m.p);
    for (int t = tid; t < nj; t += gsz) {
        const int k = a.fri[c0 + t];
        rowk[t] = make_int2(k, (int)a.Arp[k]);
        m.eoff[t] = a.feo[c0 + t];
        const int32_t src = a.fsrc[c0 + t];
        m.x[t] = src >= 0 ? a.X[src] : 0.0;  // start: X on S, zero on the rest of P
        m.r[t] = 0.0;                        // b = A_J^T e_j is written into r while staging
    }
    if (tid == 0) m.eoff[nj] = E;
    for (int i = tid; i < h; i += gsz) keys[i] = -1;
    G::sync();
    // stage the entries of rows k in J: value, run t and the table slot of the column index r
    for (int o = tid; o < E; o += gsz) {
        const int t = run_of(m.eoff, nj, o);
        const int64_t e = (int64_t)rowk[t].y + (o - m.eoff[t]);
        const int32_t rr = a.Acol[e];
        const double av = a.Aval[e];
        uint32_t s = slot_hash(rr, shift);
        for (int probe = 0;; ++probe) {
            const int32_t old = atomicCAS(keys + s, -1, rr);
            if (old == -1 || old == rr) break;
            s = (s + 1) & (uint32_t)(h - 1);
            if (probe >= h) {  // cannot happen: the table has more slots than distinct rows
                set_status(a.status, ST_INTERNAL);
                break;
            }
        }
        m.ea[o] = av;
        m.et[o] = (I)t;
        m.es[o] = (I)s;
        if (rr == j) m.r[t] = av;  // (A_J^T e_j)_t = A(j, k)
    }
    G::sync();
    // compact the occupied slots to ids 0..R-1
    for (int i = tid; i < h; i += gsz) ids[i] = keys[i] != -1 ? 1 : 0;
    G::sync();
    const int R = group_scan<G>(ids, h, tmp);
    for (int c = tid; c <= R; c += gsz) m.soff[c] = 0;
    for (int o = tid; o < E; o += gsz) m.es[o] = (I)ids[m.es[o]];
    G::sync();
    // counting sort of the entries by id
    for (int o = tid; o < E; o += gsz) atomicAdd(m.soff + m.es[o], 1);
    G::sync();
    group_scan<G>(m.soff, R, tmp);
    for (int o = tid; o < E; o += gsz) m.perm[atomicAdd(m.soff + m.es[o], 1)] = (I)o;
    G::sync();
    for (int t = tid; t < nj; t += gsz) {
        double s = 0.0;
        for (int o = m.eoff[t]; o < m.eoff[t + 1]; ++o) s += m.ea[o] * m.ea[o];
        m.dinv[t] = s != 0.0 ? 1.0 / s : 0.0;  // Jacobi: diag(B)_k = ||A e_k||^2
    }
    // this thread's share of the entries, with the id and row of its first entry
    Share sh;
    {
        const int chunk = ((E + gsz - 1) / gsz) | 1;
        sh.chunk = chunk;
        sh.lo = min(E, tid * chunk);
        sh.hi = min(E, sh.lo + chunk);
        sh.t = sh.lo < sh.hi ? run_of(m.eoff, nj, sh.lo) : 0;
        int lo = 0, hi = R - 1;  // smallest c with soff[c] > sh.lo
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (m.soff[mid] > sh.lo) hi = mid; else lo = mid + 1;
        }
        sh.c = lo;
    }
    // the CG vector work (a few vectors of nj) runs on the group's first warp; its
    // scalars reach the other threads through m.scal
    const bool vw = tid < 32;
    const int lane = tid & 31;
    // r = b - B x, z = D^{-1} r, p = z
    apply_normal<G>(m, nj, R, sh, m.x, m.q);
    if (vw) {
        double rz = 0.0;
        for (int t = lane; t < nj; t += 32) {
            const double rt = m.r[t] - m.q[t];
            const double zt = m.dinv[t] * rt;
            m.r[t] = rt;
            m.p[t] = zt;
            rz += rt * zt;
        }
        rz = WarpGroup::sum(rz, nullptr);
        if (lane == 0) m.scal[1] = rz;
    }
    G::sync();
    double rz = m.scal[1];
    for (int it = 0; it < a.iters; ++it) {
        if (rz == 0.0) break;
        apply_normal<G>(m, nj, R, sh, m.p, m.q);
        if (vw) {
            double pq = 0.0;
            for (int t = lane; t < nj; t += 32) pq += m.p[t] * m.q[t];
            pq = WarpGroup::sum(pq, nullptr);
            double rzn = 0.0;
            const bool stop = !(pq > 0.0);
            if (!stop) {
                const double alpha = rz / pq;
                for (int t = lane; t < nj; t += 32) {
                    m.x[t] += alpha * m.p[t];
                    const double rt = m.r[t] - alpha * m.q[t];
                    m.r[t] = rt;
                    rzn += rt * (m.dinv[t] * rt);
                }
                rzn = WarpGroup::sum(rzn, nullptr);
                const double beta = rzn / rz;
                for (int t = lane; t < nj; t += 32) m.p[t] = m.dinv[t] * m.r[t] + beta * m.p[t];
            }
            if (lane == 0) {
                m.scal[0] = stop ? 1.0 : 0.0;
                m.scal[1] = rzn;
            }
        }
        G::sync();
        if (m.scal[0] != 0.0) break;
        rz = m.scal[1];
        G::sync();  // every thread has read the scalars before the vector warp rewrites them
    }
    // (Y + Y^T)/2: an off-diagonal entry of P_lo gets exactly two halves (from column j
    // and from column i) added to a zeroed Y, so the result does not depend on their order
    for (int t = tid; t < nj; t += gsz) {
        const int k = a.fri[c0 + t];
        const int32_t pos = a.fpos[c0 + t];
        if (k == j) a.Y[pos] = m.x[t];
        else atomicAdd(a.Y + pos, 0.5 * m.x[t]);
    }
    G::sync();
}

__global__ void __launch_bounds__(kWarpsPerCta * 32) spai_warp_kernel(SpaiArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    using L = WarpLayout;
    unsigned char* base = smem + (size_t)(threadIdx.x >> 5) * L::kBytes;
    ColumnMem<uint16_t> m;
    m.ea = reinterpret_cast<double*>(base + L::kEa);
    m.part = reinterpret_cast<double*>(base + L::kPart);
    m.y = reinterpret_cast<double*>(base + L::kY);
    double* vec = reinterpret_cast<double*>(base + L::kVec);
    m.x = vec;
    m.r = vec + L::kJ;
    m.p = vec + 2 * L::kJ;
    m.q = vec + 3 * L::kJ;
    m.dinv = vec + 4 * L::kJ;
    m.scal = reinterpret_cast<double*>(base + L::kScal);
    m.soff = reinterpret_cast<int32_t*>(base + L::kSoff);
    m.et = reinterpret_cast<uint16_t*>(base + L::kEt);
    m.es = reinterpret_cast<uint16_t*>(base + L::kEs);
    m.perm = reinterpret_cast<uint16_t*>(base + L::kPerm);
    m.eoff = reinterpret_cast<int32_t*>(base + L::kOff);
    m.cap_h = L::kH;
    for (;;) {
        int c = 0;
        if ((threadIdx.x & 31) == 0) c = atomicAdd(a.ticket, 1);
        c = WarpGroup::broadcast(c, nullptr);
        if (c >= a.ncols) break;
        solve_column<WarpGroup>(a, a.cols[c], m, nullptr);
    }
}

template <bool kSmem>
__global__ void __launch_bounds__(kCtaThreads) spai_cta_kernel(SpaiArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double scal[2];
    __shared__ int tmp[CtaGroup::kW];
    __shared__ int cell;
    const int64_t cj = a.cap_nj, cE = a.cap_E, cH = a.cap_H;
    unsigned char* base = kSmem ? smem
                                : reinterpret_cast<unsigned char*>(a.scratch) + (size_t)blockIdx.x * (size_t)a.cta_bytes;
    ColumnMem<int32_t> m;
    m.ea = reinterpret_cast<double*>(base);
    m.part = m.ea + cE;
    m.y = m.part + cE;
    m.x = m.y + cH;
    m.r = m.x + cj;
    m.p = m.r + cj;
    m.q = m.p + cj;
    m.dinv = m.q + cj;
    m.soff = reinterpret_cast<int32_t*>(m.dinv + cj);
    m.et = m.soff + cH + 1;
    m.es = m.et + cE;
    m.perm = m.es + cE;
    m.eoff = m.perm + cE;
    m.scal = scal;
    m.cap_h = (int32_t)cH;
    for (;;) {
        int c = CtaGroup::broadcast(threadIdx.x == 0 ? atomicAdd(a.ticket + 1, 1) : 0, &cell);
        if (c >= a.ncols_cta) break;
        solve_column<CtaGroup>(a, a.cols_cta[c], m, tmp);
    }
}

}  // namespace

size_t spai_cta_bytes(int64_t cap_nj, int64_t cap_E, int64_t cap_H) {
    size_t b = sizeof(double) * (size_t)(2 * cap_E + cap_H + 5 * cap_nj) +
               sizeof(int32_t) * (size_t)((cap_H + 1) + 3 * cap_E + (cap_nj + 1));
    return (b + 255) / 256 * 256;
}

cudaError_t spai_configure() {
    cudaError_t e = cudaFuncSetAttribute(spai_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(WarpLayout::kBytes * kWarpsPerCta));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(spai_cta_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSpaiCtaSmemMax);
}

// tier C in shared memory: as many CTAs as fit on every SM; in global scratch: one per SM
int spai_cta_grid(int num_sms, int64_t ncols_cta, size_t cta_bytes) {
    int per_sm = 1;
    if (cta_bytes <= kSpaiCtaSmemMax) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spai_cta_kernel<true>, kCtaThreads, cta_bytes) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    return (int)std::min<int64_t>(ncols_cta, (int64_t)per_sm * num_sms);
}

cudaError_t spai_launch(const SpaiArgs& a, int num_sms, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(a.Y, 0, sizeof(double) * (size_t)a.nnzP, st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.ticket, 0, 2 * sizeof(int32_t), st)) != cudaSuccess) return e;
    if (a.ncols > 0) {
        int per_sm = 0;
        const size_t smem = WarpLayout::kBytes * kWarpsPerCta;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spai_warp_kernel, kWarpsPerCta * 32, smem) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        const int64_t need = (a.ncols + kWarpsPerCta - 1) / kWarpsPerCta;
        const int grid = (int)std::min<int64_t>(need, (int64_t)per_sm * num_sms);
        trace_begin("spai_warp", st);
        spai_warp_kernel<<<grid, kWarpsPerCta * 32, smem, st>>>(a);
        trace_end(st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (a.ncols_cta > 0) {
        const int grid = spai_cta_grid(num_sms, a.ncols_cta, (size_t)a.cta_bytes);
        trace_begin("spai_cta", st);
        if (a.cta_in_smem)
            spai_cta_kernel<true><<<grid, kCtaThreads, (size_t)a.cta_bytes, st>>>(a);
        else
            spai_cta_kernel<false><<<grid, kCtaThreads, 0, st>>>(a);
        trace_end(st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sinv
