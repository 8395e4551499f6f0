// Supernodal selected inversion (Section 2.1, Eqs. (4)-(5)) as one
// persistent kernel.
//
// For a supernode J (consecutive pivot blocks [s0, s0+w)) with row set C below
// it, one step of the Takahashi recurrence is
//     Lh   = L_CJ L_JJ^{-1}                         (c x w)
//     X    = -G~_CC Lh                              (G~ = G on S, 0 off S)
//     G_JJ = L_JJ^{-T} D_J^{-1} L_JJ^{-1} - Lh^T X
// and X is stored where (C[i], s0+t) is in S.  The symmetric c x c matrix G~_CC
// is read through a per-supernode list of the pairs (i, k) whose entry is in S
// (both triangles and the diagonal, sorted by i): the zeros of G~ are never
// touched.  The pairs are accumulated with shared-memory atomic adds into
// distinct rows per instruction (see accumulate_pairs).
//
// Scan form (for factors whose pair lists would not fit in memory): no list is
// stored.  A warp walks each row r = C[i] of S_lo backwards from the diagonal to
// the column C[0], looks every column up in a hash table of C built in phase A,
// and for each entry (r, C[k]) in C x C adds G(r, C[k]) Lh[i][:] into X[k] and
// G(r, C[k]) Lh[k][:] into X[i] (the symmetric pair), the latter summed over the
// warp first.  Reads of S_lo are contiguous; the plan holds nothing per pair.
//
// Scheduling: a CTA takes the next work item from a global ticket counter in
// level-major order.  An item is either one large supernode (the whole CTA
// works on it, rows split among the warps) or up to eight small ones (one per
// warp).  Before computing, the threads wait (bounded) until the supernodes
// owning the rows C have published their results; a result is published with
// a release store of the call's epoch.  A CTA only waits for items handed out
// before its own, all held by running CTAs, so the schedule cannot deadlock.
#include "device.cuh"
#include "kernels.h"
#include "plan.h"

namespace sinv {

namespace {

constexpr int kWarps = 8;          // warps per CTA
constexpr int kCW = 256;           // per-warp shared capacity for c*w values (Lh, X, output positions)
constexpr int kWMax = 16;          // supernode width limit of this kernel
constexpr int kBatch = 4;          // chunks of 32 pairs whose G loads are in flight together
constexpr int kTabW = 256;         // scan form: hash slots of C per warp in shared memory (CTA: all warps')

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

constexpr int kPairs = kWMax * (kWMax + 1) / 2;

struct WarpSmem {
    double lh[kCW];
    double x[kCW];
    double jj[kWMax * kWMax];   // L_JJ, then M = L_JJ^{-1}
    double t[kWMax * kWMax];    // D_J^{-1} M
    double red[kPairs];         // Lh^T X, lower triangle
    int32_t xpos[kCW];          // S_lo position of X[i][t] or -1
};
// a CTA-cooperative supernode lays Lh, X and the positions out over all warps' regions
static_assert(sizeof(WarpSmem) * kWarps >= (2 * sizeof(double) + sizeof(int32_t)) * kCW * kWarps, "layout");

// scan form, whole CTA: a second place for the table of C, in the warps' shared
// regions after Lh, X and the X positions of a supernode whose C x w fits them
constexpr int kCtaTabOff = kCW * kWarps * (2 * (int)sizeof(double) + (int)sizeof(int32_t));
constexpr int kCtaTabSlots = 4096;
static_assert(kCtaTabOff + 2 * kCtaTabSlots * (int)sizeof(int32_t) <= (int)sizeof(WarpSmem) * kWarps,
              "the table fits the warps' regions");

struct CtaShared {
    int item;
    int stop;
    int last;    // this CTA finishes a split supernode
    double jj[kWMax * kWMax];
    double t[kWMax * kWMax];
    double red[kWarps][kPairs];
};

// A group of threads working on one supernode: one warp, or the whole CTA.
template <bool kCta>
struct Group {
    static __device__ __forceinline__ int size() { return kCta ? kWarps * 32 : 32; }
    static __device__ __forceinline__ int rank() { return kCta ? (int)threadIdx.x : (int)(threadIdx.x & 31); }
    static __device__ __forceinline__ int nwarps() { return kCta ? kWarps : 1; }
    static __device__ __forceinline__ int warp() { return kCta ? (int)(threadIdx.x >> 5) : 0; }
    static __device__ __forceinline__ void sync() {
        if (kCta) __syncthreads(); else __syncwarp();
    }
    // vote plus a barrier that orders memory among the group's threads
    static __device__ __forceinline__ bool any(bool p) {
        if (kCta) return __syncthreads_or(p) != 0;
        const bool r = __any_sync(0xffffffffu, p);
        __syncwarp();
        return r;
    }
};

// Pairs of one warp: entries [e0, e1) of the supernode's pair list.  The first
// batch of (i, k) / position words is loaded before the dependency wait.
struct PairRange {
    int64_t e0, e1;
    uint32_t ik[kBatch];
    int32_t pos[kBatch];
};

__device__ __forceinline__ void load_pairs(const uint32_t* __restrict__ hik, const int32_t* __restrict__ hpos,
                                           int64_t base, int64_t e1, int lane, uint32_t* ik, int32_t* pos) {
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
        const int64_t e = base + u * 32 + lane;
        ik[u] = e < e1 ? hik[e] : 0xFFFFFFFFu;
        pos[u] = e < e1 ? hpos[e] : -1;
    }
}

// X -= G~_CC Lh over the pairs of this warp.  The pair list holds both (i, k) and
// (k, i), so each pair can add G(C[i], C[k]) Lh[i][:] into row k: the pairs of a
// chunk share i (sorted by i) and have distinct k, so the shared-memory atomic
// adds of one instruction hit distinct rows (FP64 and FP32 shared atomics are
// native), and no chain of dependent additions sits on the critical path.  Every
// batch issues the G loads of kBatch chunks and the pair words of the next batch
// before it computes.
template <class Form>
__device__ __forceinline__ void accumulate_pairs(PairRange& pr, const uint32_t* __restrict__ hik,
                                                 const int32_t* __restrict__ hpos, const typename Form::G* Gw,
                                                 const typename Form::R* lh, typename Form::R* x, int w, int lane,
                                                 int c, int64_t nnzS, int32_t* status) {
    using R = typename Form::R;
    for (int64_t base = pr.e0; base < pr.e1; base += 32 * kBatch) {
        R g[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
            g[u] = (pr.pos[u] >= 0 && in_range(status, pr.pos[u], 0, nnzS)) ? Form::ld(Gw + pr.pos[u]) : R(0);
        uint32_t ik_n[kBatch];
        int32_t pos_n[kBatch];
        load_pairs(hik, hpos, base + 32 * kBatch, pr.e1, lane, ik_n, pos_n);
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            if (pr.pos[u] < 0) continue;
            const int i = (int)(pr.ik[u] >> 16);
            const int k = (int)(pr.ik[u] & 0xffff);
            if (!in_range(status, i, 0, c) || !in_range(status, k, 0, c)) continue;
            if (w == 1) {
                atomicAdd(x + k, -g[u] * lh[i]);
            } else {
                for (int q = 0; q < w; ++q) atomicAdd(x + k * w + q, -g[u] * lh[i * w + q]);
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            pr.ik[u] = ik_n[u];
            pr.pos[u] = pos_n[u];
        }
    }
}

// ---- scan form --------------------------------------------------------------------
__device__ __forceinline__ uint32_t c_hash(int32_t r, uint32_t mask) { return ((uint32_t)r * 2654435761u) & mask; }

// local index of global row r in the table of C, or -1 (the table holds at most
// half as many keys as slots, so a free slot ends every probe)
__device__ __forceinline__ int c_find(const int32_t* keys, const int32_t* vals, uint32_t mask, int32_t r) {
    uint32_t h = c_hash(r, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const int32_t k = keys[h];
        if (k == r) return vals[h];
        if (k < 0) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

template <class Gr>
__device__ __forceinline__ void c_build(int32_t* keys, int32_t* vals, uint32_t mask, const int32_t* Crow, int c) {
    const int tid = Gr::rank(), gsz = Gr::size();
    for (uint32_t s = tid; s <= mask; s += gsz) keys[s] = -1;
    Gr::sync();
    for (int i = tid; i < c; i += gsz) {
        const int32_t r = Crow[i];
        uint32_t h = c_hash(r, mask);
        while (atomicCAS(keys + h, -1, r) != -1) h = (h + 1) & mask;  // rows of C are distinct
        vals[h] = i;
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// X -= G~_CC Lh for the rows [i0, i1) of C taken by this warp (rows i0 + v, then
// every nw-th).  Row r = C[i] of S_lo is read from its diagonal backwards in batches
// of kBatch x 32 entries while the columns stay >= C[0]; an entry whose column is
// C[k] adds G Lh[i][:] into X[k] (distinct k within an instruction) and G Lh[k][:]
// into X[i] (summed over the warp, one atomic add per column of the supernode).
// The warp keeps two rows in flight (two slots): the loads of both are issued
// before either is used, so one row's memory latency hides behind the other's.
struct ScanSlot {
    int i;        // local row, -1 when the slot is idle
    int64_t rs;   // first entry of the row in S_lo
    int64_t hi;   // one past the next batch's last entry
};

template <class Form>
__device__ __forceinline__ void scan_rows(const SelinvArgs& a, const typename Form::G* Gw, const int32_t* Crow, int c,
                                          int i0, int i1, int v, int nw, const int32_t* keys, const int32_t* vals,
                                          uint32_t mask, const typename Form::R* lh, typename Form::R* x, int w,
                                          int lane) {
    using R = typename Form::R;
    const int32_t c0 = c > 0 ? Crow[0] : 0;
    unsigned long long n_look = 0, n_hit = 0;
    int next = i0 + v;
    auto start = [&](ScanSlot& sl) {
        if (next < i1) {
            const int32_t r = Crow[next];
            sl.i = next;
            sl.rs = a.Srp[r];
            sl.hi = a.Sdiag[r];
            next += nw;
        } else {
            sl.i = -1;
        }
    };
    ScanSlot sl[2];
    start(sl[0]);
    start(sl[1]);
    while (sl[0].i >= 0 || sl[1].i >= 0) {
        int32_t col[2][kBatch];
        int kk[2][kBatch];
        R g[2][kBatch];
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int64_t p = sl[t].hi - 1 - lane - 32 * u;
                col[t][u] = (sl[t].i >= 0 && p >= sl[t].rs) ? __ldg(a.Sc + p) : -1;
            }
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int u = 0; u < kBatch; ++u)
                kk[t][u] = col[t][u] >= c0 ? c_find(keys, vals, mask, col[t][u]) : -1;
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int u = 0; u < kBatch; ++u)
                if (kk[t][u] >= c && !in_range(a.status, kk[t][u], 0, c)) kk[t][u] = -1;
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int u = 0; u < kBatch; ++u)
                g[t][u] = kk[t][u] >= 0 ? Form::ld(Gw + (sl[t].hi - 1 - lane - 32 * u)) : R(0);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            if (sl[t].i < 0) continue;
            const int i = sl[t].i;
            bool any = false;
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                if (kk[t][u] < 0) continue;
                any = true;
                for (int q = 0; q < w; ++q) atomicAdd(x + kk[t][u] * w + q, -g[t][u] * lh[i * w + q]);
            }
            if (__any_sync(0xffffffffu, any)) {
                for (int q = 0; q < w; ++q) {
                    R s = R(0);
#pragma unroll
                    for (int u = 0; u < kBatch; ++u)
                        if (kk[t][u] >= 0) s += g[t][u] * lh[kk[t][u] * w + q];
                    s = warp_sum(s);
                    if (lane == 0) atomicAdd(x + i * w + q, -s);
                }
            }
            if (a.counts) {
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    n_look += col[t][u] >= c0;
                    n_hit += kk[t][u] >= 0;
                }
            }
            // go on while the batch's smallest column (lane 31, last chunk) is still in range
            const int32_t last = __shfl_sync(0xffffffffu, col[t][kBatch - 1], 31);
            sl[t].hi -= 32 * kBatch;
            if (sl[t].hi <= sl[t].rs || last < c0) {
                if (lane == 0) {
                    const int64_t pd = a.Sdiag[Crow[i]];
                    const R gd = Form::ld(Gw + pd);
                    for (int q = 0; q < w; ++q) atomicAdd(x + i * w + q, -gd * lh[i * w + q]);
                }
                start(sl[t]);
            }
        }
    }
    if (a.counts) {
        n_look = (unsigned long long)warp_sum((double)n_look);
        n_hit = (unsigned long long)warp_sum((double)n_hit);
        if (lane == 0) {
            atomicAdd(a.counts, n_look);
            atomicAdd(a.counts + 1, n_hit);
        }
    }
}

// One supernode on a group (warp or CTA).  Returns false when a wait gave up.
// Phase A reads only the inputs and the plan (it overlaps the producers of C);
// phase B waits for them; phase C reads G, forms X and G_JJ and publishes.
// A supernode split over nparts CTAs (nparts > 1, CTA groups only): part `part` takes
// a range of rows of C balanced by pairs, adds its share of X into the supernode's
// global block with device atomics, and the last part to arrive (an arrival count,
// no waiting) reads the complete X back and finishes the supernode.  Blocks and
// counts are zeroed in stream order before every launch.
template <class Form, bool kCta, bool kScan>
__device__ bool process(const SelinvArgs& a, typename Form::G* Gw, int J, uint32_t epoch, WarpSmem* ws,
                        CtaShared* cs, int64_t gslot, int32_t* tab, int part = 0, int nparts = 1) {
    using R = typename Form::R;
    using Gr = Group<kCta>;
    const SnInfo I = a.sn[J];
    const int c = I.c, w = I.w, cw = c * w;
    const int tid = Gr::rank(), gsz = Gr::size(), lane = threadIdx.x & 31;
    if (tid == 0) tl_start(a.tl, J);
    const int32_t* Crow = a.Crow + I.crow_off;
    const int32_t* Lmap = a.Lmap + I.cw_off;

    // ---- phase A ---------------------------------------------------------------------
    // working arrays: shared memory of this warp (or all warps' regions for the CTA), else global scratch
    const int cap = kCta ? kCW * kWarps : kCW;
    R* lh;
    R* x;
    int32_t* xpos;
    if (cw <= cap) {
        if (kCta) {
            WarpSmem* w0 = ws - (threadIdx.x >> 5);
            double* base = reinterpret_cast<double*>(w0);
            lh = reinterpret_cast<R*>(base);
            x = reinterpret_cast<R*>(base + cap);
            xpos = reinterpret_cast<int32_t*>(base + 2 * cap);
        } else {
            lh = reinterpret_cast<R*>(ws->lh);
            x = reinterpret_cast<R*>(ws->x);
            xpos = ws->xpos;
        }
    } else {
        double* base = a.scratch + gslot * 3 * a.max_cw;
        lh = reinterpret_cast<R*>(base);
        x = reinterpret_cast<R*>(base + a.max_cw);
        xpos = reinterpret_cast<int32_t*>(base + 2 * a.max_cw);
    }
    double* jj = kCta ? cs->jj : ws->jj;
    double* tt = kCta ? cs->t : ws->t;
    for (int e = tid; e < cw; e += gsz) {
        const int q = Lmap[e];
        lh[e] = q >= 0 ? Form::from_d(a.Lval[q]) : R(0);
        xpos[e] = q >= 0 ? a.l2s[q] : -1;
        x[e] = R(0);
    }
    for (int e = tid; e < w * w; e += gsz) {
        const int q = a.JJl[I.ww_off + e];
        jj[e] = q >= 0 ? a.Lval[q] : 0.0;
    }
    // this warp's pairs: the whole list, or a contiguous range of rows balanced by pairs
    const uint32_t* hik = a.hit_ik + I.hit_off;
    const int32_t* hpos = a.hit_pos + I.hit_off;
    PairRange pr;
    pr.e0 = 0;
    pr.e1 = I.hit_cnt;
    // scan form: the table of C (this warp's or the CTA's shared slots, else a global
    // slice) and this part's rows, balanced by the row lengths of S
    int32_t* tkeys = nullptr;
    int32_t* tvals = nullptr;
    uint32_t tmask = 0;
    int r0 = 0, r1 = c;
    if (kScan) {
        uint32_t slots = 32;
        while ((int64_t)slots < 2 * (int64_t)c) slots <<= 1;
        const uint32_t avail = kCta ? kTabW * kWarps : kTabW;
        if (slots <= avail) {
            tkeys = kCta ? tab : tab + (threadIdx.x >> 5) * kTabW;
            tvals = tkeys + kTabW * kWarps;
        } else if (kCta && slots <= kCtaTabSlots) {
            // a whole-CTA supernode with C up to kCtaTabSlots / 2 rows: the table in the
            // warps' shared regions past Lh, X and their positions
            unsigned char* base = reinterpret_cast<unsigned char*>(ws - (threadIdx.x >> 5));
            tkeys = reinterpret_cast<int32_t*>(base + kCtaTabOff);
            tvals = tkeys + kCtaTabSlots;
        } else {
            tkeys = a.gtab + gslot * 2 * a.gtab_slots;
            tvals = tkeys + a.gtab_slots;
        }
        tmask = slots - 1;
        if (kCta && nparts > 1) {
            const int32_t* hrow = a.hrow + I.hrow_off;
            const int64_t E = hrow[c];
            auto row_at = [&](int64_t target) -> int {
                int lo = 0, hi = c;
                while (lo < hi) {
                    int mid = (lo + hi) >> 1;
                    if (hrow[mid] < target) lo = mid + 1; else hi = mid;
                }
                return lo;
            };
            r0 = part == 0 ? 0 : row_at(E * part / nparts);
            r1 = part == nparts - 1 ? c : row_at(E * (part + 1) / nparts);
        }
        c_build<Gr>(tkeys, tvals, tmask, Crow, c);
    } else if (kCta) {
        const int32_t* hrow = a.hrow + I.hrow_off;
        const int64_t E = I.hit_cnt;
        const int v = Gr::warp();
        auto row_start_at = [&](int64_t target) -> int64_t {
            int lo = 0, hi = c;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (hrow[mid] < target) lo = mid + 1; else hi = mid;
            }
            return hrow[lo];
        };
        // this part's rows, then this warp's share of them
        const int64_t p0 = part == 0 ? 0 : row_start_at(E * part / nparts);
        const int64_t p1 = part == nparts - 1 ? E : row_start_at(E * (part + 1) / nparts);
        pr.e0 = v == 0 ? p0 : row_start_at(p0 + (p1 - p0) * v / kWarps);
        pr.e1 = v == kWarps - 1 ? p1 : row_start_at(p0 + (p1 - p0) * (v + 1) / kWarps);
        if (pr.e1 < pr.e0) pr.e1 = pr.e0;
    }
    if (!kScan) load_pairs(hik, hpos, pr.e0, pr.e1, lane, pr.ik, pr.pos);
    Gr::sync();
    // Lh = L_CJ L_JJ^{-1}: row by row, columns from the last to the first
    if (w > 1) {
        for (int i = tid; i < c; i += gsz) {
            R* row = lh + (int64_t)i * w;
            for (int q = w - 2; q >= 0; --q) {
                R acc = row[q];
                for (int p = q + 1; p < w; ++p) acc -= row[p] * Form::from_d(jj[p * w + q]);
                row[q] = acc;
            }
        }
    }
    Gr::sync();
    // M = L_JJ^{-1} (unit lower) in place in jj (thread b owns column b), then
    // T = D_J^{-1} M with the FP64 pivot inverses (thread r owns row r)
    if (tid < 32) {
        double col[kWMax];
        if (tid < w) {
            const int b = tid;
            for (int r = 0; r < w; ++r) col[r] = 0.0;
            col[b] = 1.0;
            for (int r = b + 1; r < w; ++r) {
                double acc = 0.0;
                for (int p = b; p < r; ++p) acc -= jj[r * w + p] * col[p];
                col[r] = acc;
            }
        }
        __syncwarp();
        if (tid < w)
            for (int r = 0; r < w; ++r) jj[r * w + tid] = col[r];
        __syncwarp();
        if (tid < w) {
            const int r = tid;
            const int col_ = I.s0 + r;
            const bool first = a.pstart[col_] != 0;
            const bool two = first ? (col_ + 1 < a.n && a.pstart[col_ + 1] == 0) : true;
            const double* d = a.Dval + a.dpos[col_];
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
                double v = i_rr * jj[r * w + b];
                if (partner >= 0) v += i_rs * jj[partner * w + b];
                tt[r * w + b] = v;
            }
        }
    }

    // ---- phase B: wait until every supernode owning a row of C has published --------
    bool ok = true;
    for (int i = tid; i < c; i += gsz) {
        if (!wait_flag(a.done + a.owner[Crow[i]], epoch, a.status, a.wait_limit)) {
            ok = false;
            break;
        }
    }
    // the acquire loads above, followed by the group barrier inside any(), order
    // every thread's reads of G after the producers' release stores
    if (Gr::any(!ok)) return false;
    if (tid == 0) tl_mark(a.tl, J, 0);

    // ---- phase C ---------------------------------------------------------------------
    if (kScan)
        scan_rows<Form>(a, Gw, Crow, c, r0, r1, Gr::warp(), Gr::nwarps(), tkeys, tvals, tmask, lh, x, w, lane);
    else
        accumulate_pairs<Form>(pr, hik, hpos, Gw, lh, x, w, lane, c, a.nnzS, a.status);
    Gr::sync();
    if (tid == 0) tl_mark(a.tl, J, 1);
    if (kCta && nparts > 1) {
        double* blk = a.xsum + a.xsum_off[J];
        for (int e = tid; e < cw; e += gsz) {
            const double v = Form::to_d(x[e]);
            if (v != 0.0) atomicAdd(blk + e, v);
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) cs->last = atomicAdd(a.arrive + J, 1u) == (uint32_t)(nparts - 1) ? 1 : 0;
        __syncthreads();
        if (!cs->last) return true;  // another part finishes the supernode
        __threadfence();
        // the last part reads the complete X (the blocks and counts are cleared before each call)
        for (int e = tid; e < cw; e += gsz) x[e] = Form::from_d(__ldcg(blk + e));
        Gr::sync();
    }
    for (int e = tid; e < cw; e += gsz) {
        const int p = xpos[e];
        if (p >= 0 && in_range(a.status, p, 0, a.nnzS)) Form::st(Gw + p, x[e]);
    }
    // G_JJ[r][b] = (M^T T)[r][b] - sum_i Lh[i][r] X[i][b]   (r >= b): FP64 accumulation
    const int npair = w * (w + 1) / 2;
    for (int pidx = 0, r = 0; r < w; ++r) {
        for (int b = 0; b <= r; ++b, ++pidx) {
            double s = 0.0;
            for (int i = tid; i < c; i += gsz) s += (double)lh[i * w + r] * (double)x[i * w + b];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) {
                if (kCta) cs->red[threadIdx.x >> 5][pidx] = s;
                else ws->red[pidx] = s;
            }
        }
    }
    Gr::sync();
    for (int pidx = tid; pidx < npair; pidx += gsz) {
        int r = 0;
        while ((r + 1) * (r + 2) / 2 <= pidx) ++r;
        const int b = pidx - r * (r + 1) / 2;
        double s = 0.0;
        if (kCta) {
            for (int v = 0; v < kWarps; ++v) s += cs->red[v][pidx];
        } else {
            s = ws->red[pidx];
        }
        double m = 0.0;
        for (int p = 0; p < w; ++p) m += jj[p * w + r] * tt[p * w + b];
        const int sp = a.JJs[I.ww_off + r * w + b];
        if (sp >= 0 && in_range(a.status, sp, 0, a.nnzS)) Form::st(Gw + sp, Form::from_d(m - s));
    }
    // the barrier orders every thread's writes before thread 0's release store,
    // which publishes them (release is cumulative over the barrier)
    Gr::sync();
    if (tid == 0) {
        st_release(a.done + J, epoch);
        tl_mark(a.tl, J, 2);
    }
    return true;
}

template <class Form, bool kScan>
__global__ void __launch_bounds__(kWarps * 32, kScan ? 3 : 2) selinv_persistent(SelinvArgs a, typename Form::G* Gw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ CtaShared cs;
    WarpSmem* ws = reinterpret_cast<WarpSmem*>(smem_raw) + (threadIdx.x >> 5);
    // scan form: kWarps x kTabW keys, then as many values, after the warps' regions
    int32_t* tab = reinterpret_cast<int32_t*>(reinterpret_cast<WarpSmem*>(smem_raw) + kWarps);
    const int warp = threadIdx.x >> 5;
    const uint32_t epoch = *a.epoch;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            cs.item = a.item0 + atomicAdd(a.ticket, 1);
            cs.stop = ld_volatile(a.status) != ST_OK;
        }
        __syncthreads();
        const int item = cs.item;
        if (item >= a.nitems || cs.stop) break;
        const WorkItem it = a.items[item];
        if (it.big == 2) {
            process<Form, true, kScan>(a, Gw, a.order[it.first], epoch, ws, &cs, (int64_t)blockIdx.x * kWarps, tab,
                                       it.part, it.count);
        } else if (it.big) {
            process<Form, true, kScan>(a, Gw, a.order[it.first], epoch, ws, &cs, (int64_t)blockIdx.x * kWarps, tab);
        } else if (warp < it.count) {
            process<Form, false, kScan>(a, Gw, a.order[it.first + warp], epoch, ws, &cs,
                                        (int64_t)blockIdx.x * kWarps + warp, tab);
        }
    }
}

__global__ void prepare_kernel(uint32_t* epoch, int32_t* ticket, int32_t* ticket2) {
    uint32_t e = *epoch + 1;
    *epoch = e == 0 ? 1 : e;
    *ticket = 0;
    if (ticket2) *ticket2 = 0;
}

template <class Form>
__global__ void widen_to_double(const typename Form::G* __restrict__ src, double* __restrict__ dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = Form::to_d(src[i]);
}

size_t smem_bytes(bool scan) { return sizeof(WarpSmem) * kWarps + (scan ? 2 * sizeof(int32_t) * kWarps * kTabW : 0); }

template <class Form>
cudaError_t launch_form(const SelinvArgs& a, typename Form::G* Gw, double* G_out, cudaStream_t st, int grid) {
    if (a.scan) {
        trace_begin("selinv_scan", st);
        selinv_persistent<Form, true><<<grid, kWarps * 32, smem_bytes(true), st>>>(a, Gw);
    } else {
        trace_begin("selinv_persistent", st);
        selinv_persistent<Form, false><<<grid, kWarps * 32, smem_bytes(false), st>>>(a, Gw);
    }
    trace_end(st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((void*)Gw != (void*)G_out) {
        trace_begin("selinv_widen", st);
        widen_to_double<Form><<<a.num_sms * 8, 256, 0, st>>>(Gw, G_out, a.nnzS);
        trace_end(st);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

cudaError_t selinv_prepare(uint32_t* epoch, int32_t* ticket, cudaStream_t st, int32_t* ticket2) {
    trace_begin("selinv_prepare", st);
    prepare_kernel<<<1, 1, 0, st>>>(epoch, ticket, ticket2);
    trace_end(st);
    return cudaGetLastError();
}

int selinv_max_width() { return kWMax; }
int selinv_cw_smem() { return kCW; }
int selinv_warps_per_cta() { return kWarps; }

cudaError_t selinv_configure() {
    const int s0 = (int)smem_bytes(false), s1 = (int)smem_bytes(true);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(selinv_persistent<F64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s0)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(selinv_persistent<F32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s0)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(selinv_persistent<F64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1)) !=
            cudaSuccess)
        return e;
    return cudaFuncSetAttribute(selinv_persistent<F32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1);
}

int selinv_grid(int num_sms, bool scan) {
    int per_sm = 0;
    cudaError_t e = scan ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, selinv_persistent<F64, true>,
                                                                         kWarps * 32, smem_bytes(true))
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, selinv_persistent<F64, false>,
                                                                         kWarps * 32, smem_bytes(false));
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return per_sm * num_sms;
}

int selinv_scan_table_smem() { return kTabW; }

cudaError_t selinv_launch(const SelinvArgs& a, int prec, void* work, double* G_out, cudaStream_t st, int grid) {
    if (prec == 0) return launch_form<F64>(a, G_out, G_out, st, grid);
    return launch_form<F32>(a, reinterpret_cast<float*>(work), G_out, st, grid);
}

}  // namespace sinv
