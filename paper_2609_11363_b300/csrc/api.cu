// C ABI of libsinv (declared in include/sinv.h): handle management, the host
// symbolic analysis upload and the numeric entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/sinv.h"
#include "kernels.h"
#include "plan.h"

using namespace sinv;

namespace sinv {

// Event pairs around every kernel launch of a call, aggregated by kernel name.
struct Tracer {
    struct Rec {
        const char* name;
        cudaEvent_t a, b;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    std::map<std::string, std::pair<int64_t, double>> agg;
    int open = -1;

    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void begin(const char* name, cudaStream_t st) {
        Rec r{name, get(), get()};
        cudaEventRecord(r.a, st);
        pending.push_back(r);
        open = (int)pending.size() - 1;
    }
    void end(cudaStream_t st) {
        if (open >= 0) cudaEventRecord(pending[open].b, st);
        open = -1;
    }
    void collect() {
        for (auto& r : pending) {
            float ms = 0.f;
            if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
                auto& x = agg[r.name];
                x.first += 1;
                x.second += ms;
            }
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        pending.clear();
    }
    ~Tracer() {
        for (auto& r : pending) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

thread_local Tracer* g_tracer = nullptr;

void trace_begin(const char* name, cudaStream_t st) {
    if (g_tracer) g_tracer->begin(name, st);
}
void trace_end(cudaStream_t st) {
    if (g_tracer) g_tracer->end(st);
}

// installs the handle's tracer (if any) for the lifetime of a numeric call
struct TraceScope {
    Tracer* prev;
    explicit TraceScope(Tracer* t) : prev(g_tracer) { g_tracer = t; }
    ~TraceScope() { g_tracer = prev; }
};

}  // namespace sinv

struct sinv_handle_s {
    Tracer* tracer = nullptr;
    int device = 0;
    int num_sms = 0;
    HostPlan P;
    int64_t wait_limit = 4000000;  // polls (64 ns sleep each): a few seconds
    // device copies of the plan
    int64_t* dSrp = nullptr;
    int32_t* dSc = nullptr;
    int32_t* dSdiag = nullptr;
    int32_t* dl2s = nullptr;
    int64_t* dLrp = nullptr;
    int64_t* dLcp = nullptr;
    int32_t* dLri = nullptr;
    int32_t* dLcsr = nullptr;
    int32_t* ddpos = nullptr;
    int8_t* dpstart = nullptr;
    SnInfo* dsn = nullptr;
    int32_t* dorder = nullptr;
    int32_t* downer = nullptr;
    int32_t* dCrow = nullptr;
    int32_t* dLmap = nullptr;
    int32_t* dJJl = nullptr;
    int32_t* dJJs = nullptr;
    uint32_t* dhit_ik = nullptr;
    int32_t* dhit_pos = nullptr;
    int32_t* dhrow = nullptr;
    WorkItem* ditems = nullptr;
    int64_t* dxsum_off = nullptr;
    double* dxsum = nullptr;
    uint32_t* darrive = nullptr;
    uint32_t* ddone = nullptr;
    uint32_t* depoch = nullptr;
    int32_t* dticket = nullptr;
    int32_t* dstatus = nullptr;
    uint32_t* ddebug_flag = nullptr;
    double* dscratch = nullptr;
    // tensor-core tier of SelInv (allocated by the first call of a tensor-core form)
    WorkItem* dtc_items = nullptr;
    int32_t* dtc_map = nullptr;
    int32_t* dtc_deps = nullptr;
    int32_t* dtc_ticket = nullptr;
    double* dtc_mirror = nullptr;
    uint32_t* dtc_arrive_t = nullptr;
    double* dtc_z = nullptr;
    bool tc_ready = false;
    // NInv on its own pattern: result (CSC of N_lo) and the sizes of the last call
    int64_t* down_cp = nullptr;
    int32_t* down_r = nullptr;
    double* down_v = nullptr;
    int64_t own_nnz = 0, own_nnzW = 0;
    std::vector<int64_t> own_nnzW_steps;
    std::vector<int64_t> own_hint;  // output sizes of the last call's steps (first guesses of the next)
    // Mix on the own pattern (handle-owned CSC of the lower triangle)
    int64_t* dmix_cp = nullptr;
    int32_t* dmix_r = nullptr;
    double* dmix_v = nullptr;
    int64_t mix_nnz = -1;
    int64_t mix_gen = 0;       // bumped by every sinv_mix_own
    int64_t spai_mix_gen = -1; // the mix_gen the SPAI plan was built from (-1: not from a Mix)
    // per-supernode timeline of SelInv (allocated while enabled)
    unsigned long long* dtl_first = nullptr;
    unsigned long long* dtl_last = nullptr;
    unsigned long long* dscan_counts = nullptr;  // lookups and pairs of the scan form (with the timeline)
    // scan form of SelInv: hash tables of C in global memory for groups whose C is too large
    int32_t* dgtab = nullptr;
    int64_t gtab_slots = 0;
    void* dwork = nullptr;
    size_t work_bytes = 0;
    int grid = 0;
    // NInv pattern (built by the first sinv_ninv for a given m)
    NinvPlan W;
    // batch layout (block-diagonal concatenation of several matrices), nmat+1 offsets each
    std::vector<int64_t> b_n_off, b_L_off, b_D_off, b_S_off;
    // sinv_batch_run: device offsets and the concatenated value / output buffers
    int64_t* db_L_off = nullptr;
    int64_t* db_D_off = nullptr;
    int64_t* db_S_off = nullptr;
    double* db_L = nullptr;
    double* db_D = nullptr;
    double* db_G = nullptr;
    double* db_N = nullptr;
    int64_t* dWcp = nullptr;
    int32_t* dWr = nullptr;
    int32_t* dgrp = nullptr;
    // map form of NInv: maps of the current pattern (built by the first call of an m)
    NinvMaps X;
    int64_t index_budget = 0;   // < 0: never; 0: half the free device memory; > 0: bytes
    int index_tried_m = -1;     // m for which the index was built or found not to fit
    std::string index_note;     // why the hash form runs (empty when the maps are used)
    // SPAI refinement: analysis of the current pattern of A
    SpaiPlan Q;
    bool spai_analysed = false;  // Q holds a plan
    bool spai_ready = false;     // ... and it is on the device
    int64_t* dfcp = nullptr;
    int32_t *dfri = nullptr, *dfpos = nullptr, *dfsrc = nullptr, *dfeo = nullptr, *dfE = nullptr, *dfR = nullptr;
    int64_t* dArp = nullptr;
    int32_t *dAcol = nullptr, *dscols_w = nullptr, *dscols_c = nullptr, *dsticket = nullptr;
    double* dsscratch = nullptr;
    int64_t spai_cta_bytes = 0;
    // spectral-correction producer: analysis of the current pattern of A
    EinvPlan E;
    bool einv_analysed = false;  // E holds a plan
    bool einv_ready = false;     // ... and it is on the device
    int64_t *deArp = nullptr, *deLrp = nullptr, *defcp = nullptr;
    int32_t *deAcol = nullptr, *deLcol = nullptr, *defri = nullptr, *defpos = nullptr, *defwd = nullptr,
            *debwd = nullptr, *defwdp = nullptr, *debwdp = nullptr;
    void* dework = nullptr;
    // persistent triangular solves: per-row flags of each solve, epoch and tickets (zeroed once)
    uint32_t* detrsv = nullptr;
    int32_t einv_solver = 0;  // 0: CG with L D L^T (A SPD), 1: MINRES with L |D| L^T
    bool einv_grid_solve = false;  // the persistent grid solves even where one CTA would walk the levels
    size_t ework_bytes = 0;
    std::string last_error;
};

namespace {

void set_err(sinv_handle h, const std::string& msg) {
    if (h) h->last_error = msg;
}

sinv_status cuda_fail(sinv_handle h, cudaError_t e, const char* where) {
    set_err(h, std::string(where) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SINV_ERR_OOM : SINV_ERR_CUDA;
}

template <class T, class Alloc>
cudaError_t upload(T** dst, const std::vector<T, Alloc>& src) {
    size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void**)dst, bytes);
    if (e != cudaSuccess) return e;
    if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

void spai_free(sinv_handle h) {
    void* ptrs[] = {h->dfcp, h->dfri, h->dfpos, h->dfsrc, h->dfeo, h->dfE, h->dfR, h->dArp, h->dAcol, h->dscols_w,
                    h->dscols_c, h->dsticket, h->dsscratch};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    h->dfcp = nullptr;
    h->dfri = h->dfpos = h->dfsrc = h->dfeo = h->dfE = h->dfR = nullptr;
    h->dArp = nullptr;
    h->dAcol = h->dscols_w = h->dscols_c = h->dsticket = nullptr;
    h->dsscratch = nullptr;
    h->spai_ready = false;
    h->spai_analysed = false;
    h->Q = SpaiPlan();
}

void einv_free(sinv_handle h) {
    void* ptrs[] = {h->deArp, h->deLrp, h->defcp, h->deAcol, h->deLcol, h->defri, h->defpos, h->defwd, h->debwd,
                    h->defwdp, h->debwdp, h->dework, h->detrsv};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    h->deArp = h->deLrp = h->defcp = nullptr;
    h->deAcol = h->deLcol = h->defri = h->defpos = h->defwd = h->debwd = h->defwdp = h->debwdp = nullptr;
    h->dework = nullptr;
    h->detrsv = nullptr;
    h->ework_bytes = 0;
    h->einv_ready = false;
    h->einv_analysed = false;
    h->E = EinvPlan();
}

void free_all(sinv_handle h) {
    void* ptrs[] = {h->dSrp, h->dSc, h->dSdiag, h->dl2s, h->dLrp, h->dLcp, h->dLri, h->dLcsr, h->ddpos, h->dpstart,
                    h->dsn, h->dorder, h->downer, h->dCrow, h->dLmap, h->dJJl, h->dJJs, h->dhit_ik, h->dhit_pos,
                    h->dhrow, h->ditems, h->dxsum_off, h->dxsum, h->darrive, h->ddone, h->depoch, h->dticket, h->dstatus, h->ddebug_flag, h->dscratch, h->dwork, h->dWcp,
                    h->dWr, h->dgrp, h->dtc_items, h->dtc_map, h->dtc_deps, h->dtc_ticket, h->dtc_mirror, h->dtc_arrive_t,
                    h->dtc_z, h->dtl_first, h->dtl_last, h->dscan_counts, h->dgtab, h->dmix_cp, h->dmix_r, h->dmix_v, h->down_cp, h->down_r, h->down_v, h->db_L_off, h->db_D_off, h->db_S_off, h->db_L, h->db_D,
                    h->db_G, h->db_N};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    ninv_maps_free(h->X);
    spai_free(h);
    einv_free(h);
}

sinv_status ensure_work(sinv_handle h, size_t bytes) {
    if (bytes <= h->work_bytes) return SINV_OK;
    if (h->dwork) cudaFree(h->dwork);
    h->dwork = nullptr;
    h->work_bytes = 0;
    cudaError_t e = cudaMalloc(&h->dwork, bytes);
    if (e != cudaSuccess) return cuda_fail(h, e, "work buffer");
    h->work_bytes = bytes;
    return SINV_OK;
}

// a device buffer freed at scope exit (the own-pattern call's temporaries)
struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    template <class T>
    T* as() {
        return reinterpret_cast<T*>(p);
    }
};
cudaError_t dev_alloc(DevBuf& b, size_t bytes) { return cudaMalloc(&b.p, std::max<size_t>(bytes, 8)); }

// a handle-owned CSC result of the empty matrix: colptr = {0}, no rows or values
cudaError_t empty_csc(int64_t** cp, int32_t** rows, double** vals, cudaStream_t st) {
    if (*cp) cudaFree(*cp);
    if (*rows) cudaFree(*rows);
    if (*vals) cudaFree(*vals);
    *cp = nullptr;
    *rows = nullptr;
    *vals = nullptr;
    cudaError_t e = cudaMalloc((void**)cp, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(*cp, 0, sizeof(int64_t), st);
    return e == cudaSuccess ? cudaStreamSynchronize(st) : e;
}

bool valid_prec(int p) { return p == SINV_FP64 || p == SINV_FP32 || p == SINV_FP32X2; }
bool tc_prec(int p) { return p == SINV_TF32_FP32ACC || p == SINV_BF16_FP32ACC; }

// numeric calls need a handle that lives on a device
bool on_device(sinv_handle h) {
    if (h->device >= 0) return true;
    set_err(h, "handle was analysed host-only (device < 0): numeric calls are not available");
    return false;
}

}  // namespace

extern "C" {

const char* sinv_status_string(sinv_status s) {
    switch (s) {
        case SINV_OK: return "ok";
        case SINV_ERR_INVALID_ARG: return "invalid argument";
        case SINV_ERR_PATTERN: return "invalid sparsity pattern or pivot layout";
        case SINV_ERR_SINGULAR_PIVOT: return "singular pivot block in D";
        case SINV_ERR_OOM: return "out of memory";
        case SINV_ERR_CUDA: return "CUDA error";
        case SINV_ERR_TIMEOUT: return "device wait timed out";
        case SINV_ERR_UNSUPPORTED: return "unsupported size or option";
    }
    return "unknown status";
}

sinv_status sinv_last_error(sinv_handle h, char* buf, size_t len) {
    if (!h || !buf || len == 0) return SINV_ERR_INVALID_ARG;
    size_t n = std::min(len - 1, h->last_error.size());
    memcpy(buf, h->last_error.data(), n);
    buf[n] = 0;
    return SINV_OK;
}

sinv_status sinv_symbolic(int64_t n, const int64_t* L_rowptr, const int32_t* L_col, const int8_t* pivot_start,
                          const sinv_symbolic_opts* opts, sinv_handle* out) {
    if (!out) return SINV_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 0 || (n > 0 && (!L_rowptr || !pivot_start)) || (n > 0 && L_rowptr[n] > 0 && !L_col))
        return SINV_ERR_INVALID_ARG;
    sinv_handle h = new (std::nothrow) sinv_handle_s();
    if (!h) return SINV_ERR_OOM;
    int cap = 4;
    int64_t big_pairs = 1024;
    int64_t pair_bytes = 0;
    if (opts) {
        if (opts->supernode_cap > 0) cap = opts->supernode_cap;
        if (opts->big_pairs > 0) big_pairs = opts->big_pairs;
        h->device = opts->device;
        if (opts->wait_limit > 0) h->wait_limit = opts->wait_limit;
        h->index_budget = opts->ninv_index_bytes;
        pair_bytes = opts->selinv_pair_bytes;
    }
    cap = std::min(cap, selinv_max_width());
    const bool host_only = h->device < 0;
    cudaError_t e = cudaSuccess;
    if (!host_only && (e = cudaSetDevice(h->device)) != cudaSuccess) {
        sinv_status s = cuda_fail(h, e, "cudaSetDevice");
        *out = h;  // so that the caller can read the message
        return s;
    }
    if (!host_only) cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    // levels with fewer supernodes than SMs give each supernode a whole CTA (a sweep over
    // 0..16 x SMs on the 64^3 diffusion workload put the best at 1 x SMs)
    const int64_t thin_level = (int64_t)(h->num_sms > 0 ? h->num_sms : 148);
    std::string err;
    try {
        err = build_plan(n, L_rowptr, L_col, pivot_start, cap, big_pairs, selinv_warps_per_cta(), thin_level,
                         h->P, pair_bytes);
    } catch (const std::bad_alloc&) {
        set_err(h, "host allocation failed in the symbolic analysis");
        *out = h;
        return SINV_ERR_OOM;
    }
    if (!err.empty()) {
        set_err(h, err);
        *out = h;
        return err.find("not supported") != std::string::npos || err.find("unsupported") != std::string::npos
                   ? SINV_ERR_UNSUPPORTED
                   : SINV_ERR_PATTERN;
    }
    HostPlan& P = h->P;
    if (host_only) {
        *out = h;
        return SINV_OK;
    }
    std::vector<int64_t> Lrp(L_rowptr, L_rowptr + n + 1);
#define UP(dst, src)                                              \
    do {                                                          \
        e = upload(&h->dst, src);                                 \
        if (e != cudaSuccess) {                                   \
            *out = h;                                             \
            return cuda_fail(h, e, "upload " #dst);               \
        }                                                         \
    } while (0)
    UP(dSrp, P.Srp);
    UP(dSc, P.Sc);
    UP(dSdiag, P.Sdiag);
    UP(dl2s, P.l2s);
    UP(dLrp, Lrp);
    UP(dLcp, P.Lcp);
    UP(dLri, P.Lri);
    UP(dLcsr, P.Lcsr);
    UP(ddpos, P.dpos);
    UP(dpstart, P.pstart);
    UP(dsn, P.sn);
    UP(dorder, P.order);
    UP(downer, P.owner);
    UP(dCrow, P.Crow);
    UP(dLmap, P.Lmap);
    UP(dJJl, P.JJl);
    UP(dJJs, P.JJs);
    UP(dhit_ik, P.hit_ik);
    UP(dhit_pos, P.hit_pos);
    UP(dhrow, P.hrow);
    UP(ditems, P.items);
    UP(dxsum_off, P.xsum_off);
#undef UP
    size_t nsn = std::max<size_t>(P.sn.size(), 1);
    const size_t nxs = (size_t)std::max<int64_t>(P.xsum_total, 1);
    if ((e = cudaMalloc((void**)&h->ddone, nsn * sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMemset(h->ddone, 0, nsn * sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMalloc((void**)&h->darrive, nsn * sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMemset(h->darrive, 0, nsn * sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMalloc((void**)&h->dxsum, nxs * sizeof(double))) != cudaSuccess ||
        (e = cudaMemset(h->dxsum, 0, nxs * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc((void**)&h->depoch, 64)) != cudaSuccess || (e = cudaMemset(h->depoch, 0, 64)) != cudaSuccess ||
        (e = cudaMalloc((void**)&h->dticket, 64)) != cudaSuccess ||
        (e = cudaMemset(h->dticket, 0, 64)) != cudaSuccess ||
        (e = cudaMalloc((void**)&h->dstatus, 64)) != cudaSuccess ||
        (e = cudaMemset(h->dstatus, 0, 64)) != cudaSuccess ||
        (e = cudaMalloc((void**)&h->ddebug_flag, 64)) != cudaSuccess ||
        (e = cudaMemset(h->ddebug_flag, 0, 64)) != cudaSuccess) {
        *out = h;
        return cuda_fail(h, e, "device state");
    }
    if ((e = selinv_configure()) != cudaSuccess || (e = selinv_tc_configure()) != cudaSuccess ||
        (e = ninv_configure()) != cudaSuccess || (e = own_configure()) != cudaSuccess ||
        (e = ninv_maps_configure()) != cudaSuccess) {
        *out = h;
        return cuda_fail(h, e, "kernel attributes");
    }
    h->grid = selinv_grid(h->num_sms, P.scan != 0);
    if (P.max_cw > selinv_cw_smem()) {
        size_t bytes = (size_t)h->grid * selinv_warps_per_cta() * 3 * (size_t)P.max_cw * sizeof(double);
        if ((e = cudaMalloc((void**)&h->dscratch, bytes)) != cudaSuccess) {
            *out = h;
            return cuda_fail(h, e, "selinv scratch");
        }
    }
    if (P.scan && 2 * P.max_c > selinv_scan_table_smem()) {
        // hash tables of C for the groups whose C exceeds their shared slots
        int64_t slots = 32;
        while (slots < 2 * P.max_c) slots <<= 1;
        h->gtab_slots = slots;
        size_t bytes = (size_t)h->grid * selinv_warps_per_cta() * 2 * (size_t)slots * sizeof(int32_t);
        if ((e = cudaMalloc((void**)&h->dgtab, bytes)) != cudaSuccess) {
            *out = h;
            return cuda_fail(h, e, "selinv scan tables");
        }
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
        *out = h;
        return cuda_fail(h, e, "symbolic upload");
    }
    *out = h;
    return SINV_OK;
}

sinv_status sinv_batch_symbolic(int32_t nmat, const int64_t* n, const int64_t* const* L_rowptr,
                                const int32_t* const* L_col, const int8_t* const* pivot_start,
                                const sinv_symbolic_opts* opts, sinv_handle* out) {
    if (!out || nmat < 0 || (nmat > 0 && (!n || !L_rowptr || !L_col || !pivot_start))) return SINV_ERR_INVALID_ARG;
    *out = nullptr;
    std::vector<int64_t> n_off(nmat + 1, 0), L_off(nmat + 1, 0), D_off(nmat + 1, 0);
    for (int32_t b = 0; b < nmat; ++b) {
        if (n[b] < 0 || (n[b] > 0 && (!L_rowptr[b] || !pivot_start[b]))) return SINV_ERR_INVALID_ARG;
        const int64_t nb = n[b];
        const int64_t nnzb = nb > 0 ? L_rowptr[b][nb] : 0;
        if (nnzb > 0 && !L_col[b]) return SINV_ERR_INVALID_ARG;
        n_off[b + 1] = n_off[b] + nb;
        L_off[b + 1] = L_off[b] + nnzb;
        int64_t n2 = 0;
        for (int64_t j = 1; j < nb; ++j) n2 += pivot_start[b][j] == 0;
        D_off[b + 1] = D_off[b] + nb + n2;
    }
    const int64_t N = n_off[nmat], NNZ = L_off[nmat];
    std::vector<int64_t> rp;
    std::vector<int32_t> col;
    std::vector<int8_t> ps;
    try {
        rp.assign(N + 1, 0);
        col.resize(NNZ);
        ps.resize(N);
    } catch (const std::bad_alloc&) {
        return SINV_ERR_OOM;
    }
    for (int32_t b = 0; b < nmat; ++b) {
        const int64_t nb = n[b], r0 = n_off[b], q0 = L_off[b];
        for (int64_t i = 0; i < nb; ++i) {
            const int64_t a = L_rowptr[b][i], e = L_rowptr[b][i + 1];
            if (a < 0 || e < a || e > L_rowptr[b][nb]) return SINV_ERR_PATTERN;
            for (int64_t q = a; q < e; ++q) {
                const int32_t c = L_col[b][q];
                // checked per matrix: an entry must stay inside its own block
                if (c < 0 || c >= i) return SINV_ERR_PATTERN;
                col[q0 + q] = (int32_t)(c + r0);
            }
            rp[r0 + i + 1] = q0 + e;
        }
        if (nb > 0 && (L_rowptr[b][0] != 0 || pivot_start[b][0] != 1)) return SINV_ERR_PATTERN;
        for (int64_t j = 0; j < nb; ++j) ps[r0 + j] = pivot_start[b][j];
    }
    sinv_status st = sinv_symbolic(N, rp.data(), col.data(), ps.data(), opts, out);
    if (*out) {
        (*out)->b_n_off = n_off;
        (*out)->b_L_off = L_off;
        (*out)->b_D_off = D_off;
        (*out)->b_S_off.assign(nmat + 1, 0);
        for (int32_t b = 0; b <= nmat; ++b) (*out)->b_S_off[b] = (*out)->P.Srp.empty() ? 0 : (*out)->P.Srp[n_off[b]];
    }
    return st;
}

sinv_status sinv_batch_layout(sinv_handle h, int32_t* nmat, int64_t* n_off, int64_t* L_off, int64_t* D_off,
                              int64_t* S_off) {
    if (!h || !nmat) return SINV_ERR_INVALID_ARG;
    const int32_t nb = h->b_n_off.empty() ? 0 : (int32_t)h->b_n_off.size() - 1;
    *nmat = nb;
    if (nb == 0) return SINV_OK;
    int64_t* dst[4] = {n_off, L_off, D_off, S_off};
    const std::vector<int64_t>* src[4] = {&h->b_n_off, &h->b_L_off, &h->b_D_off, &h->b_S_off};
    for (int t = 0; t < 4; ++t)
        if (dst[t]) memcpy(dst[t], src[t]->data(), (nb + 1) * sizeof(int64_t));
    return SINV_OK;
}

sinv_status sinv_get_pattern(sinv_handle h, const int64_t** S_rowptr, const int32_t** S_col, int64_t* nnzS_lo) {
    if (!h || !S_rowptr || !S_col || !nnzS_lo) return SINV_ERR_INVALID_ARG;
    *S_rowptr = h->dSrp;
    *S_col = h->dSc;
    *nnzS_lo = h->P.nnzS;
    return SINV_OK;
}

sinv_status sinv_get_pattern_host(sinv_handle h, int64_t* S_rowptr, int32_t* S_col) {
    if (!h || !S_rowptr || (!S_col && h->P.nnzS > 0)) return SINV_ERR_INVALID_ARG;
    memcpy(S_rowptr, h->P.Srp.data(), h->P.Srp.size() * sizeof(int64_t));
    if (h->P.nnzS > 0) memcpy(S_col, h->P.Sc.data(), h->P.Sc.size() * sizeof(int32_t));
    return SINV_OK;
}

sinv_status sinv_get_stats(sinv_handle h, sinv_stats* s) {
    if (!h || !s) return SINV_ERR_INVALID_ARG;
    const HostPlan& P = h->P;
    s->n = P.n;
    s->nnz_L = P.nnzL;
    s->nnz_S_lo = P.nnzS;
    s->n_blocks = P.n_blocks;
    s->n_2x2 = P.n_2x2;
    s->n_supernodes = (int64_t)P.sn.size();
    s->n_levels = P.n_levels;
    s->max_c = P.max_c;
    s->hit_pairs = P.hit_pairs;
    s->max_width = P.max_w;
    s->nnz_W = h->W.m >= 0 ? h->W.nnzW : 0;
    s->ninv_m = h->W.m;
    s->pad = 0;
    s->horner_products = h->W.m >= 0 ? h->W.horner_products : 0;
    s->product_stream = h->W.m >= 0 ? h->W.product_stream : 0;
    s->selinv_flops = P.selinv_flops;
    s->selinv_bytes = P.selinv_bytes;
    s->ninv_index_bytes = h->X.ready ? h->X.bytes : 0;
    s->product_hits = h->X.ready ? h->X.hits : 0;
    s->spai_entries = h->spai_analysed ? h->Q.entries : 0;
    s->spai_cols_warp = h->spai_analysed ? (int64_t)h->Q.cols_w.size() : 0;
    s->spai_cols_cta = h->spai_analysed ? (int64_t)h->Q.cols_c.size() : 0;
    s->spai_nnz_P = h->spai_analysed ? h->Q.nnzP : 0;
    s->einv_levels_fwd = h->einv_analysed && !h->E.fwd_ptr.empty() ? (int64_t)h->E.fwd_ptr.size() - 1 : 0;
    s->einv_levels_bwd = h->einv_analysed && !h->E.bwd_ptr.empty() ? (int64_t)h->E.bwd_ptr.size() - 1 : 0;
    s->tc_levels = P.tc_levels;
    s->tc_supernodes = P.tc_sn;
    s->tc_pairs = P.tc_pairs;
    s->tc_mirror_bytes = P.tc_levels > 0 ? (P.n - P.tc_row0) * P.tc_width * (int64_t)sizeof(double) : 0;
    s->selinv_scan = P.scan;
    s->scan_rows_total = P.scan_rows_total;
    return SINV_OK;
}

sinv_status sinv_get_supernodes(sinv_handle h, const int32_t** sn_start, const int32_t** sn_level, int64_t* count) {
    if (!h || !sn_start || !sn_level || !count) return SINV_ERR_INVALID_ARG;
    *sn_start = h->P.sn_start.data();
    *sn_level = h->P.sn_level.data();
    *count = (int64_t)h->P.sn.size();
    return SINV_OK;
}

// device state of the tensor-core tier: its work items, ticket, mirror and partial sums
static sinv_status ensure_tc(sinv_handle h) {
    if (h->tc_ready) return SINV_OK;
    const HostPlan& P = h->P;
    cudaError_t e = upload(&h->dtc_items, P.tc_items);
    if (e == cudaSuccess) e = upload(&h->dtc_map, P.tc_map);
    if (e == cudaSuccess) e = upload(&h->dtc_deps, P.tc_deps);
    const size_t mirror = (size_t)(P.n - P.tc_row0) * (size_t)P.tc_width;
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->dtc_ticket, 64);
    if (e == cudaSuccess) e = cudaMemset(h->dtc_ticket, 0, 64);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->dtc_mirror, std::max<size_t>(mirror, 1) * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMalloc((void**)&h->dtc_arrive_t, std::max<int64_t>(P.tc_t_total, 1) * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->dtc_z, std::max<int64_t>(P.tc_z_total, 1) * sizeof(double));
    if (e != cudaSuccess) {
        if (e == cudaErrorMemoryAllocation) {
            set_err(h, "device allocation of the tensor-core tier failed");
            return SINV_ERR_OOM;
        }
        return cuda_fail(h, e, "tensor-core tier state");
    }
    h->tc_ready = true;
    return SINV_OK;
}

sinv_status sinv_selinv(sinv_handle h, const double* L_val, const double* D_val, sinv_precision prec, double* G_S,
                        void* stream) {
    if (!h || !(valid_prec(prec) || tc_prec(prec))) return SINV_ERR_INVALID_ARG;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    const HostPlan& P = h->P;
    if (P.n == 0) return SINV_OK;
    if (!D_val || !G_S || (P.nnzL > 0 && !L_val)) return SINV_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (prec == SINV_FP32) {
        sinv_status s = ensure_work(h, (size_t)P.nnzS * sizeof(float) + 256);
        if (s != SINV_OK) return s;
    }
    TraceScope trace_scope(h->tracer);
    SelinvArgs a;
    a.sn = h->dsn;
    a.order = h->dorder;
    a.items = h->ditems;
    a.nitems = (int32_t)P.items.size();
    a.nsn = (int32_t)P.sn.size();
    a.n = (int32_t)P.n;
    a.owner = h->downer;
    a.Crow = h->dCrow;
    a.Lmap = h->dLmap;
    a.JJl = h->dJJl;
    a.JJs = h->dJJs;
    a.hit_ik = h->dhit_ik;
    a.hit_pos = h->dhit_pos;
    a.hrow = h->dhrow;
    a.Sdiag = h->dSdiag;
    a.l2s = h->dl2s;
    a.dpos = h->ddpos;
    a.pstart = h->dpstart;
    a.Lval = L_val;
    a.Dval = D_val;
    a.done = h->ddone;
    a.epoch = h->depoch;
    a.ticket = h->dticket;
    a.status = h->dstatus;
    a.wait_limit = h->wait_limit;
    a.scratch = h->dscratch;
    a.max_cw = P.max_cw;
    a.nnzS = P.nnzS;
    a.num_sms = h->num_sms;
    a.xsum_off = h->dxsum_off;
    a.xsum = h->dxsum;
    a.arrive = h->darrive;
    a.item0 = 0;
    a.tl.first = h->dtl_first;
    a.tl.last = h->dtl_last;
    a.scan = P.scan;
    a.Srp = h->dSrp;
    a.Sc = h->dSc;
    a.gtab = h->dgtab;
    a.gtab_slots = h->gtab_slots;
    a.counts = h->dtl_first ? h->dscan_counts : nullptr;
    if (a.counts && (e = cudaMemsetAsync(h->dscan_counts, 0, 2 * sizeof(unsigned long long), st)) != cudaSuccess)
        return cuda_fail(h, e, "selinv counters");
    if (h->dtl_first &&
        ((e = cudaMemsetAsync(h->dtl_first, 0xFF, P.sn.size() * sizeof(unsigned long long), st)) != cudaSuccess ||
         (e = cudaMemsetAsync(h->dtl_last, 0, 3 * P.sn.size() * sizeof(unsigned long long), st)) != cudaSuccess))
        return cuda_fail(h, e, "selinv timeline");
    const bool tc = tc_prec(prec) && P.tc_levels > 0;
    if (tc) {
        sinv_status s = ensure_tc(h);
        if (s != SINV_OK) return s;
    }
    if ((e = selinv_prepare(h->depoch, h->dticket, st, tc ? h->dtc_ticket : nullptr)) != cudaSuccess)
        return cuda_fail(h, e, "selinv prepare");
    if ((P.xsum_total > 0 || tc) &&  // partial sums and arrival counts of the supernodes split over CTAs
        ((e = cudaMemsetAsync(h->dxsum, 0, (size_t)P.xsum_total * sizeof(double), st)) != cudaSuccess ||
         (e = cudaMemsetAsync(h->darrive, 0, P.sn.size() * sizeof(uint32_t), st)) != cudaSuccess))
        return cuda_fail(h, e, "selinv prepare");
    if (tc) {
        // the leading levels on the tensor cores, then the rest in FP64 from item rest_first
        const size_t mirror = (size_t)(P.n - P.tc_row0) * (size_t)P.tc_width;
        if ((e = cudaMemsetAsync(h->dtc_mirror, 0, mirror * sizeof(double), st)) != cudaSuccess ||
            (e = cudaMemsetAsync(h->dtc_arrive_t, 0, (size_t)P.tc_t_total * sizeof(uint32_t), st)) != cudaSuccess ||
            (e = cudaMemsetAsync(h->dtc_z, 0, (size_t)P.tc_z_total * sizeof(double), st)) != cudaSuccess)
            return cuda_fail(h, e, "selinv tensor-core prepare");
        TcArgs t;
        t.tcmap = h->dtc_map;
        t.deps = h->dtc_deps;
        t.items = h->dtc_items;
        t.nitems = (int32_t)P.tc_items.size();
        t.ticket = h->dtc_ticket;
        t.mirror = h->dtc_mirror;
        t.row0 = P.tc_row0;
        t.band = P.tc_band;
        t.width = P.tc_width;
        t.arrive_t = h->dtc_arrive_t;
        t.zacc = h->dtc_z;
        if ((e = selinv_tc_launch(a, t, prec == SINV_TF32_FP32ACC ? 2 : 1, G_S, st)) != cudaSuccess)
            return cuda_fail(h, e, "selinv tensor-core launch");
        a.item0 = (int32_t)P.rest_first;
        if (P.rest_first >= (int64_t)P.items.size()) return SINV_OK;
    }
    if ((e = selinv_launch(a, prec == SINV_FP32 ? 1 : 0, h->dwork, G_S, st, h->grid)) != cudaSuccess)
        return cuda_fail(h, e, "selinv launch");
    return SINV_OK;
}

static sinv_status ninv_common(sinv_handle h, const double* L_val, const double* D_val, int m, double delta,
                               sinv_precision prec, double* N_S, double* N_stack, void* stream);

sinv_status sinv_ninv(sinv_handle h, const double* L_val, const double* D_val, int m, sinv_precision prec,
                      double* N_S, void* stream) {
    return ninv_common(h, L_val, D_val, m, 0.0, prec, N_S, nullptr, stream);
}

sinv_status sinv_ninv_drop(sinv_handle h, const double* L_val, const double* D_val, int m, double delta,
                           sinv_precision prec, double* N_S, void* stream) {
    if (!(delta >= 0.0)) return SINV_ERR_INVALID_ARG;  // negative or NaN
    return ninv_common(h, L_val, D_val, m, delta, prec, N_S, nullptr, stream);
}

sinv_status sinv_ninv_stack(sinv_handle h, const double* L_val, const double* D_val, int m, sinv_precision prec,
                            double* N_stack, void* stream) {
    if (h && h->P.n > 0 && !N_stack) return SINV_ERR_INVALID_ARG;
    return ninv_common(h, L_val, D_val, m, 0.0, prec, nullptr, N_stack, stream);
}

static sinv_status ninv_common(sinv_handle h, const double* L_val, const double* D_val, int m, double delta,
                               sinv_precision prec, double* N_S, double* N_stack, void* stream) {
    if (h && tc_prec(prec)) {
        set_err(h, "the tensor-core forms apply to sinv_selinv only");
        return SINV_ERR_UNSUPPORTED;
    }
    if (!h || !valid_prec(prec) || m < 0) return SINV_ERR_INVALID_ARG;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    if (m > 30) {
        set_err(h, "m > 30 is not supported");
        return SINV_ERR_UNSUPPORTED;
    }
    const HostPlan& P = h->P;
    if (P.n == 0) return SINV_OK;
    if (!D_val || (!N_S && !N_stack) || (P.nnzL > 0 && !L_val)) return SINV_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (h->W.m != m) {
        std::string err;
        try {
            err = build_ninv_plan(P, m, h->W);
        } catch (const std::bad_alloc&) {
            set_err(h, "host allocation failed building the Neumann pattern");
            return SINV_ERR_OOM;
        }
        if (!err.empty()) {
            h->W.m = -1;
            set_err(h, err);
            return SINV_ERR_UNSUPPORTED;
        }
        ninv_maps_free(h->X);
        h->index_tried_m = -1;
        if (h->dWcp) cudaFree(h->dWcp);
        if (h->dWr) cudaFree(h->dWr);
        if (h->dgrp) cudaFree(h->dgrp);
        h->dWcp = nullptr; h->dWr = nullptr; h->dgrp = nullptr;
        if ((e = upload(&h->dWcp, h->W.Wcp)) != cudaSuccess || (e = upload(&h->dWr, h->W.Wr)) != cudaSuccess ||
            (e = upload(&h->dgrp, h->W.grp)) != cudaSuccess) {
            h->W.m = -1;
            return cuda_fail(h, e, "upload Neumann pattern");
        }
    }
    TraceScope trace_scope(h->tracer);
    NinvArgs a;
    a.n = P.n;
    a.m = m;
    a.Lcp = h->dLcp;
    a.Lri = h->dLri;
    a.Lcsr = h->dLcsr;
    a.Wcp = h->dWcp;
    a.Wr = h->dWr;
    a.grp = h->dgrp;
    a.Srp = h->dSrp;
    a.Sc = h->dSc;
    a.Lrp = h->dLrp;
    a.nnzS = P.nnzS;
    a.nnzW = h->W.nnzW;
    a.nnzL = P.nnzL;
    a.delta = delta;
    a.dpos = h->ddpos;
    a.pstart = h->dpstart;
    a.Lval = L_val;
    a.Dval = D_val;
    a.max_col = h->W.max_col;
    a.num_sms = h->num_sms;
    a.status = h->dstatus;
    // 0: FP64, 1: FP32, 2: FP64 with the product on S in pairs of floats (map form only)
    int p = prec == SINV_FP32 ? 1 : prec == SINV_FP32X2 ? 2 : 0;
    if (h->index_tried_m != m) {
        h->index_tried_m = m;
        h->index_note = "disabled";
        if (h->index_budget >= 0) {
            int64_t budget = h->index_budget;
            if (budget == 0) {
                size_t free_b = 0, total_b = 0;
                if ((e = cudaMemGetInfo(&free_b, &total_b)) != cudaSuccess) return cuda_fail(h, e, "cudaMemGetInfo");
                budget = (int64_t)(free_b / 2);
            }
            try {
                h->index_note = ninv_maps_build(a, P, h->W, budget, h->X, st, e);
            } catch (const std::bad_alloc&) {
                ninv_maps_free(h->X);
                h->index_note = "host allocation failed building the maps";
            }
            if (e != cudaSuccess && e != cudaErrorMemoryAllocation) return cuda_fail(h, e, "NInv index");
            cudaGetLastError();  // an allocation that did not fit leaves the hash form in use
        }
    }
    if (h->X.ready) {
        sinv_status s = ensure_work(h, ninv_map_work_bytes(a, p));
        if (s != SINV_OK) return s;
        if ((e = ninv_map_launch(a, h->X, p, h->dwork, N_S, st, N_stack)) != cudaSuccess)
            return cuda_fail(h, e, "ninv launch");
        return SINV_OK;
    }
    if (p == 2) p = 0;  // the hash form has no pair product: FP64 throughout
    sinv_status s = ensure_work(h, ninv_work_bytes(a, p));
    if (s != SINV_OK) return s;
    if ((e = ninv_launch(a, p, h->dwork, N_S, st, N_stack)) != cudaSuccess) return cuda_fail(h, e, "ninv launch");
    return SINV_OK;
}

sinv_status sinv_mix(sinv_handle h, const double* G_S, const double* N_S, double eps, double* M_S, void* stream) {
    if (!h) return SINV_ERR_INVALID_ARG;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    if (h->P.nnzS == 0) return SINV_OK;
    if (!G_S || !N_S || !M_S) return SINV_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    TraceScope trace_scope(h->tracer);
    if ((e = mix_launch(G_S, N_S, eps, M_S, h->P.nnzS, h->num_sms, (cudaStream_t)stream)) != cudaSuccess)
        return cuda_fail(h, e, "mix launch");
    return SINV_OK;
}

sinv_status sinv_lowrank_correct(sinv_handle h, int k, const double* V, const double* lambda, sinv_precision prec,
                                 double* X_S, void* stream) {
    if (h && tc_prec(prec)) {
        set_err(h, "the tensor-core forms apply to sinv_selinv only");
        return SINV_ERR_UNSUPPORTED;
    }
    if (!h || k < 0 || !valid_prec(prec)) return SINV_ERR_INVALID_ARG;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    if (k > kLowrankKMax) {
        set_err(h, "k > 256 is not supported");
        return SINV_ERR_UNSUPPORTED;
    }
    if (k == 0 || h->P.n == 0) return SINV_OK;
    if (!V || !lambda || !X_S) return SINV_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (prec == SINV_FP32) {
        sinv_status s = ensure_work(h, ((size_t)h->P.n * k + k) * sizeof(float) + 256);
        if (s != SINV_OK) return s;
    }
    TraceScope trace_scope(h->tracer);
    if ((e = lowrank_launch(h->P.n, h->dSrp, h->dSc, k, V, lambda, prec == SINV_FP32 ? 1 : 0, h->dwork, X_S,
                            h->num_sms, (cudaStream_t)stream)) != cudaSuccess)
        return cuda_fail(h, e, "lowrank launch");
    return SINV_OK;
}

static sinv_status spai_analyse_common(sinv_handle h, int64_t nnzA, const int64_t* A_rowptr, const int32_t* A_col,
                                       int power, int warp_entries, const int64_t* Prp, const int32_t* Pc,
                                       const int32_t* src);

sinv_status sinv_spai_analyse(sinv_handle h, int64_t nnzA, const int64_t* A_rowptr, const int32_t* A_col, int power,
                              int warp_entries) {
    if (!h || nnzA < 0 || !A_rowptr || (nnzA > 0 && !A_col) || warp_entries < 0 || power < 0)
        return SINV_ERR_INVALID_ARG;
    if (power > 8) {
        set_err(h, "power > 8 is not supported");
        return SINV_ERR_UNSUPPORTED;
    }
    return spai_analyse_common(h, nnzA, A_rowptr, A_col, power, warp_entries, nullptr, nullptr, nullptr);
}

// the SPAI plan (from S widened by `power`, or the given pattern) and its upload
static sinv_status spai_analyse_common(sinv_handle h, int64_t nnzA, const int64_t* A_rowptr, const int32_t* A_col,
                                       int power, int warp_entries, const int64_t* Prp, const int32_t* Pc,
                                       const int32_t* src) {
    cudaError_t e = cudaSuccess;
    if (h->device >= 0) {
        if ((e = cudaSetDevice(h->device)) != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(h, e, "synchronize");
    }
    spai_free(h);
    h->spai_mix_gen = -1;
    std::string err;
    try {
        const int we = warp_entries == 0 ? kSpaiWarpE : std::min(warp_entries, kSpaiWarpE);
        err = build_spai_plan(h->P, nnzA, A_rowptr, A_col, power, kSpaiWarpJ, we, kSpaiWarpH / 2, h->Q, Prp, Pc, src);
    } catch (const std::bad_alloc&) {
        h->Q = SpaiPlan();
        set_err(h, "host allocation failed in the SPAI analysis");
        return SINV_ERR_OOM;
    }
    if (!err.empty()) {
        h->Q = SpaiPlan();
        set_err(h, err);
        return err.find("not supported") != std::string::npos ? SINV_ERR_UNSUPPORTED : SINV_ERR_PATTERN;
    }
    h->spai_analysed = true;
    if (h->device < 0) return SINV_OK;  // host-only handle: the plan and the pattern, no upload
    const SpaiPlan& Q = h->Q;
    std::vector<int64_t> Arp(A_rowptr, A_rowptr + h->P.n + 1);
    std::vector<int32_t> Acol(A_col, A_col + nnzA);
    std::vector<int32_t> zero2(2, 0);
#define UPS(dst, src)                                            \
    do {                                                         \
        if ((e = upload(&h->dst, src)) != cudaSuccess) {         \
            spai_free(h);                                        \
            return cuda_fail(h, e, "upload " #dst);              \
        }                                                        \
    } while (0)
    UPS(dfcp, Q.fcp);
    UPS(dfri, Q.fri);
    UPS(dfpos, Q.fpos);
    UPS(dfsrc, Q.fsrc);
    UPS(dfeo, Q.feo);
    UPS(dfE, Q.fE);
    UPS(dfR, Q.fR);
    UPS(dArp, Arp);
    UPS(dAcol, Acol);
    UPS(dscols_w, Q.cols_w);
    UPS(dscols_c, Q.cols_c);
    UPS(dsticket, zero2);
#undef UPS
    if ((e = spai_configure()) != cudaSuccess) {
        spai_free(h);
        return cuda_fail(h, e, "kernel attributes");
    }
    h->spai_cta_bytes = 0;
    if (!Q.cols_c.empty()) {
        h->spai_cta_bytes = (int64_t)spai_cta_bytes(Q.cap_nj, Q.cap_E, Q.cap_H);
        if ((size_t)h->spai_cta_bytes > kSpaiCtaSmemMax) {
            const size_t bytes = (size_t)h->spai_cta_bytes *
                                 (size_t)spai_cta_grid(h->num_sms, (int64_t)Q.cols_c.size(), (size_t)h->spai_cta_bytes);
            if ((e = cudaMalloc((void**)&h->dsscratch, bytes)) != cudaSuccess) {
                spai_free(h);
                return cuda_fail(h, e, "SPAI scratch");
            }
        }
    }
    h->spai_ready = true;
    return SINV_OK;
}

sinv_status sinv_spai_pattern(sinv_handle h, int64_t* P_rowptr, int32_t* P_col) {
    if (!h || !P_rowptr) return SINV_ERR_INVALID_ARG;
    if (!h->spai_analysed) {
        set_err(h, "sinv_spai_pattern needs sinv_spai_analyse first");
        return SINV_ERR_INVALID_ARG;
    }
    if (h->Q.nnzP > 0 && !P_col) return SINV_ERR_INVALID_ARG;
    memcpy(P_rowptr, h->Q.Prp.data(), h->Q.Prp.size() * sizeof(int64_t));
    if (h->Q.nnzP > 0) memcpy(P_col, h->Q.Pc.data(), h->Q.Pc.size() * sizeof(int32_t));
    return SINV_OK;
}

sinv_status sinv_spai(sinv_handle h, const double* A_val, const double* X_S, int iters, double* Y_P, void* stream) {
    if (!h || iters < 0) return SINV_ERR_INVALID_ARG;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    if (!h->spai_ready) {
        set_err(h, "sinv_spai needs sinv_spai_analyse first");
        return SINV_ERR_INVALID_ARG;
    }
    if (h->Q.nnzP == 0) return SINV_OK;
    if (!X_S || !Y_P || (!A_val && h->Q.nnzA > 0)) return SINV_ERR_INVALID_ARG;
    if (X_S == Y_P) {
        set_err(h, "X_S and Y_P must not overlap");
        return SINV_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    const SpaiPlan& Q = h->Q;
    SpaiArgs a;
    a.fcp = h->dfcp;
    a.fri = h->dfri;
    a.fpos = h->dfpos;
    a.fsrc = h->dfsrc;
    a.feo = h->dfeo;
    a.fE = h->dfE;
    a.fR = h->dfR;
    a.Arp = h->dArp;
    a.Acol = h->dAcol;
    a.Aval = A_val;
    a.X = X_S;
    a.Y = Y_P;
    a.nnzP = h->Q.nnzP;
    a.iters = iters;
    a.cols = h->dscols_w;
    a.ncols = (int64_t)Q.cols_w.size();
    a.cols_cta = h->dscols_c;
    a.ncols_cta = (int64_t)Q.cols_c.size();
    a.ticket = h->dsticket;
    a.scratch = h->dsscratch;
    a.cta_bytes = h->spai_cta_bytes;
    a.cta_in_smem = (size_t)h->spai_cta_bytes <= kSpaiCtaSmemMax ? 1 : 0;
    a.cap_nj = Q.cap_nj;
    a.cap_E = Q.cap_E;
    a.cap_H = Q.cap_H;
    a.status = h->dstatus;
    TraceScope trace_scope(h->tracer);
    if ((e = spai_launch(a, h->num_sms, (cudaStream_t)stream)) != cudaSuccess) return cuda_fail(h, e, "spai launch");
    return SINV_OK;
}

sinv_status sinv_einv_analyse(sinv_handle h, int64_t nnzA, const int64_t* A_rowptr, const int32_t* A_col) {
    if (!h || nnzA < 0 || !A_rowptr || (nnzA > 0 && !A_col)) return SINV_ERR_INVALID_ARG;
    cudaError_t e = cudaSuccess;
    if (h->device >= 0) {
        if ((e = cudaSetDevice(h->device)) != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(h, e, "synchronize");
    }
    einv_free(h);
    std::string err;
    try {
        err = build_einv_plan(h->P, nnzA, A_rowptr, A_col, h->E);
    } catch (const std::bad_alloc&) {
        h->E = EinvPlan();
        set_err(h, "host allocation failed in the Lanczos analysis");
        return SINV_ERR_OOM;
    }
    if (!err.empty()) {
        h->E = EinvPlan();
        set_err(h, err);
        return err.find("not supported") != std::string::npos ? SINV_ERR_UNSUPPORTED : SINV_ERR_PATTERN;
    }
    h->einv_analysed = true;
    if (h->device < 0) return SINV_OK;  // host-only handle: the plan only
    const EinvPlan& E = h->E;
    std::vector<int64_t> Arp(A_rowptr, A_rowptr + h->P.n + 1);
    std::vector<int32_t> Acol(A_col, A_col + nnzA);
    std::vector<int64_t> Lrp(h->P.n + 1, 0);
    for (int64_t q = 0; q < h->P.nnzL; ++q) Lrp[h->P.Lri[q] + 1] += 1;
    for (int64_t i = 0; i < h->P.n; ++i) Lrp[i + 1] += Lrp[i];
#define UPE(dst, src)                                            \
    do {                                                         \
        if ((e = upload(&h->dst, src)) != cudaSuccess) {         \
            einv_free(h);                                        \
            return cuda_fail(h, e, "upload " #dst);              \
        }                                                        \
    } while (0)
    UPE(deArp, Arp);
    UPE(deAcol, Acol);
    UPE(deLrp, Lrp);
    UPE(deLcol, E.Lcol);
    UPE(defcp, E.fcp);
    UPE(defri, E.fri);
    UPE(defpos, E.fpos);
    UPE(defwd, E.fwd_rows);
    UPE(debwd, E.bwd_cols);
    UPE(defwdp, E.fwd_ptr);
    UPE(debwdp, E.bwd_ptr);
#undef UPE
    // flags of the two solves (n each), then the epoch and two tickets
    const size_t nflag = 2 * (size_t)h->P.n + 64;
    if ((e = cudaMalloc((void**)&h->detrsv, nflag * sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMemset(h->detrsv, 0, nflag * sizeof(uint32_t))) != cudaSuccess) {
        einv_free(h);
        return cuda_fail(h, e, "triangular-solve flags");
    }
    h->einv_ready = true;
    return SINV_OK;
}

sinv_status sinv_einv_set_solver(sinv_handle h, int32_t solver) {
    if (!h || (solver & ~3) != 0) return SINV_ERR_INVALID_ARG;
    h->einv_solver = solver & 1;
    h->einv_grid_solve = (solver & 2) != 0;
    return SINV_OK;
}

sinv_status sinv_einv_lanczos(sinv_handle h, const double* A_val, const double* L_val, const double* D_val,
                              const double* X_S, const double* q0, int steps, double cg_tol, int cg_maxit, int k,
                              double* lambda, double* V, int32_t* info, void* stream) {
    if (!h) return SINV_ERR_INVALID_ARG;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    if (!h->einv_ready) {
        set_err(h, "sinv_einv_lanczos needs sinv_einv_analyse first");
        return SINV_ERR_INVALID_ARG;
    }
    const int64_t n = h->P.n;
    if (k < 1 || steps < k || steps > n || !(cg_tol > 0.0) || cg_maxit < 1 || !lambda || !V || !info || !q0 ||
        !X_S || !D_val || (!A_val && h->E.nnzA > 0) || (!L_val && h->P.nnzL > 0)) {
        set_err(h, "invalid argument: need 1 <= k <= steps <= n, cg_tol > 0, cg_maxit >= 1 and all buffers");
        return SINV_ERR_INVALID_ARG;
    }
    if (steps > kEinvMaxSteps) {
        set_err(h, "steps > 256 is not supported");
        return SINV_ERR_UNSUPPORTED;
    }
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    TraceScope trace_scope(h->tracer);
    const int nb = einv_dot_blocks(h->num_sms);
    // workspace: 10 vectors, Q, D^{-1} rows, partial sums, scalars, T, U, sel, lam
    const size_t nv = (size_t)n, sq = (size_t)steps * steps;
    const size_t doubles = 10 * nv + (size_t)(steps + 1) * nv + 2 * nv + nb + 8 + (steps + 1) + 2 * sq + k;
    const size_t bytes = doubles * sizeof(double) + (nv + k + 8) * sizeof(int32_t) + 256;
    if (bytes > h->ework_bytes) {
        if (h->dework) cudaFree(h->dework);
        h->dework = nullptr;
        h->ework_bytes = 0;
        if ((e = cudaMalloc(&h->dework, bytes)) != cudaSuccess) return cuda_fail(h, e, "Lanczos workspace");
        h->ework_bytes = bytes;
    }
    double* base = reinterpret_cast<double*>(h->dework);
    double *x = base, *r = x + nv, *z = r + nv, *p = z + nv, *qv = p + nv, *y = qv + nv, *w = y + nv, *v = w + nv;
    double *u1 = v + nv, *u2 = u1 + nv;  // two more work vectors (MINRES)
    double* Q = u2 + nv;
    double* dr = Q + (size_t)(steps + 1) * nv;
    double* dp = dr + nv;
    double* partial = dp + nv;
    double* scal = partial + nb;
    double* cvec = scal + 8;
    double* T = cvec + (steps + 1);
    double* U = T + sq;
    double* lamd = U + sq;
    int32_t* part = reinterpret_cast<int32_t*>(lamd + k);
    int32_t* sel = part + nv;

    const EinvPlan& E = h->E;
    EinvArgs a;
    a.n = n;
    a.num_sms = h->num_sms;
    a.Arp = h->deArp;
    a.Acol = h->deAcol;
    a.Aval = A_val;
    a.fcp = h->defcp;
    a.fri = h->defri;
    a.fpos = h->defpos;
    a.X = X_S;
    a.Lrp = h->deLrp;
    a.Lcol = h->deLcol;
    a.Lcp = h->dLcp;
    a.Lri = h->dLri;
    a.Lcsr = h->dLcsr;
    a.Lval = L_val;
    a.dr = dr;
    a.dp = dp;
    a.part = part;
    a.fwd_rows = h->defwd;
    a.bwd_cols = h->debwd;
    a.fwd_ptr = h->defwdp;
    a.bwd_ptr = h->debwdp;
    a.nlev_fwd = h->E.fwd_ptr.empty() ? 0 : (int32_t)h->E.fwd_ptr.size() - 1;
    a.nlev_bwd = h->E.bwd_ptr.empty() ? 0 : (int32_t)h->E.bwd_ptr.size() - 1;
    // levels of fewer than 64 rows on average: one CTA walks them (a barrier per level
    // costs less than the hand-off between SMs); wider levels: the persistent grid
    a.cta_solve = (!h->einv_grid_solve && a.nlev_fwd > 0 && a.nlev_bwd > 0 &&
                   n < (int64_t)64 * std::min(a.nlev_fwd, a.nlev_bwd)) ? 1 : 0;
    a.fwd_flags = h->detrsv;
    a.bwd_flags = h->detrsv + n;
    a.tepoch = h->detrsv + 2 * n;
    a.tickets = reinterpret_cast<int32_t*>(h->detrsv + 2 * n + 16);
    a.status = h->dstatus;
    a.wait_limit = h->wait_limit;

    NinvArgs na{};
    na.n = n;
    na.dpos = h->ddpos;
    na.pstart = h->dpstart;
    na.Dval = D_val;
    na.num_sms = h->num_sms;
    na.status = h->dstatus;
    // D^{-1} (CG) or |D|^{-1} (MINRES: the SPD preconditioner L |D| L^T)
    if (h->einv_solver == 1)
        einv_absdinv(a, h->ddpos, h->dpstart, D_val, dr, dp, part, st);
    else
        ninv_dinv_launch(na, dr, dp, part, st);

    bool fail = false;
    auto chk = [&](cudaError_t err) {
        if (err != cudaSuccess && !fail) {
            fail = true;
            e = err;
        }
    };
    auto dot = [&](const double* u1, const double* u2) -> double {
        double hv = 0.0;
        chk(einv_dot(a, u1, u2, partial, scal, st));
        chk(cudaMemcpyAsync(&hv, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
        chk(cudaStreamSynchronize(st));
        return hv;
    };
    // q_0 = q0 / ||q0||
    const double n0 = std::sqrt(dot(q0, q0));
    if (fail) return cuda_fail(h, e, "Lanczos start");
    if (!(n0 > 0.0) || !std::isfinite(n0)) {
        set_err(h, "the start vector q0 must be finite and nonzero");
        return SINV_ERR_INVALID_ARG;
    }
    chk(einv_axpby(a, 1.0 / n0, q0, 0.0, q0, Q, st));
    std::vector<double> alph(steps, 0.0), beta(steps, 0.0);
    int m = steps;
    int64_t cg_total = 0;
    int cg_unconverged = 0;
    // x = A^{-1} b by preconditioned MINRES (Paige & Saunders) from x = 0 with the SPD
    // preconditioner L |D| L^T; converged when the estimate of the residual in the
    // preconditioner's inverse norm falls below tol times its start.  Returns true then.
    auto minres = [&](const double* b, double tol, int maxit) -> bool {
        double* r1 = r;
        double* r2 = z;
        double* yv = p;
        double* wv = qv;
        double* w1v = u1;
        double* w2v = u2;
        chk(cudaMemsetAsync(x, 0, nv * sizeof(double), st));
        chk(cudaMemsetAsync(wv, 0, nv * sizeof(double), st));
        chk(cudaMemsetAsync(w2v, 0, nv * sizeof(double), st));
        chk(einv_axpby(a, 1.0, b, 0.0, b, r1, st));
        chk(einv_axpby(a, 1.0, b, 0.0, b, r2, st));
        chk(einv_precond_persistent(a, r1, y, yv, st));
        const double bb = dot(r1, yv);
        if (!(bb > 0.0)) return bb == 0.0;
        const double beta1 = std::sqrt(bb);
        double oldb = 0.0, beta = beta1, dbar = 0.0, epsln = 0.0, phibar = beta1, cs = -1.0, sn = 0.0;
        for (int itn = 1; itn <= maxit && !fail; ++itn) {
            chk(einv_axpby(a, 1.0 / beta, yv, 0.0, yv, v, st));                  // v = y / beta
            chk(einv_spmv_A(a, v, yv, st));                                      // y = A v
            if (itn >= 2) chk(einv_axpby(a, 1.0, yv, -beta / oldb, r1, yv, st)); // y -= (beta/oldb) r1
            const double alfa = dot(v, yv);
            chk(einv_axpby(a, 1.0, yv, -alfa / beta, r2, yv, st));               // y -= (alfa/beta) r2
            std::swap(r1, r2);                                                   // r1 <- r2
            std::swap(r2, yv);                                                   // r2 <- y
            chk(einv_precond_persistent(a, r2, y, yv, st));                      // y = M^{-1} r2
            ++cg_total;
            oldb = beta;
            const double b2 = dot(r2, yv);
            if (!(b2 >= 0.0)) return false;  // the preconditioner lost definiteness
            beta = std::sqrt(b2);
            const double oldeps = epsln;
            const double delta = cs * dbar + sn * alfa;
            const double gbar = sn * dbar - cs * alfa;
            epsln = sn * beta;
            dbar = -cs * beta;
            const double gamma = std::max(std::sqrt(gbar * gbar + beta * beta), 1e-300);
            cs = gbar / gamma;
            sn = beta / gamma;
            const double phi = cs * phibar;
            phibar = sn * phibar;
            // w1 <- w2, w2 <- w, w = (v - oldeps w1 - delta w2) / gamma
            std::swap(w1v, w2v);
            std::swap(w2v, wv);
            chk(einv_axpby(a, 1.0 / gamma, v, -oldeps / gamma, w1v, wv, st));
            chk(einv_axpby(a, 1.0, wv, -delta / gamma, w2v, wv, st));
            chk(einv_axpby(a, 1.0, x, phi, wv, x, st));                          // x += phi w
            if (phibar <= tol * beta1 || beta == 0.0) return true;
        }
        return false;
    };
    for (int it = 0; it < steps && !fail; ++it) {
        const double* qi = Q + (size_t)it * nv;
        bool conv = false;
        if (h->einv_solver == 1) {
            conv = minres(qi, cg_tol, cg_maxit);
        } else {
            // x = A^{-1} q_i by CG preconditioned with L^{-T} D^{-1} L^{-1}, from x = 0
            chk(cudaMemsetAsync(x, 0, nv * sizeof(double), st));
            chk(einv_axpby(a, 1.0, qi, 0.0, qi, r, st));
            const double bn = std::sqrt(dot(r, r));
            chk(einv_precond_persistent(a, r, y, z, st));
            chk(einv_axpby(a, 1.0, z, 0.0, z, p, st));
            double rz = dot(r, z);
            for (int ci = 0; ci < cg_maxit && !fail; ++ci) {
                chk(einv_spmv_A(a, p, qv, st));
                const double pq = dot(p, qv);
                if (!(pq > 0.0)) break;
                const double al = rz / pq;
                chk(einv_cg_xr(a, al, p, qv, x, r, st));
                ++cg_total;
                if (std::sqrt(dot(r, r)) <= cg_tol * bn) {
                    conv = true;
                    break;
                }
                chk(einv_precond_persistent(a, r, y, z, st));
                const double rzn = dot(r, z);
                chk(einv_cg_p(a, rzn / rz, z, p, st));
                rz = rzn;
            }
        }
        if (!conv) ++cg_unconverged;
        // v = A^{-1} q_i - A^inv q_i, alpha_i = q_i . v, then v orthogonalised twice against q_0..q_i
        chk(einv_symv_X(a, qi, y, st));
        chk(einv_axpby(a, 1.0, x, -1.0, y, v, st));
        alph[it] = dot(qi, v);
        chk(einv_reorth(a, Q, it + 1, cvec, v, st));
        chk(einv_reorth(a, Q, it + 1, cvec, v, st));
        const double b = std::sqrt(dot(v, v));
        beta[it] = b;
        if (b < 1e-14 * std::max(1.0, std::fabs(alph[it]))) {
            m = it + 1;
            break;
        }
        chk(einv_axpby(a, 1.0 / b, v, 0.0, v, Q + (size_t)(it + 1) * nv, st));
    }
    if (fail) return cuda_fail(h, e, "Lanczos iteration");
    // Ritz pairs of the tridiagonal T (m x m): the k of largest |theta|
    std::vector<double> Th((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) {
        Th[(size_t)i * m + i] = alph[i];
        if (i + 1 < m) Th[(size_t)i * m + i + 1] = Th[(size_t)(i + 1) * m + i] = beta[i];
    }
    const int kk = std::min(k, m);
    chk(cudaMemcpyAsync(T, Th.data(), Th.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    chk(einv_eig(m, T, U, kk, sel, lamd, st));
    chk(cudaMemsetAsync(V, 0, nv * k * sizeof(double), st));
    chk(einv_ritz(a, m, kk, k, Q, U, sel, V, st));
    std::vector<double> lh(kk);
    chk(cudaMemcpyAsync(lh.data(), lamd, kk * sizeof(double), cudaMemcpyDeviceToHost, st));
    chk(cudaStreamSynchronize(st));
    if (fail) return cuda_fail(h, e, "Ritz pairs");
    for (int l = 0; l < k; ++l) lambda[l] = l < kk ? lh[l] : 0.0;
    info[0] = m;
    info[1] = (int32_t)std::min<int64_t>(cg_total, INT32_MAX);
    info[2] = cg_unconverged;
    return SINV_OK;
}

sinv_status sinv_sync_status(sinv_handle h, void* stream) {
    if (!h) return SINV_ERR_INVALID_ARG;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if ((e = cudaStreamSynchronize((cudaStream_t)stream)) != cudaSuccess) return cuda_fail(h, e, "synchronize");
    int32_t st = 0;
    if ((e = cudaMemcpy(&st, h->dstatus, sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(h, e, "read status");
    if (st != 0) {
        cudaMemset(h->dstatus, 0, sizeof(int32_t));
        if (st == SINV_ERR_TIMEOUT) {
            set_err(h, "a device wait exceeded its poll limit");
            return SINV_ERR_TIMEOUT;
        }
        if (st == SINV_ERR_SINGULAR_PIVOT) {
            set_err(h, "a pivot block of D is singular");
            return SINV_ERR_SINGULAR_PIVOT;
        }
        if (st == ST_BOUNDS) {
            set_err(h, "index out of range (checked build): a plan or map entry points outside its array");
            return SINV_ERR_CUDA;
        }
        set_err(h, "internal device error " + std::to_string(st));
        return SINV_ERR_CUDA;
    }
    return SINV_OK;
}

sinv_status sinv_debug_corrupt_plan(sinv_handle h) {
    if (!h) return SINV_ERR_INVALID_ARG;
#ifndef SINV_CHECKED
    set_err(h, "sinv_debug_corrupt_plan exists in the checked build only");
    return SINV_ERR_UNSUPPORTED;
#else
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    if (h->P.hit_pairs == 0 || h->P.nnzS > INT32_MAX - 1024) {
        set_err(h, "no pair lists to corrupt");
        return SINV_ERR_UNSUPPORTED;
    }
    cudaError_t e = cudaSetDevice(h->device);
    // the first pair of the first supernode that has pairs points past the end of S_lo
    int64_t at = -1;
    for (const SnInfo& I : h->P.sn)
        if (I.hit_cnt > 0) {
            at = I.hit_off;
            break;
        }
    const int32_t bad = (int32_t)(h->P.nnzS + 1000);
    if (e == cudaSuccess && at >= 0) e = cudaMemcpy(h->dhit_pos + at, &bad, sizeof(bad), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? SINV_OK : cuda_fail(h, e, "corrupt plan");
#endif
}

sinv_status sinv_debug_wait_timeout(sinv_handle h, void* stream) {
    if (!h) return SINV_ERR_INVALID_ARG;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    int64_t limit = std::min<int64_t>(h->wait_limit, 200000);
    if ((e = debug_wait_launch(h->ddebug_flag, h->dstatus, limit, (cudaStream_t)stream)) != cudaSuccess)
        return cuda_fail(h, e, "debug wait launch");
    return sinv_sync_status(h, stream);
}

sinv_status sinv_lowrank_correct_noalloc(int64_t n, const int64_t* S_rowptr, const int32_t* S_col, int k,
                                         const double* V, const double* lambda, double* X_S, void* stream) {
    if (n < 0 || k < 0) return SINV_ERR_INVALID_ARG;
    if (k > kLowrankKMax || n * (int64_t)k + k > kLowrankStaticFloats) return SINV_ERR_UNSUPPORTED;
    if (n == 0 || k == 0) return SINV_OK;
    if (!S_rowptr || !S_col || !V || !lambda || !X_S) return SINV_ERR_INVALID_ARG;
    cudaError_t e = lowrank_noalloc_launch(n, S_rowptr, S_col, k, V, lambda, X_S, (cudaStream_t)stream);
    return e == cudaSuccess ? SINV_OK : SINV_ERR_CUDA;
}

// ---- learned correction ------------------------------------------------------------
struct sinv_mlp_s {
    int device = 0;
    int num_sms = 0;
    int64_t max_batch = 0;
    int step = 0;
    float* theta = nullptr;   // FP32 master weights
    float* mom1 = nullptr;
    float* mom2 = nullptr;
    float* grad = nullptr;
    float* partial = nullptr;
    float* loss_partial = nullptr;
    int32_t* dstatus = nullptr;  // first device error of the asynchronous calls (bounded waits)
};

static uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

int32_t sinv_mlp_param_count(void) { return kMlpParams; }

void sinv_mlp_destroy(sinv_mlp m) {
    if (!m) return;
    cudaSetDevice(m->device);
    for (void* p : {(void*)m->theta, (void*)m->mom1, (void*)m->mom2, (void*)m->grad, (void*)m->partial,
                    (void*)m->loss_partial, (void*)m->dstatus})
        if (p) cudaFree(p);
    delete m;
}

sinv_status sinv_mlp_create(int32_t device, uint64_t seed, int64_t max_batch, sinv_mlp* out) {
    if (!out || max_batch <= 0 || device < 0) return SINV_ERR_INVALID_ARG;
    *out = nullptr;
    sinv_mlp m = new (std::nothrow) sinv_mlp_s();
    if (!m) return SINV_ERR_OOM;
    m->device = device;
    m->max_batch = max_batch;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, device);
    const int nblk = mlp_train_blocks(max_batch);
    const size_t P = kMlpParams * sizeof(float);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->theta, P);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->mom1, P);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->mom2, P);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->grad, P);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->partial, (size_t)nblk * P);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->loss_partial, (size_t)nblk * sizeof(float) + 16);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->dstatus, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(m->dstatus, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = mlp_configure();
    if (e != cudaSuccess) {
        sinv_mlp_destroy(m);
        return e == cudaErrorMemoryAllocation ? SINV_ERR_OOM : SINV_ERR_CUDA;
    }
    // He-uniform initial weights from a counter-based hash of (seed, index); zero biases;
    // the output layer is scaled by 0.1 so that the first predictions stay small
    std::vector<float> th(kMlpParams, 0.f);
    auto uni = [&](int p) { return (double)(splitmix64(seed * 0x100000001B3ull + (uint64_t)p) >> 11) / 9007199254740992.0; };
    for (int p = 0; p < kMlpF * kMlpH; ++p) th[kOffW1 + p] = (float)((2 * uni(p) - 1) * sqrt(6.0 / kMlpF));
    for (int p = 0; p < kMlpH * kMlpH; ++p) th[kOffW2 + p] = (float)((2 * uni(kOffW2 + p) - 1) * sqrt(6.0 / kMlpH));
    for (int p = 0; p < kMlpH; ++p) th[kOffW3 + p] = (float)(0.1 * (2 * uni(kOffW3 + p) - 1) * sqrt(6.0 / kMlpH));
    sinv_status st = sinv_mlp_set_params(m, th.data());
    if (st != SINV_OK) {
        sinv_mlp_destroy(m);
        return st;
    }
    *out = m;
    return SINV_OK;
}

sinv_status sinv_mlp_get_params(sinv_mlp m, float* theta) {
    if (!m || !theta) return SINV_ERR_INVALID_ARG;
    cudaSetDevice(m->device);
    return cudaMemcpy(theta, m->theta, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess
               ? SINV_OK
               : SINV_ERR_CUDA;
}

sinv_status sinv_mlp_set_params(sinv_mlp m, const float* theta) {
    if (!m || !theta) return SINV_ERR_INVALID_ARG;
    cudaSetDevice(m->device);
    const size_t P = kMlpParams * sizeof(float);
    if (cudaMemcpy(m->theta, theta, P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->mom1, 0, P) != cudaSuccess || cudaMemset(m->mom2, 0, P) != cudaSuccess)
        return SINV_ERR_CUDA;
    m->step = 0;
    return SINV_OK;
}

sinv_status sinv_mlp_get_state(sinv_mlp m, float* theta, float* mom1, float* mom2, int64_t* step) {
    if (!m || !theta || !mom1 || !mom2 || !step) return SINV_ERR_INVALID_ARG;
    const size_t P = kMlpParams * sizeof(float);
    if (cudaSetDevice(m->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(theta, m->theta, P, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(mom1, m->mom1, P, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(mom2, m->mom2, P, cudaMemcpyDeviceToHost) != cudaSuccess)
        return SINV_ERR_CUDA;
    *step = m->step;
    return SINV_OK;
}

sinv_status sinv_mlp_set_state(sinv_mlp m, const float* theta, const float* mom1, const float* mom2, int64_t step) {
    if (!m || !theta || !mom1 || !mom2 || step < 0 || step > INT32_MAX) return SINV_ERR_INVALID_ARG;
    const size_t P = kMlpParams * sizeof(float);
    if (cudaSetDevice(m->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(m->theta, theta, P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->mom1, mom1, P, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->mom2, mom2, P, cudaMemcpyHostToDevice) != cudaSuccess)
        return SINV_ERR_CUDA;
    m->step = (int)step;
    return SINV_OK;
}

sinv_status sinv_mlp_features(sinv_handle h, const double* N_stack, int m, const double* L_val, const double* D_val,
                              void* X, float* scale, void* stream) {
    if (!h || m < 0) return SINV_ERR_INVALID_ARG;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    if (m > kMlpF - 7) {
        set_err(h, "the feature layout holds the increments of at most 9 Neumann terms");
        return SINV_ERR_UNSUPPORTED;
    }
    if (h->P.n == 0) return SINV_OK;
    if (!N_stack || !D_val || !X || !scale || (h->P.nnzL > 0 && !L_val)) return SINV_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    TraceScope trace_scope(h->tracer);
    if ((e = mlp_features_launch(h->P.n, h->dSrp, h->dSc, h->dLrp, h->dLcp, m, N_stack, h->P.nnzS, L_val, D_val,
                                 h->ddpos, h->dpstart, X, scale, h->num_sms, (cudaStream_t)stream)) != cudaSuccess)
        return cuda_fail(h, e, "mlp features");
    return SINV_OK;
}

sinv_status sinv_mlp_targets(sinv_mlp m, int64_t count, const double* G, const double* N, const float* scale, float* y,
                             void* stream) {
    if (!m || count < 0 || (count > 0 && (!G || !N || !scale || !y))) return SINV_ERR_INVALID_ARG;
    cudaSetDevice(m->device);
    return mlp_targets_launch(count, G, N, scale, y, m->num_sms, (cudaStream_t)stream) == cudaSuccess ? SINV_OK
                                                                                                     : SINV_ERR_CUDA;
}

sinv_status sinv_mlp_grad(sinv_mlp m, const void* X, const float* y, const int64_t* idx, int64_t count, float* grad,
                          float* loss, void* stream) {
    if (!m || !X || !y || count <= 0 || count > m->max_batch) return SINV_ERR_INVALID_ARG;
    cudaSetDevice(m->device);
    return mlp_grad_launch(X, y, idx, count, m->theta, m->partial, m->loss_partial, grad ? grad : m->grad, loss,
                           (cudaStream_t)stream) == cudaSuccess
               ? SINV_OK
               : SINV_ERR_CUDA;
}

sinv_status sinv_mlp_train_step(sinv_mlp m, const void* X, const float* y, const int64_t* idx, int64_t count, float lr,
                                float* loss, void* stream) {
    sinv_status s = sinv_mlp_grad(m, X, y, idx, count, nullptr, loss, stream);
    if (s != SINV_OK) return s;
    m->step += 1;
    return mlp_adam_launch(m->theta, m->mom1, m->mom2, m->grad, lr, m->step, (cudaStream_t)stream) == cudaSuccess
               ? SINV_OK
               : SINV_ERR_CUDA;
}

sinv_status sinv_mlp_predict(sinv_mlp m, const void* X, const float* scale, const double* N, int64_t count, double* out,
                             void* stream) {
    if (!m || count < 0 || (count > 0 && (!X || !scale || !N || !out))) return SINV_ERR_INVALID_ARG;
    if (((uintptr_t)X & 15) != 0) return SINV_ERR_INVALID_ARG;  // rows are read as 16-byte vectors
    cudaSetDevice(m->device);
    return mlp_predict_launch(X, scale, N, count, m->theta, out, m->dstatus, kMlpWaitLimit, m->num_sms,
                              (cudaStream_t)stream) == cudaSuccess
               ? SINV_OK
               : SINV_ERR_CUDA;
}

sinv_status sinv_mlp_sync_status(sinv_mlp m, void* stream) {
    if (!m) return SINV_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(m->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    int32_t st = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&st, m->dstatus, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return SINV_ERR_CUDA;
    if (st != 0) {
        cudaMemset(m->dstatus, 0, sizeof(int32_t));
        return st == SINV_ERR_TIMEOUT ? SINV_ERR_TIMEOUT : SINV_ERR_CUDA;
    }
    return SINV_OK;
}

sinv_status sinv_trace_enable(sinv_handle h, int enable) {
    if (!h) return SINV_ERR_INVALID_ARG;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    if (enable && !h->tracer) h->tracer = new (std::nothrow) Tracer();
    if (enable && !h->tracer) return SINV_ERR_OOM;
    if (!enable && h->tracer) {
        cudaSetDevice(h->device);
        delete h->tracer;
        h->tracer = nullptr;
    }
    return SINV_OK;
}

sinv_status sinv_trace_read(sinv_handle h, sinv_kernel_time* out, int max_entries, int* count, int reset) {
    if (!h || !count || max_entries < 0 || (max_entries > 0 && !out)) return SINV_ERR_INVALID_ARG;
    *count = 0;
    if (!h->tracer) return SINV_OK;
    cudaSetDevice(h->device);
    h->tracer->collect();
    int c = 0;
    for (auto& kv : h->tracer->agg) {
        if (c < max_entries) {
            memset(&out[c], 0, sizeof(out[c]));
            strncpy(out[c].name, kv.first.c_str(), sizeof(out[c].name) - 1);
            out[c].launches = kv.second.first;
            out[c].total_ms = kv.second.second;
        }
        ++c;
    }
    *count = std::min(c, max_entries);
    if (reset) h->tracer->agg.clear();
    return SINV_OK;
}

sinv_status sinv_batch_run(sinv_handle h, int32_t nmat, const double* const* L_vals, const double* const* D_vals,
                           sinv_precision prec, double* const* G_outs, int m, double* const* N_outs, void* stream) {
    if (!h || nmat < 0) return SINV_ERR_INVALID_ARG;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    const int32_t nb = h->b_n_off.empty() ? 0 : (int32_t)h->b_n_off.size() - 1;
    if (nb == 0 || nmat != nb) {
        set_err(h, "sinv_batch_run needs a handle from sinv_batch_symbolic with the same number of matrices");
        return SINV_ERR_INVALID_ARG;
    }
    if (!L_vals || !D_vals || (N_outs && m < 0)) return SINV_ERR_INVALID_ARG;
    for (int32_t b = 0; b < nb; ++b) {
        const bool has_L = h->b_L_off[b + 1] > h->b_L_off[b];
        if ((has_L && !L_vals[b]) || !D_vals[b]) return SINV_ERR_INVALID_ARG;
    }
    const HostPlan& P = h->P;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (!h->db_L) {  // the first call allocates; later calls (and graph captures) do not
        if ((e = upload(&h->db_L_off, h->b_L_off)) != cudaSuccess || (e = upload(&h->db_D_off, h->b_D_off)) != cudaSuccess ||
            (e = upload(&h->db_S_off, h->b_S_off)) != cudaSuccess ||
            (e = cudaMalloc((void**)&h->db_L, std::max<int64_t>(P.nnzL, 1) * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&h->db_D, std::max<int64_t>(P.nD, 1) * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&h->db_G, std::max<int64_t>(P.nnzS, 1) * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void**)&h->db_N, std::max<int64_t>(P.nnzS, 1) * sizeof(double))) != cudaSuccess) {
            if (e == cudaErrorMemoryAllocation) {
                set_err(h, "device allocation of the batch buffers failed");
                return SINV_ERR_OOM;
            }
            return cuda_fail(h, e, "batch buffers");
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    if ((e = batch_copy_launch(nb, L_vals, h->db_L_off, 1, h->db_L, h->num_sms, st)) != cudaSuccess ||
        (e = batch_copy_launch(nb, D_vals, h->db_D_off, 1, h->db_D, h->num_sms, st)) != cudaSuccess)
        return cuda_fail(h, e, "batch gather");
    if (G_outs) {
        sinv_status s = sinv_selinv(h, h->db_L, h->db_D, prec, h->db_G, stream);
        if (s != SINV_OK) return s;
        if ((e = batch_copy_launch(nb, const_cast<const double* const*>(G_outs), h->db_S_off, 0, h->db_G, h->num_sms,
                                   st)) != cudaSuccess)
            return cuda_fail(h, e, "batch scatter");
    }
    if (N_outs) {
        sinv_status s = ninv_common(h, h->db_L, h->db_D, m, 0.0, prec, h->db_N, nullptr, stream);
        if (s != SINV_OK) return s;
        if ((e = batch_copy_launch(nb, const_cast<const double* const*>(N_outs), h->db_S_off, 0, h->db_N, h->num_sms,
                                   st)) != cudaSuccess)
            return cuda_fail(h, e, "batch scatter");
    }
    return SINV_OK;
}

sinv_status sinv_ninv_own(sinv_handle h, const double* L_val, const double* D_val, int m, double delta, void* stream) {
    if (!h || m < 0 || !(delta >= 0.0)) return SINV_ERR_INVALID_ARG;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    if (m > 30) {
        set_err(h, "m > 30 is not supported");
        return SINV_ERR_UNSUPPORTED;
    }
    const HostPlan& P = h->P;
    const int64_t n = P.n;
    if (n > 0 && (!D_val || (P.nnzL > 0 && !L_val))) return SINV_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (n == 0) {  // the empty matrix: an empty result (colptr {0}) that the size, copy and Mix calls accept
        if ((e = empty_csc(&h->down_cp, &h->down_r, &h->down_v, st)) != cudaSuccess)
            return cuda_fail(h, e, "NInv own-pattern result");
        h->own_nnz = h->own_nnzW = 0;
        h->own_nnzW_steps.assign(m + 1, 0);
        h->own_hint.clear();
        return SINV_OK;
    }
    TraceScope trace_scope(h->tracer);
    auto fail = [&](cudaError_t err, const char* what) -> sinv_status {
        if (err == cudaErrorMemoryAllocation) {
            set_err(h, std::string("device allocation failed: ") + what);
            return SINV_ERR_OOM;
        }
        return cuda_fail(h, err, what);
    };
    // a buffer that only grows
    auto ensure = [](DevBuf& b, int64_t& have, int64_t need, size_t esize) -> cudaError_t {
        if (need <= have && b.p) return cudaSuccess;
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        have = 0;
        cudaError_t err = dev_alloc(b, (size_t)std::max<int64_t>(need, 1) * esize);
        if (err == cudaSuccess) have = need;
        return err;
    };
    auto read64 = [&](const void* dptr, int64_t* out) -> cudaError_t {
        cudaError_t err = cudaMemcpyAsync(out, dptr, 8, cudaMemcpyDeviceToHost, st);
        return err == cudaSuccess ? cudaStreamSynchronize(st) : err;
    };
    DevBuf dr, dp, part, ticket, scal, stA, ctA, stB, ctB, rA, vA, rB, vB, gk, gv;
    int64_t capA = 0, capB = 0, have_gk = 0, have_gv = 0;
    if ((e = dev_alloc(dr, n * 8)) != cudaSuccess || (e = dev_alloc(dp, n * 8)) != cudaSuccess ||
        (e = dev_alloc(part, n * 4)) != cudaSuccess || (e = dev_alloc(ticket, 64)) != cudaSuccess ||
        (e = dev_alloc(scal, 64)) != cudaSuccess || (e = dev_alloc(stA, n * 8)) != cudaSuccess ||
        (e = dev_alloc(ctA, n * 8)) != cudaSuccess || (e = dev_alloc(stB, n * 8)) != cudaSuccess ||
        (e = dev_alloc(ctB, n * 8)) != cudaSuccess || (e = ensure(rA, capA, n, 4)) != cudaSuccess ||
        (e = dev_alloc(vA, n * 8)) != cudaSuccess)
        return fail(e, "NInv own-pattern work");
    int64_t* d_max = scal.as<int64_t>();
    NinvArgs na{};
    na.n = n;
    na.dpos = h->ddpos;
    na.pstart = h->dpstart;
    na.Dval = D_val;
    na.num_sms = h->num_sms;
    na.status = h->dstatus;
    ninv_dinv_launch(na, dr.as<double>(), dp.as<double>(), part.as<int32_t>(), st);
    OwnArgs a;
    a.n = n;
    a.num_sms = h->num_sms;
    a.grid = own_grid_ctas(h->num_sms);
    a.Lcp = h->dLcp;
    a.Lri = h->dLri;
    a.Lcsr = h->dLcsr;
    a.Lval = L_val;
    a.delta = delta;
    a.dr = dr.as<double>();
    a.dp = dp.as<double>();
    a.part = part.as<int32_t>();
    a.gkeys = nullptr;
    a.gvals = nullptr;
    a.gslice = 0;
    a.ticket = ticket.as<int32_t>();
    a.cursor = reinterpret_cast<unsigned long long*>(scal.as<int64_t>() + 1);
    // global hash tables of `slots` slots per CTA when shared memory is too small;
    // fewer CTAs when all of them would pass the table budget
    const int64_t table_budget = int64_t(8) << 30;
    auto tables = [&](int64_t slots, bool fits) -> cudaError_t {
        a.grid = own_grid_ctas(h->num_sms);
        a.gslice = 0;
        if (fits) return cudaSuccess;
        a.gslice = slots;
        const int64_t per = slots * (int64_t)(sizeof(int32_t) + sizeof(double));
        a.grid = (int)std::max<int64_t>(1, std::min<int64_t>(a.grid, table_budget / per));
        cudaError_t err;
        if ((err = ensure(gk, have_gk, (int64_t)a.grid * slots, 4)) != cudaSuccess ||
            (err = ensure(gv, have_gv, (int64_t)a.grid * slots, 8)) != cudaSuccess)
            return err;
        a.gkeys = gk.as<int32_t>();
        a.gvals = gv.as<double>();
        return cudaSuccess;
    };
    // W_0 = I, then m Horner steps; an output that overflows is grown to the exact
    // count the cursor reports and the step runs again
    h->own_nnzW_steps.assign(1, n);
    if ((e = own_identity_launch(n, stA.as<int64_t>(), ctA.as<int64_t>(), rA.as<int32_t>(), vA.as<double>(),
                                 h->num_sms, st)) != cudaSuccess)
        return fail(e, "NInv own-pattern identity");
    int64_t nnz_prev = n, vcapB = 0;
    for (int t = 1; t <= m; ++t) {
        int64_t maxb = 0;
        if ((e = own_bound_launch(n, h->dLcp, h->dLri, ctA.as<int64_t>(), d_max, h->num_sms, st)) != cudaSuccess ||
            (e = read64(d_max, &maxb)) != cudaSuccess ||
            (e = tables(own_table_slots(maxb), own_table_slots(maxb) <= own_horner_slots())) != cudaSuccess)
            return fail(e, "NInv own-pattern Horner tables");
        int64_t want = std::max<int64_t>(capB, 2 * nnz_prev + n);
        if ((int64_t)h->own_hint.size() > t) want = std::max<int64_t>(want, h->own_hint[t] + h->own_hint[t] / 32);
        for (int attempt = 0;; ++attempt) {
            if ((e = ensure(rB, capB, want, 4)) != cudaSuccess || (e = ensure(vB, vcapB, want, 8)) != cudaSuccess)
                return fail(e, "NInv own-pattern Horner output");
            int64_t tot = 0;
            if ((e = own_horner_launch(a, stA.as<int64_t>(), ctA.as<int64_t>(), rA.as<int32_t>(), vA.as<double>(),
                                       rB.as<int32_t>(), vB.as<double>(), stB.as<int64_t>(), ctB.as<int64_t>(),
                                       std::min(capB, vcapB), st)) != cudaSuccess ||
                (e = read64(a.cursor, &tot)) != cudaSuccess)
                return fail(e, "NInv own-pattern Horner step");
            if (tot <= std::min(capB, vcapB)) {
                nnz_prev = tot;
                break;
            }
            if (attempt > 0) {
                set_err(h, "NInv own-pattern Horner step: output count changed between runs");
                return SINV_ERR_CUDA;
            }
            // room for entries at the drop threshold that another summation order keeps
            want = tot + tot / 32 + 1024;
        }
        std::swap(stA.p, stB.p);
        std::swap(ctA.p, ctB.p);
        std::swap(rA.p, rB.p);
        std::swap(vA.p, vB.p);
        std::swap(capA, capB);
        vcapB = capB;  // the buffers swapped: r and v have the same capacity in each pair from here on
        h->own_nnzW_steps.push_back(nnz_prev);
    }
    const int64_t nnzW = nnz_prev;
    // W by rows, the diagonal of N and the bound of every column of N
    DevBuf rowcnt, rp, fill, rc, rv, diag, bound;
    if ((e = dev_alloc(rowcnt, (n + 1) * 8)) != cudaSuccess || (e = dev_alloc(rp, (n + 1) * 8)) != cudaSuccess ||
        (e = dev_alloc(fill, (n + 1) * 8)) != cudaSuccess || (e = dev_alloc(rc, nnzW * 4)) != cudaSuccess ||
        (e = dev_alloc(rv, nnzW * 8)) != cudaSuccess || (e = dev_alloc(diag, n * 8)) != cudaSuccess ||
        (e = dev_alloc(bound, (n + 1) * 8)) != cudaSuccess)
        return fail(e, "NInv own-pattern product work");
    int64_t maxct = 0, maxbound = 0;
    if ((e = own_transpose_launch(n, nnzW, stA.as<int64_t>(), ctA.as<int64_t>(), rA.as<int32_t>(), vA.as<double>(),
                                  rowcnt.as<int64_t>(), rp.as<int64_t>(), fill.as<int64_t>(), rc.as<int32_t>(),
                                  rv.as<double>(), h->num_sms, st)) != cudaSuccess ||
        (e = own_max_launch(n, ctA.as<int64_t>(), d_max, h->num_sms, st)) != cudaSuccess ||
        (e = read64(d_max, &maxct)) != cudaSuccess ||
        (e = tables(own_table_slots(2 * maxct), own_table_slots(2 * maxct) <= own_smem_slots())) != cudaSuccess ||
        (e = own_diag_launch(a, stA.as<int64_t>(), ctA.as<int64_t>(), rA.as<int32_t>(), vA.as<double>(),
                             rp.as<int64_t>(), diag.as<double>(), bound.as<int64_t>(), d_max, st)) != cudaSuccess ||
        (e = read64(d_max, &maxbound)) != cudaSuccess)
        return fail(e, "NInv own-pattern diagonal");
    // the product's tables: Y[:, j] in the first half of a CTA's slice, N's column in the second
    {
        const int64_t half = std::max<int64_t>(own_table_slots(2 * maxct), own_table_slots(std::max<int64_t>(maxbound, 1)));
        if ((e = tables(2 * half, half <= own_prod_slots())) != cudaSuccess)
            return fail(e, "NInv own-pattern product tables");
    }
    DevBuf nr, nv, stN, ctN, cpN;
    int64_t capN = 0, vcapN = 0;
    if ((e = dev_alloc(stN, n * 8)) != cudaSuccess || (e = dev_alloc(ctN, n * 8)) != cudaSuccess ||
        (e = dev_alloc(cpN, (n + 1) * 8)) != cudaSuccess)
        return fail(e, "NInv own-pattern product work");
    int64_t nnzN = 0, want = std::max<int64_t>(2 * nnzW, 2 * n);
    if ((int64_t)h->own_hint.size() > m + 1) want = std::max<int64_t>(want, h->own_hint[m + 1] + h->own_hint[m + 1] / 32);
    for (int attempt = 0;; ++attempt) {
        if ((e = ensure(nr, capN, want, 4)) != cudaSuccess || (e = ensure(nv, vcapN, want, 8)) != cudaSuccess)
            return fail(e, "NInv own-pattern product output");
        if ((e = own_product_launch(a, stA.as<int64_t>(), ctA.as<int64_t>(), rA.as<int32_t>(), vA.as<double>(),
                                    rp.as<int64_t>(), rc.as<int32_t>(), rv.as<double>(), diag.as<double>(),
                                    bound.as<int64_t>(), nr.as<int32_t>(), nv.as<double>(), stN.as<int64_t>(),
                                    ctN.as<int64_t>(), std::min(capN, vcapN), st)) != cudaSuccess ||
            (e = read64(a.cursor, &nnzN)) != cudaSuccess)
            return fail(e, "NInv own-pattern product");
        if (nnzN <= std::min(capN, vcapN)) break;
        if (attempt > 0) {
            set_err(h, "NInv own-pattern product: output count changed between runs");
            return SINV_ERR_CUDA;
        }
        want = nnzN + nnzN / 32 + 1024;
    }
    // the result, owned by the handle: CSC of the lower triangle
    if (h->down_cp) cudaFree(h->down_cp);
    if (h->down_r) cudaFree(h->down_r);
    if (h->down_v) cudaFree(h->down_v);
    h->down_cp = nullptr;
    h->down_r = nullptr;
    h->down_v = nullptr;
    if ((e = cudaMalloc((void**)&h->down_cp, (n + 1) * 8)) != cudaSuccess ||
        (e = cudaMalloc((void**)&h->down_r, std::max<int64_t>(nnzN, 1) * 4)) != cudaSuccess ||
        (e = cudaMalloc((void**)&h->down_v, std::max<int64_t>(nnzN, 1) * 8)) != cudaSuccess)
        return fail(e, "NInv own-pattern result");
    if ((e = own_scan_launch(n, ctN.as<int64_t>(), h->down_cp, st)) != cudaSuccess ||
        (e = own_compact_launch(n, stN.as<int64_t>(), h->down_cp, nr.as<int32_t>(), nv.as<double>(), h->down_r,
                                h->down_v, h->num_sms, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(e, "NInv own-pattern compaction");
    h->own_nnz = nnzN;
    h->own_nnzW = nnzW;
    h->own_hint = h->own_nnzW_steps;
    h->own_hint.push_back(nnzN);
    return SINV_OK;
}

sinv_status sinv_ninv_own_size(sinv_handle h, int64_t* nnz_N_lo, int64_t* nnz_W_steps, int32_t max_steps) {
    if (!h || !nnz_N_lo || max_steps < 0 || (max_steps > 0 && !nnz_W_steps)) return SINV_ERR_INVALID_ARG;
    if (!h->down_cp) {
        set_err(h, "sinv_ninv_own has not run");
        return SINV_ERR_INVALID_ARG;
    }
    *nnz_N_lo = h->own_nnz;
    for (int32_t t = 0; t < max_steps; ++t)
        nnz_W_steps[t] = t < (int32_t)h->own_nnzW_steps.size() ? h->own_nnzW_steps[t] : 0;
    return SINV_OK;
}

sinv_status sinv_ninv_own_copy(sinv_handle h, int64_t* N_colptr, int32_t* N_row, double* N_val, void* stream) {
    if (!h || !N_colptr || !N_row || !N_val) return SINV_ERR_INVALID_ARG;
    if (!h->down_cp) {
        set_err(h, "sinv_ninv_own has not run");
        return SINV_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(N_colptr, h->down_cp, (h->P.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && h->own_nnz > 0)
        e = cudaMemcpyAsync(N_row, h->down_r, h->own_nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && h->own_nnz > 0)
        e = cudaMemcpyAsync(N_val, h->down_v, h->own_nnz * sizeof(double), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? SINV_OK : cuda_fail(h, e, "NInv own-pattern copy");
}

sinv_status sinv_mix_own(sinv_handle h, const double* G_S, double eps, void* stream) {
    if (!h || eps != eps || (!G_S && h->P.nnzS > 0)) return SINV_ERR_INVALID_ARG;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    if (!h->down_cp) {
        set_err(h, "sinv_ninv_own has not run");
        return SINV_ERR_INVALID_ARG;
    }
    const HostPlan& P = h->P;
    const int64_t n = P.n;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (n == 0) {  // the empty matrix: an empty result
        h->mix_nnz = -1;
        if ((e = empty_csc(&h->dmix_cp, &h->dmix_r, &h->dmix_v, st)) != cudaSuccess)
            return cuda_fail(h, e, "Mix own-pattern result");
        h->mix_nnz = 0;
        h->mix_gen += 1;
        return SINV_OK;
    }
    TraceScope trace_scope(h->tracer);
    auto fail = [&](cudaError_t err, const char* what) -> sinv_status {
        if (err == cudaErrorMemoryAllocation) {
            set_err(h, std::string("device allocation failed: ") + what);
            return SINV_ERR_OOM;
        }
        return cuda_fail(h, err, what);
    };
    DevBuf ticket, scal, cnt, gk;
    int64_t maxlen = 0;
    if ((e = dev_alloc(ticket, 64)) != cudaSuccess || (e = dev_alloc(scal, 64)) != cudaSuccess ||
        (e = dev_alloc(cnt, (n + 1) * 8)) != cudaSuccess ||
        (e = own_max_col_launch(n, h->down_cp, scal.as<int64_t>(), h->num_sms, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&maxlen, scal.p, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(e, "Mix own-pattern work");
    MixOwnArgs a;
    a.n = n;
    a.grid = own_grid_ctas(h->num_sms);
    a.Ncp = h->down_cp;
    a.Nr = h->down_r;
    a.Nv = h->down_v;
    a.Srp = h->dSrp;
    a.Sdiag = h->dSdiag;
    a.Lcp = h->dLcp;
    a.Lri = h->dLri;
    a.Lcsr = h->dLcsr;
    a.l2s = h->dl2s;
    a.pstart = h->dpstart;
    a.G = G_S;
    a.eps = eps;
    a.gkeys = nullptr;
    a.gslice = 0;
    a.ticket = ticket.as<int32_t>();
    const int64_t slots = own_table_slots(maxlen);
    if (slots > own_smem_slots()) {
        // keys and positions of N's longest column per CTA, in global memory
        a.gslice = slots;
        a.grid = (int)std::max<int64_t>(1, std::min<int64_t>(a.grid, (int64_t(4) << 30) / (8 * slots)));
        if ((e = dev_alloc(gk, (size_t)a.grid * 2 * slots * sizeof(int32_t))) != cudaSuccess)
            return fail(e, "Mix own-pattern tables");
        a.gkeys = gk.as<int32_t>();
    }
    int64_t total = 0;
    if (h->dmix_cp) cudaFree(h->dmix_cp);
    h->dmix_cp = nullptr;
    h->mix_nnz = -1;
    if ((e = cudaMalloc((void**)&h->dmix_cp, (n + 1) * 8)) != cudaSuccess ||
        (e = mix_own_launch(a, false, cnt.as<int64_t>(), nullptr, nullptr, st)) != cudaSuccess ||
        (e = own_scan_launch(n, cnt.as<int64_t>(), h->dmix_cp, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&total, h->dmix_cp + n, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(e, "Mix own-pattern count");
    if (h->dmix_r) cudaFree(h->dmix_r);
    if (h->dmix_v) cudaFree(h->dmix_v);
    h->dmix_r = nullptr;
    h->dmix_v = nullptr;
    if ((e = cudaMalloc((void**)&h->dmix_r, std::max<int64_t>(total, 1) * 4)) != cudaSuccess ||
        (e = cudaMalloc((void**)&h->dmix_v, std::max<int64_t>(total, 1) * 8)) != cudaSuccess ||
        (e = mix_own_launch(a, true, h->dmix_cp, h->dmix_r, h->dmix_v, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(e, "Mix own-pattern fill");
    h->mix_nnz = total;
    h->mix_gen += 1;
    return SINV_OK;
}

sinv_status sinv_spai_analyse_mix_own(sinv_handle h, int64_t nnzA, const int64_t* A_rowptr, const int32_t* A_col,
                                      int warp_entries) {
    if (!h || nnzA < 0 || !A_rowptr || (nnzA > 0 && !A_col) || warp_entries < 0) return SINV_ERR_INVALID_ARG;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    if (h->mix_nnz < 0) {
        set_err(h, "sinv_mix_own has not run");
        return SINV_ERR_INVALID_ARG;
    }
    if (h->mix_nnz >= ((int64_t)1 << 31)) {
        set_err(h, "the Mix pattern has >= 2^31 entries: not supported");
        return SINV_ERR_UNSUPPORTED;
    }
    const int64_t n = h->P.n;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    // the Mix pattern by rows (lower triangle, sorted rows) and, per entry, its index
    // in the Mix value array
    std::vector<int64_t> cp(n + 1), Prp(n + 1, 0);
    std::vector<int32_t> rows(std::max<int64_t>(h->mix_nnz, 1)), Pc, src;
    try {
        if ((e = cudaMemcpy(cp.data(), h->dmix_cp, (n + 1) * 8, cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (h->mix_nnz > 0 &&
             (e = cudaMemcpy(rows.data(), h->dmix_r, h->mix_nnz * 4, cudaMemcpyDeviceToHost)) != cudaSuccess))
            return cuda_fail(h, e, "Mix pattern read");
        for (int64_t q = 0; q < h->mix_nnz; ++q) Prp[rows[q] + 1]++;
        for (int64_t i = 0; i < n; ++i) Prp[i + 1] += Prp[i];
        Pc.resize(h->mix_nnz);
        src.resize(h->mix_nnz);
        std::vector<int64_t> fill(Prp.begin(), Prp.end() - 1);
        for (int64_t j = 0; j < n; ++j)  // columns in increasing order: every row comes out sorted
            for (int64_t q = cp[j]; q < cp[j + 1]; ++q) {
                const int64_t d = fill[rows[q]]++;
                Pc[d] = (int32_t)j;
                src[d] = (int32_t)q;
            }
    } catch (const std::bad_alloc&) {
        set_err(h, "host allocation failed in the SPAI analysis");
        return SINV_ERR_OOM;
    }
    sinv_status s = spai_analyse_common(h, nnzA, A_rowptr, A_col, 0, warp_entries, Prp.data(), Pc.data(), src.data());
    if (s == SINV_OK) h->spai_mix_gen = h->mix_gen;
    return s;
}

sinv_status sinv_spai_mix_own(sinv_handle h, const double* A_val, const double* X_M, int iters, double* Y_P,
                              void* stream) {
    if (!h) return SINV_ERR_INVALID_ARG;
    if (h->spai_mix_gen < 0 || h->spai_mix_gen != h->mix_gen) {
        set_err(h, "sinv_spai_mix_own needs sinv_spai_analyse_mix_own on the current Mix result");
        return SINV_ERR_INVALID_ARG;
    }
    return sinv_spai(h, A_val, X_M ? X_M : h->dmix_v, iters, Y_P, stream);
}

sinv_status sinv_lowrank_correct_mix_own(sinv_handle h, int k, const double* V, const double* lambda,
                                         sinv_precision prec, void* stream) {
    if (h && tc_prec(prec)) {
        set_err(h, "the tensor-core forms apply to sinv_selinv only");
        return SINV_ERR_UNSUPPORTED;
    }
    if (!h || k < 0 || !valid_prec(prec)) return SINV_ERR_INVALID_ARG;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    if (h->mix_nnz < 0) {
        set_err(h, "sinv_mix_own has not run");
        return SINV_ERR_INVALID_ARG;
    }
    if (k > kLowrankKMax) {
        set_err(h, "k > 256 is not supported");
        return SINV_ERR_UNSUPPORTED;
    }
    if (k == 0 || h->P.n == 0) return SINV_OK;
    if (!V || !lambda) return SINV_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (prec == SINV_FP32) {
        sinv_status s = ensure_work(h, ((size_t)h->P.n * k + k) * sizeof(float) + 256);
        if (s != SINV_OK) return s;
    }
    TraceScope trace_scope(h->tracer);
    // the correction is symmetric in (i, j): the CSC of the lower triangle serves as
    // the CSR of the upper one
    if ((e = lowrank_launch(h->P.n, h->dmix_cp, h->dmix_r, k, V, lambda, prec == SINV_FP32 ? 1 : 0, h->dwork,
                            h->dmix_v, h->num_sms, (cudaStream_t)stream)) != cudaSuccess)
        return cuda_fail(h, e, "lowrank launch");
    return SINV_OK;
}

sinv_status sinv_mix_own_size(sinv_handle h, int64_t* nnz) {
    if (!h || !nnz) return SINV_ERR_INVALID_ARG;
    if (h->mix_nnz < 0) {
        set_err(h, "sinv_mix_own has not run");
        return SINV_ERR_INVALID_ARG;
    }
    *nnz = h->mix_nnz;
    return SINV_OK;
}

sinv_status sinv_mix_own_copy(sinv_handle h, int64_t* M_colptr, int32_t* M_row, double* M_val, void* stream) {
    if (!h || !M_colptr || !M_row || !M_val) return SINV_ERR_INVALID_ARG;
    if (h->mix_nnz < 0) {
        set_err(h, "sinv_mix_own has not run");
        return SINV_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(M_colptr, h->dmix_cp, (h->P.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && h->mix_nnz > 0)
        e = cudaMemcpyAsync(M_row, h->dmix_r, h->mix_nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && h->mix_nnz > 0)
        e = cudaMemcpyAsync(M_val, h->dmix_v, h->mix_nnz * sizeof(double), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? SINV_OK : cuda_fail(h, e, "Mix own-pattern copy");
}

sinv_status sinv_timeline_enable(sinv_handle h, int enable) {
    if (!h) return SINV_ERR_INVALID_ARG;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    const size_t ns = std::max<size_t>(h->P.sn.size(), 1);
    if (enable && !h->dtl_first) {
        if ((e = cudaMalloc((void**)&h->dtl_first, ns * sizeof(unsigned long long))) != cudaSuccess ||
            (e = cudaMalloc((void**)&h->dtl_last, 3 * ns * sizeof(unsigned long long))) != cudaSuccess ||
            (e = cudaMemset(h->dtl_first, 0xFF, ns * sizeof(unsigned long long))) != cudaSuccess ||
            (e = cudaMemset(h->dtl_last, 0, 3 * ns * sizeof(unsigned long long))) != cudaSuccess ||
            (e = cudaMalloc((void**)&h->dscan_counts, 2 * sizeof(unsigned long long))) != cudaSuccess ||
            (e = cudaMemset(h->dscan_counts, 0, 2 * sizeof(unsigned long long))) != cudaSuccess) {
            if (h->dtl_first) cudaFree(h->dtl_first);
            if (h->dtl_last) cudaFree(h->dtl_last);
            if (h->dscan_counts) cudaFree(h->dscan_counts);
            h->dtl_first = nullptr;
            h->dtl_last = nullptr;
            h->dscan_counts = nullptr;
            return e == cudaErrorMemoryAllocation ? SINV_ERR_OOM : cuda_fail(h, e, "timeline");
        }
    }
    if (!enable && h->dtl_first) {
        cudaFree(h->dtl_first);
        cudaFree(h->dtl_last);
        cudaFree(h->dscan_counts);
        h->dtl_first = nullptr;
        h->dtl_last = nullptr;
        h->dscan_counts = nullptr;
    }
    return SINV_OK;
}

sinv_status sinv_selinv_scan_counts(sinv_handle h, int64_t* lookups, int64_t* pairs, void* stream) {
    if (!h || !lookups || !pairs) return SINV_ERR_INVALID_ARG;
    *lookups = 0;
    *pairs = 0;
    if (!on_device(h)) return SINV_ERR_INVALID_ARG;
    if (!h->dscan_counts) return SINV_OK;
    cudaError_t e = cudaSetDevice(h->device);
    unsigned long long c[2] = {0, 0};
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemcpy(c, h->dscan_counts, sizeof(c), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "scan counters");
    *lookups = (int64_t)c[0];
    *pairs = (int64_t)c[1];
    return SINV_OK;
}

sinv_status sinv_timeline_read(sinv_handle h, uint64_t* stamps, int64_t n_supernodes, void* stream) {
    if (!h || !stamps || n_supernodes != (int64_t)h->P.sn.size()) return SINV_ERR_INVALID_ARG;
    if (!h->dtl_first) {
        set_err(h, "the timeline is not enabled");
        return SINV_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    std::vector<unsigned long long> f(n_supernodes), l(3 * n_supernodes);
    if (e == cudaSuccess && n_supernodes > 0)
        e = cudaMemcpy(f.data(), h->dtl_first, f.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && n_supernodes > 0)
        e = cudaMemcpy(l.data(), h->dtl_last, l.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "timeline read");
    for (int64_t J = 0; J < n_supernodes; ++J) {
        stamps[4 * J] = f[J];
        for (int k = 0; k < 3; ++k) stamps[4 * J + 1 + k] = l[3 * J + k];
    }
    return SINV_OK;
}

void sinv_destroy(sinv_handle h) {
    if (!h) return;
    if (h->device >= 0) {
        cudaSetDevice(h->device);
        delete h->tracer;
        h->tracer = nullptr;
        free_all(h);
    }
    delete h;
}

}  // extern "C"
