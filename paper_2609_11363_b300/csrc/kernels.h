// Launch interfaces of the device kernels (internal to libsinv).
#pragma once
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "device.cuh"
#include "plan.h"

namespace sinv {

// Optional per-kernel event timing.  The API installs a tracer for the duration
// of a numeric call when tracing is enabled on the handle; launch sites bracket
// every kernel with these two calls (no-ops otherwise).
void trace_begin(const char* name, cudaStream_t st);
void trace_end(cudaStream_t st);

struct SelinvArgs {
    const SnInfo* sn;
    const int32_t* order;
    const WorkItem* items;
    int32_t nitems;
    int32_t nsn;
    int32_t n;
    const int32_t* owner;
    const int32_t* Crow;
    const int32_t* Lmap;
    const int32_t* JJl;
    const int32_t* JJs;
    const uint32_t* hit_ik;
    const int32_t* hit_pos;
    const int32_t* hrow;
    const int32_t* Sdiag;
    const int32_t* l2s;
    const int32_t* dpos;
    const int8_t* pstart;
    const double* Lval;
    const double* Dval;
    uint32_t* done;
    const uint32_t* epoch;  // device word, bumped by selinv_prepare before each launch
    int32_t* ticket;
    int32_t* status;
    int64_t wait_limit;
    double* scratch;
    int64_t max_cw;
    int64_t nnzS;
    int32_t num_sms;
    const int64_t* xsum_off;  // per supernode: its partial-sum block when split over CTAs, else -1
    double* xsum;             // the blocks (zeroed before every launch)
    uint32_t* arrive;         // per supernode: parts arrived in this call (zeroed before every launch)
    int32_t item0;            // first work item of this launch (the tensor-core tier runs the ones before)
    Timeline tl;              // per-supernode stamps, or nulls
    // scan form (no pair lists): S_lo rows, per-group hash tables of C for groups whose
    // C exceeds shared memory (2 x gtab_slots int32 per group slot: keys, then local
    // indices), and, when not null, the call's lookups and pairs found (2 counters)
    int32_t scan;
    const int64_t* Srp;
    const int32_t* Sc;
    int32_t* gtab;
    int64_t gtab_slots;
    unsigned long long* counts;
};

// The tensor-core tier of SelInv (selinv_tc.cu): items over (supernode, row tile,
// part of C) of the leading levels whose C is contiguous.
struct TcArgs {
    const int32_t* tcmap;  // per supernode tc_c x w: CSR position of L(R[o], s0+t) or -1
    const int32_t* deps;   // per supernode: the distinct supernodes owning rows of C
    const WorkItem* items;
    int32_t nitems;
    int32_t* ticket;
    double* mirror;      // symmetric band copy of G for rows [row0, n), zeroed before every call
    int64_t row0, band, width;
    uint32_t* arrive_t;  // per row tile: parts arrived (zeroed)
    double* zacc;        // per supernode w x w: Z summed over the tiles (zeroed)
};
cudaError_t selinv_tc_configure();
// fmt: 2 = TF32, 1 = BF16 (the tcgen05 input type of the split operands)
cudaError_t selinv_tc_launch(const SelinvArgs& a, const TcArgs& t, int fmt, double* G, cudaStream_t st);

cudaError_t selinv_configure();
// epoch += 1 (skipping 0) and ticket = 0 (and ticket2 = 0 if given), in stream order:
// keeps the launch graph-capturable
cudaError_t selinv_prepare(uint32_t* epoch, int32_t* ticket, cudaStream_t st, int32_t* ticket2 = nullptr);
int selinv_grid(int num_sms, bool scan);
int selinv_scan_table_smem();  // hash slots of C per warp in shared memory (scan form)
int selinv_max_width();
int selinv_cw_smem();
int selinv_warps_per_cta();
// prec: 0 = FP64 (writes G_out directly), 1 = FP32 (working copy in `work`, |S_lo| floats)
cudaError_t selinv_launch(const SelinvArgs& a, int prec, void* work, double* G_out, cudaStream_t st, int grid);

cudaError_t mix_launch(const double* G, const double* N, double eps, double* M, int64_t nnz, int num_sms,
                       cudaStream_t st);

// per-matrix device pointers of one batched copy launch (a kernel argument)
constexpr int kBatchPtrs = 256;
struct BatchPtrs {
    const double* p[kBatchPtrs];
};
// to_cat = 1: every matrix's buffer into its range [off[b], off[b+1]) of cat; 0: back.
// A null pointer skips its matrix.  d_off: nmat+1 offsets on the device.
cudaError_t batch_copy_launch(int32_t nmat, const double* const* ptrs, const int64_t* d_off, int to_cat, double* cat,
                              int num_sms, cudaStream_t st);

// X_S += sum_l lambda_l V_il V_jl on S_lo.  prec 0: FP64; 1: FP32 products (V converted
// once into `work`, n*k floats), FP64 accumulation into X.
cudaError_t lowrank_launch(int64_t n, const int64_t* Srp, const int32_t* Sc, int k, const double* V,
                           const double* lambda, int prec, void* work, double* X, int num_sms,
                           cudaStream_t st);

struct NinvArgs {
    int64_t n;
    int m;
    const int64_t* Lcp;   // E by columns (struct(j)), CSR positions of L values
    const int32_t* Lri;
    const int32_t* Lcsr;
    const int64_t* Wcp;   // P_W by columns, grouped by first power
    const int32_t* Wr;
    const int32_t* grp;
    const int64_t* Srp;   // S_lo
    const int32_t* Sc;
    const int64_t* Lrp;   // L row pointers (CSR of the caller's L)
    int64_t nnzS;
    int64_t nnzW;
    int64_t nnzL;
    double delta;         // after every Horner step, off-diagonal |w| < delta is set to 0 (0: keep all)
    const int32_t* dpos;
    const int8_t* pstart;
    const double* Lval;
    const double* Dval;
    int64_t max_col;
    int32_t num_sms;
    int32_t* status;
};
constexpr int kIdxEnt = 5440;       // longest short column of P_W (with its partner rows)
constexpr int kIdxEntLong = 16384;  // longest column the maps handle (large shared tables)
// Map form of NInv (ninv_map.cu): per-entry positions resolved once per pattern and m.
struct NinvMaps {
    bool ready = false;
    int m = -1;
    int64_t nmap_h = 0, nmap_p = 0, bytes = 0;
    int64_t hits = 0;           // map entries with y nonzero (multiply-adds of the product)
    int64_t* moff = nullptr;    // nnz_L+1: start of the Horner map of every entry of E (CSC order)
    uint16_t* hmap = nullptr;   // position in column j of each row of column k (powers <= m-1)
    int64_t* poff = nullptr;    // |S_lo|+1: start of the product map of every entry of S_lo
    uint16_t* pmap = nullptr;   // y-table position of each row of column i (0xFFFF: y is zero)
    uint16_t* ypart = nullptr;  // nnz_W: y-table position of the partner row (2x2 rows only)
    int32_t* ynx = nullptr;     // n: extra y-table positions (partner rows outside the column)
    int32_t* cols = nullptr;    // n: the short columns, then the long ones
    int64_t n_short = 0, n_long = 0;
};
cudaError_t ninv_maps_configure();
std::string ninv_maps_build(const NinvArgs& a, const HostPlan& P, const NinvPlan& W, int64_t budget,
                            NinvMaps& x, cudaStream_t st, cudaError_t& err);
void ninv_maps_free(NinvMaps& x);
size_t ninv_map_work_bytes(const NinvArgs& a, int prec);
cudaError_t ninv_map_launch(const NinvArgs& a, const NinvMaps& x, int prec, void* work, double* N_out,
                            cudaStream_t st, double* N_stack = nullptr);
// NInv on its own pattern (ninv_own.cu)
struct OwnArgs {
    int64_t n;
    int num_sms;
    int grid;             // CTAs of the column kernels
    const int64_t* Lcp;   // E by columns: rows and CSR positions of the L values
    const int32_t* Lri;
    const int32_t* Lcsr;
    const double* Lval;
    double delta;
    const double* dr;     // D^{-1} by rows: diagonal, partner coefficient, partner
    const double* dp;
    const int32_t* part;
    int32_t* gkeys;       // per-CTA hash tables in global memory for long columns
    double* gvals;
    int64_t gslice;       // slots per CTA
    int32_t* ticket;
    unsigned long long* cursor;  // append position of the current kernel's output
};
// W columns as segments: column j = entries [st[j], st[j] + ct[j]) of (r, v)
cudaError_t own_identity_launch(int64_t n, int64_t* st, int64_t* ct, int32_t* r, double* v, int num_sms,
                                cudaStream_t s);
cudaError_t own_bound_launch(int64_t n, const int64_t* Lcp, const int32_t* Lri, const int64_t* ctIn, int64_t* maxb,
                             int num_sms, cudaStream_t s);
cudaError_t own_max_launch(int64_t n, const int64_t* x, int64_t* out, int num_sms, cudaStream_t s);
cudaError_t own_horner_launch(const OwnArgs& a, const int64_t* stIn, const int64_t* ctIn, const int32_t* rIn,
                              const double* vIn, int32_t* rOut, double* vOut, int64_t* stOut, int64_t* ctOut,
                              int64_t cap, cudaStream_t s);
cudaError_t own_scan_launch(int64_t n, const int64_t* cnt, int64_t* out, cudaStream_t s);
cudaError_t own_compact_launch(int64_t n, const int64_t* off, const int64_t* cp, const int32_t* rs, const double* vs,
                               int32_t* rd, double* vd, int num_sms, cudaStream_t s);
cudaError_t own_transpose_launch(int64_t n, int64_t nnz, const int64_t* st, const int64_t* ct, const int32_t* r,
                                 const double* v, int64_t* rowcnt, int64_t* rp, int64_t* fill, int32_t* rc,
                                 double* rv, int num_sms, cudaStream_t s);
cudaError_t own_diag_launch(const OwnArgs& a, const int64_t* st, const int64_t* ct, const int32_t* r, const double* v,
                            const int64_t* rp, double* diag, int64_t* bound, int64_t* maxb, cudaStream_t s);
cudaError_t own_product_launch(const OwnArgs& a, const int64_t* st, const int64_t* ct, const int32_t* r,
                               const double* v, const int64_t* rp, const int32_t* rc, const double* rv,
                               const double* diag, const int64_t* bound, int32_t* nr, double* nv, int64_t* stN,
                               int64_t* ctN, int64_t cap, cudaStream_t s);
// Mix on the own pattern: N (CSC of the lower triangle) and S_lo with L by columns
struct MixOwnArgs {
    int64_t n;
    int grid;
    const int64_t* Ncp;
    const int32_t* Nr;
    const double* Nv;
    const int64_t* Srp;
    const int32_t* Sdiag;
    const int64_t* Lcp;
    const int32_t* Lri;
    const int32_t* Lcsr;
    const int32_t* l2s;
    const int8_t* pstart;
    const double* G;
    double eps;
    int32_t* gkeys;  // per CTA: gslice keys then gslice positions, for columns beyond shared memory
    int64_t gslice;
    int32_t* ticket;
};
// fill = false: counts of every result column into cnt_or_cp; fill = true: the
// columns at the offsets cnt_or_cp (the scan of the counts)
cudaError_t mix_own_launch(const MixOwnArgs& a, bool fill, int64_t* cnt_or_cp, int32_t* outR, double* outV,
                           cudaStream_t s);
cudaError_t own_max_col_launch(int64_t n, const int64_t* cp, int64_t* out, int num_sms, cudaStream_t s);
int own_table_slots(int64_t entries);
int own_smem_slots();
int own_horner_slots();
int own_prod_slots();
cudaError_t own_configure();
int own_grid_ctas(int num_sms);

// D^{-1} per row (ninv.cu): diagonal, off-diagonal of its 2x2 block, partner row (-1: 1x1)
void ninv_dinv_launch(const NinvArgs& a, double* dr, double* dp, int32_t* part, cudaStream_t st);

cudaError_t ninv_configure();
size_t ninv_work_bytes(const NinvArgs& a, int prec);
// N_stack (optional): (m+1) x |S_lo| products of the truncations after 0..m steps;
// then N_out is not written (the last slice holds the full NInv)
cudaError_t ninv_launch(const NinvArgs& a, int prec, void* work, double* N_out, cudaStream_t st,
                        double* N_stack = nullptr);

// Largest rank k of the low-rank correction: lowrank_kernel stages lambda .* V_i
// in a shared row of this many values per warp.
constexpr int kLowrankKMax = 256;

// FP32 low-rank correction with its working copy in a file-scope device array
// (no allocation); k <= kLowrankKMax and n*k + k <= kLowrankStaticFloats.
constexpr int64_t kLowrankStaticFloats = int64_t(1) << 22;  // 4,194,304 floats = 16 MiB
cudaError_t lowrank_noalloc_launch(int64_t n, const int64_t* Srp, const int32_t* Sc, int k, const double* V,
                                   const double* lambda, double* X, cudaStream_t st);

// ---- SPAI refinement (spai.cu) ----
constexpr int kSpaiWarpJ = 128;   // tier W: rows of the column
constexpr int kSpaiWarpE = 704;   // tier W: staged entries of A (4 warps' columns fit twice per SM)
constexpr int kSpaiWarpH = 512;   // tier W: table slots (a tier-W column has at most kSpaiWarpH/2 rows of A)
struct SpaiArgs {
    const int64_t* fcp;   // columns of P (both triangles)
    const int32_t* fri;
    const int32_t* fpos;  // P_lo position of each entry
    const int32_t* fsrc;  // S_lo position of each entry (-1: not in S)
    const int32_t* feo;   // entry offset of each row inside its column's list
    const int32_t* fE;    // entries per column
    const int32_t* fR;    // distinct rows of A per column
    const int64_t* Arp;   // A (symmetric), CSR
    const int32_t* Acol;
    const double* Aval;
    const double* X;      // start values on S_lo
    double* Y;            // result on P_lo (zeroed by the launcher)
    int64_t nnzP;
    int iters;
    const int32_t* cols;      // tier W columns
    int64_t ncols;
    const int32_t* cols_cta;  // tier C columns
    int64_t ncols_cta;
    int32_t* ticket;          // 2 counters, zeroed by the launcher
    double* scratch;          // tier C: one block of cta_bytes per CTA (unused when it fits shared memory)
    int64_t cta_bytes;
    int cta_in_smem;          // tier C arrays in dynamic shared memory
    int64_t cap_nj, cap_E, cap_H;
    int32_t* status;
};
cudaError_t spai_configure();
size_t spai_cta_bytes(int64_t cap_nj, int64_t cap_E, int64_t cap_H);
constexpr size_t kSpaiCtaSmemMax = 200 * 1024;  // tier C blocks up to this size live in shared memory
int spai_cta_grid(int num_sms, int64_t ncols_cta, size_t cta_bytes);
cudaError_t spai_launch(const SpaiArgs& a, int num_sms, cudaStream_t st);

// ---- spectral-correction producer (einv.cu) ----
struct EinvArgs {
    int64_t n;
    int num_sms;
    const int64_t* Arp;   // A (symmetric), CSR
    const int32_t* Acol;
    const double* Aval;
    const int64_t* fcp;   // columns of S and the S_lo position of each entry
    const int32_t* fri;
    const int32_t* fpos;
    const double* X;      // A^inv on S_lo
    const int64_t* Lrp;   // L by rows
    const int32_t* Lcol;
    const int64_t* Lcp;   // L by columns, with the CSR position of each entry
    const int32_t* Lri;
    const int32_t* Lcsr;
    const double* Lval;
    const double* dr;     // D^{-1} per row: diagonal, partner coefficient, partner (-1: 1x1)
    const double* dp;
    const int32_t* part;
    const int32_t* fwd_rows;  // rows of L y = b in level order (device)
    const int32_t* bwd_cols;  // columns of L^T x = w in level order
    const int32_t* fwd_ptr;   // level starts in fwd_rows / bwd_cols (nlev + 1 each)
    const int32_t* bwd_ptr;
    int32_t nlev_fwd, nlev_bwd;
    int32_t cta_solve;        // 1: one CTA walks the levels (few rows per level), 0: persistent grid
    // persistent solves: per-row flags of each solve, their epoch, two tickets
    uint32_t* fwd_flags;
    uint32_t* bwd_flags;
    uint32_t* tepoch;
    int32_t* tickets;
    int32_t* status;
    int64_t wait_limit;
};
constexpr int kEinvMaxSteps = 256;  // Lanczos steps (the tridiagonal eigenproblem runs in one CTA)
int einv_dot_blocks(int num_sms);
cudaError_t einv_spmv_A(const EinvArgs& a, const double* x, double* y, cudaStream_t st);
cudaError_t einv_symv_X(const EinvArgs& a, const double* x, double* y, cudaStream_t st);
// z = L^{-T} D^{-1} L^{-1} r in three launches: y = L^{-1} r, then z = L^{-T} (D^{-1} y), each
// one persistent launch over all dependency levels (D^{-1}: the dr / dp / part rows given)
cudaError_t einv_precond_persistent(const EinvArgs& a, const double* r, double* y, double* z, cudaStream_t st);
// |D|^{-1} per row (diagonal, partner coefficient, partner) from D: the SPD preconditioner
// L |D| L^T of MINRES
cudaError_t einv_absdinv(const EinvArgs& a, const int32_t* dpos, const int8_t* pstart, const double* Dval, double* dr,
                         double* dp, int32_t* part, cudaStream_t st);
cudaError_t einv_dot(const EinvArgs& a, const double* x, const double* y, double* partial, double* out,
                     cudaStream_t st);
cudaError_t einv_cg_xr(const EinvArgs& a, double alpha, const double* p, const double* q, double* x, double* r,
                       cudaStream_t st);
cudaError_t einv_cg_p(const EinvArgs& a, double beta, const double* z, double* p, cudaStream_t st);
cudaError_t einv_axpby(const EinvArgs& a, double alpha, const double* x, double beta, const double* y, double* out,
                       cudaStream_t st);
// v -= Q[:, :ncols] (Q[:, :ncols]^T v)   (c: ncols work scalars)
cudaError_t einv_reorth(const EinvArgs& a, const double* Q, int ncols, double* c, double* v, cudaStream_t st);
// eigen-decomposition of the m x m symmetric T (overwritten), eigenvectors in U; the k
// eigenvalues of largest modulus and their columns into lam / sel
cudaError_t einv_eig(int m, double* T, double* U, int k, int32_t* sel, double* lam, cudaStream_t st);
cudaError_t einv_ritz(const EinvArgs& a, int m, int k, int ldv, const double* Q, const double* U,
                      const int32_t* sel, double* V, cudaStream_t st);

cudaError_t debug_wait_launch(uint32_t* flag, int32_t* status, int64_t limit, cudaStream_t st);

// ---- learned correction (mlp.cu) ----
constexpr int kMlpF = 16;  // features per entry (zero padded)
constexpr int kMlpH = 64;  // hidden width
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpF * kMlpH;
constexpr int kOffW2 = kOffB1 + kMlpH;
constexpr int kOffB2 = kOffW2 + kMlpH * kMlpH;
constexpr int kOffW3 = kOffB2 + kMlpH;
constexpr int kOffB3 = kOffW3 + kMlpH;
constexpr int kMlpParams = kOffB3 + 1;
// polls of a tensor-core completion wait before the kernel records SINV_ERR_TIMEOUT
constexpr int64_t kMlpWaitLimit = int64_t(1) << 24;
cudaError_t mlp_configure();
int mlp_train_blocks(int64_t count);
cudaError_t mlp_features_launch(int64_t n, const int64_t* Srp, const int32_t* Sc, const int64_t* Lrp,
                                const int64_t* Lcp, int m, const double* Nst, int64_t nnzS, const double* Lval,
                                const double* Dval, const int32_t* dpos, const int8_t* pstart, void* X, float* scale,
                                int num_sms, cudaStream_t st);
cudaError_t mlp_targets_launch(int64_t count, const double* G, const double* N, const float* scale, float* y,
                               int num_sms, cudaStream_t st);
cudaError_t mlp_grad_launch(const void* X, const float* y, const int64_t* idx, int64_t count, const float* theta,
                            float* partial, float* loss_partial, float* grad, float* loss, cudaStream_t st);
cudaError_t mlp_adam_launch(float* theta, float* m, float* v, const float* g, float lr, int step, cudaStream_t st);
cudaError_t mlp_predict_launch(const void* X, const float* scale, const double* N, int64_t count, const float* theta,
                               double* out, int32_t* status, int64_t wait_limit, int num_sms, cudaStream_t st);

}  // namespace sinv
