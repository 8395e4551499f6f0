// Host symbolic analysis: validation of L's pattern and the pivot layout, the
// pattern S (Section 1), pivot blocks, supernodes of the block elimination tree
// (Section 2.1, Fig. 2), dependency levels and the index maps of the numeric
// kernels.  Everything here is integer work and is deterministic.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>

#include "plan.h"

namespace sinv {

namespace {

int n_threads() {
    unsigned h = std::thread::hardware_concurrency();
    return h == 0 ? 4 : (int)std::min(h, 32u);
}

template <class F>
void parallel_for(int64_t count, F f) {
    int T = n_threads();
    if (count < 4096 || T == 1) {
        f(0, count);
        return;
    }
    std::vector<std::thread> th;
    int64_t chunk = (count + T - 1) / T;
    for (int t = 0; t < T; ++t) {
        int64_t a = t * chunk, b = std::min(count, a + chunk);
        if (a >= b) break;
        th.emplace_back([=, &f] { f(a, b); });
    }
    for (auto& x : th) x.join();
}

// The same, with items handed out in chunks of `grain` from a shared counter: for
// loops whose per-item cost varies a lot (supernodes near the root of the tree are
// the largest).  Each item must write only its own outputs.
template <class F>
void parallel_for_dynamic(int64_t count, int64_t grain, F f) {
    int T = n_threads();
    if (count < 4096 || T == 1) {
        f(0, count);
        return;
    }
    std::atomic<int64_t> next(0);
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t)
        th.emplace_back([&] {
            for (;;) {
                const int64_t a = next.fetch_add(grain);
                if (a >= count) break;
                f(a, std::min(count, a + grain));
            }
        });
    for (auto& x : th) x.join();
}

// f(t) for every t in [0, T), one thread each
template <class F>
void run_chunks(int T, F f) {
    if (T <= 1) {
        f(0);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t) th.emplace_back([=, &f] { f(t); });
    for (auto& x : th) x.join();
}

// CSR (rows 0..n-1, columns < n) to CSC, with every column's rows in increasing
// order and the CSR position of each entry: the rows are cut into T chunks of about
// equal entries; each chunk counts its entries per column, the counts become start
// positions ordered by (column, chunk), and each chunk places its own entries.  The
// result is the one a serial counting sort gives.
template <class IdxVec>
void csr_to_csc(int64_t n, const int64_t* rp, const int32_t* col, std::vector<int64_t>& cp, IdxVec& ri,
                IdxVec& pos) {
    const int64_t nnz = rp[n];
    cp.assign(n + 1, 0);
    ri.resize(nnz);
    pos.resize(nnz);
    int T = (int)std::min<int64_t>(n_threads(), std::max<int64_t>(1, nnz >> 20));
    if ((int64_t)T * n > (int64_t(1) << 30)) T = 1;  // the per-chunk counts must stay small
    std::vector<int64_t> rb(T + 1);
    for (int t = 0; t <= T; ++t)  // first row of chunk t: the first row starting at or past t nnz / T
        rb[t] = t == T ? n : std::lower_bound(rp, rp + n, (int64_t)((__int128)nnz * t / T)) - rp;
    std::vector<int64_t> start((size_t)T * n, 0);  // entries of chunk t in column j, then their start
    run_chunks(T, [&](int t) {
        int64_t* c = start.data() + (size_t)t * n;
        for (int64_t q = rp[rb[t]]; q < rp[rb[t + 1]]; ++q) c[col[q]]++;
    });
    parallel_for(n, [&](int64_t a, int64_t b) {
        for (int64_t j = a; j < b; ++j) {
            int64_t tot = 0;
            for (int t = 0; t < T; ++t) tot += start[(size_t)t * n + j];
            cp[j + 1] = tot;
        }
    });
    for (int64_t j = 0; j < n; ++j) cp[j + 1] += cp[j];
    parallel_for(n, [&](int64_t a, int64_t b) {
        for (int64_t j = a; j < b; ++j) {
            int64_t run = cp[j];
            for (int t = 0; t < T; ++t) {
                const int64_t c = start[(size_t)t * n + j];
                start[(size_t)t * n + j] = run;
                run += c;
            }
        }
    });
    run_chunks(T, [&](int t) {
        int64_t* c = start.data() + (size_t)t * n;
        for (int64_t i = rb[t]; i < rb[t + 1]; ++i)
            for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
                const int64_t d = c[col[q]]++;
                ri[d] = (int32_t)i;
                pos[d] = (int32_t)q;
            }
    });
}

// is sorted list a (minus the values in [ex0, ex1)) a subset of sorted list b?
bool subset_except(const int32_t* a, int64_t na, const int32_t* b, int64_t nb, int32_t ex0, int32_t ex1) {
    int64_t j = 0;
    for (int64_t i = 0; i < na; ++i) {
        int32_t v = a[i];
        if (v >= ex0 && v < ex1) continue;
        while (j < nb && b[j] < v) ++j;
        if (j == nb || b[j] != v) return false;
    }
    return true;
}

}  // namespace

std::string build_plan(int64_t n, const int64_t* Lrp, const int32_t* Lc, const int8_t* ps, int cap,
                       int64_t big_pairs, int group, int64_t thin_level, HostPlan& P, int64_t pair_bytes) {
    if (n < 0) return "negative n";
    if (n > INT32_MAX - 1) return "n does not fit int32 column indices";
    if (cap <= 0) cap = 16;
    if (cap > 64) cap = 64;
    P = HostPlan();
    P.n = n;
    if (n == 0) {
        P.Srp.assign(1, 0);
        P.sn_start.assign(1, 0);
        P.Lcp.assign(1, 0);
        return "";
    }
    if (Lrp[0] != 0) return "L_rowptr[0] != 0";
    for (int64_t i = 0; i < n; ++i)
        if (Lrp[i + 1] < Lrp[i]) return "L_rowptr not nondecreasing at row " + std::to_string(i);
    int64_t nnzL = Lrp[n];
    P.nnzL = nnzL;
    if (nnzL > INT32_MAX) return "nnz(L) >= 2^31 not supported";
    // rows are checked in parallel for the first bad one, whose message comes from
    // the same check in row order
    auto row_ok = [&](int64_t i) {
        for (int64_t q = Lrp[i]; q < Lrp[i + 1]; ++q) {
            const int32_t c = Lc[q];
            if (c < 0 || c >= i || (q > Lrp[i] && Lc[q - 1] >= c)) return false;
        }
        return true;
    };
    std::atomic<int64_t> first_bad(n);
    parallel_for(n, [&](int64_t a, int64_t b) {
        for (int64_t i = a; i < b; ++i)
            if (!row_ok(i)) {
                int64_t cur = first_bad.load();
                while (i < cur && !first_bad.compare_exchange_weak(cur, i)) {
                }
                return;
            }
    });
    for (int64_t i = first_bad.load(); i < n; ++i) {
        for (int64_t q = Lrp[i]; q < Lrp[i + 1]; ++q) {
            int32_t c = Lc[q];
            if (c < 0 || c >= i) return "L entry out of the strictly lower triangle at row " + std::to_string(i);
            if (q > Lrp[i] && Lc[q - 1] >= c) return "L row " + std::to_string(i) + " not strictly increasing";
        }
    }
    // pivot layout
    P.pstart.assign(ps, ps + n);
    for (int64_t j = 0; j < n; ++j) {
        if (ps[j] != 0 && ps[j] != 1) return "pivot_start values must be 0 or 1";
    }
    if (ps[0] != 1) return "pivot_start[0] must be 1";
    for (int64_t j = 1; j < n; ++j) {
        if (ps[j] == 0) {
            if (ps[j - 1] == 0) return "pivot block larger than 2x2 at column " + std::to_string(j);
            // L(j, j-1) must not be stored: last entry of row j is < j-1
            if (Lrp[j + 1] > Lrp[j] && Lc[Lrp[j + 1] - 1] == j - 1)
                return "L(j, j-1) stored inside a 2x2 pivot block at row " + std::to_string(j);
        }
    }
    P.dpos.resize(n);
    {
        int64_t off = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (ps[j]) {
                P.n_blocks++;
                bool two = (j + 1 < n) && ps[j + 1] == 0;
                P.dpos[j] = (int32_t)off;
                if (two) {
                    P.dpos[j + 1] = (int32_t)off;
                    P.n_2x2++;
                    off += 3;
                } else {
                    off += 1;
                }
            }
        }
        P.nD = off;
    }
    // S_lo: row i = L row i, then (i-1) for the second column of a 2x2 block, then i
    P.Srp.resize(n + 1);
    P.Srp[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t len = (Lrp[i + 1] - Lrp[i]) + 1 + ((i > 0 && ps[i] == 0) ? 1 : 0);
        P.Srp[i + 1] = P.Srp[i] + len;
    }
    P.nnzS = P.Srp[n];
    if (P.nnzS > INT32_MAX) return "|S_lo| >= 2^31 not supported";
    P.Sc.resize(P.nnzS);
    P.Sdiag.resize(n);
    P.l2s.resize(nnzL);
    parallel_for(n, [&](int64_t a, int64_t b) {
        for (int64_t i = a; i < b; ++i) {
            int64_t s = P.Srp[i];
            for (int64_t q = Lrp[i]; q < Lrp[i + 1]; ++q) {
                P.l2s[q] = (int32_t)s;
                P.Sc[s++] = Lc[q];
            }
            if (i > 0 && ps[i] == 0) P.Sc[s++] = (int32_t)(i - 1);
            P.Sdiag[i] = (int32_t)s;
            P.Sc[s++] = (int32_t)i;
        }
    });
    // L by columns
    csr_to_csc(n, Lrp, Lc, P.Lcp, P.Lri, P.Lcsr);
    const int64_t* Lcp = P.Lcp.data();
    const int32_t* Lri = P.Lri.data();

    // pivot blocks and their row unions U_P (rows below the block)
    std::vector<int32_t> bstart;
    for (int64_t j = 0; j < n; ++j)
        if (ps[j]) bstart.push_back((int32_t)j);
    int64_t nb = (int64_t)bstart.size();
    bstart.push_back((int32_t)n);
    auto block_union = [&](int64_t b, std::vector<int32_t>& U) {
        U.clear();
        int32_t c0 = bstart[b], c1 = bstart[b + 1];
        for (int32_t c = c0; c < c1; ++c)
            for (int64_t q = Lcp[c]; q < Lcp[c + 1]; ++q)
                if (Lri[q] >= c1) U.push_back(Lri[q]);
        std::sort(U.begin(), U.end());
        U.erase(std::unique(U.begin(), U.end()), U.end());
    };
    // merge rule between consecutive blocks b and b+1 (b+1 joins b's supernode):
    //  (a) the first column of block b+1 is in U_b (block b+1 is b's parent)
    //  (b) U_b minus block b+1 is contained in struct(c) for every column c of block b+1
    //  (c) the supernode stays within the width cap
    // Under (b) for every consecutive pair, every pair of rows (a, r) that a block of
    // the supernode reads from a later column a of the same supernode is in S, so the
    // dense supernodal step equals the scalar recurrence in exact arithmetic.
    std::vector<char> joins(nb, 0);
    parallel_for(nb - 1, [&](int64_t a, int64_t b) {
        std::vector<int32_t> U;
        for (int64_t q = a; q < b; ++q) {
            block_union(q, U);
            int32_t n0 = bstart[q + 1], n1 = bstart[q + 2];
            if (U.empty() || U[0] != n0) continue;
            bool ok = true;
            for (int32_t c = n0; c < n1 && ok; ++c)
                ok = subset_except(U.data(), (int64_t)U.size(), Lri + Lcp[c], Lcp[c + 1] - Lcp[c], n0, n1);
            joins[q] = ok;
        }
    });
    P.sn_start.clear();
    {
        int64_t b = 0;
        while (b < nb) {
            int32_t s0 = bstart[b];
            int64_t e = b + 1;
            while (e < nb && joins[e - 1] && (bstart[e + 1] - s0) <= cap) ++e;
            P.sn_start.push_back(s0);
            b = e;
        }
        P.sn_start.push_back((int32_t)n);
    }
    int64_t ns = (int64_t)P.sn_start.size() - 1;
    P.owner.resize(n);
    for (int64_t s = 0; s < ns; ++s)
        for (int32_t c = P.sn_start[s]; c < P.sn_start[s + 1]; ++c) P.owner[c] = (int32_t)s;
    // C_J per supernode
    P.sn.resize(ns);
    std::vector<std::vector<int32_t>> Cs(ns);
    parallel_for(ns, [&](int64_t a, int64_t b) {
        for (int64_t s = a; s < b; ++s) {
            int32_t s0 = P.sn_start[s], s1 = P.sn_start[s + 1];
            auto& C = Cs[s];
            for (int32_t c = s0; c < s1; ++c)
                for (int64_t q = Lcp[c]; q < Lcp[c + 1]; ++q)
                    if (Lri[q] >= s1) C.push_back(Lri[q]);
            std::sort(C.begin(), C.end());
            C.erase(std::unique(C.begin(), C.end()), C.end());
        }
    });
    // levels: 0 if C empty, else 1 + max level of the supernodes owning rows of C
    P.sn_level.assign(ns, 0);
    for (int64_t s = ns - 1; s >= 0; --s) {
        int32_t lv = -1;
        for (int32_t r : Cs[s]) lv = std::max(lv, P.sn_level[P.owner[r]]);
        P.sn_level[s] = lv + 1;
    }
    int32_t maxlev = 0;
    for (int64_t s = 0; s < ns; ++s) maxlev = std::max(maxlev, P.sn_level[s]);
    P.n_levels = ns ? maxlev + 1 : 0;
    // offsets
    int64_t crow = 0, cw = 0, ww = 0;
    for (int64_t s = 0; s < ns; ++s) {
        SnInfo& I = P.sn[s];
        I.s0 = P.sn_start[s];
        I.w = P.sn_start[s + 1] - P.sn_start[s];
        I.c = (int32_t)Cs[s].size();
        I.level = P.sn_level[s];
        if (I.c > 65535) return "a supernode touches more than 65535 rows: unsupported";
        I.crow_off = crow; crow += I.c;
        I.cw_off = cw; cw += (int64_t)I.c * I.w;
        I.ww_off = ww; ww += (int64_t)I.w * I.w;
        P.max_c = std::max<int64_t>(P.max_c, I.c);
        P.max_w = std::max<int64_t>(P.max_w, I.w);
        P.max_cw = std::max<int64_t>(P.max_cw, (int64_t)I.c * I.w);
    }
    P.Crow.resize(crow);
    P.Lmap.assign(cw, -1);
    P.JJl.assign(ww, -1);
    P.JJs.assign(ww, -1);
    // pairs of C x C in S, both triangles and the diagonal, sorted by (i, k):
    //   k < i : (C[i], C[k]) in row C[i] of S_lo            (merge with C[0..i))
    //   k = i : the diagonal of C[i]
    //   k > i : (C[k], C[i]) with C[k] in struct(C[i]) or the 2x2 partner of C[i]
    std::vector<int64_t> hits(ns, 0);
    auto pairs = [&](int64_t s, bool fill, uint32_t* ik, int32_t* pos, int32_t* hrow) {
        const auto& C = Cs[s];
        const int64_t c = (int64_t)C.size();
        int64_t cnt = 0;
        for (int64_t i = 0; i < c; ++i) {
            if (fill) hrow[i] = (int32_t)cnt;
            const int32_t r = C[i];
            // lower part
            int64_t q = P.Srp[r], qe = P.Srp[r + 1] - 1;  // exclude the diagonal
            int64_t k = 0;
            while (q < qe && k < i) {
                int32_t a = P.Sc[q], b = C[k];
                if (a == b) {
                    if (fill) { ik[cnt] = ((uint32_t)i << 16) | (uint32_t)k; pos[cnt] = (int32_t)q; }
                    ++cnt; ++q; ++k;
                } else if (a < b) {
                    ++q;
                } else {
                    ++k;
                }
            }
            // diagonal
            if (fill) { ik[cnt] = ((uint32_t)i << 16) | (uint32_t)i; pos[cnt] = P.Sdiag[r]; }
            ++cnt;
            // upper part: column r of S below the diagonal
            const bool two_first = ps[r] != 0 && r + 1 < n && ps[r + 1] == 0;
            int64_t qq = Lcp[r], qqe = Lcp[r + 1];
            k = i + 1;
            bool partner_pending = two_first;
            while (k < c) {
                int32_t b = C[k];
                // next row of column r: the 2x2 partner r+1 comes before struct(r) (all > r+1)
                int32_t a;
                int64_t apos;
                if (partner_pending) {
                    a = r + 1;
                    apos = P.Srp[r + 2] - 2;
                } else if (qq < qqe) {
                    a = Lri[qq];
                    apos = P.l2s[P.Lcsr[qq]];
                } else {
                    break;
                }
                if (a == b) {
                    if (fill) { ik[cnt] = ((uint32_t)i << 16) | (uint32_t)k; pos[cnt] = (int32_t)apos; }
                    ++cnt; ++k;
                    if (partner_pending) partner_pending = false; else ++qq;
                } else if (a < b) {
                    if (partner_pending) partner_pending = false; else ++qq;
                } else {
                    ++k;
                }
            }
        }
        if (fill) hrow[c] = (int32_t)cnt;
        return cnt;
    };
    // The pair lists take 8 B per pair.  Their number is bounded by the row lengths of
    // S over C (each lower pair is an entry of a row of C, counted once per side), and
    // measured at about a third of them on 3D factors: when even a quarter of that
    // bound would pass the budget, the lists are not built (counting them costs as
    // much as building them), else they are counted and the budget decides.
    const int64_t budget = pair_bytes > 0 ? pair_bytes : (int64_t(8) << 30);
    std::vector<int64_t> rowsum(ns, 0);
    parallel_for(ns, [&](int64_t a, int64_t b) {
        for (int64_t s = a; s < b; ++s) {
            int64_t t = 0;
            for (int32_t r : Cs[s]) t += P.Srp[r + 1] - P.Srp[r];
            rowsum[s] = t;
        }
    });
    int64_t rows_total = 0;
    for (int64_t s = 0; s < ns; ++s) rows_total += rowsum[s];
    P.scan_rows_total = rows_total;
    bool scan = pair_bytes < 0 || 8 * (rows_total / 4) > budget;
    int64_t roff = 0;
    for (int64_t s = 0; s < ns; ++s) {
        P.sn[s].hrow_off = roff;
        roff += P.sn[s].c + 1;
    }
    P.hrow.resize(roff);
    // The lists are built in one pass, into a buffer per chunk of kChunk consecutive
    // supernodes sized by an upper bound of its pairs (no-init: only the filled part
    // is touched), and then copied into place: a chunk's pairs form one contiguous
    // block of the final lists (so the lists briefly exist twice in host memory:
    // twice the budget at most).  The pass stops once the pairs pass the budget.
    constexpr int64_t kChunk = 256;
    std::vector<FillVec<uint32_t>> chunk_ik;
    std::vector<FillVec<int32_t>> chunk_pos;
    if (!scan) {
        const int64_t nchunks = (ns + kChunk - 1) / kChunk;
        chunk_ik.resize(nchunks);
        chunk_pos.resize(nchunks);
        std::atomic<int64_t> total(0);
        // pairs of row i of C: at most min(i, its S_lo row length - 1) below the
        // diagonal, the diagonal, and min(c - 1 - i, |struct| + 1) above it
        auto bound = [&](int64_t s) {
            const auto& C = Cs[s];
            const int64_t c = (int64_t)C.size();
            int64_t b = 0;
            for (int64_t i = 0; i < c; ++i) {
                const int32_t r = C[i];
                b += std::min<int64_t>(i, P.Srp[r + 1] - P.Srp[r] - 1) + 1 +
                     std::min<int64_t>(c - 1 - i, Lcp[r + 1] - Lcp[r] + 1);
            }
            return b;
        };
        parallel_for_dynamic(ns, kChunk, [&](int64_t a, int64_t b) {
            for (int64_t s0 = a; s0 < b; s0 += kChunk) {
                if (8 * total.load(std::memory_order_relaxed) > budget) return;
                const int64_t ch = s0 / kChunk, s1 = std::min(b, s0 + kChunk);
                int64_t cap = 0;
                for (int64_t s = s0; s < s1; ++s) cap += bound(s);
                chunk_ik[ch].resize(cap);
                chunk_pos[ch].resize(cap);
                int64_t off = 0;
                for (int64_t s = s0; s < s1; ++s) {
                    hits[s] = pairs(s, true, chunk_ik[ch].data() + off, chunk_pos[ch].data() + off,
                                    P.hrow.data() + P.sn[s].hrow_off);
                    off += hits[s];
                }
                total.fetch_add(off, std::memory_order_relaxed);
            }
        });
        scan = 8 * total.load() > budget;
    }
    P.scan = scan ? 1 : 0;
    int64_t hoff = 0;
    for (int64_t s = 0; s < ns; ++s) {
        SnInfo& I = P.sn[s];
        I.hit_off = scan ? 0 : hoff;
        I.hit_cnt = scan ? rowsum[s] / 3 + I.c : hits[s];
        if (!scan) hoff += hits[s];
        if (I.hit_cnt > INT32_MAX || rowsum[s] > INT32_MAX)
            return "a supernode has >= 2^31 pairs: unsupported";
    }
    P.hit_pairs = scan ? 0 : hoff;
    if (scan) {
        // work estimate: a third of the row lengths are pairs (see above); each
        // lookup reads a 4 B column index, each pair an 8 B value
        for (int64_t s = 0; s < ns; ++s) {
            const SnInfo& I = P.sn[s];
            P.selinv_flops += 2 * I.w * (rowsum[s] / 3 + I.c) + 2 * (int64_t)I.c * I.w * I.w;
            P.selinv_bytes += 4 * (rowsum[s] / 2) + 8 * ((rowsum[s] / 3 + I.c) / 2) + 16 * (int64_t)I.c * I.w;
        }
        parallel_for(ns, [&](int64_t a, int64_t b) {
            for (int64_t s = a; s < b; ++s) {
                int32_t* hr = P.hrow.data() + P.sn[s].hrow_off;
                int64_t t = 0;
                const auto& C = Cs[s];
                for (size_t i = 0; i < C.size(); ++i) {
                    hr[i] = (int32_t)t;
                    t += P.Srp[C[i] + 1] - P.Srp[C[i]];
                }
                hr[C.size()] = (int32_t)t;
            }
        });
    } else {
        for (int64_t s = 0; s < ns; ++s) {
            const SnInfo& I = P.sn[s];
            P.selinv_flops += 2 * I.w * hits[s] + 2 * (int64_t)I.c * I.w * I.w;
            P.selinv_bytes += 8 * ((hits[s] + I.c) / 2) + 16 * (int64_t)I.c * I.w;
        }
        P.hit_ik.resize(hoff);
        P.hit_pos.resize(hoff);
        const int64_t nchunks = (int64_t)chunk_ik.size();
        std::atomic<int64_t> next(0);
        run_chunks((int)std::min<int64_t>(n_threads(), nchunks), [&](int) {
            for (;;) {
                const int64_t ch = next.fetch_add(1);
                if (ch >= nchunks) break;
                const int64_t s0 = ch * kChunk, s1 = std::min(ns, s0 + kChunk);
                const int64_t cnt = P.sn[s1 - 1].hit_off + hits[s1 - 1] - P.sn[s0].hit_off;
                if (cnt > 0) {
                    std::memcpy(P.hit_ik.data() + P.sn[s0].hit_off, chunk_ik[ch].data(), cnt * sizeof(uint32_t));
                    std::memcpy(P.hit_pos.data() + P.sn[s0].hit_off, chunk_pos[ch].data(), cnt * sizeof(int32_t));
                }
                FillVec<uint32_t>().swap(chunk_ik[ch]);
                FillVec<int32_t>().swap(chunk_pos[ch]);
            }
        });
    }
    parallel_for(ns, [&](int64_t a, int64_t b) {
        for (int64_t s = a; s < b; ++s) {
            SnInfo& I = P.sn[s];
            const auto& C = Cs[s];
            std::copy(C.begin(), C.end(), P.Crow.begin() + I.crow_off);
            // Lmap: L(C[i], s0+t)
            for (int32_t t = 0; t < I.w; ++t) {
                int32_t col = I.s0 + t;
                int64_t i = 0;
                for (int64_t q = Lcp[col]; q < Lcp[col + 1]; ++q) {
                    int32_t r = Lri[q];
                    if (r < I.s0 + I.w) {
                        // inside the supernode: L_JJ(r - s0, t)
                        P.JJl[I.ww_off + (int64_t)(r - I.s0) * I.w + t] = P.Lcsr[q];
                        continue;
                    }
                    while (C[i] < r) ++i;
                    P.Lmap[I.cw_off + i * I.w + t] = P.Lcsr[q];
                }
            }
            // JJs: S positions of (s0+a, s0+b), a >= b
            for (int32_t aa = 0; aa < I.w; ++aa) {
                int32_t r = I.s0 + aa;
                for (int64_t q = P.Srp[r]; q < P.Srp[r + 1]; ++q) {
                    int32_t c = P.Sc[q];
                    if (c >= I.s0) P.JJs[I.ww_off + (int64_t)aa * I.w + (c - I.s0)] = (int32_t)q;
                }
            }
        }
    });
    // processing order: level-major, larger c first inside a level
    P.order.resize(ns);
    for (int64_t s = 0; s < ns; ++s) P.order[s] = (int32_t)(ns - 1 - s);
    std::stable_sort(P.order.begin(), P.order.end(), [&](int32_t a, int32_t b) {
        if (P.sn[a].level != P.sn[b].level) return P.sn[a].level < P.sn[b].level;
        return P.sn[a].hit_cnt > P.sn[b].hit_cnt;
    });
    // tensor-core tier: the leading levels in which every supernode has a contiguous C
    // (and width <= kTcWMax).  Its G~ reads go to a symmetric band copy of G whose
    // half-width covers every |row - column| the tier touches; the tier is cut back
    // to fewer levels while that copy would exceed kTcMirrorMax bytes.
    {
        constexpr int64_t kTcMirrorMax = int64_t(8) << 30;
        int64_t D = P.n_levels;
        for (int64_t s = 0; s < ns; ++s) {
            const auto& C = Cs[s];
            const SnInfo& I = P.sn[s];
            const int64_t range = C.empty() ? 0 : (int64_t)C.back() - C.front() + 1;
            const int64_t c = (int64_t)C.size();
            const bool ok = I.w <= kTcWMax && range <= c + std::max<int64_t>(16, c / 8);
            if (!ok) D = std::min<int64_t>(D, I.level);
        }
        // levels in processing order; shrink D until the mirror fits
        auto mirror_shape = [&](int64_t lv_end, int64_t& row0, int64_t& band) {
            row0 = n;
            band = 0;
            for (int64_t s = 0; s < ns; ++s) {
                if (P.sn[s].level >= lv_end) continue;
                const auto& C = Cs[s];
                row0 = std::min<int64_t>(row0, P.sn[s].s0);
                band = std::max<int64_t>(band, C.empty() ? P.sn[s].w - 1 : (int64_t)C.back() - P.sn[s].s0);
            }
        };
        int64_t row0 = n, band = 0;
        while (D > 0) {
            mirror_shape(D, row0, band);
            const int64_t width = ((2 * band + 136) + 3) / 4 * 4;
            if ((n - row0) * width * 8 <= kTcMirrorMax) break;
            --D;
        }
        P.tc_levels = D;
        for (int64_t s = 0; s < ns; ++s) {
            SnInfo& I = P.sn[s];
            I.tc_c = 0;
            I.tc_tiles = 0;
            I.tc_ks = 0;
            I.tc_ndep = 0;
            I.tc_t_off = I.tc_z_off = I.tc_map_off = I.tc_dep_off = -1;
        }
        if (D > 0) {
            P.tc_row0 = row0;
            P.tc_band = band;
            P.tc_width = ((2 * band + 136) + 3) / 4 * 4;
            for (int64_t t = 0; t < ns; ++t) {
                const int32_t sidx = P.order[t];
                SnInfo& I = P.sn[sidx];
                if (I.level >= D) break;  // the order is level-major
                const auto& C = Cs[sidx];
                const int64_t c = C.empty() ? 0 : (int64_t)C.back() - C.front() + 1;  // the range R
                const int64_t tiles = std::max<int64_t>(1, (c + kTcRowsTile - 1) / kTcRowsTile);
                const int64_t k0 = c > 0 ? (Cs[sidx].front() >> 2) << 2 : 0;
                const int64_t nch = c > 0 ? (Cs[sidx].front() + c - k0 + 31) / 32 : 0;
                // parts of at least 64 columns of R (two chunks) and at most kTcMaxChunks
                // chunks (their B tiles are staged at once), at most 16 parts unless needed
                int64_t ks = std::max<int64_t>(1, std::min<int64_t>({c / 64, 16, std::max<int64_t>(nch, 1)}));
                ks = std::max<int64_t>(ks, (nch + kTcMaxChunks - 1) / kTcMaxChunks);
                // the distinct supernodes owning rows of C, the latest in processing order first
                {
                    std::vector<int32_t> dep;
                    for (int32_t r : C) dep.push_back(P.owner[r]);
                    std::sort(dep.begin(), dep.end());
                    dep.erase(std::unique(dep.begin(), dep.end()), dep.end());
                    std::sort(dep.begin(), dep.end(), [&](int32_t x, int32_t y) {
                        return P.sn[x].level > P.sn[y].level || (P.sn[x].level == P.sn[y].level && x < y);
                    });
                    I.tc_dep_off = (int64_t)P.tc_deps.size();
                    I.tc_ndep = (int32_t)dep.size();
                    P.tc_deps.insert(P.tc_deps.end(), dep.begin(), dep.end());
                }
                I.tc_c = (int32_t)c;
                I.tc_map_off = (int64_t)P.tc_map.size();
                P.tc_map.resize(P.tc_map.size() + c * I.w, -1);
                for (int64_t i = 0; i < (int64_t)C.size(); ++i) {
                    const int64_t o = C[i] - C.front();
                    for (int32_t tt = 0; tt < I.w; ++tt)
                        P.tc_map[I.tc_map_off + o * I.w + tt] = P.Lmap[I.cw_off + i * I.w + tt];
                }
                I.tc_tiles = (int32_t)tiles;
                I.tc_ks = (int32_t)ks;
                I.tc_t_off = P.tc_t_total; P.tc_t_total += tiles;
                I.tc_z_off = P.tc_z_total; P.tc_z_total += (int64_t)I.w * I.w;
                P.tc_sn += 1;
                P.tc_pairs += c * c;
                for (int64_t q = 0; q < tiles * ks; ++q) {
                    WorkItem it;
                    it.first = (int32_t)t;
                    it.count = (int32_t)(tiles * ks);
                    it.big = 3;
                    it.part = (int32_t)q;
                    P.tc_items.push_back(it);
                }
            }
        }
    }
    // work items: a large supernode alone (whole CTA), else up to `group` consecutive ones.
    // Levels with fewer supernodes than thin_level sit on the critical path of the
    // dependency chain: each of their supernodes gets a whole CTA to shorten it.  A
    // supernode with more than 4 big_pairs pairs is split by rows into parts of about
    // that size (at most kMaxParts), one CTA each: the parts add their share of X into
    // a global block and the last part to arrive finishes the supernode.
    // the scan form costs more per pair (each row's lookups wait on its loads): its
    // large supernodes take smaller parts and more CTAs
    const int64_t kMaxParts = P.scan ? 32 : 16;
    const int64_t part_pairs = P.scan ? big_pairs : 4 * big_pairs;
    std::vector<int64_t> level_size(P.n_levels, 0);
    for (int64_t s = 0; s < ns; ++s) level_size[P.sn[s].level]++;
    P.items.clear();
    P.xsum_off.assign(ns, -1);
    P.xsum_total = 0;
    for (int64_t t = 0; t < ns;) {
        const SnInfo& I = P.sn[P.order[t]];
        WorkItem it;
        it.first = (int32_t)t;
        it.part = 0;
        if (I.hit_cnt >= big_pairs || level_size[I.level] < thin_level) {
            const int64_t parts = std::min<int64_t>(kMaxParts, (I.hit_cnt + part_pairs - 1) / part_pairs);
            if (parts >= 2 && I.c >= 2 * parts) {
                P.xsum_off[P.order[t]] = P.xsum_total;
                P.xsum_total += (int64_t)I.c * I.w;
                for (int64_t q = 0; q < parts; ++q) {
                    it.count = (int32_t)parts;
                    it.big = 2;
                    it.part = (int32_t)q;
                    P.items.push_back(it);
                }
                ++t;
                continue;
            }
            it.count = 1;
            it.big = 1;
            ++t;
        } else {
            int64_t e = t;
            // a group never mixes the tensor-core levels with the later ones
            const bool tc_side = I.level < P.tc_levels;
            while (e < ns && e - t < group && P.sn[P.order[e]].hit_cnt < big_pairs &&
                   level_size[P.sn[P.order[e]].level] >= thin_level &&
                   (P.sn[P.order[e]].level < P.tc_levels) == tc_side)
                ++e;
            it.count = (int32_t)(e - t);
            it.big = 0;
            t = e;
        }
        P.items.push_back(it);
    }
    P.rest_first = (int64_t)P.items.size();
    for (int64_t q = 0; q < (int64_t)P.items.size(); ++q)
        if (P.sn[P.order[P.items[q].first]].level >= P.tc_levels) {
            P.rest_first = q;
            break;
        }
    return "";
}

// Pattern of sum_{t<=m} E^t by columns: R_t(j) = {j} u union_{k in struct(j)} R_{t-1}(k),
// computed for t = 1..m, with each row tagged by the first t that reaches it.
std::string build_ninv_plan(const HostPlan& P, int m, NinvPlan& W) {
    int64_t n = P.n;
    W = NinvPlan();
    W.m = m;
    const int64_t* Lcp = P.Lcp.data();
    const int32_t* Lri = P.Lri.data();
    // Column j of the pattern, built by powers: R_t(j) = {j} + the union over k in
    // struct(j) of R_{t-1}(k).  The union of the R_{t-2}(k) is already in R_{t-1}(j), so
    // round t only propagates front[k], the rows that entered R_{t-1}(k) in round t-1,
    // and the rows it adds to column j are the group of tag t (the fewest steps that
    // reach them).  rows[j] keeps the groups one after another, each sorted, which is
    // the layout of W (grp[j] holds the group starts).
    const int G = m + 2;
    std::vector<std::vector<int32_t>> rows(n), front(n);
    W.grp.assign((size_t)n * G, 0);
    for (int64_t j = 0; j < n; ++j) {
        rows[j].push_back((int32_t)j);
        front[j].push_back((int32_t)j);
        W.grp[(size_t)j * G + 1] = 1;  // group 0 = {j}
    }
    for (int t = 1; t <= m; ++t) {
        std::vector<std::vector<int32_t>> nfront(n);
        parallel_for_dynamic(n, 512, [&](int64_t a, int64_t b) {
            // per-thread dense markers: mark[r] == j when row r is already in R_t(j)
            std::vector<int32_t> mark(n, -1);
            for (int64_t j = a; j < b; ++j) {
                auto& R = rows[j];
                for (int32_t r : R) mark[r] = (int32_t)j;
                auto& fresh = nfront[j];
                for (int64_t q = Lcp[j]; q < Lcp[j + 1]; ++q)
                    for (int32_t r : front[Lri[q]])
                        if (mark[r] != (int32_t)j) {
                            mark[r] = (int32_t)j;
                            fresh.push_back(r);
                        }
                std::sort(fresh.begin(), fresh.end());
                R.insert(R.end(), fresh.begin(), fresh.end());
                W.grp[(size_t)j * G + t + 1] = (int32_t)R.size();
            }
        });
        front.swap(nfront);
    }
    front = std::vector<std::vector<int32_t>>();
    W.Wcp.assign(n + 1, 0);
    for (int64_t j = 0; j < n; ++j) W.Wcp[j + 1] = W.Wcp[j] + (int64_t)rows[j].size();
    W.nnzW = W.Wcp[n];
    if (W.nnzW > INT32_MAX) return "pattern of the truncated Neumann series has >= 2^31 entries";
    W.Wr.resize(W.nnzW);
    // rows of 2x2 blocks carry a flag bit
    parallel_for_dynamic(n, 512, [&](int64_t a, int64_t b) {
        for (int64_t j = a; j < b; ++j) {
            int32_t* out = W.Wr.data() + W.Wcp[j];
            const auto& R = rows[j];
            for (size_t e = 0; e < R.size(); ++e) {
                const int32_t r = R[e];
                const bool two = !P.pstart[r] || (r + 1 < n && !P.pstart[r + 1]);
                out[e] = two ? (int32_t)((uint32_t)r | 0x80000000u) : r;
            }
        }
    });
    for (int64_t j = 0; j < n; ++j) W.max_col = std::max<int64_t>(W.max_col, W.Wcp[j + 1] - W.Wcp[j]);
    // work counts: step t reads groups 0..t-1 of every k in struct(j)
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t q = Lcp[j]; q < Lcp[j + 1]; ++q) {
            const int64_t k = Lri[q];
            for (int t = 1; t <= m; ++t) W.horner_products += W.grp[(size_t)k * G + t];
        }
        // column j of S_lo: j, its 2x2 partner, struct(j); each streams column i of W
        const bool two_first = P.pstart[j] && j + 1 < n && !P.pstart[j + 1];
        W.product_stream += W.Wcp[j + 1] - W.Wcp[j];
        if (two_first) W.product_stream += W.Wcp[j + 2] - W.Wcp[j + 1];
        for (int64_t q = Lcp[j]; q < Lcp[j + 1]; ++q) W.product_stream += W.Wcp[Lri[q] + 1] - W.Wcp[Lri[q]];
    }
    return "";
}

namespace {

// Checks of a symmetric matrix's CSR pattern; `sorted` receives the rows sorted.
std::string check_symmetric_pattern(int64_t n, int64_t nnzA, const int64_t* Arp, const int32_t* Ac,
                                    std::vector<int32_t>& sorted) {
    if (Arp[0] != 0 || Arp[n] != nnzA) return "A_rowptr must start at 0 and end at nnzA";
    for (int64_t i = 0; i < n; ++i)
        if (Arp[i + 1] < Arp[i]) return "A_rowptr must be non-decreasing";
    if (nnzA >= ((int64_t)1 << 31)) return "nnzA >= 2^31 is not supported";
    // rows sorted on a copy: range, duplicates and structural symmetry
    sorted.assign(Ac, Ac + nnzA);
    for (int64_t i = 0; i < n; ++i) {
        int32_t* b = sorted.data() + Arp[i];
        int32_t* e = sorted.data() + Arp[i + 1];
        std::sort(b, e);
        for (int32_t* c = b; c != e; ++c) {
            if (*c < 0 || *c >= n) return "A column index out of range";
            if (c + 1 != e && c[1] == *c) return "A has a duplicate entry";
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t q = Arp[i]; q < Arp[i + 1]; ++q) {
            const int32_t k = sorted[q];
            if (!std::binary_search(sorted.begin() + Arp[k], sorted.begin() + Arp[k + 1], (int32_t)i))
                return "the pattern of A is not symmetric";
        }
    return "";
}

}  // namespace

std::string build_spai_plan(const HostPlan& P, int64_t nnzA, const int64_t* Arp, const int32_t* Ac, int power,
                            int warp_j, int warp_e, int warp_r, SpaiPlan& X, const int64_t* Prp_given,
                            const int32_t* Pc_given, const int32_t* src_given) {
    const int64_t n = P.n;
    X = SpaiPlan();
    X.n = n;
    X.nnzA = nnzA;
    X.power = power;
    std::vector<int32_t> sorted;
    std::string err = check_symmetric_pattern(n, nnzA, Arp, Ac, sorted);
    if (!err.empty()) return err;
    // P_lo row by row: S_lo row i, and every j <= i within `power` steps of i in the graph of A
    // (or the given pattern, whose start values are read at src_given)
    X.Prp.assign(n + 1, 0);
    std::vector<int64_t> reached(n, -1);
    std::vector<int32_t> row, frontier, next;
    std::vector<int32_t> src_of;  // per P_lo entry: S_lo position or -1 (given: the caller's index)
    if (Prp_given) {
        if (Prp_given[0] != 0) return "the refinement pattern's row pointers do not start at 0";
        for (int64_t i = 0; i < n; ++i) {
            const int64_t a0 = Prp_given[i], a1 = Prp_given[i + 1];
            if (a1 <= a0 || Pc_given[a1 - 1] != i)
                return "row " + std::to_string(i) + " of the refinement pattern lacks its diagonal";
            for (int64_t p = a0 + 1; p < a1; ++p)
                if (Pc_given[p - 1] >= Pc_given[p]) return "the refinement pattern's rows are not sorted";
            if (Pc_given[a0] < 0) return "a column index of the refinement pattern is negative";
        }
        if (Prp_given[n] >= ((int64_t)1 << 31)) return "the refinement pattern has >= 2^31 entries: not supported";
        X.Prp.assign(Prp_given, Prp_given + n + 1);
        X.Pc.assign(Pc_given, Pc_given + Prp_given[n]);
        src_of.assign(src_given, src_given + Prp_given[n]);
    }
    for (int64_t i = 0; i < n && !Prp_given; ++i) {
        row.assign(P.Sc.begin() + P.Srp[i], P.Sc.begin() + P.Srp[i + 1]);
        if (power > 0) {
            reached[i] = i;
            row.push_back((int32_t)i);
            frontier.assign(1, (int32_t)i);
            for (int step = 0; step < power && !frontier.empty(); ++step) {
                next.clear();
                for (int32_t u : frontier)
                    for (int64_t q = Arp[u]; q < Arp[u + 1]; ++q) {
                        const int32_t v = sorted[q];
                        if (reached[v] == i) continue;
                        reached[v] = i;
                        next.push_back(v);
                        if (v <= i) row.push_back(v);
                    }
                frontier.swap(next);
            }
        }
        std::sort(row.begin(), row.end());
        row.erase(std::unique(row.begin(), row.end()), row.end());
        X.Prp[i + 1] = X.Prp[i] + (int64_t)row.size();
        if (X.Prp[i + 1] >= ((int64_t)1 << 31)) return "the refinement pattern has >= 2^31 entries: not supported";
        // S positions: S_lo row i is sorted and a subset of the row
        int64_t p = P.Srp[i];
        for (int32_t c : row) {
            X.Pc.push_back(c);
            if (p < P.Srp[i + 1] && P.Sc[p] == c) src_of.push_back((int32_t)p++);
            else src_of.push_back(-1);
        }
    }
    X.nnzP = X.Prp[n];
    // columns of P: row j of P_lo (rows k <= j), then the entries (i, j) of later rows i
    std::vector<int64_t> cnt(n, 0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = X.Prp[i]; p < X.Prp[i + 1]; ++p) {
            cnt[i] += 1;
            if (X.Pc[p] != i) cnt[X.Pc[p]] += 1;
        }
    X.fcp.assign(n + 1, 0);
    for (int64_t j = 0; j < n; ++j) X.fcp[j + 1] = X.fcp[j] + cnt[j];
    const int64_t nf = X.fcp[n];
    X.fri.resize(nf);
    X.fpos.resize(nf);
    X.fsrc.resize(nf);
    std::vector<int64_t> cur(n);
    for (int64_t j = 0; j < n; ++j) {
        int64_t q = X.fcp[j];
        for (int64_t p = X.Prp[j]; p < X.Prp[j + 1]; ++p, ++q) {
            X.fri[q] = X.Pc[p];
            X.fpos[q] = (int32_t)p;
            X.fsrc[q] = src_of[p];
        }
        cur[j] = q;
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = X.Prp[i]; p < X.Prp[i + 1]; ++p) {
            const int32_t j = X.Pc[p];
            if (j == i) continue;
            X.fri[cur[j]] = (int32_t)i;
            X.fpos[cur[j]] = (int32_t)p;
            X.fsrc[cur[j]] = src_of[p];
            ++cur[j];
        }
    // entry offsets, distinct rows per column and the two tiers
    X.feo.resize(nf);
    X.fE.resize(n);
    X.fR.resize(n);
    std::vector<int64_t> seen(n, -1);
    int64_t cap_R = 0;
    for (int64_t j = 0; j < n; ++j) {
        int64_t acc = 0, R = 0;
        for (int64_t q = X.fcp[j]; q < X.fcp[j + 1]; ++q) {
            X.feo[q] = (int32_t)acc;
            const int32_t k = X.fri[q];
            acc += Arp[k + 1] - Arp[k];
            if (acc >= ((int64_t)1 << 30)) return "a column of P stages more than 2^30 entries of A: not supported";
            for (int64_t e = Arp[k]; e < Arp[k + 1]; ++e)
                if (seen[Ac[e]] != j) {
                    seen[Ac[e]] = j;
                    ++R;
                }
        }
        X.fE[j] = (int32_t)acc;
        X.fR[j] = (int32_t)R;
        X.entries += acc;
        const int64_t nj = X.fcp[j + 1] - X.fcp[j];
        if (nj <= warp_j && acc <= warp_e && R <= warp_r) {
            X.cols_w.push_back((int32_t)j);
        } else {
            X.cols_c.push_back((int32_t)j);
            X.cap_nj = std::max(X.cap_nj, nj);
            X.cap_E = std::max(X.cap_E, acc);
            cap_R = std::max(cap_R, R);
        }
    }
    if (!X.cols_c.empty()) {
        X.cap_H = 32;
        while (X.cap_H < 2 * cap_R) X.cap_H <<= 1;
    }
    auto by_size = [&](int32_t a, int32_t b) { return X.fE[a] > X.fE[b]; };
    std::stable_sort(X.cols_w.begin(), X.cols_w.end(), by_size);
    std::stable_sort(X.cols_c.begin(), X.cols_c.end(), by_size);
    return "";
}

std::string build_einv_plan(const HostPlan& P, int64_t nnzA, const int64_t* Arp, const int32_t* Ac, EinvPlan& X) {
    const int64_t n = P.n;
    X = EinvPlan();
    X.n = n;
    X.nnzA = nnzA;
    std::vector<int32_t> sorted;
    std::string err = check_symmetric_pattern(n, nnzA, Arp, Ac, sorted);
    if (!err.empty()) return err;
    // columns of S: row j of S_lo (rows k <= j), then the entries (i, j) of later rows i
    std::vector<int64_t> cnt(n, 0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = P.Srp[i]; p < P.Srp[i + 1]; ++p) {
            cnt[i] += 1;
            if (P.Sc[p] != i) cnt[P.Sc[p]] += 1;
        }
    X.fcp.assign(n + 1, 0);
    for (int64_t j = 0; j < n; ++j) X.fcp[j + 1] = X.fcp[j] + cnt[j];
    X.fri.resize(X.fcp[n]);
    X.fpos.resize(X.fcp[n]);
    std::vector<int64_t> cur(n);
    for (int64_t j = 0; j < n; ++j) {
        int64_t q = X.fcp[j];
        for (int64_t p = P.Srp[j]; p < P.Srp[j + 1]; ++p, ++q) {
            X.fri[q] = P.Sc[p];
            X.fpos[q] = (int32_t)p;
        }
        cur[j] = q;
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = P.Srp[i]; p < P.Srp[i + 1]; ++p) {
            const int32_t j = P.Sc[p];
            if (j == i) continue;
            X.fri[cur[j]] = (int32_t)i;
            X.fpos[cur[j]] = (int32_t)p;
            ++cur[j];
        }
    // L by rows: the column of every CSR entry, from the CSC copy and its CSR positions
    X.Lcol.assign(P.nnzL, 0);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t q = P.Lcp[j]; q < P.Lcp[j + 1]; ++q) X.Lcol[P.Lcsr[q]] = (int32_t)j;
    std::vector<int64_t> rcnt(n + 1, 0);
    for (int64_t q = 0; q < P.nnzL; ++q) rcnt[P.Lri[q] + 1] += 1;
    for (int64_t i = 0; i < n; ++i) rcnt[i + 1] += rcnt[i];  // CSR row starts of L
    // levels: row i of L y = b needs the rows j of its entries; column j of L^T x = z
    // needs the rows i > j of column j
    std::vector<int32_t> lev(n, 0);
    int32_t nlev = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t l = 0;
        for (int64_t q = rcnt[i]; q < rcnt[i + 1]; ++q) l = std::max(l, lev[X.Lcol[q]] + 1);
        lev[i] = l;
        nlev = std::max(nlev, l + 1);
    }
    auto group = [&](std::vector<int32_t>& items, std::vector<int32_t>& ptr) {
        ptr.assign(nlev + 1, 0);
        for (int64_t i = 0; i < n; ++i) ptr[lev[i] + 1] += 1;
        for (int32_t l = 0; l < nlev; ++l) ptr[l + 1] += ptr[l];
        items.resize(n);
        std::vector<int32_t> at(ptr.begin(), ptr.end() - 1);
        for (int64_t i = 0; i < n; ++i) items[at[lev[i]]++] = (int32_t)i;
    };
    if (n > 0) group(X.fwd_rows, X.fwd_ptr);
    nlev = 0;
    for (int64_t j = n - 1; j >= 0; --j) {
        int32_t l = 0;
        for (int64_t q = P.Lcp[j]; q < P.Lcp[j + 1]; ++q) l = std::max(l, lev[P.Lri[q]] + 1);
        lev[j] = l;
        nlev = std::max(nlev, l + 1);
    }
    if (n > 0) group(X.bwd_cols, X.bwd_ptr);
    return "";
}

}  // namespace sinv
