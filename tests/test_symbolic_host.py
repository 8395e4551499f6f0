"""Host-side checks of libsinv without a GPU: exported symbols, the symbolic
analysis (S bit-exact against the oracle, supernode and level invariants) and
the pattern validation errors."""
import ctypes
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from workloads.configs import diff3d, lap2d_32, plant_2x2, random_factors

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_11363_b300.build import build_lib
    build_lib()
    from paper_2609_11363_b300 import load_library
    return load_library()


def _host_handle(f, **kw):
    from paper_2609_11363_b300 import Handle
    return Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, device=-1, **kw)


def test_library_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "sinv.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = sorted(set(re.findall(r"\b(sinv_[a-z_0-9]+)\s*\(", hdr)))
    assert len(names) >= 14
    for nm in names:
        assert hasattr(lib, nm), nm
    from paper_2609_11363_b300.binding import EXPORTS
    assert sorted(EXPORTS) == names


def test_checked_library_exports_every_declared_symbol(lib):
    """The bounds-checked build (-DSINV_CHECKED) has the same ABI."""
    import ctypes
    from paper_2609_11363_b300.binding import EXPORTS
    from paper_2609_11363_b300.build import build_lib
    path = build_lib(checked=True)
    assert path.endswith("libsinv_checked.so")
    clib = ctypes.CDLL(path)
    for nm in EXPORTS:
        assert hasattr(clib, nm), nm


CASES = {
    "lap2d": lambda: lap2d_32().factors,
    "lap2d_exact": lambda: lap2d_32(tau=0.0).factors,
    "lap2d_2x2": lambda: plant_2x2(lap2d_32().factors, 0.4, 3),
    "rand": lambda: random_factors(400, 0.03, 0.2, 8),
    "diff3d_10": lambda: plant_2x2(diff3d(10).factors, 0.05, 4),
    # 3.4 M entries of L: the analysis transposes L in several row chunks
    "rand_dense_3k": lambda: random_factors(3000, 0.75, 0.1, 9),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_pattern_bit_exact_vs_oracle(lib, name):
    f = CASES[name]()
    h = _host_handle(f)
    rp, col = h.pattern_host()
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    assert np.array_equal(rp, S[0]) and np.array_equal(col, S[1])
    st = h.stats()
    assert st["nnz_S_lo"] == len(S[1]) and st["n_2x2"] == int(np.sum(f.pivot_start == 0))


def _structs(f):
    Lc = f.L_csr().tocsc()
    Lc.sort_indices()
    return [set(Lc.indices[Lc.indptr[j]:Lc.indptr[j + 1]].tolist()) for j in range(f.n)]


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("cap", [1, 4, 16])
def test_supernode_and_level_invariants(lib, name, cap):
    f = CASES[name]()
    h = _host_handle(f, supernode_cap=cap)
    start, level = h.supernodes()
    n = f.n
    assert start[0] == 0 and start[-1] == n and np.all(np.diff(start) >= 1) and np.max(np.diff(start)) <= max(cap, 2)
    ps = f.pivot_start.astype(bool)
    # a supernode never splits a 2x2 block
    assert np.all(ps[start[:-1]])
    st = _structs(f)
    blocks = [j for j in range(n) if ps[j]] + [n]
    owner = np.repeat(np.arange(len(start) - 1), np.diff(start))
    bstart_set = set(start[:-1].tolist())
    for b in range(len(blocks) - 2):
        P = range(blocks[b], blocks[b + 1]); Q = range(blocks[b + 1], blocks[b + 2])
        U = set().union(*[st[p] for p in P]) - set(P) - set(range(blocks[b + 1]))
        U = {r for r in U if r >= blocks[b + 1]}
        joined = blocks[b + 1] not in bstart_set
        rule = (len(U) > 0 and min(U) == Q[0]) and all((U - set(Q)) <= st[c] for c in Q)
        if joined:
            assert rule, ("joined blocks violate the merge rule", b)
        else:
            width = blocks[b + 2] - start[owner[blocks[b]]]
            assert (not rule) or width > cap, ("mergeable blocks left apart", b)
    for s in range(len(start) - 1):
        cols = range(start[s], start[s + 1])
        C = set().union(*[st[c] for c in cols]) - set(range(start[s + 1] + 0)) if cols else set()
        C = {r for r in C if r >= start[s + 1]}
        want = 0 if not C else 1 + max(level[owner[r]] for r in C)
        assert level[s] == want


@pytest.mark.parametrize("name", sorted(CASES))
def test_scan_form_plan(lib, name):
    """The scan form of SelInv keeps the supernodes and levels, stores no pair list,
    and its work measure is the sum over supernodes of the S_lo row lengths of C."""
    f = CASES[name]()
    a = _host_handle(f)
    b = _host_handle(f, selinv_pair_bytes=-1)
    sa, sb = a.stats(), b.stats()
    assert sb["selinv_scan"] == 1 and sb["hit_pairs"] == 0
    # by default the pair lists, unless they would pass the memory budget (the dense
    # random case: its rows of C hold 5.0 G entries of S, so even a quarter of them
    # as 8-byte pairs passes the default 8 GB)
    assert sa["selinv_scan"] == (1 if name == "rand_dense_3k" else 0)
    for x, y in zip(a.supernodes(), b.supernodes()):
        assert np.array_equal(x, y)
    rp, _ = b.pattern_host()
    rowlen = np.diff(rp)
    start, _ = b.supernodes()
    st = _structs(f)
    want = 0
    for s_ in range(len(start) - 1):
        C = set().union(*[st[c] for c in range(start[s_], start[s_ + 1])])
        want += int(sum(rowlen[r] for r in C if r >= start[s_ + 1]))
    assert sb["scan_rows_total"] == want == sa["scan_rows_total"]


def _expect_pattern_error(n, rp, col, ps):
    from paper_2609_11363_b300 import Handle, SinvError
    with pytest.raises(SinvError) as ei:
        Handle(n, np.asarray(rp, np.int64), np.asarray(col, np.int32), np.asarray(ps, np.int8), device=-1)
    assert ei.value.name == "SINV_ERR_PATTERN"


def test_pattern_validation(lib):
    # rows: 0: -, 1: [0], 2: [0, 1]
    ok = ([0, 0, 1, 3], [0, 0, 1], [1, 1, 1])
    from paper_2609_11363_b300 import Handle
    Handle(3, np.asarray(ok[0], np.int64), np.asarray(ok[1], np.int32), np.asarray(ok[2], np.int8), device=-1)
    _expect_pattern_error(3, [0, 0, 1, 3], [0, 1, 0], [1, 1, 1])      # unsorted row
    _expect_pattern_error(3, [0, 0, 1, 3], [0, 0, 0], [1, 1, 1])      # duplicate
    _expect_pattern_error(3, [0, 0, 1, 3], [0, 0, 2], [1, 1, 1])      # diagonal stored
    _expect_pattern_error(3, [0, 0, 1, 3], [0, -1, 1], [1, 1, 1])     # negative column
    _expect_pattern_error(3, [0, 0, 2, 3], [0, 0, 1], [1, 1, 1])      # col >= row via bad rowptr
    _expect_pattern_error(3, [0, 1, 1, 3], [0, 0, 1], [1, 1, 1])      # row 0 has an entry
    _expect_pattern_error(3, [0, 0, 1, 1], [0], [0, 1, 1])            # first flag 0
    _expect_pattern_error(3, [0, 0, 0, 0], [], [1, 0, 0])             # 3x3 block
    _expect_pattern_error(3, [0, 0, 1, 1], [0], [1, 0, 1])            # L(1,0) inside a 2x2 block
    _expect_pattern_error(3, [0, 0, 0, 0], [], [1, 2, 1])             # bad flag value


def test_host_only_handle_rejects_numeric_calls(lib):
    from paper_2609_11363_b300 import SinvError
    f = lap2d_32().factors
    h = _host_handle(f)
    with pytest.raises(SinvError) as ei:
        h.sync_status()
    assert ei.value.name == "SINV_ERR_INVALID_ARG"


def test_status_strings(lib):
    for code in range(8):
        s = lib.sinv_status_string(code)
        assert s and s != b"unknown status"
    assert lib.sinv_status_string(99) == b"unknown status"


def test_batch_rejects_cross_block_entries():
    from paper_2609_11363_b300 import Handle, SinvError
    from workloads.configs import random_factors
    fs = [random_factors(50, 0.1, 0.0, 1), random_factors(60, 0.1, 0.0, 2)]
    bad = random_factors(60, 0.1, 0.0, 2)
    bad.L_col = bad.L_col.copy()
    bad.L_col[-1] = bad.L_rowptr.shape[0]  # beyond its own row
    with pytest.raises(SinvError) as ei:
        Handle.batch([fs[0], bad], device=-1)
    assert ei.value.name == "SINV_ERR_PATTERN"


def test_batch_layout_host(lib):
    from paper_2609_11363_b300 import Handle
    from workloads.configs import random_factors
    fs = [lap2d_32().factors, random_factors(300, 0.05, 0.2, 3), plant_2x2(lap2d_32().factors, 0.2, 5)]
    h = Handle.batch(fs, device=-1)
    lay = h.layout()
    rp, col = h.pattern_host()
    assert list(np.diff(lay["n"])) == [f.n for f in fs]
    assert list(np.diff(lay["L"])) == [f.nnz_L for f in fs]
    assert list(np.diff(lay["D"])) == [len(f.D_packed) for f in fs]
    for b, f in enumerate(fs):
        S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
        s0, r0 = lay["S"][b], lay["n"][b]
        assert np.array_equal(col[s0:lay["S"][b + 1]] - r0, S[1])
        assert np.array_equal(rp[r0:r0 + f.n + 1] - s0, S[0])


def _spai_cases():
    from workloads.configs import covariance
    w = lap2d_32()
    c = covariance(12)
    return {"lap2d": (w.A, w.factors), "covariance_12": (c.A, c.factors)}


@pytest.mark.parametrize("power", [0, 1, 2, 3])
@pytest.mark.parametrize("name", ["lap2d", "covariance_12"])
def test_spai_pattern_bit_exact_vs_oracle(lib, name, power):
    A, f = _spai_cases()[name]
    h = _host_handle(f)
    h.spai_analyse(A, power=power)
    rp, col = h.spai_pattern()
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    want = oracle.spai_pattern(A, S[0], S[1], power)
    assert np.array_equal(rp, want[0]) and np.array_equal(col, want[1])
    st = h.stats()
    assert st["spai_nnz_P"] == len(want[1])
    assert st["spai_cols_warp"] + st["spai_cols_cta"] == f.n
    # entries staged per B product: sum over the columns j of P of nnz(A) of their rows
    full = sp.csr_matrix((np.ones(len(col)), col, rp), shape=(f.n, f.n))
    full = full + sp.tril(full, k=-1).T
    annz = np.diff(sp.csr_matrix(A).indptr)
    assert st["spai_entries"] == int(np.asarray(full.sum(axis=0)).ravel() @ annz)


def test_spai_analysis_rejects_bad_patterns(lib):
    from paper_2609_11363_b300 import SinvError
    w = lap2d_32()
    h = _host_handle(w.factors)
    B = sp.csr_matrix(w.A, copy=True).tolil()
    B[0, w.factors.n - 1] = 1.0  # one entry without its mirror
    with pytest.raises(SinvError) as e:
        h.spai_analyse(B.tocsr())
    assert e.value.name == "SINV_ERR_PATTERN"
    with pytest.raises(SinvError) as e:
        h.spai_analyse(w.A, power=-1)
    assert e.value.name == "SINV_ERR_INVALID_ARG"
    with pytest.raises(SinvError) as e:
        h.spai_analyse(w.A, power=9)
    assert e.value.name == "SINV_ERR_UNSUPPORTED"


@pytest.mark.parametrize("name", ["lap2d", "covariance_12"])
def test_einv_solve_levels_vs_brute_force(lib, name):
    # levels of L y = b: 1 + the deepest row a row reads; of L^T x = w: 1 + the deepest
    # later row of its column
    A, f = _spai_cases()[name]
    h = _host_handle(f)
    h.einv_analyse(A)
    st = h.stats()
    L = f.L_csr()
    n = f.n
    fwd = np.zeros(n, dtype=int)
    for i in range(n):
        c = L.indices[L.indptr[i]:L.indptr[i + 1]]
        fwd[i] = fwd[c].max() + 1 if len(c) else 0
    Lc = L.tocsc()
    bwd = np.zeros(n, dtype=int)
    for j in range(n - 1, -1, -1):
        r = Lc.indices[Lc.indptr[j]:Lc.indptr[j + 1]]
        bwd[j] = bwd[r].max() + 1 if len(r) else 0
    assert st["einv_levels_fwd"] == fwd.max() + 1 and st["einv_levels_bwd"] == bwd.max() + 1


def test_spai_and_lanczos_errors_through_the_abi(lib):
    # documented error returns that need no device: calls on a host-only handle, a pattern
    # query before any analysis, bad analysis arguments
    w = lap2d_32()
    h = _host_handle(w.factors)
    rp = np.zeros(w.factors.n + 1, dtype=np.int64)
    col = np.zeros(max(1, h.nnz_S), dtype=np.int32)
    P = ctypes.c_void_p
    assert lib.sinv_spai_pattern(h._h, rp.ctypes.data_as(P), col.ctypes.data_as(P)) == 1
    assert lib.sinv_spai(h._h, None, None, 3, None, None) == 1
    lam = np.zeros(2)
    info = np.zeros(3, dtype=np.int32)
    assert lib.sinv_einv_lanczos(h._h, None, None, None, None, None, 4, 1e-10, 10, 2,
                                 lam.ctypes.data_as(P), None, info.ctypes.data_as(P), None) == 1
    A = sp.csr_matrix(w.A)
    arp = A.indptr.astype(np.int64)
    acol = A.indices.astype(np.int32)
    assert lib.sinv_spai_analyse(h._h, A.nnz, arp.ctypes.data_as(P), acol.ctypes.data_as(P), 0, -1) == 1
    assert lib.sinv_einv_analyse(h._h, -1, arp.ctypes.data_as(P), acol.ctypes.data_as(P)) == 1
    bad = arp.copy()
    bad[-1] += 1  # rowptr does not end at nnzA
    assert lib.sinv_einv_analyse(h._h, A.nnz, bad.ctypes.data_as(P), acol.ctypes.data_as(P)) == 2


def test_new_entry_points_report_errors_without_a_device(lib):
    """Documented error returns of the calls for NInv / Mix on the own pattern, the
    scan counters, the timeline and the checked-build test hook: a NULL handle, a
    host-only handle, or a call before the one it needs (no device is touched)."""
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    nnz, steps = I64(), np.zeros(4, dtype=np.int64)
    # NULL handle
    assert lib.sinv_ninv_own(None, None, None, 2, ctypes.c_double(0.1), None) == 1
    assert lib.sinv_mix_own(None, None, ctypes.c_double(0.0), None) == 1
    assert lib.sinv_mix_own_size(None, ctypes.byref(nnz)) == 1
    assert lib.sinv_lowrank_correct_mix_own(None, 4, None, None, 0, None) == 1
    assert lib.sinv_spai_mix_own(None, None, None, 3, None, None) == 1
    assert lib.sinv_selinv_scan_counts(None, ctypes.byref(nnz), ctypes.byref(nnz), None) == 1
    assert lib.sinv_debug_corrupt_plan(None) == 1
    # a host-only handle: numeric calls are refused, the results of calls that never ran too
    w = lap2d_32()
    h = _host_handle(w.factors)
    assert lib.sinv_ninv_own(h._h, None, None, 2, ctypes.c_double(0.1), None) == 1
    assert lib.sinv_ninv_own(h._h, None, None, -1, ctypes.c_double(0.1), None) == 1
    assert lib.sinv_ninv_own(h._h, None, None, 2, ctypes.c_double(-1.0), None) == 1
    assert lib.sinv_ninv_own_size(h._h, ctypes.byref(nnz), steps.ctypes.data_as(P), 4) == 1
    assert lib.sinv_mix_own(h._h, None, ctypes.c_double(float("nan")), None) == 1
    assert lib.sinv_mix_own_size(h._h, ctypes.byref(nnz)) == 1
    assert lib.sinv_lowrank_correct_mix_own(h._h, 300, None, None, 0, None) == 1
    assert lib.sinv_spai_mix_own(h._h, None, None, 3, None, None) == 1
    A = sp.csr_matrix(w.A)
    arp, acol = A.indptr.astype(np.int64), A.indices.astype(np.int32)
    assert lib.sinv_spai_analyse_mix_own(h._h, A.nnz, arp.ctypes.data_as(P), acol.ctypes.data_as(P), 0) == 1
    assert lib.sinv_timeline_enable(h._h, 1) == 1
    assert lib.sinv_debug_corrupt_plan(h._h) == 7   # the regular build never plants it
    # the network's checkpoint calls: a NULL network or buffer is refused before any device call
    buf = np.zeros(lib.sinv_mlp_param_count(), dtype=np.float32)
    bp = buf.ctypes.data_as(P)
    step = I64()
    assert lib.sinv_mlp_get_state(None, bp, bp, bp, ctypes.byref(step)) == 1
    assert lib.sinv_mlp_set_state(None, bp, bp, bp, 0) == 1


def test_empty_matrix_host_analyses(lib):
    """n = 0: the symbolic analysis, the SPAI pattern (S widened by any power) and
    the Lanczos solve levels are all empty, and no call reports an error."""
    from paper_2609_11363_b300 import Handle
    h = Handle(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int8), device=-1)
    st = h.stats()
    assert h.nnz_S == 0 and st["n_supernodes"] == 0
    A = sp.csr_matrix((0, 0))
    for power in (0, 2):
        h.spai_analyse(A, power=power)
        rp, col = h.spai_pattern()
        assert rp.tolist() == [0] and len(col) == 0 and h.stats()["spai_nnz_P"] == 0
    h.einv_analyse(A)
    st = h.stats()
    assert st["einv_levels_fwd"] == 0 and st["einv_levels_bwd"] == 0


@pytest.mark.parametrize("name", ["lap2d_exact", "diff3d_8_exact"])
def test_levels_of_exact_factors_are_elimination_tree_depths(lib, name):
    """For exact factors (a closed pattern) and one column per supernode, a column's
    level is its depth in the elimination tree (parent(j) = the first row of
    struct(j); the root has depth 0): every row of struct(j) is an ancestor of j and
    the parent is the deepest of them."""
    from workloads.configs import diff3d
    f = {"lap2d_exact": lambda: lap2d_32(tau=0.0).factors,
         "diff3d_8_exact": lambda: diff3d(8, tau=0.0, shifted=False).factors}[name]()
    assert np.all(f.pivot_start == 1)
    h = _host_handle(f, supernode_cap=1)
    start, level = h.supernodes()
    assert np.array_equal(start, np.arange(f.n + 1))
    Lc = f.L_csr().tocsc()
    Lc.sort_indices()
    depth = np.zeros(f.n, dtype=np.int64)
    for j in range(f.n - 1, -1, -1):
        rows = Lc.indices[Lc.indptr[j]:Lc.indptr[j + 1]]
        depth[j] = 0 if len(rows) == 0 else depth[rows[0]] + 1
    assert np.array_equal(np.asarray(level), depth)


@pytest.mark.parametrize("name", ["diff3d_10", "lap2d_2x2"])
def test_pair_budget_passed_while_building_gives_the_scan_form(lib, name):
    """A budget between the quick bound (a quarter of the row lengths as 8-byte
    pairs) and the real size of the lists: the lists are started, pass the budget
    while being built, and the scan form results, with the same supernodes and
    work measure as when it is asked for."""
    f = CASES[name]()
    a = _host_handle(f)
    sa = a.stats()
    lo, hi = 8 * (sa["scan_rows_total"] // 4), 8 * sa["hit_pairs"]
    assert sa["selinv_scan"] == 0 and lo < hi
    b = _host_handle(f, selinv_pair_bytes=(lo + hi) // 2)
    c = _host_handle(f, selinv_pair_bytes=-1)
    sb, sc = b.stats(), c.stats()
    assert sb["selinv_scan"] == 1 and sb["hit_pairs"] == 0
    assert sb["scan_rows_total"] == sc["scan_rows_total"] and sb["selinv_flops"] == sc["selinv_flops"]
    for x, y in zip(b.supernodes(), c.supernodes()):
        assert np.array_equal(x, y)
    # and a budget just above the lists keeps them
    d = _host_handle(f, selinv_pair_bytes=hi)
    assert d.stats()["selinv_scan"] == 0 and d.stats()["hit_pairs"] == sa["hit_pairs"]


def test_mlp_checkpoint_file_round_trip(tmp_path):
    """Mlp.save / Mlp.load carry the whole state (weights, both Adam moments, the
    step count) through an .npz file unchanged (the device calls are stood in for)."""
    from paper_2609_11363_b300 import Mlp
    rng = np.random.default_rng(0)
    m = Mlp.__new__(Mlp)   # no device: only the file format is under test
    m.n_params = 37
    state = {k: rng.standard_normal(37).astype(np.float32) for k in ("theta", "mom1", "mom2")}
    state["step"] = 12345
    m.get_state = lambda: state
    got = {}
    m.set_state = got.update
    path = str(tmp_path / "state.npz")
    m.save(path)
    m.load(path)
    assert got["step"] == 12345 and isinstance(got["step"], int)
    for k in ("theta", "mom1", "mom2"):
        assert got[k].dtype == np.float32 and np.array_equal(got[k], state[k])
    m._m = None   # nothing to free at exit
