"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: FP64 forms within 1e-10 entrywise in the scaled sense
|x_ij - r_ij| <= 1e-10 (|r_ij| + sqrt|r_ii r_jj|); the pattern S bit-exact;
Mix bit-exact (it only selects); FP32 forms normwise within the bound stated
in each test.
"""
import numpy as np
import scipy.sparse as sp
import pytest
import torch

import oracle
from tests.helpers import normwise, sel_rel_err
from workloads.configs import covariance, diff3d, elastic3d, lap2d_32, plant_2x2, random_factors, random_lowrank

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _handle(f, **kw):
    from paper_2609_11363_b300 import Handle
    return Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, **kw)


def _oracle_all(f, m):
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    N = oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, m, S)
    return S, G, N


CASES = {
    "lap2d_tau1e-2": lambda: lap2d_32().factors,
    "lap2d_exact": lambda: lap2d_32(tau=0.0).factors,
    "lap2d_planted2x2": lambda: plant_2x2(lap2d_32().factors, 0.3, 11),
    "random_nonclosed": lambda: random_factors(700, 0.02, 0.15, 5),
    "random_dense_rows": lambda: random_factors(300, 0.25, 0.1, 6, scale=0.1),
    "diff3d_12_planted": lambda: plant_2x2(diff3d(12, m=3).factors, 0.05, 13),
    # 27-point 3-dof elastic-like operator (dense 3x3 blocks, ~100 entries per row of L)
    "elastic3d_8_planted": lambda: plant_2x2(elastic3d(8).factors, 0.05, 17),
    # the covariance-type example (1 - d/3)^4 on a 24 x 24 grid
    "covariance_24": lambda: covariance(24).factors,
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    f = CASES[request.param]()
    m = 3
    S, G, N = _oracle_all(f, m)
    return request.param, f, m, S, G, N


def test_pattern_bit_exact(case):
    name, f, m, S, G, N = case
    h = _handle(f)
    rp, col = h.pattern_host()
    assert np.array_equal(rp, S[0]) and np.array_equal(col, S[1])


@pytest.mark.parametrize("cap", [1, 16])
def test_selinv_fp64(case, cap):
    name, f, m, S, G, N = case
    h = _handle(f, supernode_cap=cap)
    out = h.selinv(_dev(f.L_val), _dev(f.D_packed), "fp64")
    h.sync_status()
    err = sel_rel_err(out.cpu().numpy(), G, *S)
    assert err <= TOL64, (name, err)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_selinv_split_supernodes(case, prec):
    """A small whole-CTA threshold splits every supernode with more than 4 x 64 pairs
    over several CTAs (parts summed in a global block, finished by the last part)."""
    name, f, m, S, G, N = case
    h = _handle(f, big_pairs=64)
    Lv, Dv = _dev(f.L_val), _dev(f.D_packed)
    for _ in range(2):  # the blocks and counts are cleared before every call
        out = h.selinv(Lv, Dv, prec).cpu().numpy()
        h.sync_status()
        if prec == "fp64":
            assert sel_rel_err(out, G, *S) <= TOL64, name
        else:
            assert normwise(out, G) <= 1e-5, name


def test_selinv_repeat_is_deterministic(case):
    name, f, m, S, G, N = case
    h = _handle(f)
    Lv, Dv = _dev(f.L_val), _dev(f.D_packed)
    a = h.selinv(Lv, Dv).cpu().numpy()
    b = h.selinv(Lv, Dv).cpu().numpy()
    h.sync_status()
    assert sel_rel_err(a, G, *S) <= TOL64 and sel_rel_err(b, G, *S) <= TOL64


def test_selinv_fp32(case):
    name, f, m, S, G, N = case
    h = _handle(f)
    out = h.selinv(_dev(f.L_val), _dev(f.D_packed), "fp32")
    h.sync_status()
    assert normwise(out.cpu().numpy(), G) <= 1e-5, name


def _sum_c(f, sn_start):
    """sum over supernodes J of |C_J| (rows of L below J in J's columns)."""
    L = sp.csr_matrix((np.ones(len(f.L_col)), f.L_col, f.L_rowptr), shape=(f.n, f.n)).tocsc()
    tot = 0
    for J in range(len(sn_start) - 1):
        s0, s1 = int(sn_start[J]), int(sn_start[J + 1])
        rows = np.unique(L.indices[L.indptr[s0]:L.indptr[s1]])
        tot += int((rows >= s1).sum())
    return tot


@pytest.mark.parametrize("cap,big", [(1, 0), (16, 0), (4, 64)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_selinv_scan_form(case, cap, big, prec):
    """The scan form (no pair lists: every supernode scans its rows of S_lo against
    a hash table of C) gives the oracle's values, with whole-CTA, per-warp and split
    supernodes; the pairs it finds are exactly the pair lists' (each lower pair
    counted once: lists = 2 x pairs + the diagonals of C)."""
    name, f, m, S, G, N = case
    h = _handle(f, supernode_cap=cap, big_pairs=big, selinv_pair_bytes=-1)
    st = h.stats()
    assert st["selinv_scan"] == 1 and st["hit_pairs"] == 0
    Lv, Dv = _dev(f.L_val), _dev(f.D_packed)
    h.timeline(True)
    for _ in range(2):
        out = h.selinv(Lv, Dv, prec).cpu().numpy()
        h.sync_status()
        if prec == "fp64":
            assert sel_rel_err(out, G, *S) <= TOL64, name
        else:
            assert normwise(out, G) <= 1e-5, name
    look, pairs = h.selinv_scan_counts()
    h.timeline(False)
    ref = _handle(f, supernode_cap=cap, big_pairs=big)
    assert ref.stats()["selinv_scan"] == 0
    sn_start, _ = ref.supernodes()
    assert 2 * pairs + _sum_c(f, sn_start) == ref.stats()["hit_pairs"], name
    assert pairs <= look <= st["scan_rows_total"]


def test_selinv_scan_form_large_C():
    """Rows C of up to ~1,100 per supernode on a dense band: hash tables of C in
    global memory (beyond the shared slots of a warp and of a CTA), global X and Lh."""
    from workloads.configs import band
    f = band(4096, 1100).factors
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    for cap in (1, 4, 16):   # C x w within the shared regions (cap 1, 4) and beyond them (16)
        h = _handle(f, supernode_cap=cap, selinv_pair_bytes=-1)
        assert h.stats()["max_c"] > 1024
        out = h.selinv(_dev(f.L_val), _dev(f.D_packed), "fp64").cpu().numpy()
        h.sync_status()
        assert sel_rel_err(out, G, *S) <= TOL64, cap


def test_selinv_pair_budget_switches_to_scan_form():
    """A pair budget below the lists' size takes the scan form; the default keeps them."""
    f = lap2d_32().factors
    assert _handle(f).stats()["selinv_scan"] == 0
    assert _handle(f, selinv_pair_bytes=1024).stats()["selinv_scan"] == 1


# NInv runs in map form (maps built by the first call of an m, the default) or in
# hash form (no maps); both are checked against the oracle
FORMS = {"map": 0, "hash": -1}


def _check_form(h, form):
    st = h.stats()
    if form == "map":
        assert st["ninv_index_bytes"] > 0 and st["product_hits"] > 0
    else:
        assert st["ninv_index_bytes"] == 0


@pytest.mark.parametrize("form", sorted(FORMS))
@pytest.mark.parametrize("mm", [0, 1, 3])
def test_ninv_fp64(case, mm, form):
    name, f, m, S, G, N = case
    Nr = N if mm == m else oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, mm, S)
    h = _handle(f, ninv_index_bytes=FORMS[form])
    out = h.ninv(_dev(f.L_val), _dev(f.D_packed), mm, "fp64")
    h.sync_status()
    _check_form(h, form)
    err = sel_rel_err(out.cpu().numpy(), Nr, *S)
    assert err <= TOL64, (name, mm, form, err)


@pytest.mark.parametrize("form", sorted(FORMS))
def test_ninv_fp32(case, form):
    name, f, m, S, G, N = case
    h = _handle(f, ninv_index_bytes=FORMS[form])
    out = h.ninv(_dev(f.L_val), _dev(f.D_packed), m, "fp32")
    h.sync_status()
    _check_form(h, form)
    assert normwise(out.cpu().numpy(), N) <= 1e-5, name


@pytest.mark.parametrize("form", sorted(FORMS))
@pytest.mark.parametrize("delta", [1e-3, 1e-2, 1e-1])
def test_ninv_drop(case, delta, form):
    """NInv with the inverse tolerance (off-diagonal |w| < delta dropped after each
    Horner step) against the oracle's dropped series, in every precision form."""
    name, f, m, S, G, N = case
    Nr = oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, m, S, delta=delta)
    h = _handle(f, ninv_index_bytes=FORMS[form])
    Lv, Dv = _dev(f.L_val), _dev(f.D_packed)
    for prec in ("fp64", "fp32x2", "fp32"):
        out = h.ninv(Lv, Dv, m, prec, delta=delta).cpu().numpy()
        h.sync_status()
        if prec == "fp32":
            assert normwise(out, Nr) <= 1e-5, (name, delta, form)
        else:
            assert sel_rel_err(out, Nr, *S) <= TOL64, (name, delta, form, prec)


def test_ninv_drop_rejects_negative_tolerance():
    from paper_2609_11363_b300 import SinvError
    f = lap2d_32().factors
    h = _handle(f)
    with pytest.raises(SinvError):
        h.ninv(_dev(f.L_val), _dev(f.D_packed), 2, delta=-1.0)


@pytest.mark.parametrize("mm", [0, 1, 3])
def test_ninv_fp32x2(case, mm):
    """Product on S in pairs of floats: FP64-class, checked at the FP64 tolerance."""
    name, f, m, S, G, N = case
    Nr = N if mm == m else oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, mm, S)
    h = _handle(f)
    out = h.ninv(_dev(f.L_val), _dev(f.D_packed), mm, "fp32x2")
    h.sync_status()
    _check_form(h, "map")
    err = sel_rel_err(out.cpu().numpy(), Nr, *S)
    assert err <= TOL64, (name, mm, err)


def test_fp32x2_means_fp64_for_selinv_and_lowrank(case):
    name, f, m, S, G, N = case
    h = _handle(f)
    Lv, Dv = _dev(f.L_val), _dev(f.D_packed)
    a = h.selinv(Lv, Dv, "fp32x2").cpu().numpy()
    b = h.selinv(Lv, Dv, "fp64").cpu().numpy()
    h.sync_status()
    assert sel_rel_err(a, G, *S) <= TOL64 and sel_rel_err(b, G, *S) <= TOL64


@pytest.mark.parametrize("prec", ["fp64", "fp32x2"])
def test_ninv_map_form_is_bit_reproducible(case, prec):
    """The FP64 Horner steps sum in exact fixed point and the product reduces in a
    fixed order, so repeated calls agree bit for bit."""
    name, f, m, S, G, N = case
    h = _handle(f)
    Lv, Dv = _dev(f.L_val), _dev(f.D_packed)
    a = h.ninv(Lv, Dv, m, prec).cpu().numpy()
    b = h.ninv(Lv, Dv, m, prec).cpu().numpy()
    h.sync_status()
    assert np.array_equal(a, b), name


def test_ninv_maps_reuse_and_m_change(case):
    """Numeric reruns reuse the maps; a new m rebuilds them (and back)."""
    name, f, m, S, G, N = case
    h = _handle(f)
    Lv, Dv = _dev(f.L_val), _dev(f.D_packed)
    outs = [h.ninv(Lv, Dv, mm).cpu().numpy() for mm in (m, m, 1, m)]
    h.sync_status()
    N1 = oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, 1, S)
    for mm, out in zip((m, m, 1, m), outs):
        assert sel_rel_err(out, N if mm == m else N1, *S) <= TOL64, (name, mm)


def _arrow_factors(n, seed):
    """Column 0 of L full (an arrow): column 0 of the series pattern has n rows, and
    planted 2x2 blocks further down give it partner rows."""
    rows = np.arange(1, n)
    rng = np.random.default_rng(seed)
    L = sp.csr_matrix((rng.uniform(-1e-3, 1e-3, n - 1), (rows, np.zeros(n - 1, dtype=np.int64))), shape=(n, n))
    from workloads.factor import Factors
    f = Factors(n, L.indptr.astype(np.int64), L.indices.astype(np.int32), L.data.copy(), np.ones(n, np.int8),
                np.linspace(1.0, 2.0, n), np.zeros(n), {})
    return plant_2x2(f, 0.1, seed)


@pytest.mark.parametrize("n,form", [(6200, "map"), (17000, "hash")])
def test_ninv_long_columns(n, form):
    """A column longer than the short map tables runs in the long-column launch (map
    form); one longer than the long tables sends the whole call to the hash form."""
    f = _arrow_factors(n, 5)
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    for prec in ("fp64", "fp32x2", "fp32"):
        Nr = oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, 2, S)
        h = _handle(f)
        out = h.ninv(_dev(f.L_val), _dev(f.D_packed), 2, prec)
        h.sync_status()
        _check_form(h, form)
        if prec == "fp32":
            assert normwise(out.cpu().numpy(), Nr) <= 1e-5
        else:
            assert sel_rel_err(out.cpu().numpy(), Nr, *S) <= TOL64, prec


def test_ninv_index_over_budget_runs_hash_form():
    f = plant_2x2(lap2d_32().factors, 0.3, 11)
    S, G, N = _oracle_all(f, 3)
    h = _handle(f, ninv_index_bytes=1)
    out = h.ninv(_dev(f.L_val), _dev(f.D_packed), 3)
    h.sync_status()
    assert h.stats()["ninv_index_bytes"] == 0
    assert sel_rel_err(out.cpu().numpy(), N, *S) <= TOL64


@pytest.mark.parametrize("eps_rule", ["rel", "inf", "neg", "zero"])
def test_mix_bit_exact(case, eps_rule):
    name, f, m, S, G, N = case
    eps = {"rel": 1e-3 * np.max(np.abs(G[S[0][1:] - 1])), "inf": np.inf, "neg": -1.0, "zero": 0.0}[eps_rule]
    h = _handle(f)
    out = h.mix(_dev(G), _dev(N), eps)
    h.sync_status()
    assert np.array_equal(out.cpu().numpy(), oracle.mix(G, N, eps))


@pytest.mark.parametrize("k", [1, 16, 37])
def test_lowrank_fp64(case, k):
    name, f, m, S, G, N = case
    V, lam = random_lowrank(f.n, k, seed=100 + k)
    ref = oracle.lowrank_correct(S[0], S[1], G, V, lam)
    h = _handle(f)
    X = _dev(G.copy())
    h.lowrank_correct(_dev(V), _dev(lam), X, "fp64")
    h.sync_status()
    assert sel_rel_err(X.cpu().numpy(), ref, *S) <= 1e-12


def test_lowrank_fp32(case):
    name, f, m, S, G, N = case
    V, lam = random_lowrank(f.n, 16, seed=7)
    ref = oracle.lowrank_correct(S[0], S[1], G, V, lam)
    h = _handle(f)
    X = _dev(G.copy())
    h.lowrank_correct(_dev(V), _dev(lam), X, "fp32")
    h.sync_status()
    corr = ref - G
    assert normwise(X.cpu().numpy() - G, corr) <= 1e-5


def test_singular_pivot_reported():
    f = lap2d_32().factors
    h = _handle(f)
    D = f.D_packed.copy()
    D[5] = 0.0
    from paper_2609_11363_b300 import SinvError
    h.selinv(_dev(f.L_val), _dev(D))
    with pytest.raises(SinvError) as ei:
        h.sync_status()
    assert ei.value.name == "SINV_ERR_SINGULAR_PIVOT"
    # the handle stays usable
    out = h.selinv(_dev(f.L_val), _dev(f.D_packed))
    h.sync_status()
    S, G, _ = _oracle_all(f, 0)
    assert sel_rel_err(out.cpu().numpy(), G, *S) <= TOL64


def test_bounded_wait_reports_timeout():
    f = lap2d_32().factors
    h = _handle(f, wait_limit=20000)
    assert h.debug_wait_timeout() == 6  # SINV_ERR_TIMEOUT
    out = h.selinv(_dev(f.L_val), _dev(f.D_packed))
    h.sync_status()
    assert torch.isfinite(out).all()


def test_empty_and_tiny():
    from paper_2609_11363_b300 import Handle
    h = Handle(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int8))
    assert h.nnz_S == 0
    f = random_factors(1, 0.0, 0.0, 1)
    S, G, N = _oracle_all(f, 2)
    h = _handle(f)
    out = h.selinv(_dev(f.L_val) if f.nnz_L else torch.zeros(0, dtype=torch.float64, device="cuda"),
                   _dev(f.D_packed))
    h.sync_status()
    assert abs(out.item() - G[0]) <= 1e-15 * abs(G[0])


def test_empty_matrix_every_entry_point():
    """n = 0 through every numeric call of the path: each returns without an error
    and every result is empty (the own-pattern results are the CSC of the empty
    matrix, colptr {0})."""
    from paper_2609_11363_b300 import Handle
    h = Handle(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int8))
    e = torch.zeros(0, dtype=torch.float64, device="cuda")
    lam = torch.ones(4, dtype=torch.float64, device="cuda")
    for prec in ("fp64", "fp32", "fp32x2", "tf32", "bf16"):
        assert h.selinv(e, e, prec).numel() == 0
    for prec in ("fp64", "fp32", "fp32x2"):
        assert h.ninv(e, e, 3, prec).numel() == 0
        assert h.ninv(e, e, 3, prec, delta=1e-2).numel() == 0
        h.lowrank_correct(e, lam, e, prec)
    assert h.ninv_stack(e, e, 2).numel() == 0
    assert h.mix(e, e, 0.5).numel() == 0
    cp, rows, vals, steps = h.ninv_own(e, e, 3, 1e-1)
    assert cp.tolist() == [0] and rows.numel() == 0 and vals.numel() == 0 and steps.tolist() == [0] * 4
    cp, rows, vals = h.mix_own(e, 1e-3)
    assert cp.tolist() == [0] and rows.numel() == 0 and vals.numel() == 0 and h.mix_own_nnz() == 0
    h.lowrank_correct_mix_own(e, lam)
    A = sp.csr_matrix((0, 0))
    h.spai_analyse(A)
    assert h.spai(e, e, 3).numel() == 0
    h.spai_analyse_mix_own(A)
    assert h.spai_mix_own(e, 3).numel() == 0
    h.sync_status()


@pytest.mark.slow
def test_full_size_diff3d_64():
    """The 64^3 shifted diffusion workload at full size, in the benchmark's launch
    configuration: SelInv against the full oracle, NInv on sampled entries."""
    w = diff3d(64)
    f = plant_2x2(w.factors, 0.02, 2)
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    h = _handle(f)
    Lv, Dv = _dev(f.L_val), _dev(f.D_packed)
    out = h.selinv(Lv, Dv, "fp64")
    h.sync_status()
    assert sel_rel_err(out.cpu().numpy(), G, *S) <= TOL64
    N = h.ninv(Lv, Dv, w.m, "fp64").cpu().numpy()
    h.sync_status()
    assert h.stats()["ninv_index_bytes"] > 0  # the benchmark's form
    rng = np.random.default_rng(0)
    idx = rng.choice(len(S[1]), 64, replace=False)
    rows = np.repeat(np.arange(f.n), np.diff(S[0]))
    pairs = list(zip(rows[idx], S[1][idx]))
    Nr = oracle.ninv_entries_sampled(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, w.m, pairs)
    diag = N[S[0][1:] - 1]
    scale = np.abs(Nr) + np.sqrt(np.abs(diag[rows[idx]] * diag[S[1][idx]]))
    assert np.max(np.abs(N[idx] - Nr) / scale) <= TOL64
