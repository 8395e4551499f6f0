"""NInv on its own pattern (Section 2.2: delta sparsifies W = L^inv and the
product W^T D^{-1} W) against the oracle's ninv_own.

The pattern is decided in FP64 on both sides from sums in different orders, so
an entry whose magnitude sits at its drop threshold (within 1e-9 relative) may
fall either way; every other entry of the two patterns must agree, and the values
on the common pattern agree within 1e-10 (scaled by |N_ij| + sqrt|N_ii N_jj|, as
the other FP64 NInv tests)."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from workloads.configs import band, diff3d, lap2d_32, plant_2x2, random_factors

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _cases():
    return [("lap2d", lap2d_32().factors), ("diff3d_2x2", plant_2x2(diff3d(10, m=3).factors, 0.05, 13)),
            ("random_2x2", random_factors(400, 0.02, 0.1, 5))]


def _compare(f, m, delta, N, steps):
    R = oracle.ninv_own(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, m, delta)
    W = oracle.ninv_W(f.n, f.L_rowptr, f.L_col, f.L_val, m, delta)
    assert steps[0] == f.n and steps[m] == W.nnz
    d = R.diagonal()
    Rc, Nc = R.tocoo(), N.tocoo()
    ref = {(int(i), int(j)): v for i, j, v in zip(Rc.row, Rc.col, Rc.data)}
    got = {(int(i), int(j)): v for i, j, v in zip(Nc.row, Nc.col, Nc.data)}
    assert all(i >= j for i, j in got)
    for key in set(ref) ^ set(got):      # only entries at the threshold may differ
        v = ref.get(key, got.get(key))
        thr = delta * np.sqrt(abs(d[key[0]] * d[key[1]]))
        assert abs(abs(v) - thr) <= 1e-9 * thr, (key, v, thr)
    common = set(ref) & set(got)
    assert len(common) >= 0.999 * len(ref)
    worst = max(abs(got[k] - ref[k]) / (abs(ref[k]) + np.sqrt(abs(d[k[0]] * d[k[1]]))) for k in common)
    assert worst <= 1e-10, worst


def _gpu(h, f, m, delta):
    cp, rows, vals, steps = h.ninv_own(_dev(f.L_val), _dev(f.D_packed), m, delta)
    h.sync_status()
    cp, rows, vals = cp.cpu().numpy(), rows.cpu().numpy(), vals.cpu().numpy()
    N = sp.csc_matrix((vals, rows, cp), shape=(f.n, f.n))
    N.sort_indices()
    return N, steps


@pytest.mark.parametrize("name,f", _cases(), ids=[c[0] for c in _cases()])
@pytest.mark.parametrize("delta", [1e-1, 1e-2, 1e-3])
def test_ninv_own_matches_oracle(name, f, delta):
    from paper_2609_11363_b300 import Handle
    m = 3
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    N, steps = _gpu(h, f, m, delta)
    _compare(f, m, delta, N, steps)


def test_ninv_own_exact_series_grows_its_buffers():
    """delta = 0 on exact factors: W and the product fill in far beyond the first
    guesses of their output sizes, so every step overflows once, is grown to the
    counted size and runs again."""
    from paper_2609_11363_b300 import Handle
    f = lap2d_32(tau=0.0).factors
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    N, steps = _gpu(h, f, 3, 0.0)
    assert steps[1] > 3 * f.n
    _compare(f, 3, 0.0, N, steps)


def test_ninv_own_long_columns_use_global_tables():
    """A dense band of half-width 256: Horner bounds and product columns beyond the
    shared-memory tables (global slices per CTA)."""
    from paper_2609_11363_b300 import Handle
    f = band(2048, 256).factors
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    for delta in (1e-3, 1e-1):
        N, steps = _gpu(h, f, 2, delta)
        _compare(f, 2, delta, N, steps)


def test_fill_falls_with_delta():
    """Fewer entries in W and in the product as delta grows (the paper's fill
    behaviour), and the diagonal is always there."""
    from paper_2609_11363_b300 import Handle
    f = plant_2x2(diff3d(12, m=3).factors, 0.05, 13)
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    sizes = []
    for delta in (1e-3, 1e-2, 1e-1):
        N, steps = _gpu(h, f, 3, delta)
        assert np.all(N.diagonal() != 0)
        sizes.append((steps[3], N.nnz))
    assert sizes[0][0] > sizes[1][0] > sizes[2][0]
    assert sizes[0][1] > sizes[1][1] > sizes[2][1] >= f.n


@pytest.mark.parametrize("name,f", _cases(), ids=[c[0] for c in _cases()])
@pytest.mark.parametrize("eps_rule", ["rel", "inf", "neg", "zero"])
def test_mix_own_matches_oracle(name, f, eps_rule):
    """Mix on NInv's own pattern (delta = 1e-1, the paper's loose tolerance for Mix):
    given the oracle's SelInv values, every entry of S_eps is SelInv's value bit for
    bit; the rest is the GPU's NInv on its own pattern (as in the NInv test: values
    within 1e-10, and only entries at the drop threshold may differ in pattern)."""
    from paper_2609_11363_b300 import Handle
    m, delta = 3, 1e-1
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    eps = {"rel": 1e-3 * np.abs(G).max(), "inf": np.inf, "neg": -1.0, "zero": 0.0}[eps_rule]
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    h.ninv_own(_dev(f.L_val), _dev(f.D_packed), m, delta)
    cp, rows, vals = h.mix_own(_dev(G), eps)
    h.sync_status()
    M = sp.csc_matrix((vals.cpu().numpy(), rows.cpu().numpy(), cp.cpu().numpy()), shape=(f.n, f.n)).tocoo()
    got = {(int(i), int(j)): v for i, j, v in zip(M.row, M.col, M.data)}
    assert len(got) == M.nnz                      # no duplicate entries
    Nref = oracle.ninv_own(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, m, delta)
    R = oracle.mix_own(f.n, S[0], S[1], G, Nref, eps).tocoo()
    ref = {(int(i), int(j)): v for i, j, v in zip(R.row, R.col, R.data)}
    srow = np.repeat(np.arange(f.n), np.diff(S[0]))
    seps = {(int(i), int(j)): g for i, j, g in zip(srow, S[1], G) if abs(g) > eps}
    for k, g in seps.items():                     # S_eps: SelInv's value, bit for bit
        assert got.get(k) == g, (k, got.get(k), g)
    d = Nref.diagonal()
    for key in set(ref) ^ set(got):               # NInv's entries at its drop threshold
        assert key not in seps
        v = ref.get(key, got.get(key))
        thr = delta * np.sqrt(abs(d[key[0]] * d[key[1]]))
        assert abs(abs(v) - thr) <= 1e-9 * thr, (key, v, thr)
    rest = [k for k in set(ref) & set(got) if k not in seps]
    if rest:
        worst = max(abs(got[k] - ref[k]) / (abs(ref[k]) + np.sqrt(abs(d[k[0]] * d[k[1]]))) for k in rest)
        assert worst <= 1e-10, worst


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_lowrank_on_mix_own_pattern(prec):
    """The rank-k correction of Eq. (9) on the pattern of Mix on NInv's own pattern
    (the configuration of the 3-dof operator: Mix, then the SDDMM correction)."""
    from paper_2609_11363_b300 import Handle
    from workloads.configs import random_lowrank
    f = plant_2x2(diff3d(10, m=3).factors, 0.05, 13)
    m, delta, k = 3, 1e-1, 16
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    eps = 1e-3 * np.abs(G).max()
    V, lam = random_lowrank(f.n, k, seed=7)
    lam = lam * 1e3   # corrections of the size of the entries
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    h.ninv_own(_dev(f.L_val), _dev(f.D_packed), m, delta)
    h.mix_own(_dev(G), eps)
    h.lowrank_correct_mix_own(_dev(V), _dev(lam), prec)
    cp, rows, vals = h.mix_own_result()
    h.sync_status()
    M = sp.csc_matrix((vals.cpu().numpy(), rows.cpu().numpy(), cp.cpu().numpy()), shape=(f.n, f.n)).tocoo()
    got = {(int(i), int(j)): v for i, j, v in zip(M.row, M.col, M.data)}
    Nref = oracle.ninv_own(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, m, delta)
    R = oracle.mix_own(f.n, S[0], S[1], G, Nref, eps)
    Rv = oracle.lowrank_correct(R.indptr.astype(np.int64), R.indices.astype(np.int32), R.data, V, lam)
    Rc = sp.csc_matrix((Rv, R.indices, R.indptr), shape=(f.n, f.n)).tocoo()
    ref = {(int(i), int(j)): v for i, j, v in zip(Rc.row, Rc.col, Rc.data)}
    common = sorted(set(ref) & set(got))
    assert len(common) >= 0.999 * len(ref) and len(common) >= 0.999 * len(got)
    a = np.array([got[c] for c in common])
    b = np.array([ref[c] for c in common])
    if prec == "fp64":
        d = np.abs(R.diagonal())
        scale = np.abs(b) + np.sqrt(np.array([d[i] * d[j] for i, j in common]))
        assert np.max(np.abs(a - b) / scale) <= 1e-10
    else:
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
