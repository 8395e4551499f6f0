"""The all-threads oracle variants (SelInv by level sets, NInv in C over every
host thread) against the plain oracle and against dense definitions, and the
trailing-block sample the CPU baselines time: the oracle on the block equals the
oracle on the whole matrix restricted to the block.  CPU only."""
import numpy as np
import pytest

import oracle
from tests.helpers import sel_rel_err
from workloads.configs import diff3d, lap2d_32, plant_2x2, random_factors, random_lowrank


def _cases():
    return [
        ("lap2d_32_2x2", plant_2x2(lap2d_32().factors, 0.2, 1)),
        ("diff3d_10_2x2", plant_2x2(diff3d(10, m=3).factors, 0.05, 13)),
        ("random_nonclosed", random_factors(300, 0.03, 0.15, 21)),
    ]


@pytest.mark.parametrize("name,f", _cases())
def test_selinv_levels_is_identical_to_selinv(name, f):
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    G2, nlev = oracle.selinv_levels(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    assert np.array_equal(G, G2), name
    assert 1 <= nlev <= f.n


@pytest.mark.parametrize("name,f", _cases())
@pytest.mark.parametrize("m", [0, 1, 2, 4])
def test_ninv_threads_matches_ninv(name, f, m):
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    N = oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, m, S)
    N2 = oracle.ninv_threads(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, m, S)
    assert sel_rel_err(N2, N, *S) <= 1e-12, (name, m)


def test_ninv_threads_matches_dense_truncated_series():
    """An independent pin: W = sum_{t<=m} E^t and W^T D^{-1} W formed densely."""
    f = random_factors(60, 0.08, 0.2, 5)
    n, m = f.n, 3
    L = np.zeros((n, n))
    for i in range(n):
        L[i, f.L_col[f.L_rowptr[i]:f.L_rowptr[i + 1]]] = f.L_val[f.L_rowptr[i]:f.L_rowptr[i + 1]]
    E = -L
    W = np.eye(n)
    P = np.eye(n)
    for _ in range(m):
        P = P @ E
        W = W + P
    D = np.diag(f.d_diag)
    for j in range(n - 1):
        if not f.pivot_start[j + 1] and f.pivot_start[j]:
            D[j + 1, j] = D[j, j + 1] = f.d_off[j]
    Nd = W.T @ np.linalg.inv(D) @ W
    S = oracle.symbolic_S(n, f.L_rowptr, f.L_col, f.pivot_start)
    rows = np.repeat(np.arange(n), np.diff(S[0]))
    want = Nd[rows, S[1]]
    got = oracle.ninv_threads(n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, m, S)
    assert sel_rel_err(got, want, *S) <= 1e-12


def test_trailing_block_values_equal_the_whole_matrix_restricted():
    """The CPU baselines time the oracle on a trailing principal block of the
    workload's factors.  On that block SelInv and NInv give exactly the whole
    matrix's values (the columns of the block have no rows above it)."""
    import bench
    f = plant_2x2(diff3d(10, m=3).factors, 0.05, 13)
    V, lam = random_lowrank(f.n, 4, seed=2)
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    N = oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, 3, S)
    b = bench.trailing_block(f, V, 300)
    c0 = b["c0"]
    assert f.pivot_start[c0] == 1 and b["n"] == f.n - c0 >= 300
    Sb = oracle.symbolic_S(b["n"], b["rp"], b["col"], b["ps"])
    Gb = oracle.selinv(b["n"], b["rp"], b["col"], b["val"], b["ps"], b["dd"], b["do"], Sb)
    Nb = oracle.ninv(b["n"], b["rp"], b["col"], b["val"], b["ps"], b["dd"], b["do"], 3, Sb)
    rows = np.repeat(np.arange(f.n), np.diff(S[0]))
    sel = (rows >= c0) & (S[1] >= c0)
    # the block's S_lo is the whole S_lo restricted to the block, in the same order
    rows_b = np.repeat(np.arange(b["n"]), np.diff(Sb[0]))
    assert np.array_equal(rows[sel] - c0, rows_b) and np.array_equal(S[1][sel] - c0, Sb[1])
    assert np.array_equal(Gb, G[sel])
    assert np.allclose(Nb, N[sel], rtol=1e-13, atol=1e-15 * np.max(np.abs(N)))
    t, nS, parts = bench.oracle_step(b, lam, 3)
    assert nS == 2 * len(Sb[1]) - b["n"] and t > 0
