"""ORACLE -- test infrastructure only (see the package docstring).

FP64 throughout.  Functions take the factors as plain arrays: L strictly lower
CSR (int64 rowptr, int32 col, float64 val, unit diagonal implied), the pivot
layout ``pivot_start`` (int8[n], 1 = a pivot block starts here, a block is 2x2
iff the next flag is 0) and D as ``d_diag[n]`` / ``d_off[n]`` (``d_off[j]`` =
D(j+1, j) for the first index of a 2x2 block).  Every result on S is an array
in S_lo CSR order (row i, columns j <= i ascending).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "csrc", f) for f in ("selinv_ref.c", "ninv_ref.c")]
_LIB = os.path.join(_HERE, "_selinv_ref.so")
_lib = None


def build_lib(force: bool = False) -> str:
    """Compile the C part of the oracle in place (gcc -O2, OpenMP for the
    all-threads baseline variants)."""
    newest = max(os.path.getmtime(f) for f in _SRCS + [__file__])
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-fopenmp", "-shared", "-o", tmp] + _SRCS)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_lib())
        P = ctypes.c_void_p
        lib.oracle_selinv.argtypes = [ctypes.c_int64, P, P, P, P, P, P, P, P, P, ctypes.c_int64]
        lib.oracle_selinv.restype = ctypes.c_int
        lib.oracle_selinv_levels.argtypes = [ctypes.c_int64, P, P, P, P, P, P, P, P, P, P]
        lib.oracle_selinv_levels.restype = ctypes.c_int
        lib.oracle_ninv_threads.argtypes = [ctypes.c_int64, P, P, P, P, P, P, ctypes.c_int, P, P, P]
        lib.oracle_ninv_threads.restype = ctypes.c_int
        lib.oracle_selinv_blocks.argtypes = [ctypes.c_int64, P, P, P, P, P, P, P, P, P, P, ctypes.c_int64]
        lib.oracle_selinv_blocks.restype = ctypes.c_int
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def host_threads() -> int:
    """Threads the all-threads variants use (OpenMP's default: every host core)."""
    return int(_load().oracle_threads())


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# pattern S (Section 1: S = {(i,j): (L + D + L^T)_ij != 0})
# --------------------------------------------------------------------------
def _two_by_two_starts(pivot_start):
    ps = np.asarray(pivot_start).astype(bool)
    n = len(ps)
    two = np.zeros(n, dtype=bool)
    two[:-1] = ps[:-1] & ~ps[1:]
    return np.nonzero(two)[0]


def symbolic_S(n, L_rowptr, L_col, pivot_start):
    """Lower part S_lo of S = pattern(L + D + L^T): (rowptr int64, col int32).

    Structural: every stored entry of L counts, the diagonal always, and
    (j+1, j) for each 2x2 block of D.
    """
    L = sp.csr_matrix((np.ones(len(L_col)), np.asarray(L_col), np.asarray(L_rowptr)), shape=(n, n))
    t = _two_by_two_starts(pivot_start)
    Dp = sp.csr_matrix((np.ones(n + len(t)), (np.concatenate([np.arange(n), t + 1]),
                                               np.concatenate([np.arange(n), t]))), shape=(n, n))
    M = (L + Dp).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    return M.indptr.astype(np.int64), M.indices.astype(np.int32)


def _S_entries(Srp, Sc):
    rows = np.repeat(np.arange(len(Srp) - 1), np.diff(Srp))
    return rows, np.asarray(Sc, dtype=np.int64)


# --------------------------------------------------------------------------
# SelInv (Section 2.1)
# --------------------------------------------------------------------------
def selinv(n, L_rowptr, L_col, L_val, pivot_start, d_diag, d_off, S=None, stop_col=0):
    """Selected inverse on S by the scalar recurrence (C implementation).

    ``stop_col > 0`` runs only the pivot blocks starting at or after it (the last
    part of the recurrence), for timing a bounded sample; other entries stay 0.
    """
    lib = _load()
    if S is None:
        S = symbolic_S(n, L_rowptr, L_col, pivot_start)
    Srp, Sc = S
    Lcsc = sp.csr_matrix((np.asarray(L_val, dtype=np.float64), L_col, L_rowptr), shape=(n, n)).tocsc()
    Lcsc.sort_indices()
    cp = Lcsc.indptr.astype(np.int64); r = Lcsc.indices.astype(np.int32); v = Lcsc.data.astype(np.float64)
    ps = np.ascontiguousarray(pivot_start, dtype=np.int8)
    dd = np.ascontiguousarray(d_diag, dtype=np.float64)
    do = np.ascontiguousarray(d_off, dtype=np.float64)
    Srp = np.ascontiguousarray(Srp, dtype=np.int64); Sc = np.ascontiguousarray(Sc, dtype=np.int32)
    G = np.zeros(len(Sc))
    rc = lib.oracle_selinv(n, _p(cp), _p(r), _p(v), _p(ps), _p(dd), _p(do), _p(Srp), _p(Sc), _p(G), int(stop_col))
    if rc == -2:
        raise ZeroDivisionError("singular pivot block")
    if rc != 0:
        raise MemoryError("oracle_selinv failed")
    return G


def _csc_L(n, L_rowptr, L_col, L_val):
    Lcsc = sp.csr_matrix((np.asarray(L_val, dtype=np.float64), L_col, L_rowptr), shape=(n, n)).tocsc()
    Lcsc.sort_indices()
    return Lcsc.indptr.astype(np.int64), Lcsc.indices.astype(np.int32), Lcsc.data.astype(np.float64)


def selinv_levels(n, L_rowptr, L_col, L_val, pivot_start, d_diag, d_off, S=None):
    """``selinv`` scheduled by level sets over every host thread (the all-cores
    CPU baseline).  Each pivot block does the same arithmetic as
    in ``selinv``, so the result is identical to it.  Returns (G, levels)."""
    lib = _load()
    if S is None:
        S = symbolic_S(n, L_rowptr, L_col, pivot_start)
    cp, r, v = _csc_L(n, L_rowptr, L_col, L_val)
    ps = np.ascontiguousarray(pivot_start, dtype=np.int8)
    dd = np.ascontiguousarray(d_diag, dtype=np.float64)
    do = np.ascontiguousarray(d_off, dtype=np.float64)
    Srp = np.ascontiguousarray(S[0], dtype=np.int64); Sc = np.ascontiguousarray(S[1], dtype=np.int32)
    G = np.zeros(len(Sc))
    nlev = np.zeros(1, dtype=np.int64)
    rc = lib.oracle_selinv_levels(n, _p(cp), _p(r), _p(v), _p(ps), _p(dd), _p(do), _p(Srp), _p(Sc), _p(G),
                                  _p(nlev))
    if rc == -2:
        raise ZeroDivisionError("singular pivot block")
    if rc != 0:
        raise MemoryError("oracle_selinv_levels failed")
    return G, int(nlev[0])


def selinv_blocks(n, L_rowptr, L_col, L_val, pivot_start, d_diag, d_off, S, G, blocks):
    """The scalar recurrence of ``selinv`` on the listed pivot blocks only (each by
    its first column), in the order given, on G in place (S_lo order): the entries
    the listed blocks read must already be in G.  For checking a partition of the
    recurrence."""
    lib = _load()
    cp, r, v = _csc_L(n, L_rowptr, L_col, L_val)
    ps = np.ascontiguousarray(pivot_start, dtype=np.int8)
    dd = np.ascontiguousarray(d_diag, dtype=np.float64)
    do = np.ascontiguousarray(d_off, dtype=np.float64)
    Srp = np.ascontiguousarray(S[0], dtype=np.int64); Sc = np.ascontiguousarray(S[1], dtype=np.int32)
    bl = np.ascontiguousarray(blocks, dtype=np.int64)
    assert G.dtype == np.float64 and G.flags.c_contiguous and len(G) == len(Sc)
    rc = lib.oracle_selinv_blocks(n, _p(cp), _p(r), _p(v), _p(ps), _p(dd), _p(do), _p(Srp), _p(Sc), _p(G),
                                  _p(bl), len(bl))
    if rc == -2:
        raise ZeroDivisionError("singular pivot block")
    if rc != 0:
        raise MemoryError("oracle_selinv_blocks failed")
    return G


def ninv_W_columns(n, L_rowptr, L_col, L_val, m, cols, W_known=None):
    """Columns ``cols`` of W = sum_{t<=m} E^t (no dropping) by the column form of
    the Horner steps, W_t[:, j] = e_j + sum_{k in struct(j)} E_kj W_{t-1}[:, k]
    (Eq. (6)).  The columns it reads but does not compute come from ``W_known``:
    {column: {t: {row: value}}} for every step t = 0..m.  Plain dictionaries,
    small n.  Returns {t: {column: {row: value}}} for the computed and the known
    columns."""
    E = _E(n, L_rowptr, L_col, L_val).tocsc()
    cols = sorted(set(int(c) for c in cols), reverse=True)
    steps = {0: {}}
    known = W_known or {}
    for t in range(m + 1):
        steps.setdefault(t, {})
        for j, per_t in known.items():
            steps[t][j] = dict(per_t[t])
    for j in cols:
        steps[0][j] = {j: 1.0}
    for t in range(1, m + 1):
        for j in cols:   # a column reads columns k > j of the previous step only
            col = {j: 1.0}
            for q in range(E.indptr[j], E.indptr[j + 1]):
                k = int(E.indices[q])
                e = float(E.data[q])
                for r, w in steps[t - 1][k].items():
                    col[r] = col.get(r, 0.0) + e * w
            steps[t][j] = col
    return steps


def ninv_threads(n, L_rowptr, L_col, L_val, pivot_start, d_diag, d_off, m, S=None):
    """``ninv`` (delta = 0) in plain C over every host thread: the Horner
    columns and the entries of the product are independent (the all-cores CPU
    baseline).  Agrees with ``ninv`` to rounding."""
    lib = _load()
    if S is None:
        S = symbolic_S(n, L_rowptr, L_col, pivot_start)
    cp, r, v = _csc_L(n, L_rowptr, L_col, L_val)
    ps = np.ascontiguousarray(pivot_start, dtype=np.int8)
    dd = np.ascontiguousarray(d_diag, dtype=np.float64)
    do = np.ascontiguousarray(d_off, dtype=np.float64)
    Srp = np.ascontiguousarray(S[0], dtype=np.int64); Sc = np.ascontiguousarray(S[1], dtype=np.int32)
    N = np.zeros(len(Sc))
    rc = lib.oracle_ninv_threads(n, _p(cp), _p(r), _p(v), _p(ps), _p(dd), _p(do), int(m), _p(Srp), _p(Sc),
                                 _p(N))
    if rc == -2:
        raise ZeroDivisionError("singular pivot block")
    if rc != 0:
        raise MemoryError("oracle_ninv_threads failed")
    return N


# --------------------------------------------------------------------------
# NInv (Section 2.2)
# --------------------------------------------------------------------------
def _E(n, L_rowptr, L_col, L_val):
    """E_L with L = I - E_L: E_L = -(strict lower part of L)."""
    return sp.csr_matrix((-np.asarray(L_val, dtype=np.float64), L_col, L_rowptr), shape=(n, n))


def _Dinv(n, pivot_start, d_diag, d_off):
    """D^{-1} as a sparse block-diagonal matrix (1x1 and 2x2 blocks)."""
    rows, cols, vals = [], [], []
    ps = np.asarray(pivot_start).astype(bool)
    j = 0
    while j < n:
        if j + 1 < n and not ps[j + 1]:
            a, b, d = d_diag[j], d_off[j], d_diag[j + 1]
            inv = np.linalg.inv(np.array([[a, b], [b, d]]))
            rows += [j, j, j + 1, j + 1]; cols += [j, j + 1, j, j + 1]; vals += list(inv.ravel())
            j += 2
        else:
            rows.append(j); cols.append(j); vals.append(1.0 / d_diag[j])
            j += 1
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def _drop_offdiag(W, delta):
    """Section 2.2's inverse tolerance (reading: after each Horner step, the
    off-diagonal entries with |w| < delta are dropped)."""
    W = W.tocoo()
    keep = (W.row == W.col) | (np.abs(W.data) >= delta)
    return sp.csr_matrix((W.data[keep], (W.row[keep], W.col[keep])), shape=W.shape)


def ninv_W(n, L_rowptr, L_col, L_val, m, delta=0.0):
    """W = sum_{t=0}^{m} E_L^t (Eq. (6) truncated after the m-th power).

    Horner steps in column form, W_t = I + W_{t-1} E_L: column j of W_t is e_j
    plus E_kj times column k of W_{t-1} for the rows k of column j of E_L (the
    identity Z = I + Z E_L of Z = L^{-1}).  Without dropping this is the same sum
    as I + E_L W_{t-1}; with delta > 0 every step drops its off-diagonal entries
    below delta, and the two orders differ, so the column form is the reading.
    """
    E = _E(n, L_rowptr, L_col, L_val)
    I = sp.identity(n, format="csr")
    W = I.copy()
    for _ in range(m):
        W = (I + W @ E).tocsr()  # Horner: W_t = I + W_{t-1} E
        if delta > 0:
            W = _drop_offdiag(W, delta)
    W.sort_indices()
    return W


def ninv(n, L_rowptr, L_col, L_val, pivot_start, d_diag, d_off, m, S=None, chunk=1 << 20, delta=0.0):
    """NInv on S: N_ij = (W^T D^{-1} W)_ij for (i, j) in S_lo (Eq. (8)).

    W is the truncated series, exact for delta = 0, else with each Horner
    step's off-diagonal entries below delta dropped (ninv_W); the product is
    evaluated exactly on S, entry by entry as the dot product of column i of W
    with column j of D^{-1} W.
    """
    if S is None:
        S = symbolic_S(n, L_rowptr, L_col, pivot_start)
    W = ninv_W(n, L_rowptr, L_col, L_val, m, delta)
    Y = (_Dinv(n, pivot_start, d_diag, d_off) @ W).tocsr()
    Wt = W.T.tocsr(); Yt = Y.T.tocsr()
    rows, cols = _S_entries(*S)
    out = np.empty(len(rows))
    for s in range(0, len(rows), chunk):
        e = min(s + chunk, len(rows))
        out[s:e] = np.asarray(Wt[rows[s:e]].multiply(Yt[cols[s:e]]).sum(axis=1)).ravel()
    return out


def ninv_own(n, L_rowptr, L_col, L_val, pivot_start, d_diag, d_off, m, delta):
    """NInv on its own pattern (Section 2.2, Eq. (8)): W = ninv_W(m, delta) (the
    series with off-diagonal |w| < delta dropped after every Horner step), then
    N = W^T D^{-1} W, whose fill delta also controls.  Reading of the product's
    drop: an off-diagonal entry is dropped when |N_ij| < delta sqrt(|N_ii N_jj|)
    (relative to the diagonal, as N carries D^{-1}'s scale); the diagonal is
    always kept.  Returns the lower triangle (i >= j) as a CSC matrix with
    sorted rows."""
    W = ninv_W(n, L_rowptr, L_col, L_val, m, delta)
    Y = (_Dinv(n, pivot_start, d_diag, d_off) @ W).tocsc()
    N = sp.tril((W.T @ Y).tocsc()).tocoo()
    d = np.asarray((W.T @ Y).diagonal())
    keep = (N.row == N.col) | (np.abs(N.data) >= delta * np.sqrt(np.abs(d[N.row] * d[N.col])))
    out = sp.csc_matrix((N.data[keep], (N.row[keep], N.col[keep])), shape=(n, n))
    out.sort_indices()
    return out


def ninv_entries_sampled(n, L_rowptr, L_col, L_val, pivot_start, d_diag, d_off, m, pairs, delta=0.0):
    """N_ij for a list of (i, j) pairs, one at a time.

    delta = 0 (any n): column c of W is sum_t E^t e_c, built from sparse
    matrix-vector products.  delta > 0 (small n): the column form of ninv_W,
    column c of W_t = e_c + sum_{k in struct(c)} E_kc W_{t-1}[:, k] with the
    off-diagonal entries below delta dropped, by memoised recursion over the
    columns it reaches.
    """
    E = _E(n, L_rowptr, L_col, L_val).tocsc()
    Dinv = _Dinv(n, pivot_start, d_diag, d_off).tocsc()

    def unit(c):
        return sp.csc_matrix(([1.0], ([c], [0])), shape=(n, 1))

    memo = {}

    def wcol_drop(c, t):
        if t == 0:
            return unit(c)
        key = (c, t)
        if key not in memo:
            w = unit(c)
            for q in range(E.indptr[c], E.indptr[c + 1]):
                w = w + E.data[q] * wcol_drop(int(E.indices[q]), t - 1)
            w = w.tocoo()
            keep = (w.row == c) | (np.abs(w.data) >= delta)
            memo[key] = sp.coo_matrix((w.data[keep], (w.row[keep], w.col[keep])), shape=(n, 1)).tocsc()
        return memo[key]

    def wcol(c):
        if delta > 0:
            return wcol_drop(c, m)
        e = unit(c)
        w = e.copy()
        for _ in range(m):
            w = (e + E @ w).tocsc()
        return w

    out = np.empty(len(pairs))
    for k, (i, j) in enumerate(pairs):
        wi = wcol(int(i)); yj = Dinv @ wcol(int(j))
        out[k] = float((wi.multiply(yj)).sum())
    return out


# --------------------------------------------------------------------------
# Mix (Section 2.3) and low-rank correction (Sections 2.5-2.6)
# --------------------------------------------------------------------------
def mix(G_S, N_S, eps):
    """(A_Mix)_ij = SelInv_ij where |SelInv_ij| > eps (the set S_eps), else NInv_ij."""
    G_S = np.asarray(G_S); N_S = np.asarray(N_S)
    return np.where(np.abs(G_S) > eps, G_S, N_S)


def mix_own(n, Srp, Sc, G_S, N_lo, eps):
    """Mix on NInv's own pattern (Section 2.3): S_eps = {(i, j) in S_lo : |G_ij| > eps};
    (A_Mix)_ij = G_ij on S_eps and N_ij elsewhere on N's pattern, so the pattern
    is the union of N's pattern and S_eps.  G_S: values on S_lo (CSR order of
    Srp, Sc); N_lo: the lower triangle of NInv on its own pattern (any sparse
    format).  Returns the lower triangle as a CSC matrix with sorted rows;
    entries are kept as stored (an explicit zero of N stays an entry)."""
    G_S = np.asarray(G_S, dtype=np.float64)
    rows, cols = _S_entries(Srp, Sc)
    sel = np.abs(G_S) > eps
    Nc = sp.coo_matrix(N_lo)
    out = {}
    for i, j, v in zip(Nc.row.tolist(), Nc.col.tolist(), Nc.data.tolist()):
        out[(i, j)] = v
    for i, j, g in zip(rows[sel].tolist(), cols[sel].tolist(), G_S[sel].tolist()):
        out[(i, j)] = g
    if not out:
        return sp.csc_matrix((n, n))
    ij = np.array(list(out.keys()), dtype=np.int64)
    M = sp.csc_matrix((np.array(list(out.values())), (ij[:, 0], ij[:, 1])), shape=(n, n))
    M.sort_indices()
    return M


def lowrank_correct(Srp, Sc, X_S, V, lam):
    """(A^inv + V diag(lam) V^T)_ij for (i, j) in S_lo (Eq. (9))."""
    rows, cols = _S_entries(Srp, Sc)
    V = np.asarray(V, dtype=np.float64).reshape(len(Srp) - 1, -1)
    lam = np.asarray(lam, dtype=np.float64)
    out = np.array(X_S, dtype=np.float64, copy=True)
    if V.shape[1] == 0:
        return out
    chunk = 1 << 18
    for s in range(0, len(rows), chunk):
        e = min(s + chunk, len(rows))
        out[s:e] += np.einsum("el,l,el->e", V[rows[s:e]], lam, V[cols[s:e]])
    return out


def lowrank_diag(d_hat, V, lam):
    """Diagonal update d^k_i = d_i + sum_j lam_j v_ij^2 (Section 2.6)."""
    V = np.asarray(V, dtype=np.float64)
    return np.asarray(d_hat, dtype=np.float64) + (V * V) @ np.asarray(lam, dtype=np.float64)


# --------------------------------------------------------------------------
# spectral correction producer (Section 2.5): Lanczos on E_inv
# --------------------------------------------------------------------------
def sym_from_S(n, Srp, Sc, X_S):
    """The symmetric n x n sparse matrix whose lower part is X_S on S_lo."""
    low = sp.csr_matrix((np.asarray(X_S, dtype=np.float64), Sc, Srp), shape=(n, n))
    strict = sp.tril(low, k=-1)
    return (low + strict.T).tocsr()


def lanczos_einv(A, Ainv_sym, k, steps=None, seed=0, solve=None, q0=None):
    """k dominant (largest |lambda|) eigenpairs of E_inv = A^{-1} - A^inv.

    Matrix-free as in Section 2.5: E_inv x = A^{-1} x - A^inv x.  The first term
    is an exact sparse LU solve here (the paper uses an ILDL-preconditioned
    Krylov solve; the oracle wants the exact operator).  Lanczos with full
    reorthogonalisation, Ritz pairs of the tridiagonal matrix.
    """
    n = A.shape[0]
    if solve is None:
        lu = spla.splu(sp.csc_matrix(A))
        solve = lu.solve
    steps = min(n, steps or max(4 * k + 20, 60))
    Q = np.zeros((n, steps + 1))
    alpha = np.zeros(steps); beta = np.zeros(steps)
    q = np.random.default_rng(seed).standard_normal(n) if q0 is None else np.array(q0, dtype=np.float64)
    q /= np.linalg.norm(q)
    Q[:, 0] = q
    m = steps
    for it in range(steps):
        v = solve(Q[:, it]) - Ainv_sym @ Q[:, it]
        alpha[it] = Q[:, it] @ v
        v -= Q[:, : it + 1] @ (Q[:, : it + 1].T @ v)
        v -= Q[:, : it + 1] @ (Q[:, : it + 1].T @ v)
        b = np.linalg.norm(v)
        beta[it] = b
        if b < 1e-14 * max(1.0, abs(alpha[it])):
            m = it + 1
            break
        Q[:, it + 1] = v / b
    T = np.diag(alpha[:m]) + np.diag(beta[: m - 1], 1) + np.diag(beta[: m - 1], -1)
    th, U = np.linalg.eigh(T)
    order = np.argsort(-np.abs(th))[:k]
    lam = th[order]
    V = Q[:, :m] @ U[:, order]
    return lam, V


# --------------------------------------------------------------------------
# measures (Sections 2.6 and 3.2)
# --------------------------------------------------------------------------
def err1(d, d_hat):
    """err_1 = ||d - d_hat||_1 / ||d||_1."""
    d = np.asarray(d); d_hat = np.asarray(d_hat)
    return float(np.abs(d - d_hat).sum() / np.abs(d).sum())


def fill_fact(nnz_S_full, nnz_A):
    """nnz(L + D + L^T) / nnz(A)."""
    return nnz_S_full / nnz_A


def fill_inv(nnz_Ainv, nnz_A):
    return nnz_Ainv / nnz_A


def dodd(A):
    """Degree of diagonal dominance min_i |a_ii| / sum_{j != i} |a_ij|."""
    A = sp.csr_matrix(A)
    d = np.abs(A.diagonal())
    off = np.asarray(abs(A).sum(axis=1)).ravel() - d
    with np.errstate(divide="ignore"):
        return float(np.min(np.where(off > 0, d / off, np.inf)))


def accept_modes(d_exact, d_hat, V, lam):
    """Acceptance safeguard of Algorithm 1 step 6: modes in |lambda| order, each
    kept only if it lowers the diagonal error ||err_cand||_1 < ||err_base||_1."""
    order = np.argsort(-np.abs(lam))
    kept = []
    cur = np.asarray(d_hat, dtype=np.float64).copy()
    base = np.abs(d_exact - cur).sum()
    for l in order:
        cand = cur + lam[l] * V[:, l] ** 2
        e = np.abs(d_exact - cand).sum()
        if e < base:
            kept.append(int(l)); cur = cand; base = e
    return kept, cur
