"""ORACLE -- test infrastructure only (see the package docstring).

SPAI refinement of an approximate inverse on its own pattern (Section 2.4),
the last stage of Mix-SPAI.  For each column j the values on the fixed
pattern J_j = {i : (i, j) in S} are improved towards

    min || A m_j - e_j ||_2      over m_j supported on J_j,

by diagonally (Jacobi) preconditioned conjugate gradients on the normal
equations  B m = b  with  B = A_J^T A_J  and  b = A_J^T e_j  (A_J = the
columns J_j of A), started from the current values.  The columns are
independent; afterwards the result is symmetrised, (Y + Y^T) / 2.

Readings (the paper gives neither an iteration count nor a stopping rule):
the iteration count ``iters`` is a parameter and every column runs exactly
that many PCG steps, stopping early only when the preconditioned residual
r.z is exactly zero or the curvature p.Bp is not positive; a column of A
with no entries gets a zero preconditioner entry.

Plain dense algebra per column: B is formed explicitly with scipy and every
step is a numpy matrix-vector product or dot product.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def spai_pattern(A, Srp, Sc, power):
    """Lower CSR of P = S united with {(i, j) : dist_A(i, j) <= power}, where
    dist_A is the distance in the graph of A (power 0: P = S).  Boolean matrix
    powers: dist_A(i, j) <= p  iff  ((I + B)^p)_ij != 0, B = pattern of A."""
    n = A.shape[0]
    B = sp.csr_matrix(A, dtype=np.float64, copy=True)
    B.data[:] = 1.0
    R = sp.identity(n, format="csr")
    step = (B + sp.identity(n, format="csr")).tocsr()
    for _ in range(power):
        R = (R @ step).tocsr()
        R.data[:] = 1.0
    S = sp.csr_matrix((np.ones(len(Sc)), np.asarray(Sc), np.asarray(Srp)), shape=(n, n))
    P = sp.tril(S + R, format="csr")
    P.sort_indices()
    return P.indptr.astype(np.int64), P.indices.astype(np.int32)


def embed(Srp, Sc, X_S, Prp, Pc):
    """Values on P_lo from values on S_lo (S is a subset of P): X where (i, j) in S, else 0."""
    n = len(Srp) - 1
    X = sp.csr_matrix((np.asarray(X_S, dtype=np.float64), np.asarray(Sc), np.asarray(Srp)), shape=(n, n))
    rows = np.repeat(np.arange(n), np.diff(Prp))
    return np.asarray(X[rows, np.asarray(Pc)]).ravel()


def _full_pattern(n, Srp, Sc):
    """Column lists of the symmetric pattern S (both triangles), sorted."""
    low = sp.csr_matrix((np.ones(len(Sc)), np.asarray(Sc), np.asarray(Srp)), shape=(n, n))
    full = (low + sp.tril(low, k=-1).T).tocsc()
    full.sort_indices()
    return full.indptr, full.indices


def _sym_values(n, Srp, Sc, X_S):
    low = sp.csr_matrix((np.asarray(X_S, dtype=np.float64), np.asarray(Sc), np.asarray(Srp)), shape=(n, n))
    return (low + sp.tril(low, k=-1).T).tocsc()


def pcg_jacobi(B, b, x0, iters):
    """Jacobi-preconditioned CG on B x = b from x0, exactly ``iters`` steps
    unless r.z == 0 or p.Bp <= 0 stops it first (Hestenes-Stiefel form)."""
    d = np.diag(B).copy()
    dinv = np.where(d != 0.0, 1.0 / np.where(d != 0.0, d, 1.0), 0.0)
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - B @ x
    z = dinv * r
    p = z.copy()
    rz = r @ z
    for _ in range(iters):
        if rz == 0.0:
            break
        q = B @ p
        pq = p @ q
        if not pq > 0.0:
            break
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x


def _column_solver(A, Srp, Sc, X_S):
    """solve(j, iters) -> (J_j, m_j) for one column (see spai_columns)."""
    A = sp.csc_matrix(A, dtype=np.float64)
    Ar = sp.csr_matrix(A)
    n = A.shape[0]
    cp, ri = _full_pattern(n, Srp, Sc)
    X = _sym_values(n, Srp, Sc, X_S)

    def solve(j, iters):
        J = ri[cp[j]:cp[j + 1]]
        AJ = A[:, J]
        B = (AJ.T @ AJ).toarray()
        b = Ar[j, J].toarray().ravel()          # A_J^T e_j: row j of A on the columns J
        x0 = X[:, [j]].toarray().ravel()[J]
        return J, pcg_jacobi(B, b, x0, iters)

    return solve


def spai_columns(A, Srp, Sc, X_S, iters):
    """Per column j: (J_j, m_j) after ``iters`` PCG steps on the normal
    equations of min ||A m - e_j|| over the pattern J_j, started from the
    values of X (symmetric, given by its lower part X_S on S_lo)."""
    solve = _column_solver(A, Srp, Sc, X_S)
    return [solve(j, iters) for j in range(A.shape[0])]


def spai_entries_sampled(A, Srp, Sc, X_S, iters, pairs):
    """spai_refine at the given (i, j) in S_lo only (i >= j), solving just the
    columns those entries need."""
    solve = _column_solver(A, Srp, Sc, X_S)
    cache = {}

    def col(j):
        if j not in cache:
            J, m = solve(j, iters)
            cache[j] = dict(zip(J.tolist(), m.tolist()))
        return cache[j]

    out = np.empty(len(pairs), dtype=np.float64)
    for e, (i, j) in enumerate(pairs):
        i, j = int(i), int(j)
        out[e] = col(j)[i] if i == j else 0.5 * (col(j)[i] + col(i)[j])
    return out


def spai_refine(A, Srp, Sc, X_S, iters):
    """Mix-SPAI's refinement step on S_lo: Y_ij = (m_j[i] + m_i[j]) / 2 for
    (i, j) in S_lo, i > j, and Y_jj = m_j[j]."""
    n = A.shape[0]
    cols = spai_columns(A, Srp, Sc, X_S, iters)
    lookup = [dict(zip(J.tolist(), m.tolist())) for J, m in cols]
    Srp = np.asarray(Srp); Sc = np.asarray(Sc)
    Y = np.empty(len(Sc), dtype=np.float64)
    for i in range(n):
        for p in range(Srp[i], Srp[i + 1]):
            j = int(Sc[p])
            Y[p] = lookup[j][i] if i == j else 0.5 * (lookup[j][i] + lookup[i][j])
    return Y
