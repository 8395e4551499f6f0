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


def spai_columns(A, Srp, Sc, X_S, iters):
    """Per column j: (J_j, m_j) after ``iters`` PCG steps on the normal
    equations of min ||A m - e_j|| over the pattern J_j, started from the
    values of X (symmetric, given by its lower part X_S on S_lo)."""
    A = sp.csc_matrix(A, dtype=np.float64)
    Ar = sp.csr_matrix(A)
    n = A.shape[0]
    cp, ri = _full_pattern(n, Srp, Sc)
    X = _sym_values(n, Srp, Sc, X_S)
    out = []
    for j in range(n):
        J = ri[cp[j]:cp[j + 1]]
        AJ = A[:, J]
        B = (AJ.T @ AJ).toarray()
        b = Ar[j, J].toarray().ravel()          # A_J^T e_j: row j of A on the columns J
        x0 = X[:, [j]].toarray().ravel()[J]
        out.append((J, pcg_jacobi(B, b, x0, iters)))
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
