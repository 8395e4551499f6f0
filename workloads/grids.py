"""Seeded synthetic sparse symmetric matrices shaped like the paper's test set.

The paper measures on SuiteSparse structural/PDE matrices (Section 3, test-matrix
table) that are not available here; these closed-form generators stand in for
them.  Every random number is drawn from ``numpy.random.default_rng(seed)``
(PCG64) in the order documented on each function, so the matrices are
bit-reproducible.  Nothing in this module computes any part of the selected
inverse: it only builds the matrix A whose factors are the inputs.

Node numbering is natural (x fastest): ``i = x + nx*(y + ny*z)``; a node with
several degrees of freedom owns the consecutive indices ``dof*i .. dof*i+dof-1``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _rng(seed):
    """``seed`` is an int (a fresh PCG64 stream) or a Generator to continue."""
    return seed if isinstance(seed, np.random.Generator) else np.random.default_rng(seed)


def _coo_to_csr(rows, cols, vals, n):
    A = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def laplace2d_5pt(nx: int, ny: int, diag_shift: float = 0.1) -> sp.csr_matrix:
    """2D 5-point Dirichlet Laplacian plus ``diag_shift * I``.

    a_ii = 4 + diag_shift, a_ij = -1 for grid neighbours.  SPD.  nnz = 5n - 2(nx+ny).
    No random numbers.
    """
    n = nx * ny
    idx = np.arange(n).reshape(ny, nx)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [np.full(n, 4.0 + diag_shift)]
    for a, b in ((idx[:, :-1], idx[:, 1:]), (idx[:-1, :], idx[1:, :])):
        a = a.ravel(); b = b.ravel()
        rows += [a, b]; cols += [b, a]; vals += [-np.ones(a.size), -np.ones(a.size)]
    return _coo_to_csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)


def diffusion3d_7pt(nx: int, ny: int, nz: int, seed, sigma: float = 1.0) -> sp.csr_matrix:
    """3D 7-point cell-centred diffusion with log-normal cell coefficients.

    Draws: ``g = rng.standard_normal(n)`` in natural cell order; kappa = exp(sigma*g).
    Interior face coefficient = harmonic mean 2 k1 k2 / (k1 + k2); a Dirichlet
    boundary face contributes the cell's own kappa to the diagonal.
    a_ij = -face, a_ii = sum of the cell's face coefficients.  SPD.
    nnz = 7n - 2(nx ny + ny nz + nx nz).
    """
    rng = _rng(seed)
    n = nx * ny * nz
    kappa = np.exp(sigma * rng.standard_normal(n)).reshape(nz, ny, nx)
    idx = np.arange(n).reshape(nz, ny, nx)
    diag = np.zeros((nz, ny, nx))
    rows, cols, vals = [], [], []
    for axis in (2, 1, 0):  # x, y, z faces
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[axis] = slice(None, -1)
        sl_hi[axis] = slice(1, None)
        k1 = kappa[tuple(sl_lo)]
        k2 = kappa[tuple(sl_hi)]
        face = 2.0 * k1 * k2 / (k1 + k2)
        diag[tuple(sl_lo)] += face
        diag[tuple(sl_hi)] += face
        a = idx[tuple(sl_lo)].ravel(); b = idx[tuple(sl_hi)].ravel(); f = face.ravel()
        rows += [a, b]; cols += [b, a]; vals += [-f, -f]
        # Dirichlet boundary faces on both ends of this axis
        first = [slice(None)] * 3; first[axis] = 0
        last = [slice(None)] * 3; last[axis] = -1
        diag[tuple(first)] += kappa[tuple(first)]
        diag[tuple(last)] += kappa[tuple(last)]
    rows.append(idx.ravel()); cols.append(idx.ravel()); vals.append(diag.ravel())
    return _coo_to_csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)


def random9pt_2d(nx: int, ny: int, seed) -> sp.csr_matrix:
    """2D 9-point random-weight graph Laplacian with Dirichlet ghost edges.

    Draws: ``g = rng.standard_normal((4, ny+2, nx+2))``; edge weights w = exp(g)
    live on the grid padded by one ghost layer, one per node of the padded grid
    and forward direction d in [(1,0), (0,1), (1,1), (1,-1)] (index order of the
    first axis), the edge joining padded node (X, Y) to (X+dx, Y+dy).  Edges with
    both ends interior give a_ij = -w; every edge with an interior end adds w to
    that end's diagonal.  SPD.  nnz = (3nx-2)(3ny-2).
    """
    rng = _rng(seed)
    w = np.exp(rng.standard_normal((4, ny + 2, nx + 2)))
    n = nx * ny
    # padded index -> interior index or -1
    pid = -np.ones((ny + 2, nx + 2), dtype=np.int64)
    pid[1:-1, 1:-1] = np.arange(n).reshape(ny, nx)
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    Y, X = np.meshgrid(np.arange(ny + 2), np.arange(nx + 2), indexing="ij")
    for d, (dx, dy) in enumerate(((1, 0), (0, 1), (1, 1), (1, -1))):
        X2 = X + dx; Y2 = Y + dy
        ok = (X2 >= 0) & (X2 < nx + 2) & (Y2 >= 0) & (Y2 < ny + 2)
        a = pid[Y[ok], X[ok]]
        b = pid[Y2[ok], X2[ok]]
        ww = w[d][ok]
        ma = a >= 0
        mb = b >= 0
        np.add.at(diag, a[ma], ww[ma])
        np.add.at(diag, b[mb], ww[mb])
        both = ma & mb
        rows += [a[both], b[both]]; cols += [b[both], a[both]]; vals += [-ww[both], -ww[both]]
    rows.append(np.arange(n)); cols.append(np.arange(n)); vals.append(diag)
    return _coo_to_csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)


def elastic3d_27pt(nx: int, ny: int, nz: int, seed) -> sp.csr_matrix:
    """3D 27-point lattice-spring operator with 3 degrees of freedom per node.

    Each of the 13 forward neighbour directions d (all (dx,dy,dz) in {-1,0,1}^3
    that are lexicographically positive, in lexicographic order of (dz, dy, dx))
    joins node p to p+d with a 3x3 block K = w (0.1 I + u u^T), u = d/|d|.
    Draws: ``g = rng.standard_normal((13, nz+2, ny+2, nx+2))``; w = exp(g) per
    padded node and direction.  Assembly is the block graph Laplacian: off-diagonal
    block -K, and K added to the diagonal block of every interior end (ghost ends
    are Dirichlet).  Every neighbour pair stores its full 3x3 block (explicit
    zeros kept), so nnz = 9 (3nx-2)(3ny-2)(3nz-2).  SPD.
    """
    rng = _rng(seed)
    dirs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
            if (dz, dy, dx) > (0, 0, 0)]
    assert len(dirs) == 13
    w = np.exp(rng.standard_normal((13, nz + 2, ny + 2, nx + 2)))
    nn = nx * ny * nz
    n = 3 * nn
    pid = -np.ones((nz + 2, ny + 2, nx + 2), dtype=np.int64)
    pid[1:-1, 1:-1, 1:-1] = np.arange(nn).reshape(nz, ny, nx)
    Z, Y, X = np.meshgrid(np.arange(nz + 2), np.arange(ny + 2), np.arange(nx + 2), indexing="ij")
    dblk = np.zeros((nn, 3, 3))
    rows, cols, vals = [], [], []
    for d, (dx, dy, dz) in enumerate(dirs):
        u = np.array([dx, dy, dz], dtype=np.float64)
        u /= np.linalg.norm(u)
        K0 = 0.1 * np.eye(3) + np.outer(u, u)
        X2 = X + dx; Y2 = Y + dy; Z2 = Z + dz
        ok = (X2 >= 0) & (X2 < nx + 2) & (Y2 >= 0) & (Y2 < ny + 2) & (Z2 >= 0) & (Z2 < nz + 2)
        a = pid[Z[ok], Y[ok], X[ok]]
        b = pid[Z2[ok], Y2[ok], X2[ok]]
        ww = w[d][ok]
        ma = a >= 0
        mb = b >= 0
        np.add.at(dblk, a[ma], ww[ma, None, None] * K0)
        np.add.at(dblk, b[mb], ww[mb, None, None] * K0)
        both = ma & mb
        ab, bb, wb = a[both], b[both], ww[both]
        for r in range(3):
            for c in range(3):  # full 3x3 blocks, structural zeros kept
                rows += [3 * ab + r, 3 * bb + r]
                cols += [3 * bb + c, 3 * ab + c]
                vals += [-wb * K0[r, c], -wb * K0[r, c]]
    for r in range(3):
        for c in range(3):
            rows.append(3 * np.arange(nn) + r)
            cols.append(3 * np.arange(nn) + c)
            vals.append(dblk[:, r, c])
    return _coo_to_csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)


def covariance2d(N: int, alpha: float = 3.0, beta: float = 4.0) -> sp.csr_matrix:
    """Covariance-type matrix on an N x N grid of unit spacing (n = N^2):
    c_ij = (1 - d(i, j)/alpha)^beta for d(i, j) <= alpha, else 0, with d the
    Euclidean distance between grid points i and j (the paper's second example,
    Section 3.6, after Tang and Saad).  c_ii = 1; entries at d = alpha are 0 and
    are not stored.  The truncated power (1 - r)_+^beta is positive definite in
    the plane for beta >= 3/2 (Askey), so C is SPD for beta = 4.  No random numbers.
    """
    n = N * N
    idx = np.arange(n).reshape(N, N)
    r = int(np.floor(alpha))
    rows, cols, vals = [], [], []
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            d = float(np.hypot(dx, dy))
            if d >= alpha:
                continue
            c = (1.0 - d / alpha) ** beta
            y0, y1 = max(0, -dy), min(N, N - dy)
            x0, x1 = max(0, -dx), min(N, N - dx)
            a = idx[y0:y1, x0:x1].ravel()
            b = idx[y0 + dy:y1 + dy, x0 + dx:x1 + dx].ravel()
            rows.append(a); cols.append(b); vals.append(np.full(a.size, c))
    return _coo_to_csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)


def band_dd(n: int, b: int, dodd: float, seed) -> sp.csr_matrix:
    """Symmetric band matrix of half-bandwidth b with every entry of the band
    present, diagonally dominant with degree ``dodd`` -- the shape of the paper's
    dense-row microbenchmark matrices (n = 12,288 / 24,576, b = 1024: nnz/n =
    1963.6 / 2006.3, DoDD 1.8, SPD).

    Draws: ``u = rng.uniform(-1, 1, (b, n))``; a_{i+d, i} = a_{i, i+d} = u[d-1, i]
    for 1 <= d <= b, i + d < n.  a_ii = dodd * sum_{j != i} |a_ij|, so that
    min_i |a_ii| / sum_{j != i} |a_ij| = dodd (SPD for dodd > 1).
    nnz = n (2b + 1) - b (b + 1).
    """
    rng = _rng(seed)
    u = rng.uniform(-1.0, 1.0, (b, n))
    rows, cols, vals = [], [], []
    rowsum = np.zeros(n)
    for d in range(1, b + 1):
        i = np.arange(n - d)
        v = u[d - 1, : n - d]
        rows += [i + d, i]; cols += [i, i + d]; vals += [v, v]
        a = np.abs(v)
        rowsum[i] += a
        rowsum[i + d] += a
    rows.append(np.arange(n)); cols.append(np.arange(n)); vals.append(dodd * rowsum)
    return _coo_to_csr(np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), n)
