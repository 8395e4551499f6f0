"""The named synthetic workloads: matrix, ordering, shift and ILDL factors.

Each builder returns a ``Workload`` holding A (in nested-dissection order), the
ILDL factors (L, D) that the selected-inverse path takes as input, and the
parameters of the path (Neumann terms m, low-rank size k, Mix threshold rule).
The matrices stand in for the paper's SuiteSparse test set (Section 3), which
is not available: PDE-type operators of the same kind (structural and
diffusion problems, n in the paper's range and beyond).

Recipes (every random number from PCG64 ``numpy.random.default_rng``):

* ``lap2d_32``      2D 5-point Dirichlet Laplacian 32x32 + 0.1 I, n = 1024,
                    tau = 1e-2 (``tau=0`` gives exact factors), m = 3.
* ``diff3d``        3D 7-point diffusion, log-normal kappa (sigma = 1, seed 2),
                    shifted to A - s I with s the midpoint of the two smallest
                    eigenvalues of A (one negative eigenvalue), tau = 1e-3,
                    m = 4, k = 16.  Full size 64^3 (n = 262,144).
* ``batch9pt``      2D 9-point random-weight Laplacians, seeds 3000..3255:
                    ``rng = default_rng(seed)``, n_t = rng.integers(2048, 65536,
                    endpoint=True), nx = floor(sqrt(n_t)), ny = floor(n_t / nx),
                    then the weights from the same stream; tau = 1e-2, m = 3.
* ``diff3d_spd``    as ``diff3d`` without the shift (SPD), tau = 1e-3, m = 3:
                    48^3 training seeds 4000..4063, 128^3 inference seed 4999.
* ``elastic3d``     3D 27-point, 3 dof per node, seed 5, tau = 1e-4, m = 2, k = 64.
* ``covariance``    covariance-type matrix (1 - d/alpha)^beta on an N x N grid,
                    alpha = 3, beta = 4 (no random numbers), tau = 1e-3, m = 3:
                    the paper's second example, N = 100 and 200.
* ``band``          dense band of half-bandwidth b, DoDD 1.8, seed 6, in its
                    natural order (a band needs no reordering: its factor has
                    no fill), tau = 1e-6: the paper's dense-row microbenchmark
                    shape, n = 12,288 (b = 1024) and 24,576.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import grids
from .factor import Factors, ildl
from .nd import nd_perm


@dataclass
class Workload:
    name: str
    A: sp.csr_matrix
    factors: Factors
    tau: float
    m: int
    k: int = 0
    shift: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.A.shape[0]


def _ordered(A, shape, dof=1):
    p = nd_perm(shape, dof=dof)
    return A[p][:, p].tocsr(), p


def two_smallest_eigenvalues(A: sp.csr_matrix, tau_prec: float = 1e-3, seed: int = 0, tol: float = 1e-9):
    """lambda_1 <= lambda_2 of an SPD matrix by LOBPCG preconditioned with an ILDL.

    Block of 4 vectors from ``default_rng(seed)``; returns (l1, l2, max relative
    residual of the two pairs).
    """
    f = ildl(A, tau_prec)
    n = A.shape[0]
    M = spla.LinearOperator((n, n), matvec=lambda x: f.solve(x).ravel(), matmat=lambda X: f.solve(X),
                            dtype=np.float64)
    X0 = np.random.default_rng(seed).standard_normal((n, 4))
    w, V = spla.lobpcg(A, X0, M=M, largest=False, tol=tol, maxiter=400)
    order = np.argsort(w)
    w = w[order]; V = V[:, order]
    res = [np.linalg.norm(A @ V[:, i] - w[i] * V[:, i]) / abs(w[i]) for i in range(2)]
    return float(w[0]), float(w[1]), float(max(res))


def lap2d_32(tau: float = 1e-2, m: int = 3) -> Workload:
    A, p = _ordered(grids.laplace2d_5pt(32, 32, 0.1), (32, 32))
    return Workload("lap2d_32", A, ildl(A, tau), tau, m, meta={"shape": (32, 32), "perm": p})


def diff3d(N: int = 64, tau: float = 1e-3, m: int = 4, k: int = 16, seed: int = 2,
           shifted: bool = True) -> Workload:
    A0, p = _ordered(grids.diffusion3d_7pt(N, N, N, seed), (N, N, N))
    shift = 0.0
    meta = {"shape": (N, N, N), "perm": p, "seed": seed}
    if shifted:
        l1, l2, res = two_smallest_eigenvalues(A0)
        # rounded so that the shift does not depend on the last bits of the eigensolver
        shift = float("%.8g" % (l1 + 0.5 * (l2 - l1)))
        if not (l1 < shift < l2):
            raise RuntimeError("shift not inside the first spectral gap")
        meta.update(lambda1=l1, lambda2=l2, eig_residual=res)
    A = (A0 - shift * sp.identity(A0.shape[0], format="csr")).tocsr()
    A.sort_indices()
    f = ildl(A, tau)
    return Workload("diff3d_%d" % N, A, f, tau, m, k, shift, meta)


def batch9pt_member(seed: int, tau: float = 1e-2, m: int = 3, n_range=(2048, 65536)) -> Workload:
    rng = np.random.default_rng(seed)
    n_t = int(rng.integers(n_range[0], n_range[1], endpoint=True))
    nx = int(np.floor(np.sqrt(n_t)))
    ny = n_t // nx
    A, p = _ordered(grids.random9pt_2d(nx, ny, rng), (nx, ny))
    return Workload("9pt_%d" % seed, A, ildl(A, tau), tau, m, meta={"shape": (nx, ny), "seed": seed})


def elastic3d(N: int = 80, tau: float = 1e-4, m: int = 2, k: int = 64, seed: int = 5,
              cache_dir: str | None = None) -> Workload:
    """cache_dir: keep the ordered matrix and its factors in a file there, keyed by
    the generator, N, tau and seed (the ILDL of 80^3 nodes takes minutes on one core),
    and load them from it when present."""
    key = "elastic3d_N%d_tau%g_seed%d" % (N, tau, seed)
    cached = load_cached(cache_dir, key)
    if cached is not None:
        A, f = cached
    else:
        A, p = _ordered(grids.elastic3d_27pt(N, N, N, seed), (N, N, N), dof=3)
        f = ildl(A, tau)
        store_cached(cache_dir, key, A, f)
    return Workload("elastic3d_%d" % N, A, f, tau, m, k, meta={"shape": (N, N, N), "seed": seed})


def load_cached(cache_dir, key):
    """(A, factors) from cache_dir/key.npz, or None (no directory or no file)."""
    import os
    if not cache_dir:
        return None
    path = os.path.join(cache_dir, key + ".npz")
    if not os.path.exists(path):
        return None
    z = np.load(path)
    n = int(z["n"])
    A = sp.csr_matrix((z["A_val"], z["A_col"], z["A_rp"]), shape=(n, n))
    f = Factors(n=n, L_rowptr=z["L_rp"], L_col=z["L_col"], L_val=z["L_val"], pivot_start=z["ps"],
                d_diag=z["dd"], d_off=z["do"], stats={"cache": path})
    return A, f


def store_cached(cache_dir, key, A, f):
    """Write (A, factors) to cache_dir/key.npz (uncompressed; written to a temporary
    name first, so a reader never sees a partial file)."""
    import os
    if not cache_dir:
        return
    os.makedirs(cache_dir, exist_ok=True)
    A = sp.csr_matrix(A)
    tmp = os.path.join(cache_dir, key + ".partial.npz")
    np.savez(tmp, n=f.n, A_rp=A.indptr, A_col=A.indices, A_val=A.data, L_rp=f.L_rowptr, L_col=f.L_col,
             L_val=f.L_val, ps=f.pivot_start, dd=f.d_diag, do=f.d_off)
    os.replace(tmp, os.path.join(cache_dir, key + ".npz"))


def covariance(N: int = 200, alpha: float = 3.0, beta: float = 4.0, tau: float = 1e-3, m: int = 3) -> Workload:
    """The covariance-type example on an N x N grid (N = 100, 200 in the paper,
    alpha = 3, beta = 4, tau = 1e-3), in nested-dissection order.  m = 3 is a
    proposed NInv depth (the paper's NInv uses its inverse tolerance instead)."""
    A, p = _ordered(grids.covariance2d(N, alpha, beta), (N, N))
    return Workload("covariance_%d_a%g_b%g" % (N, alpha, beta), A, ildl(A, tau), tau, m,
                    meta={"shape": (N, N), "alpha": alpha, "beta": beta})


def band(n: int = 12288, b: int = 1024, tau: float = 1e-6, dodd: float = 1.8, seed: int = 6, m: int = 3) -> Workload:
    """The dense-row microbenchmark shape of the paper (its n12 / n24 matrices:
    n = 12,288 / 24,576, half-bandwidth 1024, DoDD 1.8, best tau = 1e-6) in
    natural order."""
    A = grids.band_dd(n, b, dodd, seed)
    return Workload("band_%d_b%d" % (n, b), A, ildl(A, tau), tau, m, meta={"n": n, "b": b, "dodd": dodd, "seed": seed})


def random_lowrank(n: int, k: int, seed: int, orthonormal: bool = True):
    """Seeded (V, lambda) for timing the low-rank correction at sizes where the
    eigenpairs of E_inv are not computed: V from ``default_rng(seed)`` standard
    normals (orthonormalised by QR if asked), lambda = standard normals * 1e-3."""
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((n, k))
    if orthonormal and k > 0:
        V, _ = np.linalg.qr(V)
    lam = rng.standard_normal(k) * 1e-3
    return np.ascontiguousarray(V), lam


def plant_2x2(f: Factors, frac: float, seed: int) -> Factors:
    """Turn a seeded fraction of adjacent 1x1 pivot pairs (j, j+1) whose L(j+1, j)
    is not stored into 2x2 blocks of D, with D(j+1, j) = 0.5 sqrt|d_j d_{j+1}| u,
    u ~ U(-1, 1) from ``default_rng(seed)``.  L is unchanged.  Used where the
    factorisation itself produces no 2x2 pivot, so that the 2x2 path runs on
    realistic factor patterns."""
    rng = np.random.default_rng(seed)
    n = f.n
    ps = f.pivot_start.astype(bool)
    Lrp, Lc = f.L_rowptr, f.L_col
    # L(j+1, j) stored?  last entry of row j+1 equals j
    last = np.full(n, -1, dtype=np.int64)
    nonempty = np.diff(Lrp) > 0
    last[nonempty] = Lc[Lrp[1:][nonempty] - 1]
    cand = np.nonzero(ps[:-1] & ps[1:] & (last[1:] != np.arange(n - 1)))[0]
    # non-overlapping pairs: keep a candidate only if the previous kept one is not j-1
    pick = cand[rng.random(len(cand)) < frac]
    keep = []
    prev = -2
    for j in pick:
        if j > prev + 1:
            keep.append(j)
            prev = j
    keep = np.array(keep, dtype=np.int64)
    ps2 = f.pivot_start.copy()
    do = f.d_off.copy()
    if len(keep):
        ps2[keep + 1] = 0
        u = rng.uniform(-1.0, 1.0, len(keep))
        do[keep] = 0.5 * np.sqrt(np.abs(f.d_diag[keep] * f.d_diag[keep + 1])) * u
    g = Factors(n=n, L_rowptr=f.L_rowptr, L_col=f.L_col, L_val=f.L_val, pivot_start=ps2, d_diag=f.d_diag.copy(),
                d_off=do, stats=dict(f.stats))
    g.stats["n_2x2"] = int(len(keep))
    g.stats["planted_2x2"] = int(len(keep))
    return g


def random_factors(n: int, density: float, frac_2x2: float, seed: int, scale: float = 0.3) -> Factors:
    """Random (L, D) with an arbitrary (generally non-closed) pattern: every
    strictly lower entry is present with probability ``density``; values
    U(-scale, scale); D diagonal U(1, 2) with random sign flips on a tenth of the
    pivots; then ``plant_2x2`` with ``frac_2x2``.  All from ``default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=rng, format="csr")
    M = sp.tril(M, k=-1).tocsr()
    M.sort_indices()
    vals = rng.uniform(-scale, scale, M.nnz)
    d = rng.uniform(1.0, 2.0, n) * np.where(rng.random(n) < 0.1, -1.0, 1.0)
    f = Factors(n=n, L_rowptr=M.indptr.astype(np.int64), L_col=M.indices.astype(np.int32), L_val=vals,
                pivot_start=np.ones(n, dtype=np.int8), d_diag=d, d_off=np.zeros(n), stats={})
    return plant_2x2(f, frac_2x2, seed + 1) if frac_2x2 > 0 else f
