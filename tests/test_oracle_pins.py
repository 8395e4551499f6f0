"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formula: each compares it with a
dense LAPACK inverse, a closed form, an invariant, a hand-derived small case
or a brute-force dense evaluation.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from workloads import grids
from workloads.configs import diff3d, lap2d_32, plant_2x2
from workloads.factor import Factors, ildl
from workloads.nd import nd_perm


def _S(f):
    return oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)


def _rows(Srp):
    return np.repeat(np.arange(len(Srp) - 1), np.diff(Srp))


def _selinv(f, S=None):
    return oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)


def _ninv(f, m, S=None):
    return oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, m, S)


def _dense_LDLt(f):
    L = (f.L_csr() + sp.identity(f.n)).toarray()
    return L @ f.D_dense_blocks().toarray() @ L.T


def _factors_from_dense(L, dblocks):
    """Factors from a dense unit-lower L (structural pattern = nonzeros) and a list
    of D blocks (scalars or 2x2 arrays)."""
    n = L.shape[0]
    low = sp.csr_matrix(np.tril(L, -1))
    low.sort_indices()
    ps = np.zeros(n, np.int8); dd = np.zeros(n); do = np.zeros(n)
    j = 0
    for b in dblocks:
        ps[j] = 1
        if np.ndim(b) == 0:
            dd[j] = b; j += 1
        else:
            dd[j], dd[j + 1], do[j] = b[0][0], b[1][1], b[1][0]; j += 2
    return Factors(n=n, L_rowptr=low.indptr.astype(np.int64), L_col=low.indices.astype(np.int32),
                   L_val=low.data.astype(np.float64), pivot_start=ps, d_diag=dd, d_off=do)


# -- S (Section 1) ----------------------------------------------------------------
def test_pattern_is_brute_force_pattern_of_L_plus_D_plus_Lt():
    f = diff3d(6, tau=1e-2, shifted=True).factors
    f2 = _factors_from_dense((f.L_csr() + sp.identity(f.n)).toarray(),
                             [f.d_diag[j] if (j + 1 == f.n or f.pivot_start[j + 1]) else
                              [[f.d_diag[j], f.d_off[j]], [f.d_off[j], f.d_diag[j + 1]]]
                              for j in range(f.n) if f.pivot_start[j]])
    Srp, Sc = _S(f2)
    B = (np.abs((f2.L_csr() + sp.identity(f.n)).toarray()) > 0) | (np.abs(f2.D_dense_blocks().toarray()) > 0)
    B = B | B.T
    low = np.tril(B)
    rows, cols = np.nonzero(low)
    assert np.array_equal(_rows(Srp), rows) and np.array_equal(Sc, cols)


# -- SelInv (Section 2.1) ------------------------------------------------------------
def test_selinv_exact_factors_equal_dense_inverse_2d():
    """Exact factors: SelInv coincides with A^{-1} on S (Section 2.1)."""
    w = lap2d_32(tau=0.0)
    f = w.factors
    Srp, Sc = _S(f)
    G = _selinv(f, (Srp, Sc))
    Ainv = np.linalg.inv(w.A.toarray())
    assert np.max(np.abs(G - Ainv[_rows(Srp), Sc])) <= 1e-12 * np.max(np.abs(Ainv))


def test_selinv_exact_indefinite_with_2x2_pivot():
    """Shifted 3D problem, exact factors with a 2x2 pivot chosen by the pivot test."""
    w = diff3d(6, tau=0.0)
    f = w.factors
    assert f.stats["n_2x2"] >= 1
    Srp, Sc = _S(f)
    G = _selinv(f, (Srp, Sc))
    Ainv = np.linalg.inv(w.A.toarray())
    assert np.max(np.abs(G - Ainv[_rows(Srp), Sc])) <= 1e-10 * np.max(np.abs(Ainv))


def test_selinv_identity_GA_diag_is_one():
    """Exact factors: pattern(A) is inside S, so (G A)_ii = 1 from entries on S only."""
    w = lap2d_32(tau=0.0)
    f = w.factors
    Srp, Sc = _S(f)
    G = _selinv(f, (Srp, Sc))
    Gs = oracle.core.sym_from_S(f.n, Srp, Sc, G)
    A = w.A
    Sset = set(zip(_rows(Srp).tolist(), Sc.tolist()))
    Alow = sp.tril(A).tocoo()
    assert all((int(i), int(j)) in Sset for i, j in zip(Alow.row, Alow.col))
    d = np.asarray(Gs.multiply(A.T).sum(axis=1)).ravel()
    assert np.max(np.abs(d - 1.0)) <= 1e-12


def test_selinv_1d_closed_form():
    """tridiag(-1, 2, -1): (A^{-1})_ij = i (n+1-j) / (n+1), 1-based, i <= j."""
    n = 50
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")
    f = ildl(A, 0.0)
    Srp, Sc = _S(f)
    G = _selinv(f, (Srp, Sc))
    r = _rows(Srp) + 1; c = Sc + 1
    i, j = np.minimum(r, c), np.maximum(r, c)
    assert np.max(np.abs(G - i * (n + 1 - j) / (n + 1))) <= 1e-12 * n


def test_selinv_2d_diagonal_closed_form_sine_expansion():
    """lap2d 32x32 + 0.1 I, exact factors: diag(A^{-1}) from the Dirichlet
    eigenbasis, d(x,y) = sum_pq phi_pq(x,y)^2 / (4 - 2cos(p pi/33) - 2cos(q pi/33) + 0.1)."""
    w = lap2d_32(tau=0.0)
    f = w.factors
    Srp, Sc = _S(f)
    G = _selinv(f, (Srp, Sc))
    diag_nd = G[Srp[1:] - 1]
    perm = w.meta["perm"]  # perm[new] = old natural index
    k = np.arange(1, 33)
    lam1 = 2 - 2 * np.cos(k * np.pi / 33)
    phi = np.sqrt(2 / 33) * np.sin(np.outer(np.arange(1, 33), k) * np.pi / 33)  # phi[x-1, p-1]
    lam = lam1[:, None] + lam1[None, :] + 0.1
    # d(x, y) = sum_pq phi[x,p]^2 phi[y,q]^2 / lam[p,q]
    d = np.einsum("xp,yq,pq->yx", phi ** 2, phi ** 2, 1.0 / lam).ravel()  # natural index y*32 + x
    assert np.max(np.abs(diag_nd - d[perm])) <= 1e-12


def test_selinv_hand_example_nonclosed():
    """n = 4, L(1,0)=a, L(2,0)=b, L(3,1)=c, L(3,2)=e: (2,1) is not in S.  By hand,
    the recurrence with the entries outside S discarded gives
      G33 = 1/d3, G32 = -e/d3, G22 = 1/d2 + e^2/d3, G31 = -c/d3, G11 = 1/d1 + c^2/d3,
      G10 = -a G11, G20 = -b G22, G00 = 1/d0 + a^2 G11 + b^2 G22,
    while the exact (LDL^T)^{-1} has G00 larger by 2 a b c e / d3."""
    a, b, c, e = 0.3, -0.7, 0.45, 0.2
    d = [2.0, 1.5, -1.25, 3.0]
    L = np.eye(4); L[1, 0] = a; L[2, 0] = b; L[3, 1] = c; L[3, 2] = e
    f = _factors_from_dense(L, d)
    Srp, Sc = _S(f)
    G = _selinv(f, (Srp, Sc))
    G33 = 1 / d[3]; G32 = -e / d[3]; G22 = 1 / d[2] + e * e / d[3]; G31 = -c / d[3]; G11 = 1 / d[1] + c * c / d[3]
    G10 = -a * G11; G20 = -b * G22; G00 = 1 / d[0] + a * a * G11 + b * b * G22
    want = {(0, 0): G00, (1, 0): G10, (1, 1): G11, (2, 0): G20, (2, 2): G22, (3, 1): G31, (3, 2): G32, (3, 3): G33}
    got = dict(zip(zip(_rows(Srp), Sc), G))
    assert set(got) == set(want)
    for key in want:
        assert abs(got[key] - want[key]) <= 1e-15 * 10, key
    exact = np.linalg.inv(_dense_LDLt(f))
    assert abs(exact[0, 0] - G00 - 2 * a * b * c * e / d[3]) <= 1e-14


def test_selinv_2x2_block_with_different_column_structures():
    """2x2 block {0,1} with struct(0) = {2}, struct(1) = {3} and (3,2) in S: the
    pattern is closed, so SelInv must equal (LDL^T)^{-1} on S.  This fixes the
    reading that the block's G11 uses X on the union of the two structures."""
    L = np.eye(4); L[2, 0] = 0.4; L[3, 1] = -0.6; L[3, 2] = 0.5
    f = _factors_from_dense(L, [[[1.5, 0.7], [0.7, -2.0]], 1.2, 2.5])
    Srp, Sc = _S(f)
    G = _selinv(f, (Srp, Sc))
    exact = np.linalg.inv(_dense_LDLt(f))
    assert np.max(np.abs(G - exact[_rows(Srp), Sc])) <= 1e-14


def test_selinv_closed_random_pattern_equals_inverse():
    """Random values on a closed pattern (the exact symbolic factor of a random
    sparse SPD matrix) and random-sign D: SelInv = (LDL^T)^{-1} on S."""
    rng = np.random.default_rng(5)
    n = 60
    B = sp.random(n, n, density=0.05, random_state=rng)
    A = (B + B.T + sp.identity(n) * 5).tocsr()
    f0 = ildl(A, 0.0, allow_2x2=False)
    # random values on the same (closed) pattern
    L = (f0.L_csr() + sp.identity(n)).toarray()
    mask = np.tril(L, -1) != 0
    L[mask] = rng.uniform(-0.5, 0.5, mask.sum())
    f = _factors_from_dense(L, list(rng.uniform(1, 2, n) * rng.choice([-1, 1], n)))
    Srp, Sc = _S(f)
    G = _selinv(f, (Srp, Sc))
    exact = np.linalg.inv(_dense_LDLt(f))
    assert np.max(np.abs(G - exact[_rows(Srp), Sc])) <= 1e-11 * np.max(np.abs(exact))


def _dense_masked_selinv(f, S):
    """The recurrence of Eqs. (4)-(5) on dense arrays, written apart from the oracle:
    pivot blocks J from the last to the first; C = the rows below J stored in L's
    columns of J; X = -G_CC L_CJ with G_CC read from the dense array, where only
    entries of S were ever written (zero off S); G_JJ = D_J^{-1} - L_CJ^T X; then only
    the entries of S kept."""
    n = f.n
    Lc = f.L_csr()
    stored = np.zeros((n, n), dtype=bool)
    stored[_rows(Lc.indptr), Lc.indices] = True
    L = Lc.toarray()
    D = f.D_dense_blocks().toarray()
    inS = np.zeros((n, n), dtype=bool)
    inS[_rows(S[0]), S[1]] = True
    inS |= inS.T
    G = np.zeros((n, n))
    starts = [j for j in range(n) if f.pivot_start[j]] + [n]
    for b in range(len(starts) - 2, -1, -1):
        J = list(range(starts[b], starts[b + 1]))
        C = [r for r in range(starts[b + 1], n) if stored[r, J].any()]
        LCJ = L[np.ix_(C, J)]
        X = -G[np.ix_(C, C)] @ LCJ
        GJJ = np.linalg.inv(D[np.ix_(J, J)]) - LCJ.T @ X
        for a, r in enumerate(C):
            for c_, c in enumerate(J):
                if inS[r, c]:
                    G[r, c] = G[c, r] = X[a, c_]
        for a, r in enumerate(J):
            for c_, c in enumerate(J):
                G[r, c] = GJJ[a, c_]
    return G[_rows(S[0]), S[1]]


@pytest.mark.parametrize("seed", [3, 8, 21])
def test_selinv_matches_a_dense_masked_recurrence(seed):
    """Incomplete (non-closed) random factors with 2x2 pivots: the oracle's sparse
    recurrence equals the same recurrence run on dense arrays, entry by entry."""
    from workloads.configs import random_factors
    f = random_factors(70, 0.08, 0.2, seed)
    S = _S(f)
    G = _selinv(f, S)
    ref = _dense_masked_selinv(f, S)
    assert np.max(np.abs(G - ref)) <= 1e-12 * np.max(np.abs(ref))
    # the pattern is not closed: the result differs from the true inverse on S
    exact = np.linalg.inv(_dense_LDLt(f))
    assert np.max(np.abs(G - exact[_rows(S[0]), S[1]])) > 1e-6 * np.max(np.abs(exact))


# -- NInv (Section 2.2) ------------------------------------------------------------------
def _brute_ninv(f, m):
    n = f.n
    E = -f.L_csr().toarray()
    W = sum(np.linalg.matrix_power(E, t) for t in range(m + 1))
    return W.T @ np.linalg.inv(f.D_dense_blocks().toarray()) @ W


@pytest.mark.parametrize("m", [0, 1, 2, 5])
def test_ninv_equals_dense_truncated_series(m):
    from workloads.configs import random_factors
    f = random_factors(120, 0.05, 0.2, 9)
    Srp, Sc = _S(f)
    N = _ninv(f, m, (Srp, Sc))
    ref = _brute_ninv(f, m)[_rows(Srp), Sc]
    assert np.max(np.abs(N - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_ninv_m0_is_Dinv_on_S():
    from workloads.configs import random_factors
    f = random_factors(80, 0.1, 0.3, 2)
    Srp, Sc = _S(f)
    N = _ninv(f, 0, (Srp, Sc))
    Dinv = np.linalg.inv(f.D_dense_blocks().toarray())
    assert np.array_equal(N == 0, Dinv[_rows(Srp), Sc] == 0)
    assert np.max(np.abs(N - Dinv[_rows(Srp), Sc])) <= 1e-15 * 4


def test_ninv_exact_when_m_reaches_depth():
    """E is nilpotent: for m >= the longest path in the graph of L the series is
    L^{-1} exactly, so NInv = (LDL^T)^{-1} on S (Section 2.2)."""
    w = lap2d_32(tau=0.0)
    f = w.factors
    Lc = f.L_csr().tocsc()
    depth = np.zeros(f.n, int)
    for j in range(f.n - 1, -1, -1):
        r = Lc.indices[Lc.indptr[j]:Lc.indptr[j + 1]]
        if len(r):
            depth[j] = 1 + depth[r].max()
    m = int(depth.max())
    Srp, Sc = _S(f)
    N = _ninv(f, m, (Srp, Sc))
    Ainv = np.linalg.inv(w.A.toarray())
    assert np.max(np.abs(N - Ainv[_rows(Srp), Sc])) <= 1e-11
    E = -f.L_csr().toarray()
    assert not np.any(np.linalg.matrix_power(E, m + 1))


def test_ninv_own_pattern_hand_example():
    """L = [[1,0,0],[0.5,1,0],[0,0.1,1]], D = I, m = 2, delta = 0.1, worked by hand:
    the Horner steps in column form give W = [[1,0,0],[-0.5,1,0],[0,-0.1,1]] (the
    second step's 0.05 in column 0 falls below delta; -0.1 is not below it), then
    N = W^T W: N_00 = 1.25, N_10 = -0.5, N_11 = 1.01, N_21 = -0.1, N_22 = 1, and the
    product's drop removes N_21 (0.1 < 0.1 sqrt(1.01)) but keeps N_10."""
    from workloads.factor import Factors
    f = Factors(n=3, L_rowptr=np.array([0, 0, 1, 2], dtype=np.int64), L_col=np.array([0, 1], dtype=np.int32),
                L_val=np.array([0.5, 0.1]), pivot_start=np.ones(3, dtype=np.int8), d_diag=np.ones(3),
                d_off=np.zeros(3))
    N = oracle.ninv_own(3, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, 2, 0.1).toarray()
    want = np.array([[1.25, 0, 0], [-0.5, 1.01, 0], [0, 0, 1.0]])
    assert np.allclose(N, want, rtol=0, atol=1e-15)
    W = oracle.ninv_W(3, f.L_rowptr, f.L_col, f.L_val, 2, 0.1).toarray()
    assert np.allclose(W, [[1, 0, 0], [-0.5, 1, 0], [0, -0.1, 1]], rtol=0, atol=1e-15)
    # with a smaller tolerance the product keeps N_21 and W keeps the 0.05
    N2 = oracle.ninv_own(3, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, 2, 0.04).toarray()
    assert np.isclose(N2[2, 1], -0.1) and np.isclose(N2[2, 0], 0.05)


def test_mix_own_hand_example():
    """S_lo = {(0,0), (1,0), (1,1), (2,1), (2,2)} with SelInv values 2, -0.004, 1.5,
    0.3, 1; NInv on its own pattern {(0,0): 1.25, (1,0): -0.5, (1,1): 1.01,
    (2,0): 0.05, (2,2): 1}; eps = 0.01.  By hand (Section 2.3): S_eps = {(0,0),
    (1,1), (2,1), (2,2)} (|-0.004| is not above eps), so Mix = G there, N at (1,0)
    and at (2,0) (outside S), and (2,1) joins the pattern from S_eps."""
    Srp = np.array([0, 1, 3, 5], dtype=np.int64)
    Sc = np.array([0, 0, 1, 1, 2], dtype=np.int32)
    G = np.array([2.0, -0.004, 1.5, 0.3, 1.0])
    N = sp.csc_matrix(([1.25, -0.5, 0.05, 1.01, 1.0], ([0, 1, 2, 1, 2], [0, 0, 0, 1, 2])), shape=(3, 3))
    M = oracle.mix_own(3, Srp, Sc, G, N, 0.01)
    assert M.nnz == 6
    assert np.array_equal(M.toarray(), [[2.0, 0, 0], [-0.5, 1.5, 0], [0.05, 0.3, 1.0]])
    # eps = +inf: NInv unchanged; eps < 0: SelInv on all of S, NInv off S
    assert np.array_equal(oracle.mix_own(3, Srp, Sc, G, N, np.inf).toarray(), N.toarray())
    Mneg = oracle.mix_own(3, Srp, Sc, G, N, -1.0)
    assert Mneg.nnz == 6
    assert np.array_equal(Mneg.toarray(), [[2.0, 0, 0], [-0.004, 1.5, 0], [0.05, 0.3, 1.0]])


def test_mix_own_on_S_reduces_to_mix():
    """With NInv given on exactly the pattern S, Mix on the own pattern is the Mix of
    Section 2.3 on S, entry by entry, for every eps rule."""
    f = plant_2x2(lap2d_32().factors, 0.3, 11)
    Srp, Sc = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    rng = np.random.default_rng(3)
    G = rng.standard_normal(len(Sc)) * np.exp(rng.standard_normal(len(Sc)) * 3)
    Nv = rng.standard_normal(len(Sc))
    rows = np.repeat(np.arange(f.n), np.diff(Srp))
    N = sp.csc_matrix((Nv, (rows, Sc)), shape=(f.n, f.n))
    for eps in (1e-3 * np.abs(G).max(), 0.0, -1.0, np.inf):
        M = oracle.mix_own(f.n, Srp, Sc, G, N, eps)
        assert M.nnz == len(Sc)
        assert np.array_equal(np.asarray(M[rows, Sc]).ravel(), oracle.mix(G, Nv, eps))


def test_ninv_own_limits():
    """delta = 0 with m >= depth and exact factors: the whole lower triangle of
    inv(A); delta huge: W = I and only the diagonal of D^{-1} is left."""
    w = lap2d_32(tau=0.0)
    f = w.factors
    Lc = f.L_csr().tocsc()
    depth = np.zeros(f.n, int)
    for j in range(f.n - 1, -1, -1):
        r = Lc.indices[Lc.indptr[j]:Lc.indptr[j + 1]]
        if len(r):
            depth[j] = 1 + depth[r].max()
    N = oracle.ninv_own(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, int(depth.max()), 0.0)
    Ainv = np.tril(np.linalg.inv(w.A.toarray()))
    assert np.max(np.abs(N.toarray() - Ainv)) <= 1e-11
    assert N.nnz == np.count_nonzero(np.abs(Ainv) > 1e-300)
    g = plant_2x2(lap2d_32().factors, 0.2, 1)
    N = oracle.ninv_own(g.n, g.L_rowptr, g.L_col, g.L_val, g.pivot_start, g.d_diag, g.d_off, 3, 1e30)
    Dinv = oracle.core._Dinv(g.n, g.pivot_start, g.d_diag, g.d_off).diagonal()
    assert N.nnz == g.n and np.allclose(N.diagonal(), Dinv, rtol=1e-15)


@pytest.mark.parametrize("m", [1, 3])
def test_ninv_own_without_dropping_is_the_dense_product(m):
    """delta = 0 on incomplete random factors with 2x2 pivots: nothing is dropped, so
    NInv on its own pattern is the lower triangle of the dense W^T D^{-1} W with
    W = sum_{t<=m} E^t, every nonzero of it present."""
    from workloads.configs import random_factors
    f = random_factors(90, 0.06, 0.2, 4)
    N = oracle.ninv_own(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, m, 0.0).toarray()
    ref = np.tril(_brute_ninv(f, m))
    assert np.max(np.abs(N - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert np.all(N[np.abs(ref) > 1e-12 * np.max(np.abs(ref))] != 0)


def test_ninv_sampled_matches_full():
    w = lap2d_32()
    f = w.factors
    Srp, Sc = _S(f)
    N = _ninv(f, 3, (Srp, Sc))
    rows = _rows(Srp)
    idx = np.arange(0, len(Sc), 37)
    Ns = oracle.ninv_entries_sampled(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, 3,
                                     list(zip(rows[idx], Sc[idx])))
    ref = _brute_ninv(f, 3)[rows[idx], Sc[idx]]
    assert np.max(np.abs(Ns - ref)) <= 1e-13 and np.max(np.abs(N[idx] - ref)) <= 1e-13


def _drop_case(e10, e21):
    """3x3 factors with E_10 = e10, E_21 = e21, no L_20 and D = diag(2, 4, 5)."""
    L = np.array([[1.0, 0.0, 0.0], [-e10, 1.0, 0.0], [0.0, -e21, 1.0]])
    return _factors_from_dense(L, [2.0, 4.0, 5.0])


@pytest.mark.parametrize("e10,e21,delta,want", [
    # exact series W = I + E + E^2 with W_20 = E_21 E_10 = 0.05
    (0.5, 0.1, 0.0, [0.5630, 0.126, 0.252, 0.02, 0.2]),
    # delta = 0.1: the second step drops W_20 = 0.05; 0.1 itself stays (strict test)
    (0.5, 0.1, 0.1, [0.5625, 0.125, 0.252, 0.02, 0.2]),
    # delta = 0.2: the first step already drops E_21 = 0.1
    (0.5, 0.1, 0.2, [0.5625, 0.125, 0.25, 0.0, 0.2]),
    # the order of the Horner product matters once entries are dropped: the first
    # step drops W_10 = 0.05, and the column form W_2 = I + W_1 E still forms
    # W_20 = W_1[2, 1] E_10 = 4 * 0.05 = 0.2 (kept), where I + E W_1 would give 0
    (0.05, 4.0, 0.0, [0.508625, 0.1725, 3.45, 0.8, 0.2]),
    (0.05, 4.0, 0.1, [0.508, 0.16, 3.45, 0.8, 0.2]),
])
def test_ninv_drop_hand_example(e10, e21, delta, want):
    """Section 2.2's inverse tolerance, read as: the Horner steps W_t = I + W_{t-1} E
    (column j from the columns of struct(j)) drop their off-diagonal |w| < delta.
    N_ij = sum_r W_ri W_rj / d_r by hand on S_lo = {(0,0), (1,0), (1,1), (2,1), (2,2)}."""
    f = _drop_case(e10, e21)
    S = _S(f)
    assert np.array_equal(S[0], [0, 1, 3, 5]) and np.array_equal(S[1], [0, 0, 1, 1, 2])
    N = oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, 2, S, delta=delta)
    assert np.allclose(N, want, rtol=0, atol=1e-14)
    pairs = list(zip(_rows(S[0]), S[1]))
    Ns = oracle.ninv_entries_sampled(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, 2,
                                     pairs, delta=delta)
    assert np.allclose(Ns, want, rtol=0, atol=1e-14)


def test_ninv_drop_limits_and_fill():
    """delta beyond every entry leaves W = I, so N = D^{-1} on S (2x2 blocks too);
    the fill of W never grows with delta; the column-wise sampled evaluation agrees
    with the matrix Horner evaluation at every delta."""
    from workloads.configs import random_factors
    f = random_factors(150, 0.05, 0.2, 12)
    Srp, Sc = _S(f)
    rows = _rows(Srp)
    Dinv = np.linalg.inv(f.D_dense_blocks().toarray())
    N = oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, 3, (Srp, Sc), delta=1e30)
    assert np.max(np.abs(N - Dinv[rows, Sc])) <= 1e-15 * 4
    fills = [oracle.ninv_W(f.n, f.L_rowptr, f.L_col, f.L_val, 3, d).nnz for d in (0.0, 1e-4, 1e-3, 1e-2, 1e-1, 1.0)]
    assert all(a >= b for a, b in zip(fills, fills[1:])) and fills[0] > fills[-1]
    idx = np.arange(0, len(Sc), 7)
    for d in (1e-3, 1e-2, 1e-1):
        N = oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, 3, (Srp, Sc), delta=d)
        Ns = oracle.ninv_entries_sampled(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, 3,
                                         list(zip(rows[idx], Sc[idx])), delta=d)
        assert np.max(np.abs(Ns - N[idx])) <= 1e-13 * max(1.0, np.max(np.abs(N)))


# -- Mix (Section 2.3) ---------------------------------------------------------------------
def test_mix_special_cases_and_hand_example():
    G = np.array([0.5, -1e-4, 2e-3, -0.2, 0.0])
    N = np.array([0.4, 7.0, 8.0, 9.0, 1.0])
    assert np.array_equal(oracle.mix(G, N, np.inf), N)
    assert np.array_equal(oracle.mix(G, N, -1.0), G)
    assert np.array_equal(oracle.mix(G, N, 1e-3), np.array([0.5, 7.0, 2e-3, -0.2, 1.0]))


# -- low-rank correction (Sections 2.5, 2.6) --------------------------------------------------
def test_lowrank_brute_force_and_diagonal_formula():
    from workloads.configs import random_factors, random_lowrank
    f = random_factors(90, 0.08, 0.1, 4)
    Srp, Sc = _S(f)
    X = np.random.default_rng(1).standard_normal(len(Sc))
    V, lam = random_lowrank(f.n, 5, seed=3, orthonormal=False)
    out = oracle.lowrank_correct(Srp, Sc, X, V, lam)
    dense = V @ np.diag(lam) @ V.T
    assert np.max(np.abs(out - X - dense[_rows(Srp), Sc])) <= 1e-14
    dd = np.diag(dense)
    # Section 2.6: d_i + sum_j lambda_j v_ij^2
    diag = oracle.lowrank_diag(X[Srp[1:] - 1], V, lam)
    assert np.max(np.abs(diag - (X[Srp[1:] - 1] + dd))) <= 1e-14
    assert np.array_equal(oracle.lowrank_correct(Srp, Sc, X, V[:, :0], lam[:0]), X)


def test_lanczos_eigenpairs_and_eckart_young():
    """Dominant eigenpairs of E_inv = A^{-1} - A^inv (Lanczos, matrix free) agree
    with a dense eigendecomposition, and the rank-k residual in the 2-norm is
    |lambda_{k+1}| (Eckart-Young, Section 2.5)."""
    A0 = grids.laplace2d_5pt(10, 10, 0.1)
    p = nd_perm((10, 10))
    A = A0[p][:, p].tocsr()
    f = ildl(A, 5e-2)
    Srp, Sc = _S(f)
    G = _selinv(f, (Srp, Sc))
    Gs = oracle.core.sym_from_S(f.n, Srp, Sc, G)
    Einv = np.linalg.inv(A.toarray()) - Gs.toarray()
    ev = np.linalg.eigvalsh(Einv)
    ev = ev[np.argsort(-np.abs(ev))]
    k = 3
    lam, V = oracle.lanczos_einv(A, Gs, k, steps=100, seed=0)
    assert np.allclose(np.sort(np.abs(lam)), np.sort(np.abs(ev[:k])), rtol=1e-9, atol=0)
    R = Einv - V @ np.diag(lam) @ V.T
    assert abs(np.linalg.norm(R, 2) - abs(ev[k])) <= 1e-8 * abs(ev[0])
    assert abs(np.linalg.norm(R, "fro") ** 2 - np.sum(ev[k:] ** 2)) <= 1e-8 * np.sum(ev ** 2)


def test_lanczos_start_vector_is_an_input():
    # a given start vector reproduces the seeded run exactly, and a scaled one gives the
    # same Ritz pairs (the first Lanczos vector is normalised)
    A = sp.csr_matrix(grids.laplace2d_5pt(8, 8, 0.1))
    f = ildl(A, 5e-2)
    Srp, Sc = _S(f)
    Gs = oracle.core.sym_from_S(f.n, Srp, Sc, _selinv(f, (Srp, Sc)))
    q = np.random.default_rng(3).standard_normal(f.n)
    lam1, V1 = oracle.lanczos_einv(A, Gs, 2, steps=20, seed=3)
    lam2, V2 = oracle.lanczos_einv(A, Gs, 2, steps=20, q0=q)
    np.testing.assert_array_equal(lam1, lam2)
    np.testing.assert_array_equal(V1, V2)
    lam3, V3 = oracle.lanczos_einv(A, Gs, 2, steps=20, q0=7.5 * q)
    np.testing.assert_allclose(lam3, lam1, rtol=1e-13)


def test_acceptance_keeps_only_improving_modes():
    d = np.array([1.0, 2.0, 3.0])
    d_hat = np.array([0.9, 2.0, 3.0])
    V = np.eye(3)[:, :2]
    lam = np.array([0.1, 0.5])  # mode 0 fixes entry 0, mode 1 spoils entry 1
    kept, cur = oracle.accept_modes(d, d_hat, V, lam)
    assert kept == [0] and np.allclose(cur, d)


# -- measures (Sections 2.6, 3.2) -----------------------------------------------------------
def test_measures():
    assert oracle.err1([1.0, -2.0], [1.0, -2.0]) == 0.0
    assert oracle.err1([1.0, 3.0], [2.0, 3.0]) == 0.25
    n = 20
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")
    assert oracle.dodd(A) == 1.0
    f = ildl(A, 0.0)
    Srp, Sc = _S(f)
    assert oracle.fill_fact(2 * len(Sc) - n, A.nnz) == 1.0


# -- the input factorisation (generator side) -------------------------------------------------
def test_ildl_exact_reconstructs_and_keeps_inertia():
    w = diff3d(6, tau=0.0)
    f = w.factors
    R = _dense_LDLt(f) - w.A.toarray()
    assert np.max(np.abs(R)) <= 1e-12 * np.max(np.abs(w.A.toarray()))
    neg_A = int(np.sum(np.linalg.eigvalsh(w.A.toarray()) < 0))
    neg_D = int(np.sum(np.linalg.eigvalsh(f.D_dense_blocks().toarray()) < 0))
    assert neg_A == neg_D == 1


# -- the learned correction's network (oracle side of the gradient check) --------------
def test_mlp_oracle_gradient_matches_finite_differences():
    from oracle import mlp as omlp
    F, H = 16, 64
    rng = np.random.default_rng(3)
    theta = rng.standard_normal(omlp.n_params(F, H)) * 0.2
    X = rng.standard_normal((40, F))
    y = rng.standard_normal(40)
    g = omlp.grad(theta, X, y, F, H)
    idx = rng.choice(len(theta), 60, replace=False)
    fd = omlp.grad_fd(theta, X, y, F, H, idx)
    assert np.max(np.abs(g[idx] - fd)) <= 1e-6 * max(1.0, np.max(np.abs(fd)))
    # Adam's first step moves every parameter by lr * sign(g) (bias-corrected moments)
    t1, m1, v1 = omlp.adam(theta, g, np.zeros_like(g), np.zeros_like(g), 1, 1e-3)
    big = np.abs(g) > 1e-3
    assert np.allclose((theta - t1)[big], 1e-3 * np.sign(g[big]), rtol=1e-4)


def test_mlp_bf16_rounding_hand_values_and_library():
    """The BF16 rounding of the hidden layer (inference on tensor cores): ties go
    to the even neighbour, and every value agrees with torch's own conversion."""
    import torch
    from oracle import mlp as omlp
    hand = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -7, 1 + 2.0 ** -8 + 2.0 ** -20, -3.0, 0.0])
    want = np.array([1.0, 1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, 1 + 2.0 ** -7, -3.0, 0.0])
    assert np.array_equal(omlp.bf16_round(hand), want)
    x = np.random.default_rng(4).standard_normal(10000) * 10.0 ** np.random.default_rng(5).integers(-8, 8, 10000)
    lib = torch.as_tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(omlp.bf16_round(x), lib)
    rng = np.random.default_rng(6)
    theta = rng.standard_normal(omlp.n_params(16, 64)) * 0.3
    X = rng.standard_normal((50, 16))
    a = omlp.forward(theta, X, 16, 64)
    b = omlp.forward(theta, X, 16, 64, act_bf16=True)
    assert 0 < np.max(np.abs(a - b)) <= 2.0 ** -7 * np.max(np.abs(a)) + 1e-3


def test_covariance_generator_matches_definition():
    """The covariance-type example entry by entry from the grid coordinates (brute
    force over all pairs), symmetric positive definite."""
    from workloads import grids
    N, alpha, beta = 7, 3.0, 4.0
    C = grids.covariance2d(N, alpha, beta).toarray()
    xy = np.array([(i % N, i // N) for i in range(N * N)], dtype=float)
    d = np.sqrt(((xy[:, None, :] - xy[None, :, :]) ** 2).sum(-1))
    ref = np.where(d <= alpha, np.clip(1.0 - d / alpha, 0.0, None) ** beta, 0.0)
    assert np.max(np.abs(C - ref)) <= 1e-15
    assert np.linalg.eigvalsh(C).min() > 0.1


# --------------------------------------------------------------------------
# SPAI refinement (Section 2.4)
# --------------------------------------------------------------------------
def _lower_pattern(M):
    low = sp.tril(sp.csr_matrix(M), format="csr")
    low.sort_indices()
    return low.indptr.astype(np.int64), low.indices.astype(np.int32)


def _spai_case(n=30, seed=11):
    """A small sparse SPD A (random symmetric couplings, diagonally dominant)
    and a pattern S = lower part of pattern(A + A^2 restricted) with the diagonal."""
    rng = np.random.default_rng(seed)
    R = sp.random(n, n, density=0.12, random_state=seed, data_rvs=lambda k: rng.uniform(-1, 1, k))
    A = (R + R.T).tocsr()
    A = A + sp.diags(np.asarray(abs(A).sum(axis=1)).ravel() + 1.0)
    P = sp.csr_matrix(A @ A)
    P.data[:] = 1.0
    keep = sp.random(n, n, density=0.5, random_state=seed + 1)
    keep = keep + keep.T
    S = P.multiply(keep != 0) + sp.identity(n)
    Srp, Sc = _lower_pattern(S)
    return sp.csr_matrix(A), Srp, Sc


def test_spai_hand_example_2x2():
    # A = [[2,1],[1,2]], full pattern, start 0.  Normal matrix B = A^T A = [[5,4],[4,5]];
    # column 0: b = [2,1], z = r/5, p = [0.4,0.2], r.z = 1, Bp = [2.8,2.6], p.Bp = 1.64,
    # x = p/1.64.  Two steps solve the 2x2 system: the inverse [[2,-1],[-1,2]]/3.
    A = sp.csr_matrix(np.array([[2.0, 1.0], [1.0, 2.0]]))
    Srp = np.array([0, 1, 3], dtype=np.int64)
    Sc = np.array([0, 0, 1], dtype=np.int32)
    Y1 = oracle.spai_refine(A, Srp, Sc, np.zeros(3), 1)
    np.testing.assert_allclose(Y1, [0.4 / 1.64, 0.2 / 1.64, 0.4 / 1.64], rtol=1e-15)
    Y2 = oracle.spai_refine(A, Srp, Sc, np.zeros(3), 2)
    np.testing.assert_allclose(Y2, [2 / 3, -1 / 3, 2 / 3], rtol=1e-14)


def test_spai_converges_to_least_squares_columns():
    # enough steps: each column is the least-squares minimiser on its pattern (LAPACK gelsd)
    A, Srp, Sc = _spai_case()
    n = A.shape[0]
    cols = oracle.spai_columns(A, Srp, Sc, np.zeros(len(Sc)), 200)
    Ad = A.toarray()
    for j, (J, m) in enumerate(cols):
        e = np.zeros(n)
        e[j] = 1.0
        ref = np.linalg.lstsq(Ad[:, J], e, rcond=None)[0]
        np.testing.assert_allclose(m, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    # and the symmetrised values are the average of the two least-squares columns
    Y = oracle.spai_refine(A, Srp, Sc, np.zeros(len(Sc)), 200)
    look = [dict(zip(J.tolist(), m.tolist())) for J, m in cols]
    rows = _rows(Srp)
    for p in range(0, len(Sc), 7):
        i, j = int(rows[p]), int(Sc[p])
        want = look[j][i] if i == j else 0.5 * (look[j][i] + look[i][j])
        assert abs(Y[p] - want) <= 1e-13 * max(1.0, abs(want))


def test_spai_full_pattern_gives_the_inverse():
    A, _, _ = _spai_case(n=14, seed=5)
    Srp, Sc = _lower_pattern(np.ones((14, 14)))
    Y = oracle.spai_refine(A, Srp, Sc, np.zeros(len(Sc)), 60)
    inv = np.linalg.inv(A.toarray())
    np.testing.assert_allclose(Y, inv[_rows(Srp), Sc], rtol=0, atol=1e-12 * np.abs(inv).max())


def test_spai_zero_steps_and_diagonal_matrix():
    A, Srp, Sc = _spai_case(n=20, seed=3)
    X = np.random.default_rng(0).standard_normal(len(Sc))
    np.testing.assert_array_equal(oracle.spai_refine(A, Srp, Sc, X, 0), X)
    # diagonal A: B = diag(a^2) is its own Jacobi preconditioner, so one step reaches
    # e_j / a_j from any start, and further steps stay there (r.z = 0)
    a = np.linspace(0.5, 3.0, 20)
    D = sp.diags(a).tocsr()
    rows = _rows(Srp)
    want = np.where(rows == Sc, 1.0 / a[rows], 0.0)
    for it in (1, 4):
        np.testing.assert_allclose(oracle.spai_refine(D, Srp, Sc, X, it), want, rtol=1e-15, atol=1e-15)


def test_spai_residual_never_grows():
    # CG minimises the B-norm of the error over growing Krylov spaces, and
    # ||A_J x - e_j||^2 = ||x - x*||_B^2 + const, so the residual cannot grow
    A, Srp, Sc = _spai_case(n=40, seed=7)
    n = A.shape[0]
    X = 0.05 * np.random.default_rng(1).standard_normal(len(Sc))
    Ad = A.toarray()
    prev = None
    for it in range(7):
        res = []
        for j, (J, m) in enumerate(oracle.spai_columns(A, Srp, Sc, X, it)):
            e = np.zeros(n)
            e[j] = 1.0
            res.append(np.linalg.norm(Ad[:, J] @ m - e))
        res = np.array(res)
        if prev is not None:
            assert np.all(res <= prev * (1 + 1e-12) + 1e-15)
        prev = res
    assert prev.max() < 0.9  # and it did move


def test_spai_sampled_entries_match_the_full_refinement():
    A, Srp, Sc = _spai_case(n=25, seed=9)
    X = 0.1 * np.random.default_rng(2).standard_normal(len(Sc))
    full = oracle.spai_refine(A, Srp, Sc, X, 3)
    rows = _rows(Srp)
    idx = np.arange(0, len(Sc), 5)
    got = oracle.spai_entries_sampled(A, Srp, Sc, X, 3, list(zip(rows[idx], Sc[idx])))
    np.testing.assert_array_equal(got, full[idx])


def test_spai_pattern_by_breadth_first_search():
    # P = S + {(i, j): graph distance <= p}: brute force by BFS on a small random graph
    A, Srp, Sc = _spai_case(n=35, seed=4)
    n = A.shape[0]
    adj = [set(A[i].indices.tolist()) - {i} for i in range(n)]
    S = set(zip(_rows(Srp).tolist(), Sc.tolist()))
    for p in (0, 1, 2, 3):
        want = set(S)
        for i in range(n):
            dist = {i: 0}
            ring = [i]
            for d in range(1, p + 1):
                ring = [v for u in ring for v in adj[u] if v not in dist]
                for v in ring:
                    dist.setdefault(v, d)
            want |= {(i, j) for j in dist if j <= i}
        Prp, Pc = oracle.spai_pattern(A, Srp, Sc, p)
        assert set(zip(_rows(Prp).tolist(), Pc.tolist())) == want
        assert np.all(Pc[Prp[1:] - 1] == np.arange(n))  # the diagonal ends every row


def test_spai_embed_places_values_on_the_wider_pattern():
    # X on S moved onto P = S + distance-1 pairs: the same values where (i, j) is in S, 0 elsewhere
    A, Srp, Sc = _spai_case(n=18, seed=12)
    X = np.random.default_rng(4).standard_normal(len(Sc))
    np.testing.assert_array_equal(oracle.embed(Srp, Sc, X, Srp, Sc), X)
    Prp, Pc = oracle.spai_pattern(A, Srp, Sc, 1)
    Y = oracle.embed(Srp, Sc, X, Prp, Pc)
    onS = dict(zip(zip(_rows(Srp).tolist(), Sc.tolist()), X.tolist()))
    for (i, j), y in zip(zip(_rows(Prp).tolist(), Pc.tolist()), Y.tolist()):
        assert y == onS.get((i, j), 0.0)
    assert len(Pc) > len(Sc)


def test_selinv_blocks_top_down_over_every_block_is_selinv():
    """The recurrence restricted to listed pivot blocks, given every block from the
    last to the first, is the whole recurrence (bit for bit); a block left out keeps
    its entries untouched (the partition of the elimination DAG relies on both)."""
    from workloads.configs import random_factors
    for f in (plant_2x2(lap2d_32().factors, 0.3, 11), random_factors(300, 0.05, 0.15, 5)):
        S = _S(f)
        G = _selinv(f, S)
        starts = np.flatnonzero(np.asarray(f.pivot_start) != 0)
        Gb = np.zeros(len(S[1]))
        oracle.selinv_blocks(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S, Gb,
                             starts[::-1])
        assert np.array_equal(Gb, G)
        # leave out the first block: its rows of S_lo (and only they) stay zero
        Gc = np.zeros(len(S[1]))
        oracle.selinv_blocks(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S, Gc,
                             starts[::-1][:-1])
        first = starts[1] if len(starts) > 1 else f.n      # columns of the first block
        col = np.asarray(S[1])
        assert np.all(Gc[col < first] == 0.0) and np.array_equal(Gc[col >= first], G[col >= first])


def test_ninv_W_columns_is_the_dense_truncated_series():
    """Columns of W_t = sum_{s<=t} E^t (E = I - L) by the column Horner steps equal
    the dense truncated series at every t; columns computed from W_known columns
    given for the rest agree with computing everything."""
    from workloads.configs import random_factors
    f = random_factors(60, 0.08, 0.1, 3)
    n, m = f.n, 3
    E = -f.L_csr().toarray()
    dense = [np.eye(n)]
    for t in range(1, m + 1):
        dense.append(np.eye(n) + E @ dense[-1])
    W = oracle.ninv_W_columns(n, f.L_rowptr, f.L_col, f.L_val, m, range(n))
    for t in range(m + 1):
        for j in range(n):
            col = np.zeros(n)
            for r, v in W[t][j].items():
                col[r] = v
            assert np.allclose(col, dense[t][:, j], rtol=0, atol=1e-13), (t, j)
    top = list(range(n // 2, n))
    known = {j: {t: W[t][j] for t in range(m + 1)} for j in top}
    W2 = oracle.ninv_W_columns(n, f.L_rowptr, f.L_col, f.L_val, m, range(n // 2), W_known=known)
    for t in range(m + 1):
        for j in range(n // 2):
            assert W2[t][j] == W[t][j]


def test_pcg_jacobi_reaches_the_solution():
    """Jacobi-PCG: n steps solve an SPD system to rounding (CG's finite termination),
    one step is exact for a diagonal matrix, and zero steps return the start."""
    from oracle.spai import pcg_jacobi
    rng = np.random.default_rng(4)
    n = 12
    Q = rng.standard_normal((n, n))
    B = Q @ Q.T + n * np.eye(n)
    b = rng.standard_normal(n)
    x = pcg_jacobi(B, b, np.zeros(n), n)
    assert np.linalg.norm(x - np.linalg.solve(B, b)) <= 1e-10 * np.linalg.norm(np.linalg.solve(B, b))
    Dg = np.diag(rng.uniform(1.0, 5.0, n))
    assert np.allclose(pcg_jacobi(Dg, b, np.zeros(n), 1), b / np.diag(Dg), rtol=1e-15, atol=0)
    x0 = rng.standard_normal(n)
    assert np.array_equal(pcg_jacobi(B, b, x0, 0), x0)


def test_fill_ratios_hand_values():
    assert oracle.fill_inv(30, 10) == 3.0 and oracle.fill_fact(25, 10) == 2.5
