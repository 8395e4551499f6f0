"""GPU parity of the SPAI refinement (Section 2.4) against the FP64 oracle.

Tolerance: FP64, entrywise |x_ij - r_ij| <= tol (|r_ij| + sqrt|r_ii r_jj|),
the rule of the other FP64 parity tests, with tol = max(1e-10, 64 sigma).
sigma is the oracle's own sensitivity to rounding: the largest change of its
result when X is perturbed by one unit in the last place (two seeded sign
patterns).  A fixed number of CG steps is a rounding-sensitive function of its
inputs while a column is still converging (the perturbation grows by a few
times per step), so sigma is about 1e-16 for a few steps and after
convergence, and larger in between; a wrong kernel is off by O(1).  iters = 0
is exact.  The start values X are seeded random symmetric values on S (the
oracle takes nothing from the CUDA path); one test runs the whole Mix-SPAI
chain on both sides.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from tests.helpers import s_rows, sel_rel_err
from workloads.configs import covariance, diff3d, elastic3d, lap2d_32, plant_2x2, random_factors

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _ldlt(f):
    L = f.L_csr() + sp.identity(f.n, format="csr")
    A = sp.csr_matrix(L @ f.D_dense_blocks() @ L.T)
    A.sum_duplicates()
    A.sort_indices()
    return A


def _case_lap2d():
    w = lap2d_32()
    return w.A, w.factors


def _case_cov():
    w = covariance(24)
    return w.A, w.factors


def _case_diff3d():
    w = diff3d(10, m=3)
    return w.A, plant_2x2(w.factors, 0.05, 4)


def _case_random():
    f = random_factors(300, 0.02, 0.1, 8)
    return _ldlt(f), f


def _case_elastic():
    w = elastic3d(5)
    return w.A, w.factors


CASES = {"lap2d": _case_lap2d, "covariance_24": _case_cov, "diff3d_10_planted": _case_diff3d,
         "random_ldlt": _case_random, "elastic3d_5": _case_elastic}


def _handle(f, **kw):
    from paper_2609_11363_b300 import Handle
    return Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, **kw)


def _start(S, seed):
    """Seeded start values on S_lo: a diagonal of about 1/a_ii scale plus small couplings."""
    rng = np.random.default_rng(seed)
    rows = s_rows(S[0])
    X = 0.05 * rng.standard_normal(len(S[1]))
    X[rows == S[1]] = rng.uniform(0.5, 1.5, int(np.sum(rows == S[1])))
    return X


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    A, f = CASES[request.param]()
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    return request.param, A, f, S


def _tolerance(A, P, X, iters, ref):
    """max(1e-10, 64 sigma): sigma = the oracle's change under a one-ulp perturbation of X
    (X and ref on the pattern P)."""
    sigma = 0.0
    for seed in (1, 2):
        sgn = np.where(np.random.default_rng(seed).random(len(X)) < 0.5, -1.0, 1.0)
        Xp = X * (1.0 + sgn * np.finfo(np.float64).eps)
        sigma = max(sigma, sel_rel_err(oracle.spai_refine(A, P[0], P[1], Xp, iters), ref, P[0], P[1]))
    return max(TOL64, 64.0 * sigma), sigma


def _oracle_on_P(A, S, X_S, power, iters):
    """(P, X on P, oracle result on P) with P from the oracle's own pattern rule."""
    P = oracle.spai_pattern(A, S[0], S[1], power)
    XP = oracle.embed(S[0], S[1], X_S, P[0], P[1])
    return P, XP, oracle.spai_refine(A, P[0], P[1], XP, iters)


@pytest.mark.parametrize("power", [0, 2])
@pytest.mark.parametrize("iters", [0, 1, 4, 15, 60])
def test_spai_parity(case, iters, power):
    name, A, f, S = case
    X = _start(S, 21)
    h = _handle(f)
    Ac = h.spai_analyse(A, power=power)
    Y = h.spai(torch.as_tensor(Ac.data, device="cuda"), torch.as_tensor(X, device="cuda"), iters)
    h.sync_status()
    P, XP, ref = _oracle_on_P(A, S, X, power, iters)
    rp, col = h.spai_pattern()
    assert np.array_equal(rp, P[0]) and np.array_equal(col, P[1])
    got = Y.cpu().numpy()
    if iters == 0:
        np.testing.assert_array_equal(got, XP)
    tol, sigma = _tolerance(A, P, XP, iters, ref) if iters > 4 else (TOL64, 0.0)
    err = sel_rel_err(got, ref, P[0], P[1])
    assert err <= tol, (name, iters, power, err, sigma)


@pytest.mark.parametrize("name", ["lap2d", "covariance_24", "elastic3d_5"])
def test_spai_cta_tier(name):
    # warp_entries = 1 moves every column that stages more than one entry to the CTA tier
    A, f = CASES[name]()
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    X = _start(S, 5)
    h = _handle(f)
    Ac = h.spai_analyse(A, power=1, warp_entries=1)
    st = h.stats()
    assert st["spai_cols_cta"] == f.n and st["spai_cols_warp"] == 0
    Y = h.spai(torch.as_tensor(Ac.data, device="cuda"), torch.as_tensor(X, device="cuda"), 6)
    h.sync_status()
    P, XP, ref = _oracle_on_P(A, S, X, 1, 6)
    tol, sigma = _tolerance(A, P, XP, 6, ref)
    assert sel_rel_err(Y.cpu().numpy(), ref, P[0], P[1]) <= tol, sigma


def test_spai_tiers_split_by_size():
    A, f = _case_elastic()
    h = _handle(f)
    h.spai_analyse(A)
    st = h.stats()
    assert st["spai_cols_warp"] + st["spai_cols_cta"] == f.n
    assert st["spai_cols_cta"] > 0  # 81 entries a row: long columns need a CTA
    A2, f2 = _case_lap2d()
    h2 = _handle(f2)
    h2.spai_analyse(A2)
    st2 = h2.stats()
    assert st2["spai_cols_warp"] == f2.n and st2["spai_entries"] > 0


def test_mix_spai_chain_lap2d():
    # SelInv, NInv (m = 3), Mix and SPAI on the GPU against the same chain in the oracle
    w = lap2d_32()
    f, A = w.factors, w.A
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    N = oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, 3, S)
    eps = 1e-3 * float(np.abs(G).max())
    Mx = oracle.mix(G, N, eps)
    ref = oracle.spai_refine(A, S[0], S[1], Mx, 10)
    tol, sigma = _tolerance(A, S, Mx, 10, ref)  # P = S here
    h = _handle(f)
    Lv = torch.as_tensor(f.L_val, device="cuda")
    Dv = torch.as_tensor(f.D_packed, device="cuda")
    Gd = h.selinv(Lv, Dv, "fp64")
    Nd = h.ninv(Lv, Dv, 3, "fp64")
    Md = h.mix(Gd, Nd, eps)
    Ac = h.spai_analyse(A)
    Y = h.spai(torch.as_tensor(Ac.data, device="cuda"), Md, 10)
    h.sync_status()
    assert sel_rel_err(Y.cpu().numpy(), ref, S[0], S[1]) <= tol, sigma


def test_mix_spai_chain_covariance_widened():
    # the covariance example with P = S + distance-2 neighbourhoods and 20 steps: the GPU
    # chain matches the oracle chain, and (as the paper reports for its covariance cases)
    # Mix-SPAI's diagonal is closer to diag(A^{-1}) than Mix's
    w = covariance(24)
    f, A = w.factors, w.A
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    N = oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, 3, S)
    eps = 1e-3 * float(np.abs(G).max())
    Mx = oracle.mix(G, N, eps)
    P, XP, ref = _oracle_on_P(A, S, Mx, 2, 20)
    tol, sigma = _tolerance(A, P, XP, 20, ref)
    h = _handle(f)
    Lv = torch.as_tensor(f.L_val, device="cuda")
    Dv = torch.as_tensor(f.D_packed, device="cuda")
    Md = h.mix(h.selinv(Lv, Dv, "fp64"), h.ninv(Lv, Dv, 3, "fp64"), eps)
    Ac = h.spai_analyse(A, power=2)
    Y = h.spai(torch.as_tensor(Ac.data, device="cuda"), Md, 20)
    h.sync_status()
    got = Y.cpu().numpy()
    assert sel_rel_err(got, ref, P[0], P[1]) <= tol, sigma
    d_exact = np.diag(np.linalg.inv(A.toarray()))
    e_mix = oracle.err1(d_exact, Mx[np.asarray(S[0][1:]) - 1])
    e_spai = oracle.err1(d_exact, got[np.asarray(P[0][1:]) - 1])
    assert e_spai < 0.2 * e_mix, (e_spai, e_mix)


def test_spai_graph_replay():
    A, f = _case_cov()
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    h = _handle(f)
    Ac = h.spai_analyse(A)
    Av = torch.as_tensor(Ac.data, device="cuda")
    X = torch.as_tensor(_start(S, 3), device="cuda")
    Y = torch.empty(h.nnz_P, dtype=torch.float64, device="cuda")
    h.spai(Av, X, 5, out=Y)
    torch.cuda.synchronize()
    want = Y.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        h.spai(Av, X, 5, out=Y, stream=s)
    Y.zero_()
    g.replay()
    torch.cuda.synchronize()
    h.sync_status()
    d = (Y - want).abs().max().item()
    assert d <= 1e-12 * want.abs().max().item()


def test_spai_errors():
    from paper_2609_11363_b300 import SinvError
    A, f = _case_lap2d()
    h = _handle(f)
    X = torch.zeros(h.nnz_S, dtype=torch.float64, device="cuda")
    Av = torch.as_tensor(sp.csr_matrix(A).data, device="cuda")
    with pytest.raises(SinvError) as e:
        h.spai(Av, X, 3)  # no analysis yet
    assert e.value.name == "SINV_ERR_INVALID_ARG"
    Ac = h.spai_analyse(A)
    Av = torch.as_tensor(Ac.data, device="cuda")
    with pytest.raises(SinvError) as e:
        h.spai(Av, X, -1)
    assert e.value.name == "SINV_ERR_INVALID_ARG"
    with pytest.raises(SinvError) as e:
        h.spai(Av, X, 3, out=X)  # in place is not allowed
    assert e.value.name == "SINV_ERR_INVALID_ARG"
    with pytest.raises(SinvError) as e:
        h.spai_analyse(A, warp_entries=-1)
    assert e.value.name == "SINV_ERR_INVALID_ARG"
    B = sp.csr_matrix(A, copy=True).tolil()
    B[0, f.n - 1] = 1.0  # one entry without its mirror
    with pytest.raises(SinvError) as e:
        h.spai_analyse(B.tocsr())
    assert e.value.name == "SINV_ERR_PATTERN"


@pytest.mark.slow
def test_full_size_64_spai_sampled():
    # the 64^3 shifted diffusion workload in the bench's launch configuration (one handle,
    # default tiers, 10 steps): 200 sampled entries against the oracle's columns, with the
    # tolerance rule above measured on the same samples
    w = diff3d(64)
    f = plant_2x2(w.factors, 0.02, 2)
    h = _handle(f)
    rp, col = h.pattern_host()
    X = _start((rp, col), 64)
    Ac = h.spai_analyse(w.A)
    Y = h.spai(torch.as_tensor(Ac.data, device="cuda"), torch.as_tensor(X, device="cuda"), 10)
    h.sync_status()
    rows = s_rows(rp)
    idx = np.random.default_rng(7).choice(len(col), 200, replace=False)
    nodes = np.unique(np.r_[rows[idx], col[idx]])
    pairs = list(zip(rows[idx], col[idx])) + [(i, i) for i in nodes]

    def sampled(Xs):
        v = oracle.spai_entries_sampled(w.A, rp, col, Xs, 10, pairs)
        diag = np.zeros(f.n)
        diag[nodes] = v[len(idx):]
        return v[:len(idx)], diag

    ref, diag = sampled(X)
    scale = np.abs(ref) + np.sqrt(np.abs(diag[rows[idx]] * diag[col[idx]]))
    sgn = np.where(np.random.default_rng(1).random(len(X)) < 0.5, -1.0, 1.0)
    pert, _ = sampled(X * (1.0 + sgn * np.finfo(np.float64).eps))
    sigma = np.max(np.abs(pert - ref) / scale)
    got = Y.cpu().numpy()[idx]
    assert np.max(np.abs(got - ref) / scale) <= max(TOL64, 64.0 * sigma), sigma


@pytest.mark.parametrize("name", ["covariance_24", "lap2d", "diff3d_10_planted"])
@pytest.mark.parametrize("iters", [0, 3, 20])
def test_mix_spai_on_mix_own_pattern(name, iters):
    """Mix-SPAI on the pattern of Mix built on NInv's own loose-tolerance pattern
    (delta = 1e-1; Sections 2.3-2.4).  The GPU's Mix pattern must be the oracle's
    (these cases have no entry at a drop threshold); the refinement then starts from
    the oracle's Mix values (given in the GPU's Mix order) and is held to the SPAI
    tolerance; from the handle's own Mix values, zero steps return those values."""
    A, f = CASES[name]()
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    eps, m, delta = 1e-3 * np.abs(G).max(), 3, 1e-1
    h = _handle(f)
    Lv = torch.as_tensor(f.L_val, device="cuda")
    Dv = torch.as_tensor(f.D_packed, device="cuda")
    h.ninv_own(Lv, Dv, m, delta)
    cp, rows, vals = h.mix_own(torch.as_tensor(G, device="cuda"), eps)
    cp, rows, vals = cp.cpu().numpy().copy(), rows.cpu().numpy().copy(), vals.cpu().numpy().copy()
    Nref = oracle.ninv_own(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, m, delta)
    R = oracle.mix_own(f.n, S[0], S[1], G, Nref, eps).tocsr()
    R.sort_indices()
    cols = np.repeat(np.arange(f.n), np.diff(cp))
    gpu_keys = set(zip(rows.tolist(), cols.tolist()))
    Rc = R.tocoo()
    assert gpu_keys == set(zip(Rc.row.tolist(), Rc.col.tolist())), name
    Ac = h.spai_analyse_mix_own(A)
    rp, col = h.spai_pattern()
    assert np.array_equal(rp, R.indptr) and np.array_equal(col, R.indices)
    Av = torch.as_tensor(Ac.data, device="cuda")
    # the oracle's Mix values in the GPU's Mix order
    X = np.asarray(R[rows, cols]).ravel()
    Y = h.spai_mix_own(Av, iters, X=torch.as_tensor(X, device="cuda")).cpu().numpy()
    h.sync_status()
    ref = oracle.spai_refine(A, R.indptr, R.indices, R.data, iters)
    tol, sigma = _tolerance(A, (R.indptr, R.indices), R.data, iters, ref) if iters > 4 else (TOL64, 0.0)
    err = sel_rel_err(Y, ref, R.indptr, R.indices)
    assert err <= tol, (name, iters, err, sigma)
    if iters == 0:
        Y0 = h.spai_mix_own(Av, 0).cpu().numpy()
        M = sp.csc_matrix((vals, rows, cp), shape=(f.n, f.n)).tocsr()
        M.sort_indices()
        np.testing.assert_array_equal(Y0, M.data)
