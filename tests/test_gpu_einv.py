"""GPU parity of the spectral-correction producer (Section 2.5): Lanczos on
E_inv = A^{-1} - A^inv with ILDL-preconditioned CG solves, against the FP64
oracle (exact sparse LU solves) from the same start vector.

Tolerance: Ritz values within 1e-9 max|lambda| and Ritz vectors within
1 - 1e-8 in |cosine|.  The CG solves stop at a relative residual of 1e-13, so
each application of E_inv differs from the oracle's by about kappa(A) 1e-13
relative; the Lanczos iteration with full reorthogonalisation is backward stable
and passes that on at the same order.  The oracle's own mirror of the GPU
arithmetic agreed to 5e-14.  A wrong kernel is off by O(1).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
import oracle.core
from workloads.configs import covariance, lap2d_32, plant_2x2

pytestmark = pytest.mark.gpu


def _handle(f):
    from paper_2609_11363_b300 import Handle
    return Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)


def _ldlt(f):
    """L D L^T, symmetrised as (M + M^T)/2: the sparse product drops exact cancellations,
    which rounding can make differ between the two triangles."""
    L = f.L_csr() + sp.identity(f.n, format="csr")
    M = sp.csr_matrix(L @ f.D_dense_blocks() @ L.T)
    A = sp.csr_matrix(0.5 * (M + M.T))
    A.sum_duplicates()
    A.sort_indices()
    return A


def _case(name):
    if name == "lap2d":
        w = lap2d_32()
        return w.A, w.factors
    if name == "covariance_24":
        w = covariance(24)
        return w.A, w.factors
    # A = L D L^T exactly, with SPD 2x2 blocks planted in D: the preconditioner is A^{-1}
    f = plant_2x2(lap2d_32().factors, 0.3, 11)
    return _ldlt(f), f


def _run(A, f, k, steps, seed=0, grid_solve=False):
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    q0 = np.random.default_rng(seed).standard_normal(f.n)
    h = _handle(f)
    Ac = h.einv_analyse(A)
    h.einv_set_solver("cg", grid_solve=grid_solve)
    lam, V, info = h.einv_lanczos(torch.as_tensor(Ac.data, device="cuda"), torch.as_tensor(f.L_val, device="cuda"),
                                  torch.as_tensor(f.D_packed, device="cuda"), torch.as_tensor(G, device="cuda"),
                                  torch.as_tensor(q0, device="cuda"), k, steps, cg_tol=1e-13, cg_maxit=3000)
    h.sync_status()
    Xs = oracle.core.sym_from_S(f.n, S[0], S[1], G)
    return lam, V.cpu().numpy(), info, S, G, Xs, q0


@pytest.mark.parametrize("grid_solve", [False, True], ids=["cta_solve", "grid_solve"])
@pytest.mark.parametrize("name", ["lap2d", "covariance_24", "exact_2x2"])
def test_lanczos_parity(name, grid_solve):
    """Both triangular solves: one CTA walking the levels (the choice for these
    factors, whose levels hold few rows) and the persistent grid."""
    A, f = _case(name)
    k, steps = 4, 40
    lam, V, info, S, G, Xs, q0 = _run(A, f, k, steps, grid_solve=grid_solve)
    lo, Vo = oracle.lanczos_einv(A, Xs, k, steps=steps, q0=q0)
    assert info["steps"] == steps and info["cg_unconverged"] == 0
    scale = np.abs(lo).max()
    np.testing.assert_allclose(lam, lo, rtol=0, atol=1e-9 * scale)
    for l in range(k):
        c = abs(V[:, l] @ Vo[:, l]) / (np.linalg.norm(V[:, l]) * np.linalg.norm(Vo[:, l]))
        assert c >= 1 - 1e-8, (l, c)


def test_exact_factors_make_cg_converge_in_one_step():
    # with A = L D L^T the preconditioner L^{-T} D^{-1} L^{-1} is A^{-1} (2x2 blocks included),
    # so every CG solve stops after one iteration: a check of the triangular solves and D^{-1}
    A, f = _case("exact_2x2")
    assert int(np.sum(f.pivot_start == 0)) > 0
    lam, V, info, *_ = _run(A, f, 2, 12)
    assert info["cg_iterations"] <= 2 * 12 and info["cg_unconverged"] == 0


def test_dominant_eigenvalue_vs_dense():
    # the dominant eigenpair of E_inv = inv(A) - A^inv from a dense eigensolver (LAPACK)
    A, f = _case("lap2d")
    lam, V, info, S, G, Xs, q0 = _run(A, f, 1, 60)
    E = np.linalg.inv(A.toarray()) - Xs.toarray()
    ev, U = np.linalg.eigh(E)
    i = np.argmax(np.abs(ev))
    assert abs(lam[0] - ev[i]) <= 1e-9 * abs(ev[i])
    c = abs(V[:, 0] @ U[:, i]) / np.linalg.norm(V[:, 0])
    assert c >= 1 - 1e-8


def test_lanczos_errors():
    from paper_2609_11363_b300 import SinvError
    A, f = _case("lap2d")
    h = _handle(f)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    Lv, Dv = dev(f.L_val), dev(f.D_packed)
    X = torch.zeros(h.nnz_S, dtype=torch.float64, device="cuda")
    q0 = torch.ones(f.n, dtype=torch.float64, device="cuda")
    Av = dev(sp.csr_matrix(A).data)
    with pytest.raises(SinvError) as e:
        h.einv_lanczos(Av, Lv, Dv, X, q0, 2, 10)  # no analysis
    assert e.value.name == "SINV_ERR_INVALID_ARG"
    Ac = h.einv_analyse(A)
    Av = dev(Ac.data)
    for k, steps, name in [(5, 4, "SINV_ERR_INVALID_ARG"), (0, 4, "SINV_ERR_INVALID_ARG"),
                           (2, 300, "SINV_ERR_UNSUPPORTED")]:
        with pytest.raises(SinvError) as e:
            h.einv_lanczos(Av, Lv, Dv, X, q0, k, steps)
        assert e.value.name == name
    with pytest.raises(SinvError) as e:
        h.einv_lanczos(Av, Lv, Dv, X, torch.zeros_like(q0), 2, 4)
    assert e.value.name == "SINV_ERR_INVALID_ARG"


def _indefinite_exact():
    """A = L D L^T exactly with an indefinite D: negated 1x1 pivots and 2x2 blocks,
    one of them indefinite (negative determinant)."""
    import dataclasses
    f = plant_2x2(lap2d_32().factors, 0.3, 11)
    dd, do = f.d_diag.copy(), f.d_off.copy()
    rng = np.random.default_rng(7)
    ones = np.nonzero((f.pivot_start == 1) & (np.r_[f.pivot_start[1:], 1] == 1))[0]
    dd[rng.choice(ones, len(ones) // 5, replace=False)] *= -1.0
    twos = np.nonzero((f.pivot_start == 1) & (np.r_[f.pivot_start[1:], 1] == 0))[0]
    assert len(twos) >= 2
    b = twos[0]
    dd[b + 1] = -abs(dd[b + 1])        # det = a d - b^2 < 0
    g = dataclasses.replace(f, d_diag=dd, d_off=do)
    return _ldlt(g), g


def _run_solver(A, f, k, steps, solver, seed=0, grid_solve=False):
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    q0 = np.random.default_rng(seed).standard_normal(f.n)
    h = _handle(f)
    Ac = h.einv_analyse(A)
    h.einv_set_solver(solver, grid_solve=grid_solve)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    lam, V, info = h.einv_lanczos(dev(Ac.data), dev(f.L_val), dev(f.D_packed), dev(G), dev(q0), k, steps,
                                  cg_tol=1e-13, cg_maxit=3000)
    h.sync_status()
    return lam, V.cpu().numpy(), info, oracle.core.sym_from_S(f.n, S[0], S[1], G), q0


def test_minres_exact_indefinite_factors_converge_in_two_steps():
    """With A = L D L^T and M = L |D| L^T, M^{-1} A has the eigenvalues +1 and -1 only,
    so every MINRES solve ends after two iterations: a check of |D|^{-1} (2x2 blocks,
    one indefinite, included) and of the persistent triangular solves."""
    A, f = _indefinite_exact()
    ev = np.linalg.eigvalsh(A.toarray())
    assert ev.min() < 0 < ev.max()
    lam, V, info, Xs, q0 = _run_solver(A, f, 2, 10, "minres")
    assert info["cg_unconverged"] == 0 and info["cg_iterations"] <= 2 * 10
    lo, Vo = oracle.lanczos_einv(A, Xs, 2, steps=10, q0=q0)
    np.testing.assert_allclose(lam, lo, rtol=0, atol=1e-9 * np.abs(lo).max())


@pytest.mark.parametrize("grid_solve", [False, True], ids=["cta_solve", "grid_solve"])
@pytest.mark.parametrize("name", ["diff3d_shifted", "lap2d"])
def test_minres_lanczos_parity(name, grid_solve):
    """Indefinite A (3D diffusion shifted into its first spectral gap, planted 2x2
    pivots) and an SPD case, MINRES inner solves against the oracle's exact ones."""
    from workloads.configs import diff3d
    if name == "lap2d":
        w = lap2d_32()
        A, f = w.A, w.factors
    else:
        w = diff3d(10, m=3)
        A, f = w.A, plant_2x2(w.factors, 0.05, 13)
    k, steps = 3, 30
    lam, V, info, Xs, q0 = _run_solver(A, f, k, steps, "minres", grid_solve=grid_solve)
    lo, Vo = oracle.lanczos_einv(A, Xs, k, steps=steps, q0=q0)
    assert info["steps"] == steps and info["cg_unconverged"] == 0
    np.testing.assert_allclose(lam, lo, rtol=0, atol=1e-8 * np.abs(lo).max())
    for l in range(k):
        c = abs(V[:, l] @ Vo[:, l]) / (np.linalg.norm(V[:, l]) * np.linalg.norm(Vo[:, l]))
        assert c >= 1 - 1e-7, (l, c)
