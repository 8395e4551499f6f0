"""Incomplete LDL^T factors (the inputs of the selected-inverse path).

The paper builds every inverse from a block ILDL with drop tolerance tau
(Section 2.1, Eq. (1); Algorithm 1, step 2).  Its JANUS implementation is not
described, so the factorisation here is a stated stand-in:

* symmetric scaling  A_hat = S A S,  S = diag(|a_ii|^{-1/2});
* left-looking ILDL^T of A_hat in the given (nested-dissection) order, with
  adjacent 1x1/2x2 pivots chosen by the Bunch-Kaufman test restricted to the
  pair (j, j+1), alpha = (1 + sqrt 17) / 8, no interchanges;
* drop |l_ij| < tau after each column (block) is formed;
* static pivot sqrt(eps) ||A_hat||_inf for pivots smaller than that;
* exact unscaling  L = S^{-1} L_hat S,  D = S^{-1} D_hat S^{-1},
  so that A ~ L D L^T and the selected-inverse path needs no scale vector.

The arithmetic runs in ``csrc/ildl.c`` (compiled on first use).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "ildl.c")
_LIB = os.path.join(_HERE, "_ildl.so")
BK_ALPHA = (1.0 + np.sqrt(17.0)) / 8.0


def build_lib(force: bool = False) -> str:
    """Compile the factorisation library in place (gcc -O3)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O3", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Result(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("cap", ctypes.c_int64),
        ("colptr", ctypes.POINTER(ctypes.c_int64)), ("row", ctypes.POINTER(ctypes.c_int32)),
        ("val", ctypes.POINTER(ctypes.c_double)), ("pivot_start", ctypes.POINTER(ctypes.c_int8)),
        ("d_diag", ctypes.POINTER(ctypes.c_double)), ("d_off", ctypes.POINTER(ctypes.c_double)),
        ("n_static", ctypes.c_int64), ("n_2x2", ctypes.c_int64),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_lib())
        P = ctypes.c_void_p
        lib.ildl_factor.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, ctypes.POINTER(_Result)]
        lib.ildl_factor.restype = ctypes.c_int
        lib.ildl_free.argtypes = [ctypes.POINTER(_Result)]
        lib.ldl_solve.argtypes = [ctypes.c_int64, P, P, P, P, P, P, P, ctypes.c_int64, ctypes.c_int64]
        lib.ldl_solve.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Factors:
    """L (strictly lower CSR, unit diagonal implied) and block-diagonal D.

    ``pivot_start[j] = 1`` when a pivot block starts at j; the block is 2x2 iff
    ``pivot_start[j+1] = 0``.  ``d_diag[j] = D(j, j)``; ``d_off[j] = D(j+1, j)``
    for the first index of a 2x2 block (0 otherwise).  ``D_packed`` lists each
    block in order: d for a 1x1 block, (d11, d21, d22) for a 2x2 block.
    """
    n: int
    L_rowptr: np.ndarray
    L_col: np.ndarray
    L_val: np.ndarray
    pivot_start: np.ndarray
    d_diag: np.ndarray
    d_off: np.ndarray
    stats: dict = field(default_factory=dict)

    @property
    def nnz_L(self) -> int:
        return int(self.L_rowptr[-1])

    @property
    def D_packed(self) -> np.ndarray:
        return pack_D(self.pivot_start, self.d_diag, self.d_off)

    def L_csr(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.L_val, self.L_col, self.L_rowptr), shape=(self.n, self.n))

    def L_csc_arrays(self):
        C = self.L_csr().tocsc()
        C.sort_indices()
        return (C.indptr.astype(np.int64), C.indices.astype(np.int32), C.data.astype(np.float64))

    def D_dense_blocks(self) -> sp.csr_matrix:
        n = self.n
        rows = [np.arange(n)]; cols = [np.arange(n)]; vals = [self.d_diag]
        two = np.nonzero(self.d_off != 0.0)[0]
        rows += [two, two + 1]; cols += [two + 1, two]; vals += [self.d_off[two], self.d_off[two]]
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))

    def solve(self, B: np.ndarray) -> np.ndarray:
        """(L D L^T)^{-1} B (B of shape (n,) or (n, k))."""
        lib = _load()
        cp, r, v = self._csc_cache()
        X = np.array(B, dtype=np.float64, order="F", copy=True)
        k = 1 if X.ndim == 1 else X.shape[1]
        lib.ldl_solve(self.n, _ptr(cp), _ptr(r), _ptr(v), _ptr(self.pivot_start), _ptr(self.d_diag),
                      _ptr(self.d_off), _ptr(X), k, self.n)
        return X

    def _csc_cache(self):
        if not hasattr(self, "_csc"):
            self._csc = self.L_csc_arrays()
        return self._csc


def pack_D(pivot_start, d_diag, d_off) -> np.ndarray:
    n = len(d_diag)
    ps = np.asarray(pivot_start).astype(bool)
    second = np.zeros(n, dtype=bool)
    second[1:] = ~ps[1:]
    out = []
    starts = np.nonzero(ps)[0]
    two = np.zeros(n, dtype=bool)
    two[:-1] = ps[:-1] & second[1:]
    vals = np.empty(n + int(two.sum()))
    # position of each block start in the packed array
    width = np.where(two[starts], 3, 1)
    pos = np.concatenate([[0], np.cumsum(width)[:-1]])
    vals[pos] = d_diag[starts]
    t = two[starts]
    vals[pos[t] + 1] = d_off[starts[t]]
    vals[pos[t] + 2] = d_diag[starts[t] + 1]
    return vals


def ildl(A: sp.spmatrix, tau: float, allow_2x2: bool = True, alpha: float = BK_ALPHA) -> Factors:
    """Incomplete LDL^T of the symmetric matrix A (already in the wanted order)."""
    lib = _load()
    A = sp.csr_matrix(A, dtype=np.float64)
    n = A.shape[0]
    dA = A.diagonal()
    if np.any(dA == 0.0):
        raise ValueError("zero diagonal entry: symmetric scaling undefined")
    s = 1.0 / np.sqrt(np.abs(dA))
    Ah = sp.diags(s) @ A @ sp.diags(s)
    norm_inf = float(abs(Ah).sum(axis=1).max())
    static_piv = np.sqrt(np.finfo(np.float64).eps) * norm_inf
    low = sp.tril(Ah).tocsc()
    low.sort_indices()
    cp = low.indptr.astype(np.int64); r = low.indices.astype(np.int32); v = low.data.astype(np.float64)
    res = _Result()
    rc = lib.ildl_factor(n, _ptr(cp), _ptr(r), _ptr(v), float(tau), float(alpha), float(static_piv),
                         int(allow_2x2), ctypes.byref(res))
    if rc != 0:
        lib.ildl_free(ctypes.byref(res))
        raise MemoryError("ildl_factor failed")
    try:
        nnz = res.nnz
        Lcp = np.ctypeslib.as_array(res.colptr, shape=(n + 1,)).copy()
        Lr = np.ctypeslib.as_array(res.row, shape=(max(nnz, 1),))[:nnz].copy()
        Lv = np.ctypeslib.as_array(res.val, shape=(max(nnz, 1),))[:nnz].copy()
        ps = np.ctypeslib.as_array(res.pivot_start, shape=(n,)).copy()
        dd = np.ctypeslib.as_array(res.d_diag, shape=(n,)).copy()
        do = np.ctypeslib.as_array(res.d_off, shape=(n,)).copy()
        stats = {"n_static": int(res.n_static), "n_2x2": int(res.n_2x2)}
    finally:
        lib.ildl_free(ctypes.byref(res))
    # unscale: L_ij = Lh_ij s_j / s_i ; D_ij = Dh_ij / (s_i s_j)
    colidx = np.repeat(np.arange(n), np.diff(Lcp))
    Lv = Lv * s[colidx] / s[Lr]
    dd = dd / (s * s)
    do_ = np.zeros(n)
    do_[:-1] = do[:-1] / (s[:-1] * s[1:])
    Lcsc = sp.csc_matrix((Lv, Lr, Lcp), shape=(n, n))
    Lcsr = Lcsc.tocsr()
    Lcsr.sort_indices()
    f = Factors(n=n, L_rowptr=Lcsr.indptr.astype(np.int64), L_col=Lcsr.indices.astype(np.int32),
                L_val=Lcsr.data.astype(np.float64), pivot_start=ps.astype(np.int8), d_diag=dd,
                d_off=do_, stats=stats)
    f.stats.update(tau=tau, nnz_L=f.nnz_L, static_piv=static_piv)
    return f
