"""The 27-point 3-dof elastic-like operator at its stated size (80^3 nodes, n =
1,536,000, ILDL tau = 1e-4), in the launch configuration the benchmark times: SelInv
(scan form: the pair lists of this factor would not fit in memory) in FP64 and in
the BF16 tensor-core form, NInv on its own pattern (m = 2, delta = 1e-1), Mix on
that pattern and the rank-64 correction on the Mix pattern.

The oracle checks the trailing principal block of the factors (the last ~4,096
columns, moved so that no 2x2 pivot is cut): the top of the elimination tree.
SelInv, the Neumann series, the product, Mix and the correction restricted to it
depend on no entry outside it, so the oracle's full computation on the block gives
the workload's own values there; the GPU's entries of the block must match them
(FP64 within 1e-10 entrywise, BF16 within 1e-5 normwise; NInv's pattern may differ
only at its drop threshold, Mix's also where |G| is at eps within rounding)."""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from tests.helpers import normwise, sel_rel_err
from workloads.configs import elastic3d, random_lowrank

pytestmark = pytest.mark.gpu

NODES = 80
BLOCK = 4096


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _block(f, nt):
    c0 = f.n - nt
    while c0 > 0 and not f.pivot_start[c0]:
        c0 -= 1
    L = sp.csr_matrix((f.L_val, f.L_col, f.L_rowptr), shape=(f.n, f.n))[c0:, c0:].tocsr()
    L.sort_indices()
    return c0, dict(n=f.n - c0, rp=L.indptr.astype(np.int64), col=L.indices.astype(np.int32), val=L.data,
                    ps=np.ascontiguousarray(f.pivot_start[c0:]), dd=np.ascontiguousarray(f.d_diag[c0:]),
                    do=np.ascontiguousarray(f.d_off[c0:]))


@pytest.fixture(scope="module")
def full():
    from paper_2609_11363_b300 import Handle
    # the ILDL at 80^3 nodes takes minutes on one host core: a factor cache
    # directory (SINV_FACTOR_CACHE) lets a run reuse the factors of an earlier one
    w = elastic3d(NODES, cache_dir=os.environ.get("SINV_FACTOR_CACHE"))
    f = w.factors
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    c0, b = _block(f, BLOCK)
    Sb = oracle.symbolic_S(b["n"], b["rp"], b["col"], b["ps"])
    Gb = oracle.selinv(b["n"], b["rp"], b["col"], b["val"], b["ps"], b["dd"], b["do"], Sb)
    return w, f, h, c0, b, Sb, Gb


def _block_of_S(h, c0, nb):
    """positions in S_lo of the block's entries, in the block's S_lo order"""
    rp, col = h.pattern_host()
    pos = []
    for i in range(c0, c0 + nb):
        cols = col[rp[i]:rp[i + 1]]
        pos.append(rp[i] + np.nonzero(cols >= c0)[0])
    return np.concatenate(pos)


def test_full_size_selinv_on_the_trailing_block(full):
    w, f, h, c0, b, Sb, Gb = full
    st = h.stats()
    assert f.n == 3 * NODES ** 3 and st["selinv_scan"] == 1
    Lv, Dv = _dev(f.L_val), _dev(f.D_packed)
    pos = _block_of_S(h, c0, b["n"])
    G = h.selinv(Lv, Dv, "fp64").cpu().numpy()
    h.sync_status()
    assert len(pos) == len(Sb[1])
    assert sel_rel_err(G[pos], Gb, *Sb) <= 1e-10
    Gh = h.selinv(Lv, Dv, "bf16").cpu().numpy()
    h.sync_status()
    assert normwise(Gh[pos], Gb) <= 1e-5
    assert np.all(np.isfinite(Gh))


def test_full_size_ninv_mix_lowrank_on_the_trailing_block(full):
    w, f, h, c0, b, Sb, Gb = full
    m, delta = w.m, 1e-1
    Lv, Dv = _dev(f.L_val), _dev(f.D_packed)
    G = h.selinv(Lv, Dv, "fp64")
    eps = 1e-3 * float(G.abs().max())
    V, lam = random_lowrank(f.n, w.k, seed=5)
    lam = lam * 1e3
    h.ninv_own(Lv, Dv, m, delta, copy=False)
    cp, rows, vals = h.mix_own(G, eps)
    before = vals.cpu().numpy().copy()
    h.lowrank_correct_mix_own(_dev(V), _dev(lam), "fp64")
    _, _, after = h.mix_own_result()
    h.sync_status()
    cp, rows, after = cp.cpu().numpy(), rows.cpu().numpy(), after.cpu().numpy()
    cols = np.repeat(np.arange(f.n), np.diff(cp))
    inb = cols >= c0
    got = {(int(i) - c0, int(j) - c0): (bv, av) for i, j, bv, av in zip(rows[inb], cols[inb], before[inb], after[inb])}
    # the oracle's chain on the block
    nb = b["n"]
    Nb = oracle.ninv_own(nb, b["rp"], b["col"], b["val"], b["ps"], b["dd"], b["do"], m, delta)
    Rb = oracle.mix_own(nb, Sb[0], Sb[1], Gb, Nb, eps)
    Rv = oracle.lowrank_correct(Rb.indptr.astype(np.int64), Rb.indices.astype(np.int32), Rb.data,
                                V[c0:], lam)
    Rc = Rb.tocoo()
    ref = {(int(i), int(j)): (x, y) for i, j, x, y in zip(Rc.row, Rc.col, Rc.data,
                                                          sp.csc_matrix((Rv, Rb.indices, Rb.indptr),
                                                                        shape=Rb.shape).tocoo().data)}
    d = np.abs(Nb.diagonal())
    srow = np.repeat(np.arange(nb), np.diff(Sb[0]))
    gmap = {(int(i), int(j)): g for i, j, g in zip(srow, Sb[1], Gb)}
    for key in set(ref) ^ set(got):   # at NInv's drop threshold, or |G| at eps
        v = (ref.get(key) or got.get(key))[0]
        g = gmap.get(key)
        thr = delta * np.sqrt(d[key[0]] * d[key[1]])
        assert abs(abs(v) - thr) <= 1e-9 * thr or (g is not None and abs(abs(g) - eps) <= 1e-9 * eps), key
    common = sorted(set(ref) & set(got))
    assert len(common) >= 0.999 * len(ref)
    scale = np.array([np.sqrt(d[i] * d[j]) for i, j in common])
    for k in (0, 1):                   # Mix, then Mix + the correction
        a = np.array([got[c][k] for c in common])
        r = np.array([ref[c][k] for c in common])
        assert np.max(np.abs(a - r) / (np.abs(r) + scale)) <= 1e-10, k
