"""Batched execution: many matrices of uneven size in one handle (block-diagonal
concatenation), one persistent SelInv launch and one launch per NInv step for
all of them, and the whole step captured and replayed as a CUDA graph."""
import numpy as np
import pytest
import torch

import oracle
from tests.helpers import normwise, sel_rel_err
from workloads.configs import batch9pt_member, plant_2x2, random_factors, random_lowrank

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _members():
    # uneven sizes: 9-point random-weight Laplacians (the batched workload's generator,
    # smaller size range) plus a random non-closed pattern with 2x2 pivots
    fs = [batch9pt_member(3000 + i, n_range=(300, 2500)).factors for i in range(5)]
    fs.append(random_factors(400, 0.03, 0.2, 21))
    fs.insert(2, plant_2x2(batch9pt_member(3100, n_range=(300, 2500)).factors, 0.1, 4))
    return fs


@pytest.fixture(scope="module")
def batch():
    from paper_2609_11363_b300 import Handle
    fs = _members()
    h = Handle.batch(fs)
    refs = []
    for f in fs:
        S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
        G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
        N = oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, 3, S)
        refs.append((S, G, N))
    Lv = _dev(np.concatenate([f.L_val for f in fs]))
    Dv = _dev(np.concatenate([f.D_packed for f in fs]))
    return fs, h, refs, Lv, Dv


def _split(x, lay, b):
    return x[lay["S"][b]:lay["S"][b + 1]]


def test_batch_layout_and_pattern(batch):
    fs, h, refs, Lv, Dv = batch
    lay = h.layout()
    rp, col = h.pattern_host()
    for b, (f, (S, G, N)) in enumerate(zip(fs, refs)):
        r0, s0 = lay["n"][b], lay["S"][b]
        assert np.array_equal(col[s0:lay["S"][b + 1]] - r0, S[1])
        assert np.array_equal(rp[r0:r0 + f.n + 1] - s0, S[0])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_selinv_ninv_match_per_matrix_oracle(batch, prec):
    fs, h, refs, Lv, Dv = batch
    lay = h.layout()
    G = h.selinv(Lv, Dv, prec).cpu().numpy()
    N = h.ninv(Lv, Dv, 3, prec).cpu().numpy()
    h.sync_status()
    for b, (S, Gr, Nr) in enumerate(refs):
        if prec == "fp64":
            assert sel_rel_err(_split(G, lay, b), Gr, *S) <= TOL64, b
            assert sel_rel_err(_split(N, lay, b), Nr, *S) <= TOL64, b
        else:
            assert normwise(_split(G, lay, b), Gr) <= 1e-5, b
            assert normwise(_split(N, lay, b), Nr) <= 1e-5, b


def test_batch_step_in_cuda_graph(batch):
    """SelInv + NInv + Mix + rank-k correction captured once, replayed twice with new
    factor values copied into the captured input buffers."""
    fs, h, refs, Lv, Dv = batch
    lay = h.layout()
    n = sum(f.n for f in fs)
    V, lam = random_lowrank(n, 8, seed=2)
    Vd, ld = _dev(V), _dev(lam)
    Lin, Din = Lv.clone(), Dv.clone()
    G = torch.empty(h.nnz_S, dtype=torch.float64, device="cuda")
    N = torch.empty_like(G)
    M = torch.empty_like(G)
    eps = 1e-3

    def step():
        h.selinv(Lin, Din, "fp64", out=G)
        h.ninv(Lin, Din, 3, "fp64", out=N)
        h.mix(G, N, eps, out=M)
        h.lowrank_correct(Vd, ld, M, "fp64")

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()  # warm-up: work buffers and the Neumann pattern exist before capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for scale in (1.0, 0.5):
        Lin.copy_(Lv * scale)
        Din.copy_(Dv)
        graph.replay()
        torch.cuda.synchronize()
        h.sync_status()
        Gh = G.cpu().numpy()
        Mh = M.cpu().numpy()
        for b, f in enumerate(fs):
            S = refs[b][0]
            Lb = f.L_val * scale
            Gr = oracle.selinv(f.n, f.L_rowptr, f.L_col, Lb, f.pivot_start, f.d_diag, f.d_off, S)
            Nr = oracle.ninv(f.n, f.L_rowptr, f.L_col, Lb, f.pivot_start, f.d_diag, f.d_off, 3, S)
            r0 = lay["n"][b]
            Mr = oracle.lowrank_correct(S[0], S[1], oracle.mix(Gr, Nr, eps), V[r0:r0 + f.n], lam)
            assert sel_rel_err(_split(Gh, lay, b), Gr, *S) <= TOL64, (scale, b)
            assert sel_rel_err(_split(Mh, lay, b), Mr, *S) <= TOL64, (scale, b)


def _gen_member(seed):
    return batch9pt_member(seed).factors


@pytest.mark.slow
def test_full_batch_256_sampled_members():
    """The 256-matrix batched workload at full size (n ~ U[2048, 65536], seeds 3000+),
    in the benchmark's form (FP32, one handle, m = 3): four members (the smallest, the
    largest and two seeded picks) against the oracle in full, and the FP64 form of the
    same members at the FP64 tolerance."""
    import multiprocessing as mp
    import os

    from paper_2609_11363_b300 import Handle
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        fs = pool.map(_gen_member, [3000 + i for i in range(256)])
    h = Handle.batch(fs)
    lay = h.layout()
    Lv = _dev(np.concatenate([f.L_val for f in fs]))
    Dv = _dev(np.concatenate([f.D_packed for f in fs]))
    G32 = h.selinv(Lv, Dv, "fp32").cpu().numpy()
    N32 = h.ninv(Lv, Dv, 3, "fp32").cpu().numpy()
    G64 = h.selinv(Lv, Dv, "fp64").cpu().numpy()
    N64 = h.ninv(Lv, Dv, 3, "fp64").cpu().numpy()
    h.sync_status()
    sizes = np.array([f.n for f in fs])
    rng = np.random.default_rng(7)
    picks = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), *rng.choice(256, 2, replace=False).tolist()})
    for b in picks:
        f = fs[b]
        S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
        G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
        N = oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, 3, S)
        assert normwise(_split(G32, lay, b), G) <= 1e-5, b
        assert normwise(_split(N32, lay, b), N) <= 1e-5, b
        assert sel_rel_err(_split(G64, lay, b), G, *S) <= TOL64, b
        assert sel_rel_err(_split(N64, lay, b), N, *S) <= TOL64, b


@pytest.mark.parametrize("prec", ["fp64", "fp32x2"])
def test_batch_run_per_matrix_buffers_and_graph(batch, prec):
    """sinv_batch_run: each matrix in its own buffers (inputs and outputs), SelInv
    and NInv (m = 3) for all of them in one call, against the oracle matrix by
    matrix; then the same call captured in a CUDA graph with new input values
    written into the same buffers, replayed, and checked again."""
    fs, h, refs, _, _ = batch
    Ls = [_dev(f.L_val) for f in fs]
    Ds = [_dev(f.D_packed) for f in fs]
    Gs = [torch.full((len(r[0][1]),), float("nan"), dtype=torch.float64, device="cuda") for r in refs]
    Ns = [torch.full((len(r[0][1]),), float("nan"), dtype=torch.float64, device="cuda") for r in refs]
    h.batch_run(Ls, Ds, prec, Gs, 3, Ns)
    h.sync_status()
    for b, (S, G, N) in enumerate(refs):
        assert sel_rel_err(Gs[b].cpu().numpy(), G, *S) <= TOL64, b
        assert sel_rel_err(Ns[b].cpu().numpy(), N, *S) <= TOL64, b
    # graph: capture once, then change the inputs in place (scaled D: G and N scale by 1/2)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        h.batch_run(Ls, Ds, prec, Gs, 3, Ns, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        h.batch_run(Ls, Ds, prec, Gs, 3, Ns, stream=torch.cuda.current_stream())
    for D in Ds:
        D.mul_(2.0)
    for x in Gs + Ns:
        x.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    h.sync_status()
    for b, (S, G, N) in enumerate(refs):
        assert sel_rel_err(Gs[b].cpu().numpy(), 0.5 * G, *S) <= TOL64, b
        assert sel_rel_err(Ns[b].cpu().numpy(), 0.5 * N, *S) <= TOL64, b


def test_batch_run_rejects_a_single_matrix_handle():
    from paper_2609_11363_b300 import Handle, SinvError
    f = _members()[0]
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    with pytest.raises(SinvError) as ei:
        h.batch_run([_dev(f.L_val)], [_dev(f.D_packed)], "fp64", [torch.empty(h.nnz_S, dtype=torch.float64,
                                                                              device="cuda")])
    assert ei.value.name == "SINV_ERR_INVALID_ARG"
