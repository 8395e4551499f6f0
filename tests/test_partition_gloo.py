"""One matrix's SelInv and NInv split over two ranks (the partition and exchange
logic of paper_2609_11363_b300.partition), run as two gloo ranks on the CPU with
the FP64 oracle as each rank's engine.

Rank 0 computes the trunk (the top of the elimination DAG) and broadcasts its
G entries and its W columns; every rank then computes its own bin.  Each rank's
part must equal the single-process oracle's entries for that part: SelInv bit
for bit (every pivot block does the same arithmetic on the same inputs), NInv
within rounding (the per-column Horner sums run in another order than the
oracle's sparse products)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    from workloads.configs import diff3d, plant_2x2
    return plant_2x2(diff3d(8, m=2).factors, 0.05, 13)


def _plan(f, world):
    import oracle
    from paper_2609_11363_b300 import Handle
    from paper_2609_11363_b300.partition import Plan
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    sn_start, _ = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, device=-1).supernodes()
    return S, Plan(f.n, f.L_rowptr, f.L_col, f.pivot_start, sn_start, S, world)


def _dinv_rows(f):
    """D^{-1} as {row: {col: value}} (1x1 and 2x2 blocks)."""
    out = {}
    j = 0
    while j < f.n:
        if j + 1 < f.n and not f.pivot_start[j + 1]:
            inv = np.linalg.inv(np.array([[f.d_diag[j], f.d_off[j]], [f.d_off[j], f.d_diag[j + 1]]]))
            out[j] = {j: inv[0, 0], j + 1: inv[0, 1]}
            out[j + 1] = {j: inv[1, 0], j + 1: inv[1, 1]}
            j += 2
        else:
            out[j] = {j: 1.0 / f.d_diag[j]}
            j += 1
    return out


def _rank_main(rank, world, port, m, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        f = _workload()
        S, P = _plan(f, world)
        P.validate()
        trunk, mine = P.parts[0], P.parts[1 + rank]
        # ---- SelInv: the trunk on rank 0, one broadcast of its entries, then each bin
        G = np.zeros(len(S[1]))
        if rank == 0:
            oracle.selinv_blocks(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S, G,
                                 trunk.blocks)
        payload = torch.as_tensor(G[trunk.s_positions].copy())
        dist.broadcast(payload, src=0)
        G[trunk.s_positions] = payload.numpy()
        oracle.selinv_blocks(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S, G, mine.blocks)
        # ---- NInv: the trunk's W columns (every step) from rank 0, then this bin's columns
        halo = [None]
        if rank == 0:
            W = oracle.ninv_W_columns(f.n, f.L_rowptr, f.L_col, f.L_val, m, trunk.columns)
            halo = [{int(j): {t: W[t][int(j)] for t in range(m + 1)} for j in trunk.columns}]
        dist.broadcast_object_list(halo, src=0)
        W = oracle.ninv_W_columns(f.n, f.L_rowptr, f.L_col, f.L_val, m, mine.columns, W_known=halo[0])[m]
        dinv = _dinv_rows(f)
        rows = np.repeat(np.arange(f.n), np.diff(S[0]))
        N = {}
        todo = list(mine.s_positions) + (list(P.parts[0].s_positions) if rank == 0 else [])
        for p in todo:                   # N_ij = W[:, i] . (D^{-1} W[:, j]); rank 0 also does the trunk
            i, j = int(rows[p]), int(S[1][p])
            y = {}
            for r, w in W[j].items():
                for c, d in dinv[r].items():
                    y[c] = y.get(c, 0.0) + d * w
            N[int(p)] = sum(w * y.get(r, 0.0) for r, w in W[i].items())
        out[rank] = (G[mine.s_positions].copy(), G[trunk.s_positions].copy(), N)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(600)
def test_selinv_and_ninv_split_over_two_ranks_match_the_oracle():
    import oracle
    world, m = 2, 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), m, out), nprocs=world, join=True)
    f = _workload()
    S, P = _plan(f, world)
    G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    Nref = oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, m, S)
    covered = np.zeros(len(S[1]), dtype=int)
    covered[P.parts[0].s_positions] += 1
    ncov = np.zeros(len(S[1]), dtype=int)
    for r in range(world):
        Gmine, Gtrunk, N = out[r]
        part = P.parts[1 + r]
        assert len(part.supernodes) > 0
        assert np.array_equal(Gmine, G[part.s_positions]), r
        assert np.array_equal(Gtrunk, G[P.parts[0].s_positions]), r
        pos = np.array(sorted(N))
        got = np.array([N[int(p)] for p in pos])
        scale = np.abs(Nref).max()
        assert np.max(np.abs(got - Nref[pos])) <= 1e-12 * scale, r
        ncov[pos] += 1
        covered[part.s_positions] += 1
    # the trunk and the bins cover every entry of S exactly once, for G and for N
    assert np.all(covered == 1) and np.all(ncov == 1)
    # the trunk is a small top part
    assert 0 < len(P.parts[0].columns) < f.n // 2


@pytest.mark.parametrize("case", ["diff3d", "lap2d", "random", "band"])
@pytest.mark.parametrize("nranks", [2, 4])
def test_partition_closure(case, nranks):
    """Every supernode depends only on the trunk or its own bin, the trunk only on
    itself, and the parts cover each supernode, column and S entry once -- on a 3D
    and a 2D nested-dissection factor, a random non-closed pattern and a band (a
    chain: no independent subtrees, so everything stays in the trunk)."""
    from workloads.configs import band, diff3d, lap2d_32, random_factors
    f = {"diff3d": lambda: diff3d(8, m=2).factors, "lap2d": lambda: lap2d_32().factors,
         "random": lambda: random_factors(300, 0.02, 0.1, 3), "band": lambda: band(400, 20).factors}[case]()
    S, P = _plan(f, nranks)
    assert P.validate()
    cols = np.concatenate([p.columns for p in P.parts])
    assert np.array_equal(np.sort(cols), np.arange(f.n))
    pos = np.concatenate([p.s_positions for p in P.parts])
    assert np.array_equal(np.sort(pos), np.arange(len(S[1])))
    if case in ("diff3d", "lap2d"):
        assert sum(len(p.supernodes) > 0 for p in P.parts[1:]) == nranks


@pytest.mark.parametrize("nranks", [1, 3, 8, 64])
def test_partition_any_rank_count(nranks):
    """One rank (everything in its bin), an odd count, and more ranks than there are
    independent subtrees (some bins stay empty): the parts still cover every column
    and S entry once and pass the closure check."""
    from workloads.configs import lap2d_32, random_factors
    for f in (lap2d_32().factors, random_factors(5, 0.3, 0.0, 1)):
        S, P = _plan(f, nranks)
        assert P.validate() and len(P.parts) == nranks + 1
        assert np.array_equal(np.sort(np.concatenate([p.columns for p in P.parts])), np.arange(f.n))
        assert np.array_equal(np.sort(np.concatenate([p.s_positions for p in P.parts])), np.arange(len(S[1])))
