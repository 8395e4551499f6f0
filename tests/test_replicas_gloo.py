"""The multi-GPU path of the benchmark is replicas only: every rank runs its own
matrix and the ranks meet once, to take the slowest rank's time.  These tests run
that host logic as two gloo ranks on the CPU."""
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2609_11363_b300 import Handle
        from workloads.configs import batch9pt_member
        # replica work: the symbolic analysis of this rank's own matrix (host only)
        f = batch9pt_member(3000 + rank, n_range=(2048, 4096)).factors
        h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, device=-1)
        st = h.stats()
        stats = torch.tensor([st["n"], st["nnz_S_lo"], st["n_levels"]], dtype=torch.int64)
        gathered = [torch.zeros_like(stats) for _ in range(world)]
        dist.all_gather(gathered, stats)
        # timing aggregation: rank r took 100 + 50 r ms for 4 steps of 10 units each
        ms, value = bench.aggregate_ranks(100.0 + 50.0 * rank, 10, 4, world, "cpu")
        out[rank] = [ms, value] + [int(v) for g in gathered for v in g]
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_replicas_aggregate_and_stay_independent():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    slowest = 100.0 + 50.0 * (world - 1)
    for r in range(world):
        ms, value = out[r][:2]
        assert ms == pytest.approx(slowest / 4)
        assert value == pytest.approx(world * 10 * 4 / (slowest / 1e3))
    # every rank sees the same per-replica statistics, each from its own matrix, equal to
    # the single-process analysis of that matrix
    from paper_2609_11363_b300 import Handle
    from workloads.configs import batch9pt_member
    for r in range(world):
        f = batch9pt_member(3000 + r, n_range=(2048, 4096)).factors
        st = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, device=-1).stats()
        want = [st["n"], st["nnz_S_lo"], st["n_levels"]]
        for rank in range(world):
            assert out[rank][2 + 3 * r: 5 + 3 * r] == want
    assert out[0][2:5] != out[0][5:8]
