"""The allocation-free FP32 low-rank correction (sinv_lowrank_correct_noalloc).

Callers that cannot allocate device memory use this entry point: it takes the
pattern and the vectors as device pointers, needs no handle, and keeps its FP32
working copy in an array built into the library.  Its result must match the
handle-based FP32 form (sinv_lowrank_correct with SINV_FP32) within the FP32
tolerance of the other tests, on two calls in a row (the second call reuses the
array the first one wrote).  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from tests.helpers import normwise
from workloads.configs import diff3d, lap2d_32, plant_2x2, random_lowrank


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.gpu
def test_noalloc_matches_handle_fp32_on_two_calls():
    from paper_2609_11363_b300 import Handle, lowrank_correct_noalloc

    f = plant_2x2(diff3d(12, m=3).factors, 0.05, 13)
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    rp, col = h.pattern_host()
    S_rp, S_col = _dev(rp), _dev(col)
    rng = np.random.default_rng(5)
    X0 = rng.standard_normal(h.nnz_S)
    for call, k in enumerate((16, 7)):
        V, lam = random_lowrank(f.n, k, seed=40 + call)
        want = _dev(X0.copy())
        h.lowrank_correct(_dev(V), _dev(lam), want, "fp32")
        got = _dev(X0.copy())
        lowrank_correct_noalloc(S_rp, S_col, _dev(V), _dev(lam), got)
        torch.cuda.synchronize()
        h.sync_status()
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert normwise(g - X0, w - X0) <= 1e-5, call
        assert np.allclose(g, w, rtol=1e-6, atol=1e-9), call


@pytest.mark.gpu
def test_noalloc_rejects_oversized_request():
    from paper_2609_11363_b300 import LOWRANK_NOALLOC_MAX, SinvError, lowrank_correct_noalloc

    f = lap2d_32().factors
    from paper_2609_11363_b300 import Handle
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    rp, col = h.pattern_host()
    k = LOWRANK_NOALLOC_MAX // f.n + 1
    V = torch.zeros(f.n * k, dtype=torch.float64, device="cuda")
    lam = torch.zeros(k, dtype=torch.float64, device="cuda")
    X = torch.zeros(h.nnz_S, dtype=torch.float64, device="cuda")
    with pytest.raises(SinvError) as ei:
        lowrank_correct_noalloc(_dev(rp), _dev(col), V, lam, X)
    assert ei.value.name == "SINV_ERR_UNSUPPORTED"
    assert torch.count_nonzero(X).item() == 0
