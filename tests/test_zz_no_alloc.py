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


def test_noalloc_rejects_rank_above_256_before_reading_pointers():
    """k > 256 does not fit the kernel's shared row of lambda .* V_i: the entry
    point must refuse it before it looks at any pointer, so NULL pointers give
    SINV_ERR_UNSUPPORTED (a regression would give SINV_ERR_INVALID_ARG) and
    nothing reaches a GPU.  Runs without a GPU."""
    from paper_2609_11363_b300.binding import LOWRANK_NOALLOC_KMAX, load_library

    lib = load_library()
    for n, k in ((100, 257), (1024, 300), (100, 1000), (0, 257)):
        assert lib.sinv_lowrank_correct_noalloc(n, None, None, k, None, None, None, None) == 7, (n, k)
    assert LOWRANK_NOALLOC_KMAX == 256
    # within both limits, NULL pointers are an invalid argument, not a launch
    assert lib.sinv_lowrank_correct_noalloc(100, None, None, 256, None, None, None, None) == 1
    assert lib.sinv_lowrank_correct_noalloc(-1, None, None, 4, None, None, None, None) == 1


@pytest.mark.gpu
def test_noalloc_rank_257_leaves_X_unchanged():
    from paper_2609_11363_b300 import Handle, SinvError, lowrank_correct_noalloc
    from paper_2609_11363_b300.binding import load_library

    # the same request with NULL pointers first: if the rank check ever went
    # missing this returns SINV_ERR_INVALID_ARG and the test stops here, before
    # a kernel could be launched with a rank its shared row cannot hold
    assert load_library().sinv_lowrank_correct_noalloc(1024, None, None, 257, None, None, None, None) == 7
    f = lap2d_32().factors
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    rp, col = h.pattern_host()
    k = 257
    assert f.n * k + k <= 1 << 22   # inside the array: only the rank limit applies
    V, lam = random_lowrank(f.n, k, seed=9)
    X0 = np.random.default_rng(3).standard_normal(h.nnz_S)
    X = _dev(X0)
    with pytest.raises(SinvError) as ei:
        lowrank_correct_noalloc(_dev(rp), _dev(col), _dev(V), _dev(lam), X)
    assert ei.value.name == "SINV_ERR_UNSUPPORTED"
    torch.cuda.synchronize()
    assert np.array_equal(X.cpu().numpy(), X0)
