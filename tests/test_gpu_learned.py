"""Learned correction: NInv truncation stack, BF16 MLP gradients against the FP64
oracle, one Adam step, and the gain of a trained network over plain NInv on a
held-out matrix (SelInv as the reference)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp as omlp
from tests.helpers import sel_rel_err
from workloads.configs import diff3d, plant_2x2

pytestmark = pytest.mark.gpu

F, H = 16, 64


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _bf16_round(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("index_bytes,prec", [(0, "fp64"), (-1, "fp64"), (0, "fp32x2")])
def test_ninv_stack_matches_each_truncation(index_bytes, prec):
    """Map form (0), hash form (-1) and the map form in pairs of floats."""
    from paper_2609_11363_b300 import Handle
    f = plant_2x2(diff3d(10, shifted=False, m=3).factors, 0.05, 3)
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, ninv_index_bytes=index_bytes)
    st = h.ninv_stack(_dev(f.L_val), _dev(f.D_packed), 3, prec).cpu().numpy()
    h.sync_status()
    for t in range(4):
        ref = oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, t, S)
        assert sel_rel_err(st[t], ref, *S) <= 1e-10, t


def test_mlp_checkpoint_resumes_training_bit_for_bit(tmp_path):
    """A checkpoint holds the whole training state: a network restored from it (built
    with other initial weights) and the original, trained on with the same
    mini-batches, end with the same weights bit for bit (the gradient sums run in a
    fixed order); a restart from the weights alone, with Adam's moments reset, does
    not."""
    from paper_2609_11363_b300 import Mlp
    rng = np.random.default_rng(11)
    B = 2048
    X = torch.as_tensor(rng.standard_normal((B, F)).astype(np.float32)).to(torch.bfloat16).cuda()
    y = _dev(rng.standard_normal(B).astype(np.float32))
    idx = torch.arange(B, dtype=torch.int64, device="cuda")
    a = Mlp(seed=3, max_batch=B)
    for _ in range(3):
        a.train_step(X, y, idx, 1e-3)
    path = str(tmp_path / "mlp_state.npz")
    a.save(path)
    b = Mlp(seed=99, max_batch=B)
    b.load(path)
    c = Mlp(seed=99, max_batch=B)
    c.set_params(a.get_params())
    for _ in range(2):
        for net in (a, b, c):
            net.train_step(X, y, idx, 1e-3)
    torch.cuda.synchronize()
    assert np.array_equal(a.get_params(), b.get_params())
    assert not np.array_equal(a.get_params(), c.get_params())
    assert a.get_state()["step"] == b.get_state()["step"] == 5 and c.get_state()["step"] == 2


def test_mlp_gradient_matches_oracle_and_adam_step():
    from paper_2609_11363_b300 import Mlp
    rng = np.random.default_rng(0)
    B = 1000
    Xf = rng.standard_normal((B, F)).astype(np.float32)
    y = rng.standard_normal(B).astype(np.float32)
    net = Mlp(seed=7, max_batch=4096)
    th = net.get_params().astype(np.float64)
    Xb = torch.as_tensor(Xf).to(torch.bfloat16).cuda()
    g, loss = net.grad(Xb, _dev(y))
    torch.cuda.synchronize()
    # the oracle sees the same BF16-rounded weights and features
    Xr = Xb.float().cpu().numpy().astype(np.float64)
    thr = _bf16_round(th)
    g_ref = omlp.grad(thr, Xr, y.astype(np.float64), F, H)
    l_ref = omlp.loss(thr, Xr, y.astype(np.float64), F, H)
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - l_ref) <= 1e-4 * max(1.0, abs(l_ref))
    assert np.linalg.norm(gg - g_ref) <= 1e-3 * np.linalg.norm(g_ref)
    # one Adam step on the FP32 master weights
    idx = torch.arange(B, dtype=torch.int64, device="cuda")
    net.train_step(Xb, _dev(y), idx, 1e-3)
    th1 = net.get_params().astype(np.float64)
    want, _, _ = omlp.adam(th, gg, np.zeros_like(th), np.zeros_like(th), 1, 1e-3)
    assert np.max(np.abs(th1 - want)) <= 1e-6


def _assert_predict_close(got, N, sc, theta_bf16, Xr):
    """Entry by entry against N + s * oracle.mlp.forward(theta, X, act_bf16=True):
    BF16 weights and features, the first hidden layer rounded to BF16 (the
    operand of the tensor-core layer).  The sums are FP32 (tensor-core
    accumulators and the output dot product): three layers of at most 65 terms,
    so f is off by at most a few units of 2^-24 times the sum of the magnitudes
    of the terms (|h|.|W|, from the oracle in FP64) -- the tight bound.  Where the
    device's FP32 sum and the exact one straddle a BF16 rounding boundary, the two
    sides round that hidden unit one BF16 unit (2^-8 relative) apart: the loose
    bound allows that for every unit; at most 2 % of the entries may need it."""
    W1, b1, W2, b2, W3, b3 = omlp.split(theta_bf16, F, H)
    h1 = omlp.bf16_round(np.maximum(Xr @ W1 + b1, 0.0))
    h2 = np.maximum(h1 @ W2 + b2, 0.0)
    f_ref = h2 @ W3 + b3[0]
    assert np.array_equal(f_ref, omlp.forward(theta_bf16, Xr, F, H, act_bf16=True))
    aW2, aW3 = np.abs(W2), np.abs(W3)
    mag = ((np.abs(Xr) @ np.abs(W1) + np.abs(b1)) @ aW2) @ aW3      # layer-1 sums carried through
    mag += (np.abs(h1) @ aW2 + np.abs(b2)) @ aW3                      # layer-2 sums
    mag += np.abs(h2) @ aW3 + abs(b3[0])                              # output sum
    tight = 2 * (H + 1) * 2.0 ** -24 * mag + 1e-30
    loose = tight + 2.0 ** -8 * (np.abs(h1) @ aW2) @ aW3
    f_got = (got - N) / sc.astype(np.float64)
    err = np.abs(f_got - f_ref)
    assert np.all(err <= loose), float(np.max(err / loose))
    assert np.mean(err <= tight) >= 0.98, float(np.mean(err <= tight))


@pytest.mark.parametrize("count", [1, 127, 128, 1000, 4099, 300001])
def test_mlp_predict_matches_oracle_entry_by_entry(count):
    """sinv_mlp_predict against N + s * oracle.mlp.forward(bf16(theta), bf16(X)) on
    random features and weights: every entry, full tiles and a ragged tail."""
    from paper_2609_11363_b300 import Mlp
    rng = np.random.default_rng(11 + count)
    net = Mlp(seed=3, max_batch=4096)
    th = rng.standard_normal(net.n_params).astype(np.float32) * 0.3
    net.set_params(th)
    Xb = torch.as_tensor(rng.standard_normal((count, F)).astype(np.float32)).to(torch.bfloat16).cuda()
    sc = rng.uniform(0.5, 2.0, count).astype(np.float32)
    N = rng.standard_normal(count)
    got = net.predict(Xb, _dev(sc), _dev(N)).cpu().numpy()
    net.sync_status()
    Xr = Xb.float().cpu().numpy().astype(np.float64)
    _assert_predict_close(got, N, sc, _bf16_round(th), Xr)


def test_mlp_predict_on_diffusion_features():
    """The same comparison on the features of a 3D diffusion case (the inputs the
    learned correction sees), after a few training steps so the weights are not
    the initial ones."""
    from paper_2609_11363_b300 import Handle, Mlp
    f = plant_2x2(diff3d(9, shifted=False, m=3).factors, 0.05, 8)
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    Lv, Dv = _dev(f.L_val), _dev(f.D_packed)
    st = h.ninv_stack(Lv, Dv, 3)
    X, sc = h.mlp_features(st, 3, Lv, Dv)
    G = h.selinv(Lv, Dv)
    net = Mlp(seed=5, max_batch=1 << 15)
    y = net.targets(G, st[3].contiguous(), sc)
    idx = torch.arange(min(X.shape[0], 1 << 15), dtype=torch.int64, device="cuda")
    for _ in range(5):
        net.train_step(X, y, idx, 3e-3)
    N = st[3].contiguous()
    got = net.predict(X, sc, N).cpu().numpy()
    h.sync_status()
    net.sync_status()
    th = _bf16_round(net.get_params())
    Xr = X.float().cpu().numpy().astype(np.float64)
    _assert_predict_close(got, N.cpu().numpy(), sc.cpu().numpy(), th, Xr)


def test_features_match_their_definition():
    from paper_2609_11363_b300 import Handle
    f = plant_2x2(diff3d(8, shifted=False, m=3).factors, 0.1, 5)
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    Lv, Dv = _dev(f.L_val), _dev(f.D_packed)
    st = h.ninv_stack(Lv, Dv, 3)
    X, sc = h.mlp_features(st, 3, Lv, Dv)
    h.sync_status()
    X = X.float().cpu().numpy()
    sc = sc.cpu().numpy()
    Nst = st.cpu().numpy()
    rows = np.repeat(np.arange(f.n), np.diff(S[0]))
    cols = S[1].astype(np.int64)
    N = Nst[3]
    diag = N[S[0][1:] - 1]
    s = np.sqrt(np.abs(diag[rows] * diag[cols]))
    assert np.allclose(sc, s, rtol=1e-6)
    assert np.allclose(X[:, 0], _bf16_round(N / s), rtol=1e-2, atol=1e-3)
    for t in range(1, 4):
        assert np.allclose(X[:, t], _bf16_round((Nst[t] - Nst[t - 1]) / s), rtol=1e-2, atol=1e-3)
    assert np.array_equal(X[:, 5], (rows == cols).astype(np.float32))


def test_trained_network_beats_plain_ninv_on_held_out_matrix():
    """Train on three 3D diffusion matrices, judge on a fourth: the corrected NInv is
    closer to SelInv than NInv itself."""
    from paper_2609_11363_b300 import Handle
    from paper_2609_11363_b300.learned import LearnedCorrection
    lc = LearnedCorrection(m=3, seed=1, batch=4096)
    sets = []
    for seed in (4000, 4001, 4002, 4003):
        f = diff3d(14, shifted=False, m=3, seed=seed).factors
        h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
        sets.append(lc.prepare(h, _dev(f.L_val), _dev(f.D_packed)))
    lc.fit(sets[:3], epochs=12, lr=3e-3)
    ev = lc.evaluate(sets[3])
    assert ev["err_learned"] < 0.8 * ev["err_ninv"], ev


@pytest.mark.slow
def test_full_size_128_ninv_stack_sampled():
    """The learned correction's inference matrix at full size (3D diffusion 128^3,
    n = 2,097,152, m = 3): the NInv truncation stack on sampled entries against the
    oracle, entry by entry, in the form the benchmark runs."""
    from paper_2609_11363_b300 import Handle
    f = diff3d(128, shifted=False, m=3, seed=4999).factors
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    Lv, Dv = _dev(f.L_val), _dev(f.D_packed)
    st = h.ninv_stack(Lv, Dv, 3).cpu().numpy()
    h.sync_status()
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    rp_h, col_h = h.pattern_host()
    assert np.array_equal(rp_h, S[0]) and np.array_equal(col_h, S[1])
    rng = np.random.default_rng(3)
    idx = rng.choice(len(S[1]), 24, replace=False)
    rows = np.repeat(np.arange(f.n), np.diff(S[0]))
    pairs = list(zip(rows[idx], S[1][idx]))
    for t in (1, 3):
        ref = oracle.ninv_entries_sampled(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, t,
                                          pairs)
        diag = st[t][S[0][1:] - 1]
        scale = np.abs(ref) + np.sqrt(np.abs(diag[rows[idx]] * diag[S[1][idx]]))
        assert np.max(np.abs(st[t][idx] - ref) / scale) <= 1e-10, t
