"""The bounds-checked build (libsinv_checked.so, compiled with -DSINV_CHECKED).

In a fresh process that loads the checked library: the path gives the oracle's
results with no index out of range (SelInv with pair lists and in the scan form,
NInv in map and hash form, NInv and Mix on NInv's own pattern, the rank-k
correction); a pair position planted past the end of S_lo is reported by
sinv_sync_status as an out-of-range index, the access skipped (nothing faults),
and a new handle works again.  The regular build refuses to plant it."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, ROOT)
import numpy as np, torch
import oracle
from paper_2609_11363_b300 import binding
binding.use_checked_library()
from paper_2609_11363_b300 import Handle, SinvError
from tests.helpers import sel_rel_err
from workloads.configs import diff3d, lap2d_32, plant_2x2, random_lowrank
assert binding.load_library()._name.endswith("libsinv_checked.so")
dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
for f in (plant_2x2(lap2d_32().factors, 0.3, 11), plant_2x2(diff3d(10, m=3).factors, 0.05, 13)):
    S = oracle.symbolic_S(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    G = oracle.selinv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, S)
    N = oracle.ninv(f.n, f.L_rowptr, f.L_col, f.L_val, f.pivot_start, f.d_diag, f.d_off, 3, S)
    Lv, Dv = dev(f.L_val), dev(f.D_packed)
    for pb in (0, -1):
        h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, selinv_pair_bytes=pb)
        g = h.selinv(Lv, Dv, "fp64").cpu().numpy()
        h.sync_status()
        assert sel_rel_err(g, G, *S) <= 1e-10
    for budget in (0, -1):
        h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, ninv_index_bytes=budget)
        nn = h.ninv(Lv, Dv, 3, "fp64").cpu().numpy()
        h.sync_status()
        assert sel_rel_err(nn, N, *S) <= 1e-10
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    Gd = h.selinv(Lv, Dv, "fp64")
    h.ninv_own(Lv, Dv, 3, 0.1)
    h.mix_own(Gd, 1e-3 * float(Gd.abs().max()))
    V, lam = random_lowrank(f.n, 8, seed=3)
    h.lowrank_correct_mix_own(dev(V), dev(lam), "fp64")
    h.sync_status()
# a planted out-of-range pair position: reported, not used
f = plant_2x2(lap2d_32().factors, 0.3, 11)
h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
assert h.debug_corrupt_plan() == 0
h.selinv(dev(f.L_val), dev(f.D_packed), "fp64")
try:
    h.sync_status()
    raise AssertionError("the out-of-range index was not reported")
except SinvError as e:
    assert "out of range" in str(e), str(e)
h2 = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
h2.selinv(dev(f.L_val), dev(f.D_packed), "fp64")
h2.sync_status()
print("checked build ok")
"""


def test_checked_build_parity_and_out_of_range_report():
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], capture_output=True, text=True,
                       cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked build ok" in r.stdout


def test_regular_build_refuses_to_plant_a_bad_index():
    from paper_2609_11363_b300 import Handle
    from workloads.configs import lap2d_32
    f = lap2d_32().factors
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start)
    assert h.debug_corrupt_plan() == 7   # SINV_ERR_UNSUPPORTED: nothing changed
