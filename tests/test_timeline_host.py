"""Host side of the SelInv timeline: the dependency lists against a brute-force
recomputation of C_J, and the critical-path walk on a hand-made timeline."""
import numpy as np

from paper_2609_11363_b300.timeline import critical_path, dependencies
from workloads.configs import diff3d, plant_2x2


def test_dependencies_match_brute_force():
    from paper_2609_11363_b300 import Handle
    f = plant_2x2(diff3d(8, m=3).factors, 0.05, 3)
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, device=-1)
    sn_start, _ = h.supernodes()
    deps = dependencies(f.n, f.L_rowptr, f.L_col, sn_start)
    owner = np.repeat(np.arange(len(sn_start) - 1), np.diff(sn_start))
    cols = [[] for _ in range(f.n)]
    for i in range(f.n):
        for q in range(f.L_rowptr[i], f.L_rowptr[i + 1]):
            cols[f.L_col[q]].append(i)
    for J in range(len(sn_start) - 1):
        C = {r for c in range(sn_start[J], sn_start[J + 1]) for r in cols[c] if r >= sn_start[J + 1]}
        assert sorted(deps[J]) == sorted({int(owner[r]) for r in C}), J


def test_critical_path_on_a_hand_timeline():
    # chain 2 -> 1 -> 0 (0 depends on 1, 1 on 2); 3 is independent and early
    deps = [[1], [2], [], []]
    st = np.array([[5000, 9000, 12000, 13000],     # hand-off 9000-8000, contraction 3000, finish 1000
                   [3000, 5500, 7000, 8000],       # hand-off 5500-5000
                   [1000, 1000, 4000, 5000],       # no dependency: from its own start
                   [1000, 1000, 2000, 2500]], dtype=np.uint64)
    out = critical_path(st, deps)
    assert out["chain_length"] == 3
    assert out["span_us"] == 12.0
    assert np.isclose(out["handoff_us"], (0 + 500 + 1000) / 1e3)
    assert np.isclose(out["contraction_us"], (3000 + 1500 + 3000) / 1e3)
    assert np.isclose(out["finish_us"], (1000 + 1000 + 1000) / 1e3)


def test_totals_sum_the_phases_of_every_supernode():
    import numpy as np
    from paper_2609_11363_b300.timeline import totals
    st = np.array([[0, 10, 30, 35], [5, 40, 50, 60], [2**64 - 1, 0, 0, 0]], dtype=np.uint64)  # the last never ran
    t = totals(st)
    assert t["supernodes"] == 2
    assert abs(t["span_us"] - 0.060) < 1e-12
    assert abs(t["wait_us"] - 0.045) < 1e-12 and abs(t["contraction_us"] - 0.030) < 1e-12
    assert abs(t["finish_us"] - 0.015) < 1e-12
