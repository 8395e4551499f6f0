"""Critical path of one SelInv call from its per-supernode timeline.

SelInv (Section 2.1) processes supernode J once the supernodes owning its rows
C_J have published.  ``Handle.timeline()`` makes the kernels stamp, per
supernode, when its first work item started, when its dependencies had
published (as seen by the kernel), when its contraction was done and when it
published.  ``critical_path`` walks back from the last publication through the
dependency that published last, and splits the chain into

* hand-off: from the dependency's publication to the moment the waiting work
  item saw it (the cost of the flag protocol and of the item's position in the
  schedule);
* contraction: from then to the end of the contraction (the gathers of G~_CC
  and the products);
* finish: from there to the publication (X and G_JJ written, parts combined).

Usage (one GPU)::

    python -m paper_2609_11363_b300.timeline --workload diff3d --size 64 --prec fp64
    python -m paper_2609_11363_b300.timeline --workload band --n 12288 --b 1024 --tau 0 --prec tf32 --cap 16
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np


def dependencies(n, L_rowptr, L_col, sn_start):
    """For every supernode, the distinct supernodes owning the rows of its C."""
    sn_start = np.asarray(sn_start, dtype=np.int64)
    ns = len(sn_start) - 1
    owner = np.repeat(np.arange(ns), np.diff(sn_start))
    rows = np.repeat(np.arange(n), np.diff(np.asarray(L_rowptr)))
    cols = np.asarray(L_col, dtype=np.int64)
    js = owner[cols]
    below = rows >= sn_start[js + 1]
    # distinct (J, K) pairs, sorted by J then K, as one int64 key per pair
    key = np.unique(js[below].astype(np.int64) * ns + owner[rows[below]].astype(np.int64))
    J, K = key // ns, key % ns
    cuts = np.searchsorted(J, np.arange(1, ns))
    return [a.tolist() for a in np.split(K, cuts)]


def critical_path(stamps, deps, levels=None):
    """Walk back from the last publication.  stamps: [ns, 4] (start, ready, done,
    published) in ns.  Returns a summary dict (totals in microseconds and the
    per-step medians)."""
    st = np.asarray(stamps, dtype=np.float64)
    pub = st[:, 3]
    valid = pub > 0
    t0 = float(np.min(np.where(st[:, 0] < 1.8e19, st[:, 0], np.inf)))
    J = int(np.argmax(np.where(valid, pub, -1)))
    path = []
    while True:
        d = [k for k in deps[J] if valid[k]]
        K = max(d, key=lambda k: pub[k]) if d else None
        ready, done, p = st[J, 1], st[J, 2], st[J, 3]
        hand = ready - (pub[K] if K is not None else st[J, 0])
        path.append((J, hand, done - ready, p - done))
        if K is None:
            break
        J = K
    path.reverse()
    arr = np.array([[h, c, f] for _, h, c, f in path]) / 1e3
    total = (float(np.max(pub[valid])) - t0) / 1e3
    out = {
        "supernodes": int(st.shape[0]), "chain_length": len(path), "span_us": total,
        "handoff_us": float(arr[:, 0].sum()), "contraction_us": float(arr[:, 1].sum()),
        "finish_us": float(arr[:, 2].sum()),
        "median_step_us": {"handoff": float(np.median(arr[:, 0])), "contraction": float(np.median(arr[:, 1])),
                           "finish": float(np.median(arr[:, 2]))},
    }
    if levels is not None:
        lv = np.asarray(levels)
        out["levels"] = int(lv.max()) + 1 if len(lv) else 0
    return out


def totals(stamps):
    """Sums over all supernodes (microseconds): waiting for dependencies after the
    first work item started (ready - start), contraction (done - ready) and finish
    (published - done); with the span, what the CTAs spent on each.  For a supernode
    split over several CTAs the stamps cover all its parts."""
    st = np.asarray(stamps, dtype=np.float64)
    ok = (st[:, 3] > 0) & (st[:, 0] < 1.8e19)
    st = st[ok]
    t0, t1 = float(st[:, 0].min()), float(st[:, 3].max())
    return {"supernodes": int(st.shape[0]), "span_us": (t1 - t0) / 1e3,
            "wait_us": float((st[:, 1] - st[:, 0]).sum()) / 1e3,
            "contraction_us": float((st[:, 2] - st[:, 1]).sum()) / 1e3,
            "finish_us": float((st[:, 3] - st[:, 2]).sum()) / 1e3}


def _workload(args):
    from workloads.configs import band, diff3d, elastic3d, plant_2x2
    if args.workload == "band":
        return band(args.n, args.b, tau=args.tau).factors
    if args.workload == "elastic":
        return elastic3d(args.size, cache_dir=args.factor_cache).factors
    return plant_2x2(diff3d(args.size).factors, 0.02, 2)


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--workload", default="diff3d", choices=["diff3d", "band", "elastic"])
    p.add_argument("--size", type=int, default=64)
    p.add_argument("--n", type=int, default=12288)
    p.add_argument("--b", type=int, default=1024)
    p.add_argument("--tau", type=float, default=1e-6)
    p.add_argument("--cap", type=int, default=0)
    p.add_argument("--prec", default="fp64", choices=["fp64", "fp32", "tf32", "bf16"])
    p.add_argument("--totals-only", action="store_true",
                   help="only the sums over all supernodes (no dependency walk: fast at any size)")
    p.add_argument("--factor-cache", default=None, help="elastic: directory of the on-disk factor cache")
    p.add_argument("--pair-bytes", type=int, default=0,
                   help="memory the SelInv pair lists may take (0: default, < 0: the scan form)")
    args = p.parse_args(argv)
    import torch
    from paper_2609_11363_b300 import Handle
    f = _workload(args)
    h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, supernode_cap=args.cap, selinv_pair_bytes=args.pair_bytes)
    Lv = torch.as_tensor(f.L_val, device="cuda")
    Dv = torch.as_tensor(f.D_packed, device="cuda")
    G = torch.empty(h.nnz_S, dtype=torch.float64, device="cuda")
    for _ in range(3):
        h.selinv(Lv, Dv, args.prec, out=G)
    h.sync_status()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    h.selinv(Lv, Dv, args.prec, out=G)
    e1.record()
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    h.timeline(True)
    h.selinv(Lv, Dv, args.prec, out=G)
    h.sync_status()
    stamps = h.timeline_read()
    h.timeline(False)
    if args.totals_only:
        out = {"totals": totals(stamps)}
    else:
        sn_start, sn_level = h.supernodes()
        deps = dependencies(f.n, f.L_rowptr, f.L_col, sn_start)
        out = critical_path(stamps, deps, sn_level)
        out["totals"] = totals(stamps)
    out.update(workload=args.workload, prec=args.prec, n=f.n, cap=args.cap, ms_without_timeline=ms_plain,
               stats={k: v for k, v in h.stats().items()
                      if k in ("n_supernodes", "n_levels", "tc_levels", "selinv_scan", "max_c")})
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
