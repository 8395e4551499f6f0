"""Autotuner for the schedule of the persistent SelInv kernel.

The kernel's "tile" is the work unit a CTA takes: one supernode for the whole
CTA, or a group of small supernodes one per warp.  Two symbolic options decide
the shape: the supernode width cap (columns merged into one dense step) and the
pair count above which a supernode gets a whole CTA.  This module times the
real numeric call for each candidate on the caller's matrix (or batch) with
CUDA events and returns the fastest setting; the handle it returns was built
with that setting.
"""
from __future__ import annotations

import itertools
import time

import numpy as np
import torch

from .binding import Handle

DEFAULT_CAPS = (1, 4, 16)
DEFAULT_BIG = (512, 2048, 8192)


def _time_selinv(h, Lv, Dv, prec, reps):
    out = torch.empty(h.nnz_S, dtype=torch.float64, device=Lv.device)
    h.selinv(Lv, Dv, prec, out=out)  # warm-up
    h.sync_status()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        h.selinv(Lv, Dv, prec, out=out)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    h.sync_status()
    return float(np.median(ts))


def tune_selinv(factors, L_val, D_val, prec="fp64", caps=DEFAULT_CAPS, bigs=DEFAULT_BIG, reps=3, device=0):
    """Return (best_handle, best_params, table).

    ``factors``: one object with n, L_rowptr, L_col, pivot_start, or a list of
    them (batched handle).  ``L_val`` / ``D_val``: the matching device tensors.
    ``table`` lists (cap, big_pairs, median ms, symbolic s) for every candidate.
    """
    batch = isinstance(factors, (list, tuple))
    table = []
    best = None
    for cap, big in itertools.product(caps, bigs):
        t0 = time.time()
        if batch:
            h = Handle.batch(factors, supernode_cap=cap, big_pairs=big, device=device)
        else:
            f = factors
            h = Handle(f.n, f.L_rowptr, f.L_col, f.pivot_start, supernode_cap=cap, big_pairs=big, device=device)
        t_sym = time.time() - t0
        ms = _time_selinv(h, L_val, D_val, prec, reps)
        table.append((cap, big, ms, t_sym))
        if best is None or ms < best[0]:
            if best is not None:
                best[2].close()
            best = (ms, {"supernode_cap": cap, "big_pairs": big}, h)
        else:
            h.close()
    return best[2], best[1], table
