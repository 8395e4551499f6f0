"""Shared test helpers: tolerance checks on S and small input builders."""
from __future__ import annotations

import numpy as np


def s_rows(Srp):
    return np.repeat(np.arange(len(Srp) - 1), np.diff(Srp))


def sel_rel_err(x, r, Srp, Sc):
    """Entrywise error scaled as in the tolerance rule of the selected inverse:
    |x_ij - r_ij| / (|r_ij| + sqrt(|r_ii r_jj|)), max over S_lo."""
    x = np.asarray(x); r = np.asarray(r)
    rows = s_rows(Srp)
    diag = r[np.asarray(Srp[1:]) - 1]  # the diagonal is the last entry of each S_lo row
    scale = np.abs(r) + np.sqrt(np.abs(diag[rows] * diag[Sc]))
    scale = np.where(scale == 0, 1.0, scale)
    return float(np.max(np.abs(x - r) / scale)) if len(x) else 0.0


def normwise(x, r):
    r = np.asarray(r); x = np.asarray(x)
    d = np.linalg.norm(r)
    return float(np.linalg.norm(x - r) / (d if d > 0 else 1.0))
