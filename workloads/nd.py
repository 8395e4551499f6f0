"""Geometric nested-dissection ordering on a box of grid nodes.

The paper factors in a fill-reducing order (the block elimination tree of its
Fig. 2 comes from it) but does not say which; this module fixes one:
recursive bisection of the box, splitting the longest axis (ties broken
x, then y, then z) at ``mid = lo + (hi - lo) // 2``.  The separator plane at
``mid`` is numbered after both halves; a box with at most 8 nodes is a leaf and
is numbered in ascending natural index.  A node's degrees of freedom stay
consecutive.  A single plane separates 5-, 7-, 9- and 27-point stencils alike.
"""
from __future__ import annotations

import numpy as np


def nd_perm(shape, dof: int = 1, leaf: int = 8) -> np.ndarray:
    """Return ``perm`` with ``perm[new] = old`` (natural index, x fastest).

    ``shape`` is (nx, ny) or (nx, ny, nz).  ``A_nd = A[perm][:, perm]``.
    """
    shape = tuple(int(s) for s in shape)
    dim = len(shape)
    strides = [1]
    for s in shape[:-1]:
        strides.append(strides[-1] * s)
    strides = np.array(strides, dtype=np.int64)

    def box_nodes(lo, hi):
        axes = [np.arange(lo[a], hi[a], dtype=np.int64) * strides[a] for a in range(dim)]
        grid = axes[0]
        for a in range(1, dim):
            grid = (axes[a][:, None] + grid[None, :]).ravel()
        return grid  # ascending natural index because higher axes are outer

    out = []
    # explicit stack of (lo, hi, state); state 0 = expand, 1 = emit separator
    stack = [(tuple([0] * dim), shape, None)]
    while stack:
        lo, hi, sep = stack.pop()
        if sep is not None:
            out.append(sep)
            continue
        ext = [hi[a] - lo[a] for a in range(dim)]
        if min(ext) <= 0:
            continue
        count = int(np.prod(ext))
        if count <= leaf:
            out.append(box_nodes(lo, hi))
            continue
        ax = int(np.argmax(ext))  # first maximum: x before y before z
        mid = lo[ax] + (hi[ax] - lo[ax]) // 2
        lo_l, hi_l = list(lo), list(hi)
        hi_l[ax] = mid
        lo_r, hi_r = list(lo), list(hi)
        lo_r[ax] = mid + 1
        lo_s, hi_s = list(lo), list(hi)
        lo_s[ax] = mid
        hi_s[ax] = mid + 1
        sep_nodes = box_nodes(lo_s, hi_s)
        # pushed in reverse: left first, then right, then separator
        stack.append((lo, hi, sep_nodes))
        stack.append((tuple(lo_r), tuple(hi_r), None))
        stack.append((tuple(lo_l), tuple(hi_l), None))
    nodes = np.concatenate(out) if out else np.zeros(0, dtype=np.int64)
    if dof == 1:
        return nodes
    return (dof * nodes[:, None] + np.arange(dof)[None, :]).ravel()
