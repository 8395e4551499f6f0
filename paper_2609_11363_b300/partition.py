"""Splitting one matrix's SelInv and NInv over ranks (host logic).

SelInv (Section 2.1) finishes supernode J once the supernodes owning its rows
C_J have finished: a dependency DAG from the root separators down to the
leaves.  NInv's Horner steps (Eq. (6)) read, for column j, the columns of
struct(j), which belong to the same supernodes.  A partition therefore takes

* a trunk T: the top of the DAG, closed under dependencies (every supernode a
  trunk supernode depends on is in T), computed by rank 0 first;
* one bin per rank: subtrees hanging below T; a bin's supernodes depend only on
  T and on their own bin.

The exchange is one broadcast from rank 0: the G entries of the trunk's
columns for SelInv, and the trunk's W columns (every Horner step) for NInv.
Then every rank finishes its bin with no further communication.  Rank r then
holds the entries of the trunk's columns and of its bin's columns; their union
over ranks is the whole result.

``split`` builds the partition from the supernode partition and the
dependencies; ``Plan`` derives the pivot blocks, columns and S_lo positions of
every part.  The arithmetic of each part is whatever engine the caller runs on
it (the tests use the FP64 oracle on gloo ranks).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .timeline import dependencies


def _parents(deps, ns):
    """Nearest dependency of every supernode (the owner of the first row of C_J,
    the elimination-tree parent for exact factors), -1 for roots."""
    return np.array([min(d) if d else -1 for d in deps], dtype=np.int64)


def split(sn_start, deps, work, nranks, max_trunk_frac=0.5, tol=0.1):
    """Trunk and nranks bins of supernodes.  work[J]: the cost of supernode J.

    The trunk starts empty and the frontier at the roots; while the frontier's
    subtrees cannot be packed into nranks bins within (1 + tol) of the mean
    (largest subtree first into the lightest bin), the heaviest frontier subtree
    moves its root into the trunk.  Dependencies that leave a bin are then pulled
    into the trunk with everything they depend on.  Returns (trunk, bins) as
    sorted int arrays."""
    ns = len(sn_start) - 1
    work = np.asarray(work, dtype=np.float64)
    par = _parents(deps, ns)
    children = [[] for _ in range(ns)]
    for j in range(ns):
        if par[j] >= 0:
            children[par[j]].append(j)
    sub = work.copy()
    for j in range(ns):          # children have smaller indices than their parent
        if par[j] >= 0:
            sub[par[j]] += sub[j]
    total = float(work.sum())
    trunk = set()
    frontier = [j for j in range(ns) if par[j] < 0]

    def pack(front):
        bins = [[] for _ in range(nranks)]
        load = np.zeros(nranks)
        for j in sorted(front, key=lambda x: -sub[x]):
            b = int(np.argmin(load))
            bins[b].append(j)
            load[b] += sub[j]
        return bins, load

    while True:
        bins, load = pack(frontier)
        mean = load.sum() / nranks
        tw = sum(work[j] for j in trunk)
        if load.max() <= (1 + tol) * mean or not frontier or tw > max_trunk_frac * total:
            break
        top = max(frontier, key=lambda x: sub[x])
        frontier.remove(top)
        trunk.add(top)
        frontier.extend(children[top])
    owner_bin = np.full(ns, -1, dtype=np.int64)

    def mark(j, b):
        stack = [j]
        while stack:
            x = stack.pop()
            owner_bin[x] = b
            stack.extend(children[x])

    for b, roots in enumerate(bins):
        for j in roots:
            mark(j, b)
    for j in trunk:
        owner_bin[j] = -1
    # repair: a dependency outside T and outside J's own bin moves into T with its closure
    changed = True
    while changed:
        changed = False
        for j in range(ns):
            b = owner_bin[j]
            for k in deps[j]:
                if owner_bin[k] >= 0 and (b < 0 or owner_bin[k] != b):
                    stack = [k]
                    while stack:
                        x = stack.pop()
                        if owner_bin[x] >= 0:
                            owner_bin[x] = -1
                            changed = True
                            stack.extend(deps[x])
    trunk = np.nonzero(owner_bin < 0)[0]
    return trunk, [np.nonzero(owner_bin == b)[0] for b in range(nranks)]


@dataclass
class Part:
    supernodes: np.ndarray   # in processing order (decreasing supernode index: dependencies first)
    blocks: np.ndarray       # pivot blocks (first column), processing order
    columns: np.ndarray      # columns of the part, ascending
    s_positions: np.ndarray  # S_lo positions whose column is in the part


class Plan:
    """The parts of one matrix for nranks ranks: parts[0] is the trunk, parts[1 + r]
    rank r's bin.  ``validate`` checks the closure properties."""

    def __init__(self, n, L_rowptr, L_col, pivot_start, sn_start, S, nranks, work=None):
        self.n = n
        self.sn_start = np.asarray(sn_start, dtype=np.int64)
        ns = len(self.sn_start) - 1
        self.deps = dependencies(n, L_rowptr, L_col, self.sn_start)
        if work is None:   # |C_J|^2 |J|: the size of the supernode's contraction
            rows = [set() for _ in range(ns)]
            owner = np.repeat(np.arange(ns), np.diff(self.sn_start))
            rr = np.repeat(np.arange(n), np.diff(np.asarray(L_rowptr)))
            for r, c in zip(rr, np.asarray(L_col)):
                J = owner[c]
                if r >= self.sn_start[J + 1]:
                    rows[J].add(int(r))
            work = np.array([len(rows[J]) ** 2 * (self.sn_start[J + 1] - self.sn_start[J]) + 1 for J in range(ns)],
                            dtype=np.float64)
        trunk, bins = split(self.sn_start, self.deps, work, nranks)
        ps = np.asarray(pivot_start)
        Srp, Sc = S
        col_of = np.asarray(Sc, dtype=np.int64)
        self.parts = []
        for sns in [trunk] + list(bins):
            sns = np.sort(np.asarray(sns, dtype=np.int64))[::-1]
            cols = np.concatenate([np.arange(self.sn_start[J], self.sn_start[J + 1]) for J in sns]) \
                if len(sns) else np.zeros(0, dtype=np.int64)
            cols = np.sort(cols)
            blocks = np.array([c for c in cols[::-1] if ps[c]], dtype=np.int64)
            inpart = np.zeros(n, dtype=bool)
            inpart[cols] = True
            spos = np.nonzero(inpart[col_of])[0]
            self.parts.append(Part(sns, blocks, cols, spos))
        self.nranks = nranks

    def validate(self):
        """Every supernode depends only on its own part or the trunk, and the trunk only
        on itself; the parts cover every supernode once."""
        ns = len(self.sn_start) - 1
        where = np.full(ns, -1)
        for p, part in enumerate(self.parts):
            assert np.all(where[part.supernodes] == -1)
            where[part.supernodes] = p
        assert np.all(where >= 0)
        for J in range(ns):
            for K in self.deps[J]:
                assert where[K] == 0 or where[K] == where[J], (J, K)
        return True
