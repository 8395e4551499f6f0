"""ORACLE -- test infrastructure only.

Plain, slow, obviously correct FP64 CPU implementations of what the selected-
inverse path computes, written from the paper (Akter, Bollhoefer, Schenk,
"Scalable Approximate Selected Inversion Based on Single-Level Incomplete
LDL^T Factorization and Spectral Corrections"):

* ``symbolic_S``      -- S = {(i,j): (L+D+L^T)_ij != 0}   (Section 1)
* ``selinv``          -- scalar Takahashi recurrence, Eqs. (4)-(5) with the
                         restriction to S of Section 2.1       (C, csrc/selinv_ref.c)
* ``ninv``            -- truncated Neumann series L^{-1} ~ sum_{t<=m} E_L^t,
                         Eq. (6), and (L^inv)^T D^{-1} L^inv, Eq. (8), on S
* ``ninv_own``        -- the same with the inverse tolerance delta on its own
                         pattern (the product's fill controlled by delta too)
* ``mix``             -- Mix approximation (Section 2.3), on S
* ``mix_own``         -- the same on NInv's own pattern: the union of that
                         pattern and S_eps
* ``lowrank_correct`` -- A^inv + V_k Lambda_k V_k^T on S, Eq. (9); diagonal
                         update formula of Section 2.6
* ``spai_refine``     -- SPAI refinement on a fixed pattern by Jacobi-PCG on
                         each column's normal equations, then (Y + Y^T)/2
                         (Section 2.4; Mix-SPAI = spai_refine(Mix)); the
                         pattern is S or S widened by ``spai_pattern``
* ``lanczos_einv``    -- dominant eigenpairs of E_inv = A^{-1} - A^inv
                         (Section 2.5, Algorithm 1 step 5)
* measures            -- err_1, fill_fact, fill_inv, DoDD (Sections 2.6, 3.2)
* ``selinv_blocks``, ``ninv_W_columns`` -- the same recurrence on a list of
                         pivot blocks, and the series on a set of columns
                         given the columns they read (to check a partition)
* ``selinv_levels``, ``ninv_threads`` -- the same SelInv and NInv on every
                         host thread (OpenMP over level sets / independent
                         columns and entries; C, csrc/): the all-cores CPU
                         baseline, checked against ``selinv`` and ``ninv``

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: the one thing both sides use is the seeded input generator package
``workloads`` (matrices, ordering and the ILDL factors, none of the selected-
inverse arithmetic).

Parity pins: see ``tests/test_oracle_pins.py``.  Every function here is pinned
by at least one check that is not a re-typing of its own formula.
"""
from .core import (  # noqa: F401
    symbolic_S,
    selinv,
    ninv,
    ninv_W,
    ninv_own,
    ninv_entries_sampled,
    mix,
    mix_own,
    lowrank_correct,
    lowrank_diag,
    lanczos_einv,
    err1,
    fill_fact,
    fill_inv,
    dodd,
    accept_modes,
    build_lib,
    selinv_levels,
    ninv_threads,
    host_threads,
    selinv_blocks,
    ninv_W_columns,
)
from .spai import spai_columns, spai_refine, spai_entries_sampled, spai_pattern, embed, pcg_jacobi  # noqa: F401
