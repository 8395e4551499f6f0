"""Values the paper prints, kept as text fixtures under tests/golden/ (each file
cites the table or figure it copies), checked against the input generators and
the oracle's measured quantities: the shape and diagonal dominance of the
microbenchmark band, the DoDD convention for a diagonal matrix, and the sizes
of the covariance example."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from workloads import grids

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [line.split() for line in fh if line.strip() and not line.startswith("#")]


@pytest.mark.parametrize("row", _rows("microbench_matrices.txt"), ids=lambda r: r[0])
def test_microbench_band_matches_the_printed_table(row):
    name, n, nnz_per_row, definiteness, dodd = row
    n, nnz_per_row, dodd = int(n), float(nnz_per_row), float(dodd)
    A = grids.band_dd(n, 1024, dodd, seed=6)
    assert A.shape == (n, n)
    assert round(A.nnz / n, 1) == nnz_per_row
    assert abs(oracle.dodd(A) - dodd) <= 1e-12 * dodd
    # SPD: a symmetric matrix with a positive diagonal and DoDD > 1 (Gershgorin)
    assert definiteness == "SPD"
    assert abs(A - A.T).max() == 0.0 and A.diagonal().min() > 0.0 and oracle.dodd(A) > 1.0


def test_dodd_of_a_diagonal_matrix_is_infinite():
    name, n, nnz_per_row, definiteness, dodd = _rows("test_matrices_diagonal.txt")[0]
    n = int(n)
    d = np.random.default_rng(0).uniform(-2.0, 2.0, n)
    d[d == 0] = 1.0
    A = sp.diags(d).tocsr()
    assert round(A.nnz / n, 1) == float(nnz_per_row)
    assert oracle.dodd(A) == float(dodd) == np.inf


@pytest.mark.parametrize("row", _rows("covariance_sizes.txt"), ids=lambda r: "N" + r[0])
def test_covariance_example_sizes(row):
    N, alpha, beta, n = (int(v) for v in row)
    C = grids.covariance2d(N, float(alpha), float(beta))
    assert C.shape == (n, n)
    assert np.all(C.diagonal() == 1.0)              # d(i, i) = 0
    assert abs(C - C.T).max() == 0.0
