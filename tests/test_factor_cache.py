"""The on-disk cache of generated factors (keyed by generator, size, tolerance and
seed): a second build loads exactly the first one's matrix and factors."""
import numpy as np

from workloads.configs import elastic3d


def test_factor_cache_round_trip(tmp_path):
    a = elastic3d(5, cache_dir=str(tmp_path))
    files = list(tmp_path.iterdir())
    assert len(files) == 1 and files[0].name == "elastic3d_N5_tau0.0001_seed5.npz"
    b = elastic3d(5, cache_dir=str(tmp_path))
    assert b.factors.stats.get("cache") == str(files[0])
    fa, fb = a.factors, b.factors
    for name in ("L_rowptr", "L_col", "L_val", "pivot_start", "d_diag", "d_off"):
        x, y = getattr(fa, name), getattr(fb, name)
        assert x.dtype == y.dtype and np.array_equal(x, y), name
    assert (a.A != b.A).nnz == 0
    # another seed is another key
    elastic3d(5, seed=6, cache_dir=str(tmp_path))
    assert len(list(tmp_path.iterdir())) == 2
