"""The built-in fill-reducing ordering (glu_order_nd), host only.

It must return a permutation, deterministically; reduce fill well below the
natural order on a grid; set the high-degree supply-net vertices last; give
no more fill than the generator's geometric nested dissection on the mesh
workloads; and the analysis under it must match the oracle bit for bit."""
import numpy as np
import pytest

import oracle
import synth
from paper_1908_00204_gb300 import glu


def fill(n, cp, ri, perm):
    h = glu.glu_analyze(n, cp, ri, perm, glu.default_options(host_only=1))
    try:
        return glu.glu_get_stats(h)["nnz_lu"]
    finally:
        glu.glu_destroy(h)


def test_permutation_and_deterministic():
    m = synth.make("mesh100x200_nets64", 1)
    p1 = glu.glu_order_nd(m.n, m.colptr, m.rowidx)
    p2 = glu.glu_order_nd(m.n, m.colptr.copy(), m.rowidx.copy())
    assert np.array_equal(np.sort(p1), np.arange(m.n))
    assert np.array_equal(p1, p2)


def test_grid_fill_far_below_natural():
    m = synth.make("grid32_natural", 0)
    p = glu.glu_order_nd(m.n, m.colptr, m.rowidx)
    assert fill(m.n, m.colptr, m.rowidx, p) < 0.5 * fill(m.n, m.colptr, m.rowidx, None)   # 25k vs 64,574


def test_supply_nets_ordered_last_and_fill_vs_generator():
    m = synth.make("mesh100x200_nets64", 1)
    p = glu.glu_order_nd(m.n, m.colptr, m.rowidx)
    nets = set(range(m.n - 64, m.n))          # the generator numbers the nets after the mesh nodes
    assert set(p[-64:].tolist()) == nets
    assert fill(m.n, m.colptr, m.rowidx, p) <= fill(m.n, m.colptr, m.rowidx, m.perm)


@pytest.mark.parametrize("seed", range(3))
def test_analysis_under_the_order_matches_oracle(seed):
    cp, ri, v = synth.random_pattern_matrix(120, 0.05, 70 + seed)
    p = glu.glu_order_nd(120, cp, ri)
    f = oracle.Factorization(120, cp, ri, p)
    h = glu.glu_analyze(120, cp, ri, p, glu.default_options(host_only=1))
    try:
        fcp, fri = glu.glu_get_fill(h)
        assert np.array_equal(fcp, f.lu_colptr) and np.array_equal(fri, f.lu_rowidx)
        lp, lc = glu.glu_get_levels(h)
        assert np.array_equal(lp, f.level_ptr) and np.array_equal(lc, f.level_cols)
    finally:
        glu.glu_destroy(h)


def test_disconnected_and_tiny_and_invalid():
    # two disconnected paths and isolated vertices
    n = 70
    rows, cols = list(range(n)), list(range(n))
    for i in range(29):
        rows += [i, i + 1]
        cols += [i + 1, i]
    for i in range(40, 68):
        rows += [i, i + 1]
        cols += [i + 1, i]
    import scipy.sparse as sp
    A = sp.csc_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    p = glu.glu_order_nd(n, A.indptr, A.indices)
    assert np.array_equal(np.sort(p), np.arange(n))
    assert glu.glu_order_nd(1, np.array([0, 1]), np.array([0])).tolist() == [0]
    assert glu.glu_order_nd(0, np.array([0]), np.array([], np.int32)).size == 0
    with pytest.raises(glu.GluError):
        glu.glu_order_nd(3, np.array([0, 1, 2, 3]), np.array([0, 5, 2]))
