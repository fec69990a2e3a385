"""Static pivoting with scaling (glu_static_pivot), host only.

The row matching must maximize the product of the diagonal magnitudes (brute
force over all permutations for small n; scipy's minimum-weight full
bipartite matching on larger ones), the scalings must put magnitude 1 on
the matching and at most 1 everywhere, structurally singular inputs must be
reported, and a matrix whose diagonal was scrambled must go through
pivoting, ordering, analysis and the oracle's factorization to a solution of
the original system."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import min_weight_full_bipartite_matching

import oracle
import synth
from paper_1908_00204_gb300 import glu


def random_nonsingular(n, density, seed):
    """Random magnitudes over six decades, a random permutation's entries
    present (so a perfect matching exists), no dominant diagonal."""
    rng = np.random.default_rng(seed)
    M = (rng.random((n, n)) < density) * 10.0 ** rng.uniform(-3, 3, (n, n)) * rng.choice([-1, 1], (n, n))
    p = rng.permutation(n)
    M[p, np.arange(n)] = 10.0 ** rng.uniform(-3, 3, n)
    A = sp.csc_matrix(M)
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.copy(), M


def log_product(M, rows_of_cols):
    return float(np.sum(np.log(np.abs(M[rows_of_cols, np.arange(M.shape[0])]))))


@pytest.mark.parametrize("seed", range(30))
def test_matching_is_optimal_by_brute_force(seed):
    n = 2 + seed % 6
    cp, ri, v, M = random_nonsingular(n, 0.5, seed)
    rp, rs, cs = glu.glu_static_pivot(n, cp, ri, v)
    assert sorted(rp.tolist()) == list(range(n))
    assert (M[rp, np.arange(n)] != 0).all()
    best = max(log_product(M, np.array(q)) for q in itertools.permutations(range(n))
               if (M[np.array(q), np.arange(n)] != 0).all())
    assert abs(log_product(M, rp) - best) <= 1e-9 * max(1.0, abs(best))
    # the scalings: magnitude 1 on the matching, at most 1 anywhere
    S = np.abs(rs[:, None] * M * cs[None, :])
    assert np.allclose(S[rp, np.arange(n)], 1.0, rtol=1e-12)
    assert (S <= 1.0 + 1e-12).all()


@pytest.mark.parametrize("n,density", [(300, 0.02), (1000, 0.005), (2000, 0.003)])
def test_matches_scipy_matching(n, density):
    # most columns need an augmenting path here: magnitudes spread over six
    # decades, no dominant diagonal
    cp, ri, va, M = random_nonsingular(n, density, 7 + n)
    rp, rs, cs = glu.glu_static_pivot(n, cp, ri, va)
    colmax = np.log(np.abs(M).max(axis=0))
    cost = sp.csc_matrix((colmax[np.repeat(np.arange(n), np.diff(cp))] - np.log(np.abs(va)) + 1.0, ri, cp),
                         shape=(n, n))
    r, c = min_weight_full_bipartite_matching(cost.T.tocsr())     # rows of cost^T are A's columns
    want = log_product(M, c[np.argsort(r)])
    assert abs(log_product(M, rp) - want) <= 1e-9 * max(1.0, abs(want))
    S = np.abs(rs[:, None] * M * cs[None, :])
    assert np.allclose(S[rp, np.arange(n)], 1.0, rtol=1e-12) and (S <= 1.0 + 1e-12).all()


def test_scrambled_mesh_gets_its_diagonal_back():
    m = synth.make("mesh100x200_nets64", 1)
    v = m.values(3)
    scramble = np.random.default_rng(4).permutation(m.n)          # row k of A is row scramble[k]
    A = sp.csc_matrix((v, m.rowidx, m.colptr), shape=(m.n, m.n))[scramble, :].tocsc()
    A.sort_indices()
    rp, rs, cs = glu.glu_static_pivot(m.n, A.indptr, A.indices, A.data)
    # the mesh is diagonally dominant by columns' largest entries: the
    # matching undoes the scramble
    assert np.array_equal(scramble[rp], np.arange(m.n))
    S = abs(sp.diags(rs) @ A @ sp.diags(cs))
    assert S.max() <= 1.0 + 1e-12
    assert np.allclose(np.asarray(S[rp, np.arange(m.n)]).ravel(), 1.0, rtol=1e-12)


def test_pivot_order_analyze_factor_solve_on_cpu():
    # rows scrambled: the analysis refuses the matrix (no diagonal); after
    # static pivoting and ordering it factors, and the solution of the
    # original system follows from the transformed one
    m = synth.CircuitMatrix(synth.CircuitSpec(20, 25, 4, 30, 0.02, 0.05, "nd"), 7)
    v = m.values(5)
    rng = np.random.default_rng(2)
    A = sp.csc_matrix((v, m.rowidx, m.colptr), shape=(m.n, m.n))[rng.permutation(m.n), :].tocsc()
    A.sort_indices()
    cp, ri, va = A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data
    with pytest.raises(glu.GluError) as e:
        glu.glu_analyze(m.n, cp, ri, None, glu.default_options(host_only=1))
    assert e.value.code == glu.GLU_ERR_STRUCT_SINGULAR
    rp, rs, cs = glu.glu_static_pivot(m.n, cp, ri, va)
    bcp, bri, bva = glu.apply_static_pivot(m.n, cp, ri, va, rp, rs, cs)
    perm = glu.glu_order_nd(m.n, bcp, bri)
    h = glu.glu_analyze(m.n, bcp, bri, perm, glu.default_options(host_only=1))
    f = oracle.Factorization(m.n, bcp, bri, perm, bva)
    fcp, fri = glu.glu_get_fill(h)
    glu.glu_destroy(h)
    assert np.array_equal(fcp, f.lu_colptr) and np.array_equal(fri, f.lu_rowidx)
    # A x = b  <=>  B y = P_r D_r b with x = D_c y
    b = synth.rhs(m.n, 1, 3).reshape(-1)
    y = np.asarray(f.solve((rs * b)[rp])).reshape(-1)
    x = cs * y
    assert np.abs(A @ x - b).max() <= 1e-10 * (np.abs(A).max() * np.abs(x).max() + np.abs(b).max())


def test_singular_and_invalid_inputs():
    # two columns whose only entries share one row: no perfect matching
    cp = np.array([0, 1, 2, 4], np.int32)
    ri = np.array([0, 0, 1, 2], np.int32)
    with pytest.raises(glu.GluError) as e:
        glu.glu_static_pivot(3, cp, ri, np.ones(4))
    assert e.value.code == glu.GLU_ERR_STRUCT_SINGULAR
    # an empty column, and a column of explicit zeros
    with pytest.raises(glu.GluError) as e:
        glu.glu_static_pivot(2, np.array([0, 1, 1], np.int32), np.array([0], np.int32), np.ones(1))
    assert e.value.code == glu.GLU_ERR_STRUCT_SINGULAR
    with pytest.raises(glu.GluError) as e:
        glu.glu_static_pivot(2, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, 0.0]))
    assert e.value.code == glu.GLU_ERR_STRUCT_SINGULAR
    for bad_ri, bad_v in (([0, 2], [1.0, 1.0]), ([0, 1], [1.0, np.nan])):
        with pytest.raises(glu.GluError) as e:
            glu.glu_static_pivot(2, np.array([0, 1, 2], np.int32), np.array(bad_ri, np.int32), np.array(bad_v))
        assert e.value.code == glu.GLU_ERR_INVALID
    assert glu.glu_static_pivot(0, np.array([0], np.int32), np.array([], np.int32), np.array([]))[0].size == 0


def test_deterministic():
    cp, ri, v, _ = random_nonsingular(60, 0.08, 11)
    a = glu.glu_static_pivot(60, cp, ri, v)
    b = glu.glu_static_pivot(60, cp.copy(), ri.copy(), v.copy())
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_apply_static_pivot_matches_scipy():
    """glu_apply_static_pivot against the same product formed with scipy:
    B = P_r D_r A D_c, rows ascending in every column."""
    cp, ri, v, A = random_nonsingular(80, 0.06, 21)
    rp, rs, cs = glu.glu_static_pivot(80, cp, ri, v)
    bcp, bri, bva = glu.glu_apply_static_pivot(80, cp, ri, v, rp, rs, cs)
    want = (sp.diags(rs) @ sp.csc_matrix(A) @ sp.diags(cs)).tocsr()[rp, :].tocsc()
    want.sort_indices()
    assert np.array_equal(bcp, want.indptr) and np.array_equal(bri, want.indices)
    np.testing.assert_allclose(bva, want.data, rtol=1e-15, atol=0)
    assert np.all(np.diff(bri[bcp[0]:bcp[1]]) > 0)
    # without scalings: a pure row permutation
    bcp, bri, bva = glu.glu_apply_static_pivot(80, cp, ri, v, rp)
    want = sp.csc_matrix(A).tocsr()[rp, :].tocsc()
    want.sort_indices()
    assert np.array_equal(bri, want.indices) and np.array_equal(bva, want.data)


def test_apply_static_pivot_invalid():
    cp = np.array([0, 2, 3], np.int32)
    ri = np.array([0, 1, 1], np.int32)
    v = np.ones(3)
    for rp in ([0, 0], [0, 2], [-1, 1]):        # not a permutation
        with pytest.raises(glu.GluError) as e:
            glu.glu_apply_static_pivot(2, cp, ri, v, np.array(rp, np.int32))
        assert e.value.code == glu.GLU_ERR_INVALID
    with pytest.raises(glu.GluError) as e:          # a row twice in one column
        glu.glu_apply_static_pivot(2, cp, np.array([1, 1, 0], np.int32), v, np.array([1, 0], np.int32))
    assert e.value.code == glu.GLU_ERR_INVALID
