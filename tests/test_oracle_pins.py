"""Pins for the CPU oracle: each check rests on something other than the oracle.

* fill: brute-force boolean dense elimination; closed forms (tridiagonal,
  arrow, dense first row/column);
* numeric: exact rational elimination (fractions.Fraction), scipy's LU on
  column-dominant matrices (partial pivoting then never swaps), the Thomas
  recurrence for tridiagonal matrices, and ||B - L U|| / ||B||;
* dependencies: GLU2.0's double-U search (Algorithm 3) and GLU1.0's
  up-looking rule must be contained in Algorithm 4's sets; a level-hazard
  checker (no column of a level reads what another column of that level
  writes during the right-looking update, Section II-C);
* levels: closed forms (diagonal, tridiagonal, block-tridiagonal, arrow) and
  the 32x32 natural-order grid (1024 levels of width 1);
* the paper's worked example (Figs. 2-4, 8, 9) from ``golden/paper_example.json``;
* solve: identity matrix, numpy's dense solve, backward error.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp

import oracle
import synth
from conftest import csc_from_mask, dense_from_csc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- brute force
def bool_fill(mask):
    """Structural no-pivot elimination of a dense boolean pattern."""
    M = mask.copy()
    n = M.shape[0]
    for k in range(n):
        M[k + 1:, k + 1:] |= np.outer(M[k + 1:, k], M[k, k + 1:])
    return M


def oracle_pattern_dense(n, colptr, rowidx, perm=None):
    f = oracle.Factorization(n, colptr, rowidx, perm)
    return f, dense_from_csc(n, f.lu_colptr, f.lu_rowidx).astype(bool)


def random_mask(n, density, seed):
    rng = np.random.default_rng(seed)
    m = rng.random((n, n)) < density
    np.fill_diagonal(m, True)
    return m


# ---------------------------------------------------------------------- fill
@pytest.mark.parametrize("seed", range(40))
def test_fill_matches_boolean_elimination_random(seed):
    n = 4 + seed % 37
    mask = random_mask(n, [0.05, 0.1, 0.2, 0.4][seed % 4], seed)
    cp, ri = csc_from_mask(mask)
    _, got = oracle_pattern_dense(n, cp, ri)
    assert np.array_equal(got, bool_fill(mask))


def test_fill_matches_boolean_elimination_permuted():
    rng = np.random.default_rng(7)
    n = 120
    mask = random_mask(n, 0.03, 7)
    perm = rng.permutation(n).astype(np.int32)
    cp, ri = csc_from_mask(mask)
    _, got = oracle_pattern_dense(n, cp, ri, perm)
    B = mask[np.ix_(perm, perm)]          # B(i,j) = A(perm i, perm j)
    assert np.array_equal(got, bool_fill(B))


def test_fill_grid32_brute_force(grid32):
    m = grid32
    mask = dense_from_csc(m.n, m.colptr, m.rowidx).astype(bool)
    want = bool_fill(mask)
    f, got = oracle_pattern_dense(m.n, m.colptr, m.rowidx, m.perm)
    assert np.array_equal(got, want)
    assert f.nnz == int(want.sum()) == 64574
    # flops from the brute-force pattern: sum_j l_j + 2 l_j u_j
    lj = np.tril(want, -1).sum(0)
    uj = np.triu(want, 1).sum(1)
    F = int((lj + 2 * lj * uj).sum())
    assert F == 2043613
    assert f.flops() == F


def test_fill_closed_forms():
    n = 50
    tri = np.eye(n, dtype=bool) | np.eye(n, k=1, dtype=bool) | np.eye(n, k=-1, dtype=bool)
    f, got = oracle_pattern_dense(n, *csc_from_mask(tri))
    assert f.nnz == 3 * n - 2 and np.array_equal(got, tri)
    arrow_last = np.eye(n, dtype=bool)
    arrow_last[-1, :] = arrow_last[:, -1] = True
    f, got = oracle_pattern_dense(n, *csc_from_mask(arrow_last))
    assert f.nnz == 3 * n - 2 and np.array_equal(got, arrow_last)
    arrow_first = np.eye(n, dtype=bool)
    arrow_first[0, :] = arrow_first[:, 0] = True
    f, _ = oracle_pattern_dense(n, *csc_from_mask(arrow_first))
    assert f.nnz == n * n


def test_fill_explicit_zero_is_structural():
    # an explicit zero entry still creates fill
    cp = np.array([0, 2, 4, 5], np.int32)
    ri = np.array([0, 2, 0, 1, 2], np.int32)   # (2,0) and (0,1) present
    f = oracle.Factorization(3, cp, ri, None, np.array([1.0, 0.0, 0.0, 1.0, 1.0]))
    pat = dense_from_csc(3, f.lu_colptr, f.lu_rowidx).astype(bool)
    assert pat[2, 1]  # fill from (2,0) x (0,1)


# ------------------------------------------------------------------- numeric
def exact_lu(Mq):
    """Doolittle elimination in rationals; returns the combined L+U-I."""
    n = len(Mq)
    A = [row[:] for row in Mq]
    for k in range(n):
        for i in range(k + 1, n):
            if A[i][k] != 0:
                A[i][k] = A[i][k] / A[k][k]
                for j in range(k + 1, n):
                    A[i][j] -= A[i][k] * A[k][j]
    return A


@pytest.mark.parametrize("seed", range(12))
def test_numeric_matches_exact_rational_lu(seed):
    n = 3 + seed % 6
    cp, ri, v = synth.random_pattern_matrix(n, 0.5, 100 + seed, dominant=(seed % 3 != 0))
    D = dense_from_csc(n, cp, ri, v)
    ex = exact_lu([[Fraction(x) for x in row] for row in D])
    f = oracle.Factorization(n, cp, ri, None, v)
    for j in range(n):
        for p in range(f.lu_colptr[j], f.lu_colptr[j + 1]):
            i = f.lu_rowidx[p]
            want = float(ex[i][j])
            assert abs(f.lu_val[p] - want) <= 1e-13 * max(1.0, abs(want)), (i, j)


@pytest.mark.parametrize("seed", range(8))
def test_numeric_matches_scipy_lu_on_dominant(seed):
    n = 30 + 10 * seed
    cp, ri, v = synth.random_pattern_matrix(n, 0.08, 200 + seed)
    D = dense_from_csc(n, cp, ri, v)
    P, L, U = scipy.linalg.lu(D)
    assert np.array_equal(P, np.eye(n))         # column dominance: no swaps
    f = oracle.Factorization(n, cp, ri, None, v)
    got = dense_from_csc(n, f.lu_colptr, f.lu_rowidx, f.lu_val)
    want = np.tril(L, -1) + U
    pat = dense_from_csc(n, f.lu_colptr, f.lu_rowidx).astype(bool)
    assert np.all(want[~pat] == 0.0)            # nothing outside the fill
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)


def test_numeric_thomas_tridiagonal():
    n = 200
    rng = np.random.default_rng(3)
    a = rng.uniform(3, 4, n)            # diagonal
    b = rng.uniform(-1, 1, n - 1)       # super-diagonal
    c = rng.uniform(-1, 1, n - 1)       # sub-diagonal
    D = np.diag(a) + np.diag(b, 1) + np.diag(c, -1)
    mask = D != 0
    cp, ri = csc_from_mask(mask)
    vals = np.concatenate([D[ri[cp[j]:cp[j + 1]], j] for j in range(n)])
    f = oracle.Factorization(n, cp, ri, None, vals)
    d = np.empty(n)
    l = np.empty(n - 1)
    d[0] = a[0]
    for i in range(1, n):
        l[i - 1] = c[i - 1] / d[i - 1]
        d[i] = a[i] - l[i - 1] * b[i - 1]
    got = dense_from_csc(n, f.lu_colptr, f.lu_rowidx, f.lu_val)
    np.testing.assert_allclose(np.diag(got), d, rtol=1e-14)
    np.testing.assert_allclose(np.diag(got, -1), l, rtol=1e-14)
    np.testing.assert_allclose(np.diag(got, 1), b, rtol=0)


def lu_residual(f, values):
    """||B - L U||_F / ||B||_F on the filled pattern."""
    n = f.n
    cp, ri, lv = f.lu_colptr, f.lu_rowidx, f.lu_val
    cols = np.repeat(np.arange(n), np.diff(cp))
    low = ri > cols
    L = sp.csc_matrix((lv[low], (ri[low], cols[low])), shape=(n, n)) + sp.identity(n)
    U = sp.csc_matrix((lv[~low], (ri[~low], cols[~low])), shape=(n, n))
    bc = np.repeat(np.arange(n), np.diff(f.bcolptr))
    B = sp.csc_matrix((np.asarray(values)[f.bsrc], (f.browidx, bc)), shape=(n, n))
    R = B - L @ U
    return sp.linalg.norm(R) / sp.linalg.norm(B)


def test_invariant_grid32(grid32):
    v = grid32.values(1)
    f = oracle.Factorization(grid32.n, grid32.colptr, grid32.rowidx, grid32.perm, v)
    assert lu_residual(f, v) <= 1e-13


def test_invariant_mesh_nd_small():
    m = synth.CircuitMatrix(synth.CircuitSpec(24, 30, 4, 20, 0.02, 0.05, "nd"), 5)
    v = m.values(11)
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm, v)
    assert lu_residual(f, v) <= 1e-13


def test_zero_and_nonfinite_pivot():
    cp = np.array([0, 2, 4], np.int32)
    ri = np.array([0, 1, 0, 1], np.int32)
    with pytest.raises(oracle.OracleError) as e:
        oracle.Factorization(2, cp, ri, None, np.array([1.0, 2.0, 3.0, 6.0]))  # pivot 6-2*3 = 0
    assert e.value.code == -3 and e.value.column == 1
    with pytest.raises(oracle.OracleError) as e:
        oracle.Factorization(2, cp, ri, None, np.array([np.nan, 2.0, 3.0, 6.0]))
    assert e.value.code == -4 and e.value.column == 0


def test_invalid_inputs():
    with pytest.raises(oracle.OracleError) as e:   # missing diagonal
        oracle.permute(2, np.array([0, 1, 2]), np.array([1, 0]))
    assert e.value.code == -2
    with pytest.raises(oracle.OracleError):        # unsorted rows
        oracle.permute(2, np.array([0, 2, 3]), np.array([1, 0, 1]))
    with pytest.raises(oracle.OracleError):        # bad permutation
        oracle.permute(2, np.array([0, 1, 2]), np.array([0, 1]), np.array([0, 0]))


# ---------------------------------------------------------------------- deps
def alg3_pairs(M):
    """GLU2.0 double-U detection (Algorithm 3): i -> t when rows i and j
    share a column k > t, for t with A_s(t,i) != 0 and j with A_s(j,t) != 0."""
    n = M.shape[0]
    out = set()
    rows = [set(np.nonzero(M[i])[0]) for i in range(n)]
    for i in range(n):
        for t in range(i + 1, n):
            if not M[t, i]:
                continue
            for j in range(t + 1, n):
                if M[j, t] and any(k > t for k in rows[i] & rows[j]):
                    out.add((i, t))
    return out


def uplooking_pairs(M):
    """GLU1.0: k depends on i < k if U(i,k) != 0 and column i of L is not empty."""
    n = M.shape[0]
    hasl = [M[i + 1:, i].any() for i in range(n)]
    return {(i, k) for k in range(n) for i in range(k) if M[i, k] and hasl[i]}


def dep_pairs(f):
    return {(int(i), k) for k in range(f.n) for i in f.dep_idx[f.dep_ptr[k]:f.dep_ptr[k + 1]]}


def level_hazards(M, level_of):
    """Entries written by one source of a level and read as an input by
    another source of the same level during the right-looking update
    (Algorithm 2): a source j reads L(:,j), the pivot and U(j,:), and writes
    L(:,j) and the submatrix entries (i,k).  Two sources subtracting from the
    same (i,k) commute and are not a hazard."""
    n = M.shape[0]
    bad = []
    for lv in range(level_of.max() + 1):
        cols = np.nonzero(level_of == lv)[0]
        reads, writes = {}, {}
        for j in cols:
            Lj = np.nonzero(M[j + 1:, j])[0] + j + 1
            Uj = np.nonzero(M[j, j + 1:])[0] + j + 1
            r = {(i, j) for i in Lj} | {(j, j)}
            w = {(i, j) for i in Lj}
            if Lj.size:
                r |= {(j, k) for k in Uj}
                w |= {(i, k) for i in Lj for k in Uj}
            reads[j], writes[j] = r, w
        for a in cols:
            for b in cols:
                if a != b and writes[a] & reads[b]:
                    bad.append((lv, a, b))
    return bad


@pytest.mark.parametrize("seed", range(30))
def test_deps_superset_and_hazard_free(seed):
    n = 5 + seed % 20
    mask = random_mask(n, [0.1, 0.2, 0.3][seed % 3], 1000 + seed)
    cp, ri = csc_from_mask(mask)
    f, M = oracle_pattern_dense(n, cp, ri)
    d = dep_pairs(f)
    assert alg3_pairs(M) <= d
    assert uplooking_pairs(M) <= d
    # Algorithm 4 literally: look up (with non-empty L) and look left
    hasl = [M[i + 1:, i].any() for i in range(n)]
    want = {(i, k) for k in range(n) for i in range(k) if (M[i, k] and hasl[i]) or M[k, i]}
    assert d == want
    assert level_hazards(M, f.level_of) == []


def test_uplooking_alone_has_hazards():
    # the hazard checker is not vacuous: GLU1.0's levels race on this pattern
    found = False
    for seed in range(60):
        n = 8 + seed % 10
        mask = random_mask(n, 0.25, 5000 + seed)
        M = bool_fill(mask)
        up = uplooking_pairs(M)
        lv = np.zeros(n, np.int64)
        for k in range(n):
            lv[k] = 1 + max([lv[i] for (i, kk) in up if kk == k], default=-1)
        if level_hazards(M, lv):
            found = True
            break
    assert found


def test_paper_example():
    g = json.load(open(os.path.join(GOLDEN, "paper_example.json")))
    n = g["n"]
    mask = np.zeros((n, n), bool)
    for r, c in g["entries_1based"]:
        mask[r - 1, c - 1] = True
    cp, ri = csc_from_mask(mask)
    f, M = oracle_pattern_dense(n, cp, ri)
    assert np.array_equal(M, bool_fill(mask))
    e = g["expect"]
    hasl = [M[i + 1:, i].any() for i in range(n)]
    # Algorithm 1 on column 7 uses k with A_s(k,7) != 0 and a non-empty L(:,k)
    assert [k + 1 for k in range(6) if M[k, 6] and hasl[k]] == e["gp_column7_sources_1based"]
    assert [k + 1 for k in range(3, n) if M[2, k]] == e["column3_subcolumns_1based"]
    deps6 = set(f.dep_idx[f.dep_ptr[5]:f.dep_ptr[6]] + 1)
    up6 = {i + 1 for i in range(5) if M[i, 5] and hasl[i]}
    left6 = {i + 1 for i in range(5) if M[5, i]}
    assert sorted(up6) == e["column6_uplooking_deps_1based"]
    assert sorted(left6) == e["column6_leftlooking_deps_1based"]
    assert deps6 == up6 | left6
    du = sorted([i + 1, t + 1] for i, t in alg3_pairs(M))
    assert du == e["double_u_pairs_1based"]
    # levels from GLU2.0's exact set (up-looking + double-U) equal Algorithm 4's
    exact = uplooking_pairs(M) | alg3_pairs(M)
    lv = np.zeros(n, np.int64)
    for k in range(n):
        lv[k] = 1 + max([lv[i] for (i, kk) in exact if kk == k], default=-1)
    assert np.array_equal(lv, f.level_of) == e["levels_equal_glu2"]
    assert dep_pairs(f) > exact   # strictly more edges: the redundant ones


# -------------------------------------------------------------------- levels
def test_levels_closed_forms():
    n = 40
    f = oracle.Factorization(n, *csc_from_mask(np.eye(n, dtype=bool)))
    assert f.nlevels == 1 and np.array_equal(f.level_cols, np.arange(n))
    tri = np.eye(n, dtype=bool) | np.eye(n, k=1, dtype=bool) | np.eye(n, k=-1, dtype=bool)
    f = oracle.Factorization(n, *csc_from_mask(tri))
    assert f.nlevels == n and np.array_equal(f.level_of, np.arange(n))
    # b disjoint tridiagonal blocks of size m, interleaved: m levels of width b
    b, m = 5, 8
    blk = np.zeros((b * m, b * m), bool)
    for t in range(b):
        idx = np.arange(m) * b + t
        blk[np.ix_(idx, idx)] = (np.eye(m, dtype=bool) | np.eye(m, k=1, dtype=bool)
                                 | np.eye(m, k=-1, dtype=bool))
    f = oracle.Factorization(b * m, *csc_from_mask(blk))
    assert f.nlevels == m and np.all(np.diff(f.level_ptr) == b)
    arrow = np.eye(n, dtype=bool)
    arrow[-1, :] = arrow[:, -1] = True
    f = oracle.Factorization(n, *csc_from_mask(arrow))
    assert f.nlevels == 2 and list(np.diff(f.level_ptr)) == [n - 1, 1]


def test_levels_grid32(grid32):
    f = oracle.Factorization(grid32.n, grid32.colptr, grid32.rowidx, grid32.perm)
    assert f.nlevels == 1024 and np.all(np.diff(f.level_ptr) == 1)


def test_levels_longest_path_definition():
    mask = random_mask(60, 0.05, 42)
    f = oracle.Factorization(60, *csc_from_mask(mask))
    for k in range(60):
        d = f.dep_idx[f.dep_ptr[k]:f.dep_ptr[k + 1]]
        assert f.level_of[k] == (1 + f.level_of[d].max() if d.size else 0)
    for lv in range(f.nlevels):
        cols = f.level_cols[f.level_ptr[lv]:f.level_ptr[lv + 1]]
        assert np.all(np.diff(cols) > 0) and np.all(f.level_of[cols] == lv)


# --------------------------------------------------------------------- solve
def test_solve_identity():
    n = 17
    f = oracle.Factorization(n, *csc_from_mask(np.eye(n, dtype=bool)), None, np.ones(n))
    b = np.random.default_rng(0).uniform(-1, 1, (3, n))
    assert np.array_equal(f.solve(b), b)


@pytest.mark.parametrize("seed", range(6))
def test_solve_matches_dense(seed):
    n = 20 + 15 * seed
    cp, ri, v = synth.random_pattern_matrix(n, 0.1, 300 + seed)
    perm = np.random.default_rng(seed).permutation(n).astype(np.int32)
    D = dense_from_csc(n, cp, ri, v)
    f = oracle.Factorization(n, cp, ri, perm, v)
    b = np.random.default_rng(seed + 9).uniform(-1, 1, (2, n))
    x = f.solve(b)
    want = np.linalg.solve(D, b.T).T
    np.testing.assert_allclose(x, want, rtol=1e-10, atol=1e-12)


def test_solve_backward_error_grid32(grid32):
    v = grid32.values(1)
    f = oracle.Factorization(grid32.n, grid32.colptr, grid32.rowidx, grid32.perm, v)
    b = synth.rhs(grid32.n, 1, 7)
    x = f.solve(b)
    D = dense_from_csc(grid32.n, grid32.colptr, grid32.rowidx, v)
    r = b[0] - D @ x[0]
    berr = np.abs(r).max() / (np.abs(D).sum(1).max() * np.abs(x).max() + np.abs(b).max())
    assert berr <= 1e-12
    np.testing.assert_allclose(oracle.residual(grid32.n, grid32.colptr, grid32.rowidx, v, b, x)[0],
                               r, atol=1e-13)


def test_solve_levels_closed_forms():
    n = 30
    tri = np.eye(n, dtype=bool) | np.eye(n, k=1, dtype=bool) | np.eye(n, k=-1, dtype=bool)
    cp, ri = csc_from_mask(tri)
    f = oracle.Factorization(n, cp, ri)
    lf, lb = oracle.solve_levels(n, f.lu_colptr, f.lu_rowidx)
    assert np.array_equal(lf, np.arange(n)) and np.array_equal(lb, np.arange(n)[::-1])
    f = oracle.Factorization(n, *csc_from_mask(np.eye(n, dtype=bool)))
    lf, lb = oracle.solve_levels(n, f.lu_colptr, f.lu_rowidx)
    assert not lf.any() and not lb.any()
