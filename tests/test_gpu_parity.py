"""GPU parity: the CUDA library against the CPU oracle on the same seeded inputs.

Bars: fill, dependencies and levels bit-exact; FP64 factors within 1e-10
relative per entry (cancellation rule in ``parity.factor_mismatches``);
FP64 solves with a normwise backward error <= 1e-12.
"""
import numpy as np
import pytest

import oracle
import synth
from parity import BERR_TOL, backward_error, factor_mismatches

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def glu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_00204_gb300 as g
    g.build.build()
    g.load_library()
    torch.cuda.init()
    return g


def run_case(g, n, colptr, rowidx, perm, values, rhs, opts=None, device_inputs=False):
    f = oracle.Factorization(n, colptr, rowidx, perm, values)
    h = g.glu_analyze(n, colptr, rowidx, perm, opts)
    cp, ri = g.glu_get_fill(h)
    assert np.array_equal(cp, f.lu_colptr) and np.array_equal(ri, f.lu_rowidx)
    dp, di = g.glu_get_deps(h)
    assert np.array_equal(dp, f.dep_ptr) and np.array_equal(di, f.dep_idx)
    lp, lc = g.glu_get_levels(h)
    assert np.array_equal(lp, f.level_ptr) and np.array_equal(lc, f.level_cols)
    if device_inputs:
        g.glu_factor(h, torch.from_numpy(values).cuda())
        g.glu_sync(h)
    else:
        g.glu_factor(h, values)
    got = g.glu_get_factors(h)
    bad, _ = factor_mismatches(f.lu_colptr, f.lu_rowidx, got, f.lu_val)
    assert bad.size == 0, f"{bad.size} factor entries off, first {bad[:5]}"
    if device_inputs:
        x = g.glu_solve(h, torch.from_numpy(rhs).cuda()).cpu().numpy()
    else:
        x = g.glu_solve(h, rhs)
    assert backward_error(n, colptr, rowidx, values, rhs, x) <= BERR_TOL
    xr = f.solve(rhs)
    np.testing.assert_allclose(x, xr, rtol=1e-8, atol=1e-12)
    return h, got, f


def test_grid32(glu):
    m = synth.make("grid32_natural", 0)
    run_case(glu, m.n, m.colptr, m.rowidx, m.perm, m.values(1), synth.rhs(m.n, 1, 2))


@pytest.mark.parametrize("seed", range(6))
def test_random_small(glu, seed):
    n = [1, 2, 7, 33, 65, 150][seed]
    cp, ri, v = synth.random_pattern_matrix(n, 0.15, 40 + seed)
    perm = np.random.default_rng(seed).permutation(n).astype(np.int32)
    run_case(glu, n, cp, ri, perm, v, synth.rhs(n, 3, seed))


def test_mesh_small_nd_with_nets(glu):
    m = synth.CircuitMatrix(synth.CircuitSpec(30, 40, 8, 60, 0.02, 0.05, "nd"), 3)
    run_case(glu, m.n, m.colptr, m.rowidx, m.perm, m.values(5), synth.rhs(m.n, 2, 5))


def test_mesh100x200(glu):
    m = synth.make("mesh100x200_nets64", 1)
    run_case(glu, m.n, m.colptr, m.rowidx, m.perm, m.values(2001), synth.rhs(m.n, 4, 2001),
             device_inputs=True)


def test_mesh100x200_under_builtin_order(glu):
    # the same matrix in the library's own nested-dissection order
    m = synth.make("mesh100x200_nets64", 1)
    perm = glu.glu_order_nd(m.n, m.colptr, m.rowidx)
    run_case(glu, m.n, m.colptr, m.rowidx, perm, m.values(2002), synth.rhs(m.n, 2, 2002))


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_mode_invariance(glu, mode):
    m = synth.CircuitMatrix(synth.CircuitSpec(20, 30, 4, 30, 0.02, 0.05, "nd"), 9)
    v = m.values(3)
    base = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    glu.glu_factor(base, v)
    ref = glu.glu_get_factors(base)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(mode_force=mode))
    glu.glu_factor(h, v)
    assert np.array_equal(glu.glu_get_factors(h), ref)


def test_refactor_new_values_and_determinism(glu):
    m = synth.make("mesh100x200_nets64", 1)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm)
    for s in (11, 12):
        v = m.values(s)
        glu.glu_factor(h, v)
        a = glu.glu_get_factors(h)
        glu.glu_factor(h, v)
        assert np.array_equal(glu.glu_get_factors(h), a)   # run-to-run identical
        bad, _ = factor_mismatches(f.lu_colptr, f.lu_rowidx, a, f.factor(v))
        assert bad.size == 0


def test_zero_pivot_reported(glu):
    cp = np.array([0, 2, 4, 5], np.int32)
    ri = np.array([0, 1, 0, 1, 2], np.int32)
    h = glu.glu_analyze(3, cp, ri)
    with pytest.raises(glu.GluError) as e:
        glu.glu_factor(h, np.array([1.0, 2.0, 3.0, 6.0, 1.0]))
    assert e.value.code == glu.glu.GLU_ERR_ZERO_PIVOT and e.value.column == 1
    with pytest.raises(glu.GluError) as e:
        glu.glu_factor(h, np.array([np.nan, 2.0, 3.0, 7.0, 1.0]))
    assert e.value.code == glu.glu.GLU_ERR_NONFINITE and e.value.column == 0
    # a good refactorization afterwards works again
    glu.glu_factor(h, np.array([4.0, 1.0, 1.0, 4.0, 1.0]))
    x = glu.glu_solve(h, np.array([1.0, 2.0, 3.0]))
    np.testing.assert_allclose(x, np.linalg.solve(np.array([[4, 1, 0], [1, 4, 0], [0, 0, 1.0]]),
                                                  [1, 2, 3]), rtol=1e-14)


def test_solve_before_factor_and_empty(glu):
    m = synth.make("grid32_natural", 0)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    with pytest.raises(glu.GluError) as e:
        glu.glu_solve(h, np.zeros(m.n))
    assert e.value.code == glu.glu.GLU_ERR_NOT_FACTORED
    glu.glu_factor(h, m.values(1))
    x = glu.glu_solve(h, np.zeros((0, m.n)), nrhs=0)
    assert x.shape == (0, m.n)


def test_mesh400x500_full(glu):
    """The 200k-unknown workload at full size, the whole factor compared."""
    m = synth.make("mesh400x500_nets64", 1)
    run_case(glu, m.n, m.colptr, m.rowidx, m.perm, m.values(1001), synth.rhs(m.n, 1, 1001),
             device_inputs=True)


def test_graph_and_direct_launches_identical(glu):
    """The CUDA-graph path and the direct-launch path give bit-identical
    factors and solutions (several right-hand-side counts, repeated calls)."""
    m = synth.make("mesh100x200_nets64", 1)
    v = m.values(77)
    hg = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(use_graph=1))
    hd = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(use_graph=0))
    for h in (hg, hd):
        glu.glu_factor(h, v)
    assert np.array_equal(glu.glu_get_factors(hg), glu.glu_get_factors(hd))
    for k in (1, 4, 2, 4):
        b = synth.rhs(m.n, k, 100 + k)
        xg = glu.glu_solve(hg, b)
        xd = glu.glu_solve(hd, b)
        assert np.array_equal(xg, xd)
        assert backward_error(m.n, m.colptr, m.rowidx, v, b, xg) <= BERR_TOL


def test_multiple_rhs_device(glu):
    m = synth.CircuitMatrix(synth.CircuitSpec(40, 50, 16, 100, 0.02, 0.05, "nd"), 21)
    v = m.values(4)
    b = synth.rhs(m.n, 8, 4)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    glu.glu_factor(h, torch.from_numpy(v).cuda())
    x = glu.glu_solve(h, torch.from_numpy(b).cuda()).cpu().numpy()
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm, v)
    np.testing.assert_allclose(x, f.solve(b), rtol=1e-9, atol=1e-12)
    assert backward_error(m.n, m.colptr, m.rowidx, v, b, x) <= BERR_TOL


@pytest.mark.parametrize("spec", [(16, 20, 900, 15), (16, 20, 1700, 10)])
def test_dense_tail_factor(glu, spec):
    """A trailing dense block of ~900 / ~1700 columns (panel widths 16 and 8)
    factored by the dense kernel: factors against the oracle, and against the
    level sweep run over the same block (factor_tail=0)."""
    m = synth.CircuitMatrix(synth.CircuitSpec(spec[0], spec[1], spec[2], spec[3], 0.02, 0.05, "nd"), 3)
    v = m.values(8)
    h, got, _ = run_case(glu, m.n, m.colptr, m.rowidx, m.perm, v, synth.rhs(m.n, 2, 8))
    assert glu.glu_get_stats(h)["factor_tail_cols"] >= 800
    h0 = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(factor_tail=0))
    assert glu.glu_get_stats(h0)["factor_tail_cols"] == 0
    glu.glu_factor(h0, v)
    ref = glu.glu_get_factors(h0)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-14 * np.abs(ref).max())


def test_dense_tail_factor_mesh100x200(glu):
    m = synth.make("mesh100x200_nets64", 1)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    assert glu.glu_get_stats(h)["factor_tail_cols"] >= 64
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm)
    v = m.values(31)
    glu.glu_factor(h, v)
    got = glu.glu_get_factors(h)
    bad, _ = factor_mismatches(f.lu_colptr, f.lu_rowidx, got, f.factor(v))
    assert bad.size == 0
    # the pipelined (persistent) mode before the block, and the FP32 path
    hp = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(tail_threshold=4))
    glu.glu_factor(hp, v)
    assert np.array_equal(glu.glu_get_factors(hp), got)
    glu.glu_factor_f32(h, v)
    b = synth.rhs(m.n, 2, 5)
    x, info = glu.glu_solve_refine(h, b, tol=1e-12, maxit=10)
    assert info["converged"] == 1 and backward_error(m.n, m.colptr, m.rowidx, v, b, x) <= BERR_TOL


def test_dense_tail_nonfinite_pivot_reported(glu):
    """A non-finite pivot inside the dense block is reported with its column
    (the numbering of P A P^T), and a good refactorization works afterwards."""
    m = synth.CircuitMatrix(synth.CircuitSpec(16, 20, 900, 15, 0.02, 0.05, "nd"), 3)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    t = glu.glu_get_stats(h)["factor_tail_cols"]
    assert t >= 800
    c = m.n - t // 2                          # a column inside the block
    old = int(m.perm[c])                      # B(c, c) = A(old, old)
    q = m.colptr[old] + int(np.searchsorted(m.rowidx[m.colptr[old]:m.colptr[old + 1]], old))
    assert m.rowidx[q] == old
    v = m.values(8)
    v2 = v.copy()
    v2[q] = np.nan
    with pytest.raises(glu.GluError) as e:
        glu.glu_factor(h, v2)
    assert e.value.code == glu.glu.GLU_ERR_NONFINITE and e.value.column == c
    glu.glu_factor(h, v)
    b = synth.rhs(m.n, 1, 3)
    assert backward_error(m.n, m.colptr, m.rowidx, v, b, glu.glu_solve(h, b)) <= BERR_TOL


@pytest.mark.parametrize("case", ["grid32", "random", "mesh_small", "mesh100x200", "dense900"])
def test_block_factor_parity(glu, case):
    """The supernodal factorization (factor_blocks=1) against the oracle."""
    opts = glu.default_options(factor_blocks=1)
    if case == "grid32":
        m = synth.make("grid32_natural", 0)
        args = (m.n, m.colptr, m.rowidx, m.perm, m.values(1), synth.rhs(m.n, 1, 2))
    elif case == "random":
        cp, ri, v = synth.random_pattern_matrix(150, 0.15, 45)
        perm = np.random.default_rng(5).permutation(150).astype(np.int32)
        args = (150, cp, ri, perm, v, synth.rhs(150, 3, 5))
    elif case == "mesh_small":
        m = synth.CircuitMatrix(synth.CircuitSpec(30, 40, 8, 60, 0.02, 0.05, "nd"), 3)
        args = (m.n, m.colptr, m.rowidx, m.perm, m.values(5), synth.rhs(m.n, 2, 5))
    elif case == "mesh100x200":
        m = synth.make("mesh100x200_nets64", 1)
        args = (m.n, m.colptr, m.rowidx, m.perm, m.values(2001), synth.rhs(m.n, 4, 2001))
    else:
        m = synth.CircuitMatrix(synth.CircuitSpec(16, 20, 900, 15, 0.02, 0.05, "nd"), 3)
        args = (m.n, m.colptr, m.rowidx, m.perm, m.values(8), synth.rhs(m.n, 2, 8))
    h, got, f = run_case(glu, *args, opts=opts)
    # deterministic: the same factors again
    glu.glu_factor(h, args[4])
    assert np.array_equal(glu.glu_get_factors(h), got)
    # the FP32 path through the same schedule, refined to 1e-12
    glu.glu_factor_f32(h, args[4])
    x, info = glu.glu_solve_refine(h, args[5], tol=1e-12, maxit=10)
    assert info["converged"] == 1
    assert backward_error(args[0], args[1], args[2], args[4], args[5], x) <= BERR_TOL


def test_block_factor_mesh400x500_full(glu):
    """The 200k-unknown workload through the supernodal factorization."""
    m = synth.make("mesh400x500_nets64", 1)
    run_case(glu, m.n, m.colptr, m.rowidx, m.perm, m.values(1001), synth.rhs(m.n, 1, 1001),
             opts=glu.default_options(factor_blocks=1), device_inputs=True)
