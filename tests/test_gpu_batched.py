"""Batched refactorization: B value sets of one pattern in one graph launch,
FP64 (factors against the oracle per set, solves by backward error) and
FP32 + FP64 refinement (every side of every set reaches the FP64 bound)."""
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
    return g


def value_sets(m, B, base=5):
    return np.stack([m.values(100 + b, sigma=0.1, base_seed=base) for b in range(B)])


@pytest.mark.parametrize("name,B", [("small", 40), ("mesh100x200_nets64", 64)])
def test_batched_fp64(glu, name, B):
    if name == "small":
        m = synth.CircuitMatrix(synth.CircuitSpec(30, 40, 8, 60, 0.02, 0.05, "nd"), 8)
    else:
        m = synth.make(name, 1)
    V = value_sets(m, B)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    glu.glu_factor_batched(h, torch.from_numpy(V).cuda())
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm)
    for b in sorted({0, 1, B // 2, B - 1}):
        got = glu.glu_get_factors_batched(h, b)
        bad, _ = factor_mismatches(f.lu_colptr, f.lu_rowidx, got, f.factor(V[b]))
        assert bad.size == 0, (b, bad[:5])
    rhs = np.stack([synth.rhs(m.n, 2, 300 + b) for b in range(B)])       # (B, 2, n)
    x = glu.glu_solve_batched(h, torch.from_numpy(rhs).cuda()).cpu().numpy()
    for b in range(B):
        assert backward_error(m.n, m.colptr, m.rowidx, V[b], rhs[b], x[b]) <= BERR_TOL, b


def test_batched_matches_single(glu):
    m = synth.CircuitMatrix(synth.CircuitSpec(20, 30, 4, 30, 0.02, 0.05, "nd"), 2)
    B = 33
    V = value_sets(m, B)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    glu.glu_factor_batched(h, V)          # host values
    hs = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    for b in (0, 17, 32):
        glu.glu_factor(hs, V[b])
        np.testing.assert_allclose(glu.glu_get_factors_batched(h, b), glu.glu_get_factors(hs),
                                   rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("B", [32, 256])
def test_batched_fp32_refine(glu, B):
    m = synth.make("mesh100x200_nets64", 1)
    V = value_sets(m, B)
    rhs = np.stack([synth.rhs(m.n, 4, 700 + b) for b in range(B)])
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    glu.glu_factor_batched_f32(h, torch.from_numpy(V).cuda())
    x, info = glu.glu_solve_batched_refine(h, torch.from_numpy(rhs).cuda(), tol=1e-12, maxit=20)
    x = x.cpu().numpy()
    assert info["converged"] == 1, info
    worst = 0.0
    for b in range(0, B, max(1, B // 16)):
        e = backward_error(m.n, m.colptr, m.rowidx, V[b], rhs[b], x[b])
        worst = max(worst, e)
    assert worst <= BERR_TOL
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm, V[0])
    xr = f.solve(rhs[0])
    rel = np.abs(x[0] - xr).max() / np.abs(xr).max()
    print(f"B={B}: IR iterations {info['iterations']}, berr {info['berr']:.2e}, set 0 rel err vs FP64 oracle {rel:.2e}")
    assert rel <= 1e-9


def test_batched_errors(glu):
    m = synth.make("grid32_natural", 0)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    with pytest.raises(glu.GluError) as e:
        glu.glu_solve_batched(h, np.zeros((2, 1, m.n)))
    assert e.value.code == glu.glu.GLU_ERR_NOT_FACTORED
    V = np.stack([m.values(1), m.values(2)])
    V[1, :] = 0.0                         # set 1 is all zeros: zero pivot at column 0
    with pytest.raises(glu.GluError) as e:
        glu.glu_factor_batched(h, V)
    assert e.value.code == glu.glu.GLU_ERR_ZERO_PIVOT and e.value.column == 0


@pytest.mark.parametrize("nrhs", [1, 3, 5, 8])
def test_batched_solve_nrhs(glu, nrhs):
    """The batched dataflow solve for right-hand-side counts that exercise
    every path: fewer sides than copies of a dense block item (idle copies
    still publish the block), more (a copy takes sides q and q + 4), and the
    four/two/one-side forms of the row items; 40 sets, so two lane groups and
    padded lanes."""
    m = synth.make("mesh100x200_nets64", 1)
    B = 40
    V = value_sets(m, B, base=9)
    rhs = np.stack([synth.rhs(m.n, nrhs, 900 + b) for b in range(B)])    # (B, nrhs, n)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    glu.glu_factor_batched(h, torch.from_numpy(V).cuda())
    x = glu.glu_solve_batched(h, torch.from_numpy(rhs).cuda()).cpu().numpy()
    for b in range(B):
        assert backward_error(m.n, m.colptr, m.rowidx, V[b], rhs[b], x[b]) <= BERR_TOL, b
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm, V[B - 1])
    xr = f.solve(rhs[B - 1])
    assert np.abs(x[B - 1] - xr).max() <= 1e-10 * np.abs(xr).max()
