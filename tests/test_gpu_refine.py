"""FP32 factorization + FP64 iterative refinement: every result reaches the
FP64 backward-error bound, and its error against the FP64 oracle is stated
(and bounded) per case."""
import numpy as np
import pytest

import oracle
import synth
from parity import BERR_TOL, backward_error

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


CASES = [("grid32_natural", 1), ("mesh100x200_nets64", 4), ("mesh400x500_nets64", 1)]


@pytest.mark.parametrize("name,nrhs", CASES)
def test_fp32_factor_fp64_refinement(glu, name, nrhs):
    m = synth.make(name, 1)
    v = m.values(1001)
    b = synth.rhs(m.n, nrhs, 77)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    glu.glu_factor_f32(h, torch.from_numpy(v).cuda())
    x, info = glu.glu_solve_refine(h, torch.from_numpy(b).cuda(), tol=1e-12, maxit=20)
    x = x.cpu().numpy()
    assert info["converged"] == 1, info
    berr = backward_error(m.n, m.colptr, m.rowidx, v, b, x)
    assert berr <= BERR_TOL, (berr, info)
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm, v)
    xr = f.solve(b)
    rel = np.abs(x - xr).max() / np.abs(xr).max()
    print(f"{name}: IR iterations {info['iterations']}, berr {berr:.2e}, max rel err vs FP64 oracle {rel:.2e}")
    assert rel <= 1e-9


def test_fp32_factor_close_to_oracle(glu):
    m = synth.CircuitMatrix(synth.CircuitSpec(30, 40, 8, 60, 0.02, 0.05, "nd"), 17)
    v = m.values(5)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    glu.glu_factor_f32(h, v)
    x, info = glu.glu_solve_refine(h, synth.rhs(m.n, 2, 5), maxit=0)   # one FP32 solve, no correction
    # a single FP32 solve is accurate to FP32 level, not FP64
    assert 1e-12 < info["berr"] < 1e-5 and info["iterations"] == 0


def test_refine_host_buffers_and_not_factored(glu):
    m = synth.make("grid32_natural", 0)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    with pytest.raises(glu.GluError) as e:
        glu.glu_solve_refine(h, np.zeros(m.n))
    assert e.value.code == glu.glu.GLU_ERR_NOT_FACTORED
    v = m.values(2)
    glu.glu_factor_f32(h, v)
    b = synth.rhs(m.n, 3, 1)
    x, info = glu.glu_solve_refine(h, b)
    assert info["converged"] == 1
    assert backward_error(m.n, m.colptr, m.rowidx, v, b, x) <= BERR_TOL
