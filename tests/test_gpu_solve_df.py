"""Dataflow solve (with and without the one-block dense tail and the
one-warp dense diagonal blocks): the same results as the level-by-level
solve up to rounding order, and a bounded wait
that runs out (a row flag that nothing sets) returns GLU_ERR_TIMEOUT with the
context still usable.  No GPU fault is involved: the missing flag is
a host-chosen test hook and every device wait has a time limit."""
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


@pytest.mark.parametrize("name,nrhs", [("grid32_natural", 1), ("mesh100x200_nets64", 3),
                                       ("mesh400x500_nets64", 2)])
def test_dataflow_equals_level_solve(glu, name, nrhs):
    m = synth.make(name, 1)
    v = m.values(9)
    b = synth.rhs(m.n, nrhs, 9)
    hs = {}
    for key, opts in (("levels", dict(solve_mode=0)), ("df", dict(solve_mode=1, solve_tail=0, solve_blocks=0)),
                      ("df+tail", dict(solve_mode=1, solve_tail=1, solve_blocks=0)),
                      ("df+blocks+tail", dict(solve_mode=1, solve_tail=1, solve_blocks=1))):
        h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(**opts))
        glu.glu_factor(h, torch.from_numpy(v).cuda())
        hs[key] = glu.glu_solve(h, torch.from_numpy(b).cuda()).cpu().numpy()
        glu.glu_sync(h)
        if key == "df+tail" and name != "grid32_natural":
            assert glu.glu_get_stats(h)["tail_rows"] >= 32
    assert np.array_equal(hs["levels"], hs["df"])          # same per-row summation order
    np.testing.assert_allclose(hs["df+tail"], hs["df"], rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(hs["df+blocks+tail"], hs["df"], rtol=1e-10, atol=1e-14)
    for x in hs.values():
        assert backward_error(m.n, m.colptr, m.rowidx, v, b, x) <= BERR_TOL


def test_dataflow_repeated_and_host_buffers(glu):
    m = synth.CircuitMatrix(synth.CircuitSpec(30, 40, 8, 60, 0.02, 0.05, "nd"), 13)
    v = m.values(2)
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm, v)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    glu.glu_factor(h, v)
    for k in (1, 5, 1):
        b = synth.rhs(m.n, k, 40 + k)
        x = glu.glu_solve(h, b)
        np.testing.assert_allclose(x, f.solve(b), rtol=1e-9, atol=1e-12)


def test_wait_timeout_is_reported_and_context_survives(glu):
    m = synth.make("mesh100x200_nets64", 1)
    v = m.values(3)
    b = torch.from_numpy(synth.rhs(m.n, 1, 3)).cuda()
    bad = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm,
                          glu.default_options(fault_row=m.n // 2, spin_limit_us=20000))
    glu.glu_factor(bad, torch.from_numpy(v).cuda())
    glu.glu_sync(bad)
    x = torch.empty_like(b)
    glu.glu_solve(bad, b, x)
    with pytest.raises(glu.GluError) as e:
        glu.glu_sync(bad)
    assert e.value.code == glu.glu.GLU_ERR_TIMEOUT
    # the context still works: a fresh handle solves correctly
    good = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    glu.glu_factor(good, torch.from_numpy(v).cuda())
    xg = glu.glu_solve(good, b).cpu().numpy()
    glu.glu_sync(good)
    assert backward_error(m.n, m.colptr, m.rowidx, v, b.cpu().numpy(), xg) <= BERR_TOL


@pytest.mark.parametrize("seed", range(8))
def test_dataflow_unsymmetric_patterns(glu, seed):
    """Unsymmetric patterns: a backward row can be ready while forward rows
    still read the forward value of that row."""
    n = 20 + 23 * seed
    cp, ri, v = synth.random_pattern_matrix(n, 0.12, 900 + seed)
    perm = np.random.default_rng(seed).permutation(n).astype(np.int32)
    f = oracle.Factorization(n, cp, ri, perm, v)
    b = synth.rhs(n, 2, seed)
    h = glu.glu_analyze(n, cp, ri, perm)
    glu.glu_factor(h, v)
    x = glu.glu_solve(h, b)
    np.testing.assert_allclose(x, f.solve(b), rtol=1e-9, atol=1e-12)
