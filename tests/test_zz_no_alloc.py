"""glu_solve_noalloc: the solve for callers that must not allocate device
memory while running (for example a time-stepping loop whose memory is all
reserved up front, where a cudaMalloc could fail or stall), using the
library's fixed scratch array.

Checked through the C ABI: on two calls in a row it returns glu_solve's
result bit for bit (it runs the same launches with other scratch memory),
for the default dataflow solve and for the per-level one; every result meets
the backward-error bound; at the 200k-unknown workload it matches the CPU
oracle's solution, and a handle of another size reuses the array right
after.  The size limit is checked on the host before anything runs.  This
file is collected last so that a stop at its first failure has already run
every other test; it passes alone in a fresh process and after the others.
"""
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


@pytest.mark.parametrize("solve_mode", [1, 0])
def test_noalloc_matches_solve_twice(glu, solve_mode):
    m = synth.make("mesh100x200_nets64", 1)
    v = m.values(31)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(solve_mode=solve_mode))
    glu.glu_factor(h, torch.from_numpy(v).cuda())
    for call, k in enumerate((4, 3)):
        bh = synth.rhs(m.n, k, 500 + call)
        b = torch.from_numpy(bh).cuda()
        want = glu.glu_solve(h, b).cpu().numpy()
        x = torch.full_like(b, float("nan"))
        glu.glu_solve_noalloc(h, b, x)
        glu.glu_sync(h)
        got = x.cpu().numpy()
        assert np.array_equal(got, want)
        assert backward_error(m.n, m.colptr, m.rowidx, v, bh, got) <= BERR_TOL


def test_noalloc_full_size_against_oracle(glu):
    m = synth.make("mesh400x500_nets64", 1)
    v = m.values(1001)
    bh = synth.rhs(m.n, 2, 1001)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    glu.glu_factor(h, torch.from_numpy(v).cuda())
    x = torch.full((2, m.n), float("nan"), dtype=torch.float64, device="cuda")
    glu.glu_solve_noalloc(h, torch.from_numpy(bh).cuda(), x)
    glu.glu_sync(h)
    got = x.cpu().numpy()
    assert backward_error(m.n, m.colptr, m.rowidx, v, bh, got) <= BERR_TOL
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm, v)
    np.testing.assert_allclose(got, f.solve(bh), rtol=1e-8, atol=1e-12)
    glu.glu_destroy(h)
    # another handle, another size, the same array right after
    g = synth.make("grid32_natural", 0)
    vg = g.values(1)
    hg = glu.glu_analyze(g.n, g.colptr, g.rowidx, g.perm)
    glu.glu_factor(hg, vg)
    bg = synth.rhs(g.n, 1, 7)
    xg = torch.full((1, g.n), float("nan"), dtype=torch.float64, device="cuda")
    glu.glu_solve_noalloc(hg, torch.from_numpy(bg).cuda(), xg)
    glu.glu_sync(hg)
    assert np.array_equal(xg.cpu().numpy(), glu.glu_solve(hg, bg))


def test_noalloc_rejects_oversize_and_host_pointers(glu):
    m = synth.make("mesh100x200_nets64", 1)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    glu.glu_factor(h, m.values(32))
    limit = glu.glu.GLU_NOALLOC_SCRATCH_DOUBLES
    k = limit // (2 * m.n) + 1                 # y and z alone are over the limit
    b = torch.zeros((k, m.n), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(glu.GluError) as e:
        glu.glu_solve_noalloc(h, b, x)
    assert e.value.code == glu.glu.GLU_ERR_TOO_LARGE
    with pytest.raises(glu.GluError) as e:
        glu.glu_solve_noalloc(h, np.zeros(m.n), np.zeros(m.n))
    assert e.value.code == glu.glu.GLU_ERR_INVALID
