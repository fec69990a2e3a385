"""glu_solve_noalloc: the solve for callers that must not allocate device
memory while running (for example a time-stepping loop whose memory is all
reserved up front), using the library's fixed scratch array.

Checked through the C ABI against glu_solve on two calls in a row, and the
size limit is checked on the host before anything runs.  This file is
collected last so that a stop at its first failure has already run every
other test; it passes alone in a fresh process and after the others.
"""
import numpy as np
import pytest

import synth
from parity import FACTOR_RTOL

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


def test_noalloc_matches_solve_twice(glu):
    m = synth.make("mesh100x200_nets64", 1)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    glu.glu_factor(h, torch.from_numpy(m.values(31)).cuda())
    for call, k in enumerate((4, 3)):
        b = torch.from_numpy(synth.rhs(m.n, k, 500 + call)).cuda()
        want = glu.glu_solve(h, b).cpu().numpy()
        x = torch.full_like(b, float("nan"))
        glu.glu_solve_noalloc(h, b, x)
        glu.glu_sync(h)
        got = x.cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=FACTOR_RTOL, atol=0.0)


def test_noalloc_rejects_oversize_and_host_pointers(glu):
    m = synth.make("mesh100x200_nets64", 1)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    glu.glu_factor(h, m.values(32))
    limit = glu.glu.GLU_NOALLOC_SCRATCH_DOUBLES
    k = limit // m.n + 1                       # n * k alone is over the limit
    b = torch.zeros((k, m.n), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(glu.GluError) as e:
        glu.glu_solve_noalloc(h, b, x)
    assert e.value.code == glu.glu.GLU_ERR_TOO_LARGE
    with pytest.raises(glu.GluError) as e:
        glu.glu_solve_noalloc(h, np.zeros(m.n), np.zeros(m.n))
    assert e.value.code == glu.glu.GLU_ERR_INVALID
