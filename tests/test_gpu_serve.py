"""Serving loop: requests for several patterns with new values and 1-4
right-hand sides, submitted while others run.  Every result meets the FP64
backward-error bound and equals the result of the same request served alone:
FP64 within 1e-10 relative (the batched and single kernels differ only in
rounding order); FP32 + refinement, refined to a backward error of 1e-14 in
both runs, within 1e-8 relative (two solutions with backward error <= 1e-14
differ by at most about cond(A) * 1e-14, and cond(A) < 1e5 here)."""
import numpy as np
import pytest

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


def mixed_requests(n_req=60, seed=0):
    from paper_1908_00204_gb300.serve import Request
    mats = {f"p{k}": synth.CircuitMatrix(synth.CircuitSpec(r, c, 8, nf, 0.02, 0.05, "nd"), 10 + k)
            for k, (r, c, nf) in enumerate([(20, 25, 10), (30, 40, 20), (40, 50, 30)])}
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n_req):
        key = f"p{rng.integers(3)}"
        m = mats[key]
        k = int(rng.integers(1, 5))
        reqs.append(Request(i, key, m.values(5000 + i, sigma=0.1, base_seed=3), synth.rhs(m.n, k, 9000 + i)))
    return mats, reqs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mix_equals_alone(glu, precision):
    from paper_1908_00204_gb300.serve import Request, Server
    mats, reqs = mixed_requests()
    tol = 1e-14 if precision == "fp32" else 1e-12
    rtol = 1e-8 if precision == "fp32" else 1e-10
    srv = Server(device_budget_bytes=8e9, max_batch=16, slots=3, precision=precision, tol=tol, maxit=20)
    for key, m in mats.items():
        srv.register(key, m.n, m.colptr, m.rowidx, m.perm)
    arrivals = np.cumsum(np.random.default_rng(1).exponential(1 / 2000.0, len(reqs)))
    srv.run(list(arrivals), lambda i: reqs[i])
    assert len(srv.done) == len(reqs) and srv.batches < len(reqs)   # some batching happened
    alone = Server(device_budget_bytes=8e9, max_batch=1, slots=1, precision=precision, tol=tol, maxit=20)
    for key, m in mats.items():
        alone.register(key, m.n, m.colptr, m.rowidx, m.perm)
    for r in reqs:
        m = mats[r.key]
        assert backward_error(m.n, m.colptr, m.rowidx, r.values, r.b, r.x) <= BERR_TOL
        single = Request(r.rid, r.key, r.values, r.b)
        alone.submit(single)
        alone.drain()
        np.testing.assert_allclose(r.x, single.x, rtol=rtol, atol=1e-13)
    lat = srv.latencies()
    assert lat.size == len(reqs) and np.all(lat > 0)


def test_budget_evicts_idle_patterns(glu):
    from paper_1908_00204_gb300.serve import Server
    mats, reqs = mixed_requests(12, seed=4)
    # a budget that holds roughly one pattern forces evictions between patterns
    one = max(glu.glu_get_stats(glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm))["device_bytes"]
              for m in mats.values())
    srv = Server(device_budget_bytes=1.2 * one, max_batch=1, slots=1)
    for key, m in mats.items():
        srv.register(key, m.n, m.colptr, m.rowidx, m.perm)
    for r in reqs:
        srv.submit(r)
    srv.drain()
    assert len(srv.done) == len(reqs)
    assert srv.evictions > 0 and srv._bytes_in_use() <= srv.budget


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_zero_pivot_reaches_its_request(glu, precision):
    """A request whose values make the first pivot exactly zero comes back with
    GLU_ERR_ZERO_PIVOT and column 0 (read from the device error word, also when
    it ran inside a batch); every other request still gets its solution."""
    from paper_1908_00204_gb300.serve import Server
    mats, reqs = mixed_requests(24, seed=6)
    bad = {3, 11}
    for i in bad:
        m = mats[reqs[i].key]
        p0 = int(m.perm[0])          # B(0, 0) = A(perm[0], perm[0]): the first pivot
        cb, ce = int(m.colptr[p0]), int(m.colptr[p0 + 1])
        v = reqs[i].values.copy()
        v[cb + int(np.searchsorted(m.rowidx[cb:ce], p0))] = 0.0
        reqs[i].values = v
    tol = 1e-14 if precision == "fp32" else 1e-12
    srv = Server(device_budget_bytes=8e9, max_batch=16, slots=2, precision=precision, tol=tol, maxit=5)
    for key, m in mats.items():
        srv.register(key, m.n, m.colptr, m.rowidx, m.perm)
    for r in reqs:
        srv.submit(r)
    srv.drain()
    assert sorted(r.rid for r in srv.done) == list(range(len(reqs)))
    for r in srv.done:
        if r.rid in bad:
            assert r.status == glu.glu.GLU_ERR_ZERO_PIVOT and r.error_column == 0 and r.x is None
        else:
            m = mats[r.key]
            assert r.status == 0 and r.error_column == -1
            assert backward_error(m.n, m.colptr, m.rowidx, r.values, r.b, r.x) <= BERR_TOL
