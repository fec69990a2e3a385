"""The serving loop's host logic on CPU, against a fake device.

The continuous-batching loop (paper_1908_00204_gb300/serve.py) decides which
pattern runs next, how many same-pattern requests form a batch, which idle
pattern to evict when the device-memory budget is short, and when a slot's
work is finished.  Here torch's CUDA calls and the library are replaced by
fakes that solve each system on the host (scipy) and finish a slot's work
only after it has been polled a few times, so requests overlap.  Checked:
every request gets the solution of its own system; a pattern is never evicted
while its work is in flight; the budget is respected; a batch holds at most
max_batch requests of one pattern; the pattern whose oldest request waited
longest runs first; a request whose factorization meets a zero pivot gets
that status and column (its batch is rerun one request at a time, so the
others still get their solutions).
"""
import contextlib
import sys
import types

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth


class FakeTensor:
    def __init__(self, a):
        self.a = np.asarray(a)

    @property
    def shape(self):
        return self.a.shape

    def to(self, *args, **kw):
        return self

    def cpu(self):
        return self

    def numpy(self):
        return self.a


GLU_OK, GLU_ERR_ZERO_PIVOT = 0, -3


class GluError(RuntimeError):
    def __init__(self, code, where, column=-1):
        super().__init__(where)
        self.code, self.column = code, column


class FakeDevice:
    """Handles, in-flight work and events of the fake GPU.  A value set whose
    first entry is exactly zero stands for one with a zero pivot in column 0:
    the device error word is set and read at the next sync."""

    GLU_OK = GLU_OK
    GluError = GluError

    def __init__(self, bytes_per_entry=8):
        self.bytes_per_entry = bytes_per_entry
        self.live = {}
        self.last = None
        self.analyses = 0
        self.log = []          # (pattern n, batch size) per launch

    # -- the library's calls used by the loop
    def glu_analyze(self, n, colptr, rowidx, perm=None, options=None):
        h = types.SimpleNamespace(n=n, colptr=np.asarray(colptr), rowidx=np.asarray(rowidx),
                                  perm=perm, inflight=False, vals=None, err=GLU_OK)
        self.live[id(h)] = h
        self.analyses += 1
        return h

    def glu_get_stats(self, h):
        nnz = int(h.colptr[-1])
        return {"device_bytes": nnz * self.bytes_per_entry, "nnz_lu": 4 * nnz}

    def glu_destroy(self, h):
        assert not h.inflight, "a pattern was evicted while its work was in flight"
        del self.live[id(h)]

    def glu_set_stream(self, h, stream):
        pass

    def _solve(self, h, vals, b):
        A = sp.csc_matrix((vals, h.rowidx, h.colptr), shape=(h.n, h.n))
        lu = spla.splu(A.tocsc())
        return np.stack([lu.solve(bi) for bi in np.atleast_2d(b)])

    def _launch(self, h, batch):
        assert not h.inflight
        h.inflight = True
        self.last = h
        self.log.append((h.n, batch))

    def glu_sync_status(self, h):
        code, h.err = h.err, GLU_OK
        return code, (0 if code != GLU_OK else -1)

    def glu_factor(self, h, v):
        self._launch(h, 1)
        h.vals = v.a
        if v.a[0] == 0.0:
            h.err = GLU_ERR_ZERO_PIVOT

    def glu_factor_f32(self, h, v):
        self.glu_factor(h, v)

    def glu_solve(self, h, b):
        if h.err != GLU_OK:
            return FakeTensor(np.full(b.a.shape, np.nan))
        return FakeTensor(self._solve(h, h.vals, b.a).reshape(b.a.shape))

    def glu_solve_refine(self, h, b, tol=1e-12, maxit=10):
        if h.err != GLU_OK:     # the library's refinement synchronizes and raises
            code, h.err = h.err, GLU_OK
            raise GluError(code, "glu_solve_refine", 0)
        return self.glu_solve(h, b), {"iterations": 1, "converged": 1}

    def glu_factor_batched(self, h, V):
        self._launch(h, V.a.shape[0])
        h.vals = V.a
        if np.any(V.a[:, 0] == 0.0):
            h.err = GLU_ERR_ZERO_PIVOT

    def glu_factor_batched_f32(self, h, V):
        self.glu_factor_batched(h, V)

    def glu_solve_batched(self, h, B):
        if h.err != GLU_OK:
            return FakeTensor(np.full(B.a.shape, np.nan))
        return FakeTensor(np.stack([self._solve(h, h.vals[i], B.a[i]) for i in range(B.a.shape[0])]))

    def glu_solve_batched_refine(self, h, B, tol=1e-12, maxit=10):
        if h.err != GLU_OK:
            code, h.err = h.err, GLU_OK
            raise GluError(code, "glu_solve_batched_refine", 0)
        return self.glu_solve_batched(h, B), {"iterations": 1, "converged": 1}


def fake_torch(dev, polls=3):
    class Event:
        def __init__(self):
            self.h, self.left = None, polls

        def record(self, stream):
            self.h = dev.last

        def query(self):
            self.left -= 1
            if self.left > 0:
                return False
            self.h.inflight = False
            return True

    cuda = types.SimpleNamespace(Stream=lambda device=None: object(), Event=Event,
                                 stream=lambda s: contextlib.nullcontext())
    return types.SimpleNamespace(cuda=cuda, device=lambda *a: "fake", from_numpy=FakeTensor)


@pytest.fixture
def server(monkeypatch):
    from paper_1908_00204_gb300 import serve
    dev = FakeDevice()
    monkeypatch.setitem(sys.modules, "torch", fake_torch(dev))
    monkeypatch.setattr(serve, "_glu", dev)

    def make(**kw):
        srv = serve.Server(**kw)
        return srv, dev
    return make


def patterns():
    return {f"p{k}": synth.CircuitMatrix(synth.CircuitSpec(r, c, 4, nf, 0.02, 0.05, "nd"), 20 + k)
            for k, (r, c, nf) in enumerate([(8, 10, 6), (10, 12, 8), (12, 14, 10)])}


def requests(mats, n_req, seed=0):
    from paper_1908_00204_gb300.serve import Request
    rng = np.random.default_rng(seed)
    keys = sorted(mats)
    out = []
    for i in range(n_req):
        key = keys[int(rng.integers(len(keys)))]
        m = mats[key]
        out.append(Request(i, key, m.values(700 + i, sigma=0.1, base_seed=2),
                           synth.rhs(m.n, int(rng.integers(1, 4)), 800 + i)))
    return out


def check_results(mats, done, n_req, failed=()):
    assert sorted(r.rid for r in done) == list(range(n_req))
    for r in done:
        if r.rid in failed:
            assert r.status == GLU_ERR_ZERO_PIVOT and r.error_column == 0 and r.x is None
            continue
        assert r.status == GLU_OK and r.error_column == -1
        m = mats[r.key]
        A = sp.csc_matrix((r.values, m.rowidx, m.colptr), shape=(m.n, m.n))
        x = np.atleast_2d(r.x)
        assert x.shape == np.atleast_2d(r.b).shape
        for xi, bi in zip(x, np.atleast_2d(r.b)):
            assert np.abs(A @ xi - bi).max() <= 1e-9 * (np.abs(bi).max() + 1.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_every_request_gets_its_own_solution(server, precision):
    mats = patterns()
    srv, dev = server(device_budget_bytes=1e12, max_batch=8, slots=3, precision=precision)
    for k, m in mats.items():
        srv.register(k, m.n, m.colptr, m.rowidx, m.perm)
    reqs = requests(mats, 60)
    for r in reqs[:30]:
        srv.submit(r)
    for _ in range(5):             # some work in flight, then the rest arrives
        srv.step()
    for r in reqs[30:]:
        srv.submit(r)
    srv.drain()
    check_results(mats, srv.done, 60)
    assert dev.analyses == 3 and srv.evictions == 0        # every pattern analysed once
    assert all(b <= 8 for b in srv.batch_sizes)
    assert any(b > 1 for b in srv.batch_sizes)             # same-pattern requests were batched
    assert all(b in (1, 32) for _, b in dev.log)           # batches padded to the 32-set lane groups


def test_budget_evicts_idle_patterns_only(server):
    mats = patterns()
    dev_bytes = {k: int(m.colptr[-1]) * 8 for k, m in mats.items()}
    # room for the two largest patterns' analyses, not for all three (and no
    # batch buffers: batches shrink to single requests)
    big = sorted(dev_bytes.values())
    budget = big[-1] + big[-2] + big[0] // 2
    srv, dev = server(device_budget_bytes=budget, max_batch=4, slots=2)
    for k, m in mats.items():
        srv.register(k, m.n, m.colptr, m.rowidx, m.perm)
    reqs = requests(mats, 40, seed=3)
    for r in reqs:
        srv.submit(r)
        srv.step()
        assert srv._bytes_in_use() <= budget
    srv.drain()
    check_results(mats, srv.done, 40)
    assert srv.evictions > 0 and dev.analyses > 3            # patterns came back after eviction
    assert len(dev.live) == len(srv.resident) <= 2
    assert all(b == 1 for b in srv.batch_sizes)


def test_oldest_waiting_pattern_runs_first(server):
    mats = patterns()
    srv, dev = server(device_budget_bytes=1e12, max_batch=16, slots=1)
    for k, m in mats.items():
        srv.register(k, m.n, m.colptr, m.rowidx, m.perm)
    from paper_1908_00204_gb300.serve import Request
    order = ["p2", "p0", "p1", "p0"]
    for i, key in enumerate(order):
        m = mats[key]
        srv.submit(Request(i, key, m.values(i), synth.rhs(m.n, 1, i)))
    srv.drain()
    # one slot: p2 first, then p0 (its oldest request is older than p1's) as a batch of two, then p1
    assert [n for n, _ in dev.log] == [mats["p2"].n, mats["p0"].n, mats["p1"].n]
    assert srv.batch_sizes == [1, 2, 1]
    check_results(mats, srv.done, 4)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_zero_pivot_reaches_its_request(server, precision):
    mats = patterns()
    srv, dev = server(device_budget_bytes=1e12, max_batch=8, slots=2, precision=precision)
    for k, m in mats.items():
        srv.register(k, m.n, m.colptr, m.rowidx, m.perm)
    reqs = requests(mats, 24, seed=5)
    bad = {reqs[3].rid, reqs[17].rid}
    for r in reqs:
        if r.rid in bad:
            r.values = r.values.copy()
            r.values[0] = 0.0
        srv.submit(r)
    srv.drain()
    check_results(mats, srv.done, 24, failed=bad)
    assert any(b > 1 for b in srv.batch_sizes)  # batches ran, and the failed ones again one by one


def test_replicas_run_one_pattern_concurrently(server):
    """With replicas, requests of one pattern below the batching threshold run
    at the same time on separate handles (never two launches on one busy
    handle), within the budget; results are each request's own."""
    mats = patterns()
    srv, dev = server(device_budget_bytes=1e12, max_batch=8, slots=4, replicas=3, batch_min=100)
    key = "p1"
    m = mats[key]
    srv.register(key, m.n, m.colptr, m.rowidx, m.perm)
    from paper_1908_00204_gb300.serve import Request
    reqs = [Request(i, key, m.values(900 + i), synth.rhs(m.n, 2, 950 + i)) for i in range(9)]
    for r in reqs:
        srv.submit(r)
    srv.step()
    assert sum(h.inflight for h in dev.live.values()) == 3          # three handles busy at once
    srv.drain()
    assert dev.analyses == 3 and len(srv.resident[key].hs) == 3
    assert all(b == 1 for b in srv.batch_sizes)
    check_results({key: m}, srv.done, 9)


def test_prepare_makes_replicas_and_keeps_no_results(server):
    mats = patterns()
    srv, dev = server(device_budget_bytes=1e12, max_batch=16, slots=3, replicas=2, batch_min=4)
    key = "p0"
    m = mats[key]
    srv.register(key, m.n, m.colptr, m.rowidx, m.perm)
    assert srv.prepare(key, m.values(1), synth.rhs(m.n, 1, 1))
    assert len(srv.resident[key].hs) == 2 and dev.analyses == 2
    assert srv.done == [] and not any(srv.queues.values())
    assert 4 in srv.batch_sizes                       # a batch ran (its graph exists)
