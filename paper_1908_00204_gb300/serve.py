"""Continuous-batching request loop for refactor + solve requests.

Each request carries a sparsity pattern (by key), new values and 1-8
right-hand sides.  The loop:

* analyses each pattern once (glu_analyze) and keeps the handle -- the
  pattern's fill, dependencies, levels and schedule -- resident on the device
  (the paper's flow repeats only the numeric part for a fixed pattern,
  Section III), evicting the least recently used idle pattern when the
  device-memory budget would be exceeded;
* keeps up to ``replicas`` handles per pattern (each its own numeric
  workspace, the budget permitting), so several requests of one pattern can
  run at once through the single-matrix path;
* once ``batch_min`` or more requests of one pattern wait, groups them into a
  batch (up to ``max_batch``) and runs it as one batched refactorization +
  solve (glu_factor_batched / glu_solve_batched, or the FP32 +
  FP64-refinement pair) on the pattern's first handle; the batched kernels
  run 32 value sets per lane group whatever the batch, so a batch is padded
  to a multiple of 32 with copies of its last request (one captured graph per
  padded size, the padding's results discarded);
* runs work of different patterns and handles at the same time on separate
  CUDA streams ("slots"); a request that arrives while others run is
  admitted as soon as a slot and the memory budget allow it;
* records each request's latency from submission to result-ready, and its
  status: a zero or non-finite pivot (or another device error) reaches the
  request as ``status`` / ``error_column`` instead of a solution.  A batch
  shares one device error word, so a failed batch is run again one request
  at a time and each request gets its own status.

The host side is plain Python (argument marshalling and bookkeeping); every
numeric step runs in the CUDA library.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Dict, List, Optional

import numpy as np

from . import glu as _glu


@dataclasses.dataclass
class Pattern:
    key: str
    n: int
    colptr: np.ndarray
    rowidx: np.ndarray
    perm: Optional[np.ndarray]


@dataclasses.dataclass
class Request:
    rid: int
    key: str
    values: np.ndarray          # nnz(A) doubles
    b: np.ndarray               # (nrhs, n)
    t_submit: float = 0.0
    t_done: float = 0.0
    x: Optional[np.ndarray] = None
    info: Optional[dict] = None
    status: int = 0             # GLU_OK, or the GLU_ERR_* code of its factorization / solve
    error_column: int = -1      # the failing pivot's column for GLU_ERR_ZERO_PIVOT / NONFINITE
    solo: bool = False          # run alone (set when its batch failed)


class _Resident:
    """A pattern's handles on the device (replicas of one analysis, each with
    its own numeric workspace), which of them are running, and its last use.
    Batches run on the first handle."""

    def __init__(self, pat: Pattern, handle):
        self.pat = pat
        self.hs = [handle]
        self.busy_h = [False]
        self.last_use = time.perf_counter()
        st = _glu.glu_get_stats(handle)
        self.one_bytes = int(st["device_bytes"])
        self.nnz_lu = int(st["nnz_lu"])
        self.batch_bytes = 0

    @property
    def h(self):
        return self.hs[0]

    @property
    def busy(self) -> bool:
        return any(self.busy_h)

    @property
    def base_bytes(self) -> int:
        return self.one_bytes * len(self.hs)

    def free_handle(self) -> int:
        return next((i for i, b in enumerate(self.busy_h) if not b), -1)


class _Slot:
    def __init__(self, torch, device):
        self.stream = torch.cuda.Stream(device=device)
        self.event = None
        self.res: Optional[_Resident] = None
        self.hi = 0             # which of the pattern's handles
        self.reqs: List[Request] = []
        self.out = None
        self.info = None
        self.error = None       # (code, column) raised while enqueueing
        self.pinned = {}        # page-locked staging buffers of this slot, by use


class Server:
    """Continuous batching over patterns; see the module docstring."""

    def __init__(self, device_budget_bytes: float = 60e9, max_batch: int = 64, slots: int = 4,
                 precision: str = "fp64", tol: float = 1e-12, maxit: int = 10, device: int = 0,
                 replicas: int = 1, batch_min: int = 2):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.budget = int(device_budget_bytes)
        self.max_batch = max_batch
        self.replicas = max(1, replicas)
        self.batch_min = max(2, batch_min)
        self.precision = precision
        self.tol = tol
        self.maxit = maxit
        self.patterns: Dict[str, Pattern] = {}
        self.resident: "collections.OrderedDict[str, _Resident]" = collections.OrderedDict()
        self.queues: Dict[str, collections.deque] = collections.defaultdict(collections.deque)
        self.slots = [_Slot(torch, self.device) for _ in range(slots)]
        self.done: List[Request] = []
        self.analyses = 0
        self.evictions = 0
        self.batches = 0
        self.batch_sizes: List[int] = []     # requests per launch, in launch order

    # ------------------------------------------------------------ patterns
    def register(self, key: str, n: int, colptr, rowidx, perm=None) -> None:
        self.patterns[key] = Pattern(key, n, np.asarray(colptr, np.int32), np.asarray(rowidx, np.int32),
                                     None if perm is None else np.asarray(perm, np.int32))

    def _bytes_in_use(self) -> int:
        return sum(r.base_bytes + r.batch_bytes for r in self.resident.values())

    def _batch_bytes(self, res: _Resident, batch: int, nrhs: int) -> int:
        s = (batch + 31) // 32 * 32
        per_value = 8 if self.precision == "fp64" else 4
        a = int(res.pat.colptr[-1])
        return int(res.nnz_lu * s * per_value + 3 * a * s * 8 + 8 * res.pat.n * nrhs * s * 8)

    def _make_room(self, need: int, keep: str) -> bool:
        while self._bytes_in_use() + need > self.budget:
            victim = next((k for k, r in self.resident.items() if not r.busy and k != keep), None)
            if victim is None:
                return False
            for h in self.resident.pop(victim).hs:
                _glu.glu_destroy(h)
            self.evictions += 1
        return True

    def _add_replica(self, res: _Resident) -> int:
        """Another handle for the pattern when the budget leaves room for it
        without evicting anything; its index, or -1."""
        if len(res.hs) >= self.replicas or self._bytes_in_use() + res.one_bytes > self.budget:
            return -1
        pat = res.pat
        res.hs.append(_glu.glu_analyze(pat.n, pat.colptr, pat.rowidx, pat.perm))
        res.busy_h.append(False)
        self.analyses += 1
        return len(res.hs) - 1

    def _resident(self, key: str) -> Optional[_Resident]:
        if key in self.resident:
            self.resident.move_to_end(key)
            return self.resident[key]
        pat = self.patterns[key]
        h = _glu.glu_analyze(pat.n, pat.colptr, pat.rowidx, pat.perm)
        self.analyses += 1
        res = _Resident(pat, h)
        if not self._make_room(res.base_bytes, key):
            _glu.glu_destroy(h)
            return None
        self.resident[key] = res
        return res

    def prepare(self, key: str, values: np.ndarray, b: np.ndarray) -> bool:
        """Make a pattern resident before traffic: its analysis, every
        replica the budget allows, and one refactorization + solve on each
        handle and one padded batch on the first (so the captured graphs
        exist); a server keeps no result of these.  False if the budget has
        no room for the pattern."""
        res = self._resident(key)
        if res is None:
            return False
        while self._add_replica(res) >= 0:
            pass
        warm = [Request(-1 - i, key, values, b) for i in range(max(len(res.hs), self.batch_min))]
        q = self.queues[key]
        for r in warm[: len(res.hs)]:
            q.append(r)
        self.drain()
        for r in warm:
            q.append(r)
        self.drain()
        self.done = [r for r in self.done if r.rid >= 0]
        return True

    # ------------------------------------------------------------ requests
    def submit(self, req: Request) -> None:
        req.t_submit = time.perf_counter()
        self.queues[req.key].append(req)

    def _launch(self, slot: _Slot) -> bool:
        # the pattern whose oldest waiting request is oldest, among those with
        # a handle free (or room for another one)
        best = None
        for key, q in self.queues.items():
            if not q:
                continue
            res = self.resident.get(key)
            if res is not None and res.free_handle() < 0 and len(res.hs) >= self.replicas:
                continue
            if best is None or q[0].t_submit < self.queues[best][0].t_submit:
                best = key
        if best is None:
            return False
        q = self.queues[best]
        res = self._resident(best)
        if res is None:
            return False
        take = 1 if q[0].solo else min(len(q), self.max_batch)
        if take < self.batch_min or res.busy_h[0]:
            take = 1                        # too few for a batch, or the batch handle is running
        hi = 0 if take > 1 else res.free_handle()
        if hi < 0:
            hi = self._add_replica(res)
            if hi < 0:
                return False
        nrhs = max(r.b.shape[0] for r in list(q)[:take])
        # a batch never evicts other patterns: it shrinks to what the budget
        # leaves (batch buffers stay with the pattern until it is evicted)
        free = self.budget - self._bytes_in_use()
        while take > 1 and self._batch_bytes(res, take, nrhs) - res.batch_bytes > free:
            take //= 2
        reqs = [q.popleft() for _ in range(take)]
        if any(r.solo for r in reqs[1:]):
            for r in reversed(reqs[1:]):
                q.appendleft(r)
            reqs, take = reqs[:1], 1
        nrhs = max(r.b.shape[0] for r in reqs)
        torch = self.torch
        res.busy_h[hi] = True
        res.last_use = time.perf_counter()
        slot.res, slot.hi, slot.reqs = res, hi, reqs
        h = res.hs[hi]
        slot.error = None
        with torch.cuda.stream(slot.stream):
            _glu.glu_set_stream(h, slot.stream)
            try:
                self._enqueue(slot, res, reqs, nrhs)
            except _glu.GluError as e:
                slot.error = (e.code, e.column)
                slot.out = None
            slot.event = torch.cuda.Event()
            slot.event.record(slot.stream)
        self.batches += 1
        self.batch_sizes.append(take)
        return True

    def _staged(self, slot: _Slot, name: str, shape):
        """A host buffer of `shape` doubles for one copy to the device:
        page-locked and kept by the slot (grown when too small), so the copy
        runs asynchronously on the slot's stream; reused only once the slot's
        work has finished.  Returns its numpy view and its tensor."""
        torch = self.torch
        count = int(np.prod(shape))
        if not hasattr(torch, "empty"):          # a host-only stand-in for torch
            a = np.empty(shape)
            return a, torch.from_numpy(a)
        buf = slot.pinned.get(name)
        if buf is None or buf.numel() < count:
            buf = torch.empty(max(count, 1), dtype=torch.float64, pin_memory=True)
            slot.pinned[name] = buf
        t = buf[:count].view(*shape)
        return t.numpy(), t

    def _enqueue(self, slot: _Slot, res: _Resident, reqs: List[Request], nrhs: int) -> None:
        """The batch's factorization and solve, on the slot's stream."""
        torch = self.torch
        h = res.hs[slot.hi]
        take = len(reqs)
        if take == 1:
            r = reqs[0]
            va, vt = self._staged(slot, "v", r.values.shape)
            va[...] = r.values
            ba, bt = self._staged(slot, "b", r.b.shape)
            ba[...] = r.b
            v = vt.to(self.device, non_blocking=True)
            bb = bt.to(self.device, non_blocking=True)
            if self.precision == "fp64":
                _glu.glu_factor(h, v)
                x = _glu.glu_solve(h, bb)
                slot.info = None
            else:
                _glu.glu_factor_f32(h, v)
                x, slot.info = _glu.glu_solve_refine(h, bb, tol=self.tol, maxit=self.maxit)
            slot.out = x
        else:
            # padded to the batched kernels' 32-set lane groups with copies of
            # the last request (their results are discarded)
            S = (take + 31) // 32 * 32
            res.batch_bytes = max(res.batch_bytes, self._batch_bytes(res, S, nrhs))
            V, Vt = self._staged(slot, "V", (S, reqs[0].values.size))
            Bt, Btt = self._staged(slot, "B", (S, nrhs, res.pat.n))
            for i in range(S):
                r = reqs[min(i, take - 1)]
                V[i] = r.values
                Bt[i, : r.b.shape[0]] = r.b
                Bt[i, r.b.shape[0]:] = 0.0
            Vd = Vt.to(self.device, non_blocking=True)
            Bd = Btt.to(self.device, non_blocking=True)
            if self.precision == "fp64":
                _glu.glu_factor_batched(h, Vd)
                x = _glu.glu_solve_batched(h, Bd)
                slot.info = None
            else:
                _glu.glu_factor_batched_f32(h, Vd)
                x, slot.info = _glu.glu_solve_batched_refine(h, Bd, tol=self.tol, maxit=self.maxit)
            slot.out = x

    def _finish(self, slot: _Slot) -> None:
        # the device error word of the handle: pivots of the factorization,
        # bounded waits of the solve (device inputs leave it unread until here)
        code, col = slot.error if slot.error is not None else _glu.glu_sync_status(slot.res.hs[slot.hi])
        if code != _glu.GLU_OK and len(slot.reqs) > 1:
            q = self.queues[slot.res.pat.key]
            for r in reversed(slot.reqs):
                r.solo = True
                q.appendleft(r)
            self._release(slot)
            return
        x = slot.out.cpu().numpy() if code == _glu.GLU_OK else None
        now = time.perf_counter()
        for i, r in enumerate(slot.reqs):
            if x is not None:
                r.x = x if len(slot.reqs) == 1 else x[i, : r.b.shape[0]].copy()
            r.status, r.error_column = code, (col if code != _glu.GLU_OK else -1)
            r.info = slot.info
            r.t_done = now
            self.done.append(r)
        self._release(slot)

    def _release(self, slot: _Slot) -> None:
        slot.res.busy_h[slot.hi] = False
        slot.res = None
        slot.reqs = []
        slot.event = None
        slot.out = None

    def step(self) -> bool:
        """One pass: retire finished slots, fill free ones.  True if anything ran."""
        active = False
        for slot in self.slots:
            if slot.event is not None:
                if slot.event.query():
                    self._finish(slot)
                else:
                    active = True
        for slot in self.slots:
            if slot.event is None and self._launch(slot):
                active = True
        return active

    def drain(self) -> None:
        while self.step() or any(self.queues.values()):
            pass

    def run(self, arrivals: List[float], make_request: Callable[[int], Request]) -> None:
        """Replay arrival times (seconds from now): requests are submitted at
        their time while the loop keeps slots busy.  A request's latency
        counts from its scheduled arrival, so time it waited for the loop to
        notice it is included."""
        t0 = time.perf_counter()
        i = 0
        while i < len(arrivals) or self.step() or any(self.queues.values()):
            now = time.perf_counter() - t0
            while i < len(arrivals) and arrivals[i] <= now:
                req = make_request(i)
                self.submit(req)
                req.t_submit = t0 + arrivals[i]
                i += 1
            self.step()

    # ------------------------------------------------------------ reporting
    def latencies(self, skip: int = 0) -> np.ndarray:
        reqs = sorted(self.done, key=lambda r: r.rid)[skip:]
        return np.array([r.t_done - r.t_submit for r in reqs])
