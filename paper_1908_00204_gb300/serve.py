"""Continuous-batching request loop for refactor + solve requests.

Each request carries a sparsity pattern (by key), new values and 1-8
right-hand sides.  The loop:

* analyses each pattern once (glu_analyze) and keeps the handle -- the
  pattern's fill, dependencies, levels and schedule -- resident on the device
  (the paper's flow repeats only the numeric part for a fixed pattern,
  Section III), evicting the least recently used idle pattern when the
  device-memory budget would be exceeded;
* groups waiting requests of one pattern into a batch (up to ``max_batch``)
  and runs it as one batched refactorization + solve (glu_factor_batched /
  glu_solve_batched, or the FP32 + FP64-refinement pair), or through the
  single-matrix path for a batch of one;
* runs batches of different patterns at the same time on separate CUDA
  streams ("slots"); a request that arrives while others run is admitted as
  soon as a slot and the memory budget allow it;
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
    """A pattern's handle on the device, plus its last use."""

    def __init__(self, pat: Pattern, handle):
        self.pat = pat
        self.h = handle
        self.last_use = time.perf_counter()
        self.busy = False
        st = _glu.glu_get_stats(handle)
        self.base_bytes = int(st["device_bytes"])
        self.nnz_lu = int(st["nnz_lu"])
        self.batch_bytes = 0


class _Slot:
    def __init__(self, torch, device):
        self.stream = torch.cuda.Stream(device=device)
        self.event = None
        self.res: Optional[_Resident] = None
        self.reqs: List[Request] = []
        self.out = None
        self.info = None
        self.error = None       # (code, column) raised while enqueueing


class Server:
    """Continuous batching over patterns; see the module docstring."""

    def __init__(self, device_budget_bytes: float = 60e9, max_batch: int = 64, slots: int = 4,
                 precision: str = "fp64", tol: float = 1e-12, maxit: int = 10, device: int = 0):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.budget = int(device_budget_bytes)
        self.max_batch = max_batch
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
            _glu.glu_destroy(self.resident.pop(victim).h)
            self.evictions += 1
        return True

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

    # ------------------------------------------------------------ requests
    def submit(self, req: Request) -> None:
        req.t_submit = time.perf_counter()
        self.queues[req.key].append(req)

    def _launch(self, slot: _Slot) -> bool:
        # the pattern whose oldest waiting request is oldest, not already running
        best = None
        for key, q in self.queues.items():
            if q and not (key in self.resident and self.resident[key].busy):
                if best is None or q[0].t_submit < self.queues[best][0].t_submit:
                    best = key
        if best is None:
            return False
        q = self.queues[best]
        res = self._resident(best)
        if res is None:
            return False
        take = 1 if q[0].solo else min(len(q), self.max_batch)
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
        res.busy = True
        res.last_use = time.perf_counter()
        slot.res, slot.reqs = res, reqs
        h = res.h
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
        return True

    def _enqueue(self, slot: _Slot, res: _Resident, reqs: List[Request], nrhs: int) -> None:
        """The batch's factorization and solve, on the slot's stream."""
        torch = self.torch
        h = res.h
        take = len(reqs)
        if take == 1:
            r = reqs[0]
            v = torch.from_numpy(r.values).to(self.device, non_blocking=True)
            bb = torch.from_numpy(np.ascontiguousarray(r.b)).to(self.device, non_blocking=True)
            if self.precision == "fp64":
                _glu.glu_factor(h, v)
                x = _glu.glu_solve(h, bb)
                slot.info = None
            else:
                _glu.glu_factor_f32(h, v)
                x, slot.info = _glu.glu_solve_refine(h, bb, tol=self.tol, maxit=self.maxit)
            slot.out = x
        else:
            res.batch_bytes = max(res.batch_bytes, self._batch_bytes(res, take, nrhs))
            V = np.stack([r.values for r in reqs])
            Bt = np.zeros((take, nrhs, res.pat.n))
            for i, r in enumerate(reqs):
                Bt[i, : r.b.shape[0]] = r.b
            Vd = torch.from_numpy(V).to(self.device, non_blocking=True)
            Bd = torch.from_numpy(Bt).to(self.device, non_blocking=True)
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
        code, col = slot.error if slot.error is not None else _glu.glu_sync_status(slot.res.h)
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
        slot.res.busy = False
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
        their time while the loop keeps slots busy."""
        t0 = time.perf_counter()
        i = 0
        while i < len(arrivals) or self.step() or any(self.queues.values()):
            now = time.perf_counter() - t0
            while i < len(arrivals) and arrivals[i] <= now:
                self.submit(make_request(i))
                i += 1
            self.step()

    # ------------------------------------------------------------ reporting
    def latencies(self, skip: int = 0) -> np.ndarray:
        reqs = sorted(self.done, key=lambda r: r.rid)[skip:]
        return np.array([r.t_done - r.t_submit for r in reqs])
