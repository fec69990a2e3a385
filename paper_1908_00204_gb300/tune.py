"""Autotuner: picks the execution knobs of one sparsity pattern by timing.

Knobs (all fields of ``glu_options``):

* ``piece_updates``, ``src_min``, ``lane_max``, ``lane_segs`` -- the task
  shapes of the level schedule: updates per warp task, the source count from
  which a target column is cut into 32-position chunk tasks, and the size of
  the tasks that run on a single lane;
* ``row_lookup`` -- how the level kernels find a row in its target column
  (position map, or run table);
* ``tail_threshold`` -- levels with at most this many columns run in the
  pipelined mode (one dataflow launch for a run of them) instead of one
  launch per level: the per-level mode choice (the paper's stream-mode
  threshold, Section III-B.2);
* ``solve_tail`` / ``factor_tail`` -- the dense trailing block solved by one
  block, or factored by the dense kernel, or not.

Two searches: a fixed list of candidates, or a coordinate descent that
starts from the defaults and, knob by knob, keeps the fastest value.  A
candidate is analysed, factorized and solved on the current GPU with new
values (``batch`` > 0: the batched refactorization + solve of that many
value sets instead); its median time over a few runs (CUDA events) counts
only if its factors match the default candidate's (1e-10 relative; each
candidate's factors are also checked against the CPU oracle by the tests).
Results are cached in a JSON file keyed by a hash of the pattern and
permutation (and the batch size), so a pattern is tuned once.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Dict, List, Optional

import numpy as np

from . import glu as _glu

DEFAULT_CANDIDATES: List[Dict[str, int]] = [
    {"tail_threshold": 0, "piece_updates": 1024, "solve_tail": 1},
    {"tail_threshold": 0, "piece_updates": 2048, "solve_tail": 1},
    {"tail_threshold": 0, "piece_updates": 512, "solve_tail": 1},
    {"tail_threshold": 4, "piece_updates": 1024, "solve_tail": 1},
    {"tail_threshold": 0, "piece_updates": 1024, "solve_tail": 0},
    {"tail_threshold": 0, "piece_updates": 1024, "factor_tail": 0},
]

# the coordinate search, in this order; the first value of each is the default
KNOBS: List[tuple] = [
    ("piece_updates", [1024, 512, 2048, 4096]),
    ("src_min", [5, 3, 8]),
    ("lane_max", [32, 16, 64]),
    ("lane_segs", [2, 1, 4]),
    ("row_lookup", [1, 2]),
    ("tail_threshold", [0, 4]),
    ("factor_tail", [1, 0]),
]


def pattern_key(n, colptr, rowidx, perm=None) -> str:
    h = hashlib.sha256()
    h.update(np.int64(n).tobytes())
    h.update(np.ascontiguousarray(colptr, np.int32).tobytes())
    h.update(np.ascontiguousarray(rowidx, np.int32).tobytes())
    if perm is not None:
        h.update(np.ascontiguousarray(perm, np.int32).tobytes())
    return h.hexdigest()[:24]


def _cache_key(n, colptr, rowidx, perm, batch) -> str:
    k = pattern_key(n, colptr, rowidx, perm)
    return k if batch <= 0 else f"{k}|batch{batch}"


def _time_candidate(torch, n, colptr, rowidx, perm, values, b, opts, reps):
    """Median ms of one refactorization + solve, and the factors."""
    h = _glu.glu_analyze(n, colptr, rowidx, perm, _glu.default_options(**opts))
    try:
        v = torch.from_numpy(values).cuda()
        bb = torch.from_numpy(b).cuda()
        x = torch.empty_like(bb)
        for _ in range(2):
            _glu.glu_factor(h, v)
            _glu.glu_solve(h, bb, x)
        _glu.glu_sync(h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for _ in range(reps):
            e0.record()
            _glu.glu_factor(h, v)
            _glu.glu_solve(h, bb, x)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        _glu.glu_sync(h)
        return float(np.median(ts)), _glu.glu_get_factors(h)
    finally:
        _glu.glu_destroy(h)


def _time_batched(torch, n, colptr, rowidx, perm, V, b, opts, reps):
    """Median ms of one batched refactorization + solve of the value sets V
    (batch, nnz) with right-hand sides b (batch, nrhs, n), and set 0's factors."""
    h = _glu.glu_analyze(n, colptr, rowidx, perm, _glu.default_options(**opts))
    try:
        vd = torch.from_numpy(V).cuda()
        bd = torch.from_numpy(b).cuda()
        for _ in range(2):
            _glu.glu_factor_batched(h, vd)
            _glu.glu_solve_batched(h, bd)
        _glu.glu_sync(h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for _ in range(reps):
            e0.record()
            _glu.glu_factor_batched(h, vd)
            _glu.glu_solve_batched(h, bd)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        _glu.glu_sync(h)
        return float(np.median(ts)), _glu.glu_get_factors_batched(h, 0)
    finally:
        _glu.glu_destroy(h)


def tune(n, colptr, rowidx, perm, values, cache_path: Optional[str] = None,
         candidates: Optional[List[Dict[str, int]]] = None, reps: int = 3, nrhs: int = 1,
         seed: int = 0, search: str = "list", batch: int = 0) -> Dict:
    """Best options for this pattern: {"options": {...}, "ms": ..., "table": [...]}.

    search="list": time ``candidates`` (default DEFAULT_CANDIDATES);
    search="descent": coordinate descent over KNOBS from the defaults.
    batch > 0: time the batched path on ``batch`` value sets (values: one
    set, perturbed per set, or an array (batch, nnz))."""
    import torch
    key = _cache_key(n, colptr, rowidx, perm, batch)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return cache[key]
    rng = np.random.default_rng(seed)
    values = np.ascontiguousarray(values, np.float64)
    if batch > 0:
        V = values if values.ndim == 2 else \
            np.ascontiguousarray(values[None, :] * rng.uniform(0.9, 1.1, (batch, values.size)))
        b = rng.uniform(-1.0, 1.0, (batch, nrhs, n))

        def timed(opts):
            return _time_batched(torch, n, colptr, rowidx, perm, V, b, opts, reps)
    else:
        b = rng.uniform(-1.0, 1.0, (nrhs, n))

        def timed(opts):
            return _time_candidate(torch, n, colptr, rowidx, perm, values, b, opts, reps)
    table, ref = [], None

    def run(opts):
        nonlocal ref
        ms, lu = timed(opts)
        if ref is None:
            ref = lu
        ok = bool(np.allclose(lu, ref, rtol=1e-10, atol=0.0))
        table.append({"options": dict(opts), "ms": ms, "factors_match": ok})
        return ms, ok

    if search == "descent":
        best_opts: Dict[str, int] = {}
        best_ms, _ = run(best_opts)
        for knob, vals in KNOBS:
            for v in vals[1:]:
                trial = dict(best_opts, **{knob: v})
                ms, ok = run(trial)
                if ok and ms < best_ms:
                    best_ms, best_opts = ms, trial
        best = {"options": best_opts, "ms": best_ms}
    else:
        for opts in candidates or DEFAULT_CANDIDATES:
            run(opts)
        best = min((t for t in table if t["factors_match"]), key=lambda t: t["ms"])
    result = {"options": best["options"], "ms": best["ms"], "table": table, "search": search, "batch": batch}
    if cache_path:
        cache[key] = result
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return result


def options_for(n, colptr, rowidx, perm=None, cache_path: Optional[str] = None, batch: int = 0):
    """glu_options from the cache (defaults when the pattern was never tuned)."""
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        hit = cache.get(_cache_key(n, colptr, rowidx, perm, batch))
        if hit:
            return _glu.default_options(**hit["options"])
    return _glu.default_options()
