"""Autotuner: picks the execution knobs of one sparsity pattern by timing.

Knobs (all fields of ``glu_options``):

* ``tail_threshold`` -- levels with at most this many columns run in the
  pipelined mode (one persistent launch with grid barriers) instead of one
  launch per level (the paper's stream-mode threshold, Section III-B.2);
* ``piece_updates`` -- target updates per row task (work split size);
* ``solve_tail`` -- dense trailing block solved by one block, or not;
* ``factor_tail`` -- dense trailing block factored by the dense kernel, or
  one level per column.

Each candidate is analysed, factorized and solved on the current GPU with
new values; the fastest refactor + solve (median of a few runs, CUDA events)
wins.  Results are cached in a JSON file keyed by a hash of the pattern and
permutation, so a pattern is tuned once.  Every candidate's factors are
checked against the first candidate's (same pattern, same values) before its
time counts.
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


def pattern_key(n, colptr, rowidx, perm=None) -> str:
    h = hashlib.sha256()
    h.update(np.int64(n).tobytes())
    h.update(np.ascontiguousarray(colptr, np.int32).tobytes())
    h.update(np.ascontiguousarray(rowidx, np.int32).tobytes())
    if perm is not None:
        h.update(np.ascontiguousarray(perm, np.int32).tobytes())
    return h.hexdigest()[:24]


def _time_candidate(torch, n, colptr, rowidx, perm, values, b, opts, reps):
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


def tune(n, colptr, rowidx, perm, values, cache_path: Optional[str] = None,
         candidates: Optional[List[Dict[str, int]]] = None, reps: int = 3, nrhs: int = 1,
         seed: int = 0) -> Dict:
    """Best options for this pattern: {"options": {...}, "ms": ..., "table": [...]}."""
    import torch
    key = pattern_key(n, colptr, rowidx, perm)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return cache[key]
    cands = candidates or DEFAULT_CANDIDATES
    b = np.random.default_rng(seed).uniform(-1.0, 1.0, (nrhs, n))
    table, ref = [], None
    for opts in cands:
        ms, lu = _time_candidate(torch, n, colptr, rowidx, perm, np.ascontiguousarray(values, np.float64), b,
                                 opts, reps)
        if ref is None:
            ref = lu
        ok = bool(np.allclose(lu, ref, rtol=1e-10, atol=0.0))
        table.append({"options": opts, "ms": ms, "factors_match": ok})
    best = min((t for t in table if t["factors_match"]), key=lambda t: t["ms"])
    result = {"options": best["options"], "ms": best["ms"], "table": table}
    if cache_path:
        cache[key] = result
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return result


def options_for(n, colptr, rowidx, perm=None, cache_path: Optional[str] = None):
    """glu_options from the cache (defaults when the pattern was never tuned)."""
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        hit = cache.get(pattern_key(n, colptr, rowidx, perm))
        if hit:
            return _glu.default_options(**hit["options"])
    return _glu.default_options()
