"""Autotuner: the cache key depends on the pattern and permutation only, the
cache round-trips, and (GPU) tuning picks a candidate whose factors match."""
import json

import numpy as np
import pytest

import synth


def test_pattern_key_and_cache(tmp_path):
    from paper_1908_00204_gb300 import tune
    m = synth.make("grid32_natural", 0)
    k1 = tune.pattern_key(m.n, m.colptr, m.rowidx, m.perm)
    assert k1 == tune.pattern_key(m.n, m.colptr.copy(), m.rowidx.copy(), m.perm.copy())
    assert k1 != tune.pattern_key(m.n, m.colptr, m.rowidx, m.perm[::-1].copy())
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({k1: {"options": {"piece_updates": 777, "solve_tail": 0}, "ms": 1.0, "table": []}}))
    o = tune.options_for(m.n, m.colptr, m.rowidx, m.perm, str(path))
    assert o.piece_updates == 777 and o.solve_tail == 0
    o = tune.options_for(m.n, m.colptr, m.rowidx, None, str(path))      # another pattern: defaults
    assert o.piece_updates == 1024 or o.piece_updates == 2048 or o.piece_updates > 0


def test_tune_selection_and_cache_with_fake_timings(tmp_path, monkeypatch):
    # the tuner's choice on the host: the fastest candidate whose factors
    # match the first candidate's (1e-10 relative) wins; a faster one with
    # different factors is rejected; the result is cached and reused
    from paper_1908_00204_gb300 import tune
    m = synth.make("grid32_natural", 0)
    ref = np.linspace(1.0, 2.0, 50)
    cands = [{"piece_updates": 1024}, {"piece_updates": 512}, {"piece_updates": 2048}, {"piece_updates": 64}]
    plan = {1024: (3.0, ref), 512: (2.0, ref * (1 + 1e-13)), 2048: (2.5, ref), 64: (1.0, ref * 1.001)}
    calls = []

    def fake(torch, n, cp, ri, perm, values, b, opts, reps):
        calls.append(opts["piece_updates"])
        return plan[opts["piece_updates"]]
    monkeypatch.setattr(tune, "_time_candidate", fake)
    path = str(tmp_path / "tune.json")
    r = tune.tune(m.n, m.colptr, m.rowidx, m.perm, m.values(1), cache_path=path, candidates=cands)
    assert r["options"] == {"piece_updates": 512} and r["ms"] == 2.0
    assert [t["factors_match"] for t in r["table"]] == [True, True, True, False]
    assert calls == [1024, 512, 2048, 64]
    again = tune.tune(m.n, m.colptr, m.rowidx, m.perm, m.values(1), cache_path=path, candidates=cands)
    assert again["options"] == r["options"] and calls == [1024, 512, 2048, 64]     # from the cache
    assert tune.options_for(m.n, m.colptr, m.rowidx, m.perm, path).piece_updates == 512


@pytest.mark.gpu
def test_tune_on_gpu(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_00204_gb300 import build, tune
    build.build()
    m = synth.CircuitMatrix(synth.CircuitSpec(30, 40, 8, 60, 0.02, 0.05, "nd"), 3)
    path = str(tmp_path / "tune.json")
    r = tune.tune(m.n, m.colptr, m.rowidx, m.perm, m.values(1), cache_path=path, reps=2)
    assert all(t["factors_match"] for t in r["table"])
    assert r["ms"] == min(t["ms"] for t in r["table"])
    again = tune.tune(m.n, m.colptr, m.rowidx, m.perm, m.values(1), cache_path=path)
    assert again == json.load(open(path))[tune.pattern_key(m.n, m.colptr, m.rowidx, m.perm)]
