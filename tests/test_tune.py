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


def test_descent_keeps_fastest_matching_value_per_knob(tmp_path, monkeypatch):
    # coordinate descent on the host with fake timings: per knob the fastest
    # value whose factors match is kept, later knobs start from it; a faster
    # value with other factors is rejected; batched results cache apart
    from paper_1908_00204_gb300 import tune
    m = synth.make("grid32_natural", 0)
    ref = np.linspace(1.0, 2.0, 20)
    calls = []

    def fake(torch, n, cp, ri, perm, values, b, opts, reps):
        calls.append(dict(opts))
        ms = 10.0
        ms -= {512: 1.0, 2048: -1.0, 4096: -2.0}.get(opts.get("piece_updates"), 0.0)
        ms -= 0.5 if opts.get("src_min") == 8 else 0.0
        lu = ref * (1.001 if opts.get("row_lookup") == 2 else 1.0)    # wrong factors: rejected
        ms -= 5.0 if opts.get("row_lookup") == 2 else 0.0
        return ms, lu
    monkeypatch.setattr(tune, "_time_candidate", fake)
    monkeypatch.setattr(tune, "_time_batched", lambda *a: fake(*a))
    path = str(tmp_path / "tune.json")
    r = tune.tune(m.n, m.colptr, m.rowidx, m.perm, m.values(1), cache_path=path, search="descent")
    assert r["options"] == {"piece_updates": 512, "src_min": 8}
    assert r["ms"] == 8.5
    assert calls[0] == {} and len(calls) == 1 + sum(len(v) - 1 for _, v in tune.KNOBS)
    assert any(t["options"].get("row_lookup") == 2 and not t["factors_match"] for t in r["table"])
    rb = tune.tune(m.n, m.colptr, m.rowidx, m.perm, m.values(1), cache_path=path, search="descent", batch=8)
    assert rb["batch"] == 8 and len(calls) == 2 * (1 + sum(len(v) - 1 for _, v in tune.KNOBS))
    assert tune.options_for(m.n, m.colptr, m.rowidx, m.perm, path).piece_updates == 512
    assert tune.options_for(m.n, m.colptr, m.rowidx, m.perm, path, batch=8).src_min == 8


@pytest.mark.gpu
@pytest.mark.parametrize("batch", [0, 8])
def test_descent_on_gpu_choice_matches_oracle(tmp_path, batch):
    """The coordinate search on the GPU (single matrix and batched): the
    options it picks give factors that match the CPU oracle's."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from parity import factor_mismatches
    from paper_1908_00204_gb300 import build, glu, tune
    build.build()
    m = synth.CircuitMatrix(synth.CircuitSpec(30, 40, 8, 60, 0.02, 0.05, "nd"), 3)
    v = m.values(1)
    r = tune.tune(m.n, m.colptr, m.rowidx, m.perm, v, cache_path=str(tmp_path / "t.json"), reps=1,
                  search="descent", batch=batch)
    assert r["ms"] == min(t["ms"] for t in r["table"] if t["factors_match"])
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, tune.options_for(m.n, m.colptr, m.rowidx, m.perm,
                                                                          str(tmp_path / "t.json"), batch=batch))
    glu.glu_factor(h, v)
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm, v)
    bad, _ = factor_mismatches(f.lu_colptr, f.lu_rowidx, glu.glu_get_factors(h), f.lu_val)
    assert bad.size == 0
