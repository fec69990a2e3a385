"""Every execution path of the factorization and the solves against the CPU
oracle, entry by entry, at two sizes (the 20k- and the 200k-unknown power-grid
workloads).

The default path is covered by ``test_gpu_parity.py``; here each non-default
option -- forced level modes (Section III-B.2's three modes as reinterpreted:
0 warp-per-column, 1 block-per-column, 2 pipelined), the pipelined persistent
mode for narrow levels, the level sweep over the dense trailing block instead
of the dense kernel, direct launches instead of the CUDA graph, the per-level
solve, the solve without its one-block tail or its dense diagonal blocks, and
every candidate the autotuner times -- gets the same bars: fill, dependencies
and levels bit-exact, FP64 factors within 1e-10 relative per entry, solve
backward error <= 1e-12 and solution close to the oracle's.  The FP32
factorizations (single and batched) are checked entry by entry by
``parity.fp32_factor_check``: their componentwise backward error within the
rounding-error bound of LU in FP32 on every entry, and their difference from
the FP64 oracle's factors: on the entries without cancellation, at least
99.9% within the FP32 rounding of their own recurrence and all within 1e-3."""
import numpy as np
import pytest

import oracle
import synth
from parity import BERR_TOL, U32, backward_error, factor_mismatches, fp32_factor_check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WORKLOADS = ["mesh100x200_nets64", "mesh400x500_nets64"]

OPTIONS = {
    "mode0_warp_per_column": dict(mode_force=0),
    "mode1_block_per_column": dict(mode_force=1),
    "mode2_pipelined_all": dict(mode_force=2),
    "pipelined_narrow_4": dict(tail_threshold=4),
    "pipelined_narrow_32": dict(tail_threshold=32),
    "level_sweep_over_dense_block": dict(factor_tail=0),
    "direct_launches": dict(use_graph=0),
    "per_level_solve": dict(solve_mode=0),
    "solve_without_tail": dict(solve_tail=0),
    "solve_without_dense_blocks": dict(solve_blocks=0),
    "supernodal": dict(factor_blocks=1),
    "position_map_lookup": dict(row_lookup=1),
    "run_table_lookup": dict(row_lookup=2),
    "run_table_pipelined_narrow_32": dict(row_lookup=2, tail_threshold=32),
    "run_table_level_sweep_over_dense_block": dict(row_lookup=2, factor_tail=0),
    "run_table_mode0": dict(row_lookup=2, mode_force=0),
    "gpu_dependency_analysis": dict(gpu_analysis=1),
}


def _tuner_candidates():
    from paper_1908_00204_gb300 import tune
    return {f"tune_candidate_{i}": c for i, c in enumerate(tune.DEFAULT_CANDIDATES)}


@pytest.fixture(scope="module")
def glu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_00204_gb300 as g
    g.build.build()
    g.load_library()
    return g


_REF = {}


def reference(name):
    """The workload, its values and right-hand sides, and the oracle's
    factorization and solution (computed once per workload)."""
    if name not in _REF:
        m = synth.make(name, 1)
        v = m.values(3001)
        b = synth.rhs(m.n, 2, 3001)
        f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm, v)
        _REF[name] = (m, v, b, f, f.solve(b))
    return _REF[name]


def check_against_oracle(g, name, opts):
    m, v, b, f, xr = reference(name)
    h = g.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, g.default_options(**opts))
    try:
        st = g.glu_get_stats(h)
        if opts.get("factor_blocks", 0) == 0:
            want = {1: 1, 2: 2}.get(opts.get("row_lookup", 0), 1)   # auto: the map fits at these sizes
            assert st["row_lookup"] == want, st
            assert (st["n_runs"] > 0) == (want == 2) and st["lookup_bytes"] > 0
        cp, ri = g.glu_get_fill(h)
        assert np.array_equal(cp, f.lu_colptr) and np.array_equal(ri, f.lu_rowidx)
        dp, di = g.glu_get_deps(h)
        assert np.array_equal(dp, f.dep_ptr) and np.array_equal(di, f.dep_idx)
        lp, lc = g.glu_get_levels(h)
        assert np.array_equal(lp, f.level_ptr) and np.array_equal(lc, f.level_cols)
        g.glu_factor(h, torch.from_numpy(v).cuda())
        g.glu_sync(h)
        got = g.glu_get_factors(h)
        bad, _ = factor_mismatches(f.lu_colptr, f.lu_rowidx, got, f.lu_val)
        assert bad.size == 0, f"{opts}: {bad.size} factor entries off, first {bad[:5]}"
        x = g.glu_solve(h, torch.from_numpy(b).cuda()).cpu().numpy()
        assert backward_error(m.n, m.colptr, m.rowidx, v, b, x) <= BERR_TOL
        np.testing.assert_allclose(x, xr, rtol=1e-8, atol=1e-12)
    finally:
        g.glu_destroy(h)


@pytest.mark.parametrize("name", WORKLOADS)
@pytest.mark.parametrize("key", sorted(OPTIONS))
def test_option_path_matches_oracle(glu, name, key):
    check_against_oracle(glu, name, OPTIONS[key])


@pytest.mark.parametrize("name", WORKLOADS)
@pytest.mark.parametrize("idx", range(6))
def test_tuner_candidate_matches_oracle(glu, name, idx):
    cands = _tuner_candidates()
    key = f"tune_candidate_{idx}"
    if key not in cands:
        pytest.skip("fewer tuner candidates")
    check_against_oracle(glu, name, cands[key])


def _check_fp32(m, v, perm, f, got, ref, cols=None):
    r = fp32_factor_check(m.n, m.colptr, m.rowidx, v, perm, f.lu_colptr, f.lu_rowidx, got, ref, cols)
    print(f"FP32 factors: {r}")
    assert r["backward_worst"] <= 1.0, r                   # Higham's componentwise bound, every entry
    assert r["forward_within"] >= 0.999, r                 # FP32-level agreement with the FP64 oracle
    assert r["forward_worst_rel"] <= 1e-3, r
    assert r["clean_entries"] >= 0.5 * r["entries"], r     # the forward check covers most entries
    assert r["max_rel_err"] > U32 / 4, r                   # not vacuous: these are FP32 values


@pytest.mark.parametrize("name,lookup", [(w, 0) for w in WORKLOADS] + [("mesh100x200_nets64", 2)])
def test_fp32_factors_match_oracle(glu, name, lookup):
    """glu_factor_f32's factors: backward error bound and FP64-oracle
    comparison, on every column (20k) or on 3,000 sampled columns plus the
    last 600 (200k)."""
    m, v, b, f, xr = reference(name)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(row_lookup=lookup))
    glu.glu_factor_f32(h, torch.from_numpy(v).cuda())
    got = glu.glu_get_factors_f32(h).astype(np.float64)
    glu.glu_destroy(h)
    cols = None
    if m.n > 50000:
        rng = np.random.default_rng(0)
        cols = np.union1d(rng.choice(m.n - 600, 3000, replace=False), np.arange(m.n - 600, m.n))
    _check_fp32(m, v, m.perm, f, got, f.lu_val, cols)


@pytest.mark.parametrize("lookup", [0, 2])
def test_fp32_batched_factors_match_oracle(glu, lookup):
    """glu_factor_batched_f32's factors of several sets, checked the same way
    against the FP64 oracle's factorization of the same sets."""
    m = synth.make("mesh100x200_nets64", 1)
    B = 40
    V = np.stack([m.values(100 + s, sigma=0.1, base_seed=5) for s in range(B)])
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(row_lookup=lookup))
    glu.glu_factor_batched_f32(h, torch.from_numpy(V).cuda())
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm)
    for s in (0, 17, B - 1):
        got = glu.glu_get_factors_batched_f32(h, s).astype(np.float64)
        _check_fp32(m, V[s], m.perm, f, got, f.factor(V[s]))
    glu.glu_destroy(h)


def test_batched_fp64_run_table_matches_oracle(glu):
    """The batched FP64 refactorization through the run table: factors of
    several sets against the oracle's, solves by backward error."""
    m = synth.make("mesh100x200_nets64", 1)
    B = 40
    V = np.stack([m.values(200 + s, sigma=0.1, base_seed=6) for s in range(B)])
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(row_lookup=2))
    glu.glu_factor_batched(h, torch.from_numpy(V).cuda())
    assert glu.glu_get_stats(h)["row_lookup"] == 2
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm)
    for s in (0, 21, B - 1):
        bad, _ = factor_mismatches(f.lu_colptr, f.lu_rowidx, glu.glu_get_factors_batched(h, s), f.factor(V[s]))
        assert bad.size == 0, (s, bad[:5])
    rhs = np.stack([synth.rhs(m.n, 2, 400 + s) for s in range(B)])
    x = glu.glu_solve_batched(h, torch.from_numpy(rhs).cuda()).cpu().numpy()
    for s in (0, 21, B - 1):
        assert backward_error(m.n, m.colptr, m.rowidx, V[s], rhs[s], x[s]) <= BERR_TOL
    glu.glu_destroy(h)


@pytest.mark.parametrize("name", WORKLOADS)
@pytest.mark.parametrize("opts", [dict(tail_threshold=16), dict(mode_force=2)])
def test_dataflow_levels_equal_level_launches(glu, name, opts):
    """The pipelined levels run as one dataflow launch per run of narrow levels
    (mode_force=2: every level in one launch).  Every target entry takes its
    additions in the same order as with one launch per level, so the factors
    are bitwise equal."""
    m, v, b, f, xr = reference(name)
    base = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm)
    glu.glu_factor(base, torch.from_numpy(v).cuda())
    ref = glu.glu_get_factors(base)
    glu.glu_destroy(base)
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(**opts))
    assert glu.glu_get_stats(h)["levels_by_mode"][2] > 0
    for _ in range(2):
        glu.glu_factor(h, torch.from_numpy(v).cuda())
        assert np.array_equal(glu.glu_get_factors(h), ref)
    glu.glu_destroy(h)


def test_dataflow_factor_wait_timeout_reported_and_context_survives(glu):
    """A dataflow wait that can never be met (the test hook: the tasks that
    update one column never publish) ends the launch with GLU_ERR_TIMEOUT
    after the configured bound; a fresh handle then factors correctly."""
    m = synth.make("mesh100x200_nets64", 1)
    v = m.values(5)
    bad = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm,
                          glu.default_options(mode_force=2, factor_tail=0, fault_row=m.n - 1,
                                              spin_limit_us=100000))
    with pytest.raises(glu.GluError) as e:
        glu.glu_factor(bad, v)
    assert e.value.code == glu.glu.GLU_ERR_TIMEOUT
    glu.glu_destroy(bad)
    good = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(mode_force=2, factor_tail=0))
    glu.glu_factor(good, v)
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm, v)
    bad_entries, _ = factor_mismatches(f.lu_colptr, f.lu_rowidx, glu.glu_get_factors(good), f.lu_val)
    assert bad_entries.size == 0
    glu.glu_destroy(good)
