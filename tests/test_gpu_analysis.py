"""Algorithm 4 and the levels on the GPU (option gpu_analysis): the
dependency lists and the levels equal the host analysis's and the CPU
oracle's bit for bit on small, random, unsymmetric and degenerate patterns
(the full-size workloads are in tests/test_gpu_paths.py)."""
import numpy as np
import pytest

import oracle
import synth

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


def cases():
    out = []
    m = synth.make("grid32_natural", 0)
    out.append((m.n, m.colptr, m.rowidx, m.perm))
    m = synth.CircuitMatrix(synth.CircuitSpec(30, 40, 8, 60, 0.02, 0.05, "nd"), 3)
    out.append((m.n, m.colptr, m.rowidx, m.perm))
    for seed, n in enumerate([1, 2, 7, 65, 300]):
        cp, ri, _ = synth.random_pattern_matrix(n, 0.08, 60 + seed)
        out.append((n, cp, ri, np.random.default_rng(seed).permutation(n).astype(np.int32)))
    cp, ri, _ = synth.random_pattern_matrix(50, 1.0, 5)          # fully dense: a chain
    out.append((50, cp, ri, None))
    n = 40                                                          # diagonal: one level
    out.append((n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), None))
    return out


@pytest.mark.parametrize("idx", range(9))
def test_gpu_deps_and_levels_equal_host_and_oracle(glu, idx):
    n, cp, ri, perm = cases()[idx]
    hh = glu.glu_analyze(n, cp, ri, perm, glu.default_options(host_only=1))
    hg = glu.glu_analyze(n, cp, ri, perm, glu.default_options(gpu_analysis=1))
    for get in (glu.glu_get_deps, glu.glu_get_levels):
        a, b = get(hh), get(hg)
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
    f = oracle.Factorization(n, cp, ri, perm)
    dp, di = glu.glu_get_deps(hg)
    lp, lc = glu.glu_get_levels(hg)
    assert np.array_equal(dp, f.dep_ptr) and np.array_equal(di, f.dep_idx)
    assert np.array_equal(lp, f.level_ptr) and np.array_equal(lc, f.level_cols)
