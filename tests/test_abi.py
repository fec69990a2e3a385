"""CPU checks of the boundary: the library loads, exports every symbol that
include/glu.h declares, and its host analysis matches the oracle bit for bit
(run with host_only=1, no device touched)."""
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def glu():
    import paper_1908_00204_gb300 as g
    g.build.build()
    g.load_library()
    return g


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(glu_\w+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol(glu):
    lib = glu.load_library()
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_strerror_and_options(glu):
    assert glu.glu_strerror(0) == "ok"
    assert "pivot" in glu.glu_strerror(-3)
    o = glu.default_options()
    assert o.tail_threshold == 0 and o.mode_force == -1


def host(glu, n, cp, ri, perm=None):
    return glu.glu_analyze(n, cp, ri, perm, glu.default_options(host_only=1))


@pytest.mark.parametrize("name", ["grid32_natural", "mesh100x200_nets64"])
def test_host_analysis_bit_exact(glu, name):
    m = synth.make(name, 1)
    h = host(glu, m.n, m.colptr, m.rowidx, m.perm)
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm)
    cp, ri = glu.glu_get_fill(h)
    dp, di = glu.glu_get_deps(h)
    lp, lc = glu.glu_get_levels(h)
    assert np.array_equal(cp, f.lu_colptr) and np.array_equal(ri, f.lu_rowidx)
    assert np.array_equal(dp, f.dep_ptr) and np.array_equal(di, f.dep_idx)
    assert np.array_equal(lp, f.level_ptr) and np.array_equal(lc, f.level_cols)
    st = glu.glu_get_stats(h)
    assert st["flops"] == f.flops() and st["nnz_lu"] == f.nnz and st["nlevels"] == f.nlevels


@pytest.mark.parametrize("seed", range(25))
def test_host_analysis_random(glu, seed, monkeypatch):
    # the analysis runs on host threads: vary their number (1, 3, 16)
    monkeypatch.setenv("GLU_ANALYZE_THREADS", str([1, 3, 16][(seed // 3) % 3]))
    n = 1 + seed * 7
    cp, ri, _ = synth.random_pattern_matrix(n, [0.02, 0.1, 0.3][seed % 3], 700 + seed, extra=2)
    perm = np.random.default_rng(seed).permutation(n).astype(np.int32)
    h = host(glu, n, cp, ri, perm)
    f = oracle.Factorization(n, cp, ri, perm)
    cp2, ri2 = glu.glu_get_fill(h)
    dp, di = glu.glu_get_deps(h)
    lp, lc = glu.glu_get_levels(h)
    assert np.array_equal(cp2, f.lu_colptr) and np.array_equal(ri2, f.lu_rowidx)
    assert np.array_equal(dp, f.dep_ptr) and np.array_equal(di, f.dep_idx)
    assert np.array_equal(lp, f.level_ptr) and np.array_equal(lc, f.level_cols)


def test_invalid_inputs_rejected(glu):
    bad = [
        (2, [0, 1, 2], [1, 0], None, glu.glu.GLU_ERR_STRUCT_SINGULAR),   # no diagonal
        (2, [0, 2, 3], [1, 0, 1], None, glu.glu.GLU_ERR_INVALID),        # unsorted rows
        (2, [0, 2, 3], [0, 0, 1], None, glu.glu.GLU_ERR_INVALID),        # duplicate row
        (2, [0, 1, 2], [0, 2], None, glu.glu.GLU_ERR_INVALID),           # row out of range
        (2, [1, 1, 2], [0, 1], None, glu.glu.GLU_ERR_INVALID),           # colptr[0] != 0
        (2, [0, 1, 2], [0, 1], [0, 0], glu.glu.GLU_ERR_INVALID),         # not a permutation
        (-1, [0], [], None, glu.glu.GLU_ERR_INVALID),
    ]
    for n, cp, ri, perm, code in bad:
        with pytest.raises(glu.GluError) as e:
            host(glu, n, np.array(cp), np.array(ri, np.int32),
                 None if perm is None else np.array(perm))
        assert e.value.code == code, (cp, ri, perm)


def test_empty_matrix(glu):
    h = host(glu, 0, np.zeros(1, np.int32), np.zeros(0, np.int32))
    assert glu.glu_get_stats(h)["nlevels"] == 0


def test_schedule_covers_every_update_once(glu):
    """Host logic of the level schedule: re-derive, from the analysis, that
    the per-level work items touch every (i, j, k) update exactly once."""
    m = synth.CircuitMatrix(synth.CircuitSpec(12, 14, 3, 10, 0.03, 0.05, "nd"), 4)
    h = host(glu, m.n, m.colptr, m.rowidx, m.perm)
    st = glu.glu_get_stats(h)
    f = oracle.Factorization(m.n, m.colptr, m.rowidx, m.perm)
    cp, ri = f.lu_colptr, f.lu_rowidx
    col = np.repeat(np.arange(m.n), np.diff(cp))
    l = np.bincount(col[ri > col], minlength=m.n)
    u = np.bincount(ri[ri < col], minlength=m.n)
    assert st["n_updates"] == int((l * u).sum())
    assert st["n_pairs"] == int(((ri < col) & (l[ri] > 0)).sum())
