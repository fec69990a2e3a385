"""Algorithm 4 on the GPU (``csrc/analyze_gpu.cu``), its index arithmetic on
the CPU: the union of a column's up-looking candidates (rows above the
diagonal whose L column is not empty) and row k of L, formed by ranks --
a kept candidate a not in row k lands at (kept candidates before it) +
(row-k entries below a), a row-k entry b at its index + (kept candidates
below b) -- equals the host analysis's dependency lists (the merge of the
two sorted lists).  The GPU result itself is compared with the oracle by
tests/test_gpu_paths.py and tests/test_gpu_analysis.py."""
import numpy as np
import pytest

import synth
from paper_1908_00204_gb300 import glu


def rank_union(A, keep, B):
    add = np.array([keep[i] and not (np.searchsorted(B, a) < len(B) and B[np.searchsorted(B, a)] == a)
                    for i, a in enumerate(A)], bool)
    S = np.concatenate([[0], np.cumsum(add)])[:-1] if len(A) else np.zeros(0, np.int64)
    carry = int(add.sum())
    out = np.full(carry + len(B), -1, np.int64)
    for t, a in enumerate(A):
        if add[t]:
            out[S[t] + np.searchsorted(B, a)] = a
    for j, b in enumerate(B):
        p = np.searchsorted(A, b)
        out[j + (S[p] if p < len(A) else carry)] = b
    assert (out >= 0).all()
    return out


@pytest.mark.parametrize("case", ["grid", "mesh", "random"])
def test_rank_union_equals_host_dependencies(case):
    if case == "grid":
        m = synth.make("grid32_natural", 0)
        n, cp, ri, perm = m.n, m.colptr, m.rowidx, m.perm
    elif case == "mesh":
        m = synth.CircuitMatrix(synth.CircuitSpec(20, 30, 6, 40, 0.02, 0.05, "nd"), 4)
        n, cp, ri, perm = m.n, m.colptr, m.rowidx, m.perm
    else:
        n = 120
        cp, ri, _ = synth.random_pattern_matrix(n, 0.05, 17)
        perm = np.random.default_rng(3).permutation(n).astype(np.int32)
    h = glu.glu_analyze(n, cp, ri, perm, glu.default_options(host_only=1))
    fcp, fri = glu.glu_get_fill(h)
    dp, di = glu.glu_get_deps(h)
    glu.glu_destroy(h)
    col = np.repeat(np.arange(n), np.diff(fcp))
    diag = np.array([fcp[j] + np.searchsorted(fri[fcp[j]:fcp[j + 1]], j) for j in range(n)])
    keep_col = fcp[1:] - 1 > diag                      # column i of L not empty
    low = fri > col
    order = np.lexsort((col[low], fri[low]))           # row view of L, columns ascending
    lrows, lcols = fri[low][order], col[low][order]
    for k in range(n):
        A = fri[fcp[k]:diag[k]]
        B = lcols[lrows == k]
        got = rank_union(A, keep_col[A], B)
        assert np.array_equal(got, di[dp[k]:dp[k + 1]]), k
