"""Host-side check of the supernodal factorization schedule (no GPU).

The analysis's block schedule (option factor_blocks) is replayed on the CPU
with the index arithmetic the kernels use -- diagonal blocks, panel rows
L21 = A21 U11^-1, target rows U12 = L11^-1 A12, and the per-task updates
A(R_B, k) -= L21 U12(:, k) through the row map -- level by level, on the
CSC values.  The result must match the oracle's factors, and every
supernode must be a run with a dense diagonal block and equal rows below.
The dump is the library's diagnostic copy of the schedule (environment
variable GLU_DUMP_BLOCKS at glu_analyze).
"""
import numpy as np
import pytest

import oracle
import synth
from paper_1908_00204_gb300 import glu
from parity import factor_mismatches


def load_blocks(path):
    w = np.fromfile(path, np.int64)
    nsn, nbl, nd, ni, npairs, nseg, ntask = (int(x) for x in w[:7])
    q = 7

    def take(k):
        nonlocal q
        v = w[q:q + k]
        q += k
        return v
    d = {}
    d["sn_c0"] = take(nsn + 1)
    d["sn_r"] = take(nsn)
    d["bdiag_ptr"] = take(nbl + 1)
    d["bdiag"] = take(nd)
    d["bitem_ptr"] = take(nbl + 1)
    d["bitems"] = take(4 * ni).reshape(ni, 4)
    d["bpairs"] = take(5 * npairs).reshape(npairs, 5)
    d["bsegs"] = take(3 * nseg).reshape(nseg, 3)
    d["btask_ptr"] = take(nbl + 1)
    d["btasks"] = take(2 * ntask).reshape(ntask, 2)
    d["nbl"] = nbl
    return d


def replay(cp, ri, diag, lu, d):
    """The kernels' arithmetic, sequentially, on the CSC values lu."""
    c0v, rv = d["sn_c0"], d["sn_r"]
    pairs = d["bpairs"]
    # the row map: offsets in column k of the rows R_B
    def rows_below(q):
        r = rv[q]
        e = cp[c0v[q + 1]]
        return ri[e - r:e]
    for l in range(d["nbl"]):
        for it in range(d["bdiag_ptr"][l], d["bdiag_ptr"][l + 1]):
            q = d["bdiag"][it]
            c0, s = c0v[q], c0v[q + 1] - c0v[q]
            idx = np.array([[diag[c0 + m] - m + rr for m in range(s)] for rr in range(s)])
            X = lu[idx].copy()
            for jj in range(s - 1):
                X[jj + 1:, jj] /= X[jj, jj]
                X[jj + 1:, jj + 1:] -= np.outer(X[jj + 1:, jj], X[jj, jj + 1:])
            lu[idx] = X
        for it in range(d["bitem_ptr"][l], d["bitem_ptr"][l + 1]):
            q, kind, a, b = d["bitems"][it]
            c0, s, r = c0v[q], c0v[q + 1] - c0v[q], rv[q]
            if kind == 0:
                for t in range(a, b):
                    pos = [cp[c0 + m + 1] - r + t for m in range(s)]
                    x = lu[pos].copy()
                    for jj in range(s):
                        x[jj] /= lu[diag[c0 + jj]]
                        for m in range(jj + 1, s):
                            x[m] -= x[jj] * lu[diag[c0 + m] - m + jj]
                    lu[pos] = x
            else:
                sn, k, f, upos, mb = pairs[a]
                pos = [upos + (m - f) for m in range(f, s)]
                x = lu[pos].copy()
                for jj in range(f, s - 1):
                    for m in range(jj + 1, s):
                        x[m - f] -= lu[diag[c0 + jj] + (m - jj)] * x[jj - f]
                lu[pos] = x
        for it in range(d["btask_ptr"][l], d["btask_ptr"][l + 1]):
            s0, s1 = d["btasks"][it]
            for sg in range(s0, s1):
                p, t0, t1 = d["bsegs"][sg]
                sn, k, f, upos, mb = pairs[p]
                c0, s, r = c0v[sn], c0v[sn + 1] - c0v[sn], rv[sn]
                R = rows_below(sn)
                kr = ri[cp[k]:cp[k + 1]]
                for t in range(t0, t1):
                    acc = 0.0
                    for m in range(f, s):
                        acc += lu[cp[c0 + m + 1] - r + t] * lu[upos + (m - f)]
                    off = int(np.searchsorted(kr, R[t]))
                    assert kr[off] == R[t], "row of R_B missing from the target column"
                    lu[cp[k] + off] -= acc
    return lu


@pytest.mark.parametrize("case", ["random", "mesh_nets", "arrow", "dense"])
def test_block_schedule_replay_matches_oracle(tmp_path, monkeypatch, case):
    if case == "dense":
        # degenerate: every column in supernodes of 32 with nothing below the last
        n = 100
        cp, ri, v = synth.random_pattern_matrix(n, 1.0, 9)
        perm = None
    elif case == "random":
        n = 60
        cp, ri, v = synth.random_pattern_matrix(n, 0.12, 7)
        perm = np.random.default_rng(3).permutation(n).astype(np.int32)
    elif case == "mesh_nets":
        m = synth.CircuitMatrix(synth.CircuitSpec(10, 12, 4, 12, 0.02, 0.05, "nd"), 5)
        n, cp, ri, perm, v = m.n, m.colptr, m.rowidx, m.perm, m.values(2)
    else:
        # dense last row and column: one supernode at the end
        n = 40
        rows, cols = [], []
        for j in range(n):
            rows += [j] + ([n - 1] if j < n - 1 else [])
            cols += [j] + ([j] if j < n - 1 else [])
            if j < n - 1:
                rows.append(j)
                cols.append(n - 1)
        import scipy.sparse as sp
        A = sp.csc_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
        A.sum_duplicates()
        A.sort_indices()
        cp, ri = A.indptr.astype(np.int32), A.indices.astype(np.int32)
        v = np.random.default_rng(1).uniform(0.1, 1.0, len(ri))
        v[[np.searchsorted(ri[cp[j]:cp[j + 1]], j) + cp[j] for j in range(n)]] += n
        perm = None
    path = tmp_path / "blocks.bin"
    monkeypatch.setenv("GLU_DUMP_BLOCKS", str(path))
    h = glu.glu_analyze(n, cp, ri, perm, glu.default_options(host_only=1, factor_blocks=1))
    fcp, fri = glu.glu_get_fill(h)
    glu.glu_destroy(h)
    d = load_blocks(path)
    fcp, fri = np.asarray(fcp, np.int64), np.asarray(fri, np.int64)
    diag = np.array([fcp[j] + np.searchsorted(fri[fcp[j]:fcp[j + 1]], j) for j in range(n)])
    c0v = d["sn_c0"]
    assert c0v[0] == 0 and c0v[-1] == n and (np.diff(c0v) >= 1).all() and (np.diff(c0v) <= 32).all()
    for q in range(len(c0v) - 1):
        c0, c1 = c0v[q], c0v[q + 1]
        R = fri[fcp[c1] - d["sn_r"][q]:fcp[c1]]
        for j in range(c0, c1):
            col = fri[fcp[j]:fcp[j + 1]]
            assert set(range(c0, c1)) <= set(col.tolist())          # dense diagonal block
            assert np.array_equal(col[col >= c1], R)                # equal rows below
    f = oracle.Factorization(n, cp, ri, perm, v)
    # the values gathered into the filled pattern (B = P A P^T), as the library does
    B_vals = np.zeros(len(fri))
    pinv = np.arange(n) if perm is None else np.argsort(perm)
    for jo in range(n):
        for p in range(cp[jo], cp[jo + 1]):
            i, j = pinv[ri[p]], pinv[jo]
            B_vals[fcp[j] + np.searchsorted(fri[fcp[j]:fcp[j + 1]], i)] = v[p]
    lu = replay(fcp, fri, diag, B_vals, d)
    bad, _ = factor_mismatches(f.lu_colptr, f.lu_rowidx, lu, f.lu_val)
    assert bad.size == 0
    assert d["nbl"] <= n


def test_block_levels_contract_separator_chains(tmp_path, monkeypatch):
    m = synth.make("mesh100x200_nets64", 1)
    path = tmp_path / "blocks.bin"
    monkeypatch.setenv("GLU_DUMP_BLOCKS", str(path))
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(host_only=1, factor_blocks=1))
    nl = glu.glu_get_stats(h)["nlevels"]
    glu.glu_destroy(h)
    d = load_blocks(path)
    assert d["nbl"] * 4 < nl                  # 482 column levels, about 70 block levels
    assert (np.diff(d["sn_c0"]) == 32).sum() > 10
