"""Host-side check of the column-level factorization schedule (no GPU).

The level kernel's work lists are replayed on the CPU with the kernels' own
index arithmetic: each pair's run table as its build kernel defines it (a
run starts at every row of L(:,j) whose position in column k is not the
previous row's plus one), each segment's run range as the segment pass picks
it, and each row's position found as the kernels find it -- the 32-run
window, ballots and OR-reduction of a warp over rows (ROW tasks), the
one-lane walk (SRC and LANE tasks) -- checked against the plain definition
(the offset of row L(:,j)[t] in column k past U(j,k), by binary search).
Then level by level the normalization items of the previous level and the
update tasks, each segment applying A_s(i,k) -= A_s(i,j) * (A_s(j,k) /
A_s(j,j)) for its rows t0..t1-1 (Algorithm 5, Eq. 3), then the dense
trailing block as a dense LU without pivoting, or the final normalization
pass.  The result must match the oracle's factors.

Because the replay applies a level's tasks one after the other while the
GPU runs them at once, it also checks what makes the two the same: within a
level no task writes a position that another task writes or that any task
reads, and the normalization items touch neither; a KIND_SRC task's targets
lie in its 32 positions.  Every update (i,j,k) whose source j lies before the
dense block is applied exactly once, and every L entry outside the block is
divided exactly once.  The library's value gather map must place A's values
where the replay's own gather does.  The dump is the library's diagnostic
copy of the schedule (environment variable GLU_DUMP_COLUMNS at glu_analyze).
"""
import numpy as np
import pytest

import oracle
import synth
from paper_1908_00204_gb300 import glu
from parity import factor_mismatches

KIND_ROW, KIND_SRC, KIND_LANE = 0, 1, 2
SRC_SLOTS = 32


def load_columns(path):
    w = np.fromfile(path, np.int64)
    nl, npairs, nseg, ntask, nnorm, ft0, flev = (int(x) for x in w[:7])
    q = 7

    def take(k, width=1):
        nonlocal q
        v = w[q:q + k * width]
        q += k * width
        return v.reshape(k, width) if width > 1 else v
    d = dict(nl=nl, ftail_t0=ft0, ftail_level=flev)
    d["task_ptr"] = take(nl + 1)
    d["row_ptr"] = take(nl)
    d["lane_ptr"] = take(nl)
    d["norm_ptr"] = take(nl + 2)
    d["pairs"] = take(npairs, 4).reshape(npairs, 4)
    d["segs"] = take(nseg, 5).reshape(nseg, 5)
    d["tasks"] = take(ntask, 5).reshape(ntask, 5)
    d["norms"] = take(nnorm, 3).reshape(nnorm, 3)
    d["gsrc"] = w[q:]
    return d


def position_map(fcp, fri, diag, pairs):
    """The position map as the map-build kernel defines it."""
    lcount = fcp[1:] - diag - 1
    total = int(pairs[-1, 3] + lcount[pairs[-1, 0]]) if len(pairs) else 0
    mp = np.full(total, -1, np.int64)
    nxt = 0
    for j, k, pos, mb in pairs:
        assert mb == nxt                      # map blocks are consecutive, in pair order
        lj = int(lcount[j])
        nxt = mb + lj
        rows = fri[diag[j] + 1:fcp[j + 1]]
        col = fri[pos + 1:fcp[k + 1]]
        off = np.searchsorted(col, rows)
        assert (off < col.size).all() and (col[np.minimum(off, col.size - 1)] == rows).all()
        mp[mb:mb + lj] = off
    return mp


def runs_of(offsets):
    """A pair's runs (ts, off) from its rows' offsets, as the build kernel writes them."""
    t = np.arange(offsets.size)
    start = np.ones(offsets.size, bool)
    start[1:] = offsets[1:] != offsets[:-1] + 1
    return np.stack([t[start], offsets[start]], 1)


def segment_runs(runs, t0, t1):
    """The segment pass: the first run overlapping t0..t1-1 and their count."""
    rb = int(np.searchsorted(runs[:, 0], t0, side="right")) - 1
    re = int(np.searchsorted(runs[:, 0], t1, side="left"))
    return rb, re - rb


def offsets_warp(runs, rb, nr, t0, t1, rows_per_batch=256):
    """row_segment's lookup: lanes hold runs wb..wb+31; per group of 32 rows
    one ballot for the run holding the group's first row, an OR of the bits
    of the runs starting inside the group, a popcount per lane."""
    INF = 2**31 - 1
    rend = rb + nr

    def window(wb):
        w = np.full((32, 2), [INF, 0], np.int64)
        k = max(0, min(32, rend - wb))
        w[:k] = runs[wb:wb + k]
        return w
    wb = rb
    w = window(wb)
    out = np.empty(t1 - t0, np.int64)
    for g0 in range(t0, t1, 32):
        glast = min(g0 + 31, t1 - 1)
        if wb + 32 < rend and w[31, 0] <= glast:
            wb += int((w[:, 0] <= g0).sum()) - 1
            w = window(wb)
        a = int((w[:, 0] <= g0).sum()) - 1
        starts = 0
        for ts in w[:, 0]:
            if g0 < ts <= glast:
                starts |= 1 << int(ts - g0)
        for lane in range(32):
            t = g0 + lane
            if t >= t1:
                break
            idx = a + bin(starts & ((1 << (lane + 1)) - 1)).count("1")
            assert 0 <= idx < 32
            out[t - t0] = w[idx, 1] + (t - w[idx, 0])
    return out


def offsets_walk(runs, rb, nr, t0, t1):
    """lane_task / src_task's lookup: one lane walks the runs in order."""
    INF = 2**31 - 1
    rend = rb + nr
    r = rb
    cur = runs[r]
    nxt = runs[r + 1] if r + 1 < rend else (INF, 0)
    out = np.empty(t1 - t0, np.int64)
    for t in range(t0, t1):
        while t >= nxt[0]:
            cur, r = nxt, r + 1
            nxt = runs[r + 1] if r + 1 < rend else (INF, 0)
        out[t - t0] = cur[1] + (t - cur[0])
    return out


def replay(fcp, fri, diag, lu, d):
    n = diag.size
    nl, t0b, lend = d["nl"], d["ftail_t0"], d["ftail_level"]
    dense = t0b < n
    if not dense:
        lend = nl
    pairs, segs, tasks, norms = d["pairs"], d["segs"], d["tasks"], d["norms"]
    mp = position_map(fcp, fri, diag, pairs)
    lcount = fcp[1:] - diag - 1
    pair_runs = [runs_of(mp[mb:mb + lcount[j]]) for j, k, pos, mb in pairs]
    applied = np.zeros(mp.size, np.int64)          # uses of each map entry
    divided = np.zeros(lu.size, np.int64)          # divisions of each L entry
    kinds = np.zeros(3, np.int64)

    def normalize(lo, hi):
        written = []
        for col, a, b in norms[lo:hi]:
            p = diag[col] + 1 + np.arange(a, b)
            lu[p] /= lu[diag[col]]
            divided[p] += 1
            written.append(p)
        return np.concatenate(written) if written else np.zeros(0, np.int64)

    for l in range(lend):
        nw = normalize(d["norm_ptr"][l], d["norm_ptr"][l + 1])
        reads, writes, owner = [], [], []
        for ti in range(d["task_ptr"][l], d["task_ptr"][l + 1]):
            sb, se, kind, nslots, base = tasks[ti]
            want = KIND_SRC if ti < d["row_ptr"][l] else KIND_ROW if ti < d["lane_ptr"][l] else KIND_LANE
            assert kind == want
            kinds[kind] += 1
            assert se > sb
            for pos, dj, pair, a, b in segs[sb:se]:
                assert b > a
                j, k, ppos, mb = pairs[pair]
                assert ppos == pos and diag[j] == dj and b <= lcount[j]
                t = np.arange(a, b)
                src = dj + 1 + t
                runs = pair_runs[pair]
                rb, nr = segment_runs(runs, a, b)
                look = offsets_warp if kind == KIND_ROW else offsets_walk
                off = look(runs, rb, nr, a, b)
                assert np.array_equal(off, mp[mb + t])         # the kernels' lookup = the definition
                tgt = pos + 1 + off
                if kind == KIND_SRC:
                    assert 1 <= nslots <= SRC_SLOTS and (tgt >= base).all() and (tgt < base + nslots).all()
                f = lu[pos] / lu[dj]
                lu[tgt] -= lu[src] * f
                applied[mb + t] += 1
                reads.append(np.concatenate([src, [pos, dj]]))
                writes.append(tgt)
                owner.append(np.full(tgt.size, ti))
        if writes:
            wr, ow, rd = np.concatenate(writes), np.concatenate(owner), np.concatenate(reads)
            # one owner per written position
            order = np.argsort(wr, kind="stable")
            same = wr[order][1:] == wr[order][:-1]
            assert (ow[order][1:][same] == ow[order][:-1][same]).all(), f"level {l}: a position has two owners"
            assert not np.isin(rd, wr).any(), f"level {l}: a task reads what another writes"
            assert not np.isin(nw, wr).any() and not np.isin(nw, rd).any(), f"level {l}: normalization overlaps"
    if dense:
        normalize(d["norm_ptr"][lend], d["norm_ptr"][lend + 1])
        T = n - t0b
        idx = np.array([[fcp[j + 1] - T + r for j in range(t0b, n)] for r in range(T)])
        assert (fri[idx] == np.arange(t0b, n)[:, None]).all()       # the block is dense
        X = lu[idx].copy()
        for c in range(T - 1):
            X[c + 1:, c] /= X[c, c]
            X[c + 1:, c + 1:] -= np.outer(X[c + 1:, c], X[c, c + 1:])
        lu[idx] = X
    else:
        normalize(d["norm_ptr"][nl], d["norm_ptr"][nl + 1])
    # completeness: every update from a source before the block once, the
    # others never; every L entry outside the block divided once
    from_outside = np.zeros(mp.size, bool)
    for j, k, pos, mb in pairs:
        if j < t0b:
            from_outside[mb:mb + lcount[j]] = True
    assert (applied[from_outside] == 1).all() and (applied[~from_outside] == 0).all()
    is_l = np.zeros(lu.size, bool)
    for j in range(min(t0b, n)):
        is_l[diag[j] + 1:fcp[j + 1]] = True
    assert (divided[is_l] == 1).all() and (divided[~is_l] == 0).all()
    return lu, kinds


CASES = {
    "grid32_natural": lambda: synth.make("grid32_natural", 0),
    "mesh30x40_nets8": lambda: synth.CircuitMatrix(synth.CircuitSpec(30, 40, 8, 60, 0.02, 0.05, "nd"), 3),
    "mesh60x60_nets16": lambda: synth.CircuitMatrix(synth.CircuitSpec(60, 60, 16, 200, 0.02, 0.05, "nd"), 4),
}


def run_case(tmp_path, monkeypatch, m, values, mutate=None, **opts):
    path = tmp_path / "columns.bin"
    monkeypatch.setenv("GLU_DUMP_COLUMNS", str(path))
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(host_only=1, **opts))
    try:
        fcp, fri = glu.glu_get_fill(h)
    finally:
        glu.glu_destroy(h)
    d = load_columns(path)
    fcp, fri = np.asarray(fcp, np.int64), np.asarray(fri, np.int64)
    n = m.n
    if mutate is not None:
        mutate(d, fcp)
    diag = np.array([fcp[j] + np.searchsorted(fri[fcp[j]:fcp[j + 1]], j) for j in range(n)])
    # the values gathered into the filled pattern (B = P A P^T)
    lu = np.zeros(fri.size)
    pinv = np.arange(n) if m.perm is None else np.argsort(m.perm)
    cp, ri = m.colptr, m.rowidx
    for jo in range(n):
        for p in range(cp[jo], cp[jo + 1]):
            i, j = pinv[ri[p]], pinv[jo]
            lu[fcp[j] + np.searchsorted(fri[fcp[j]:fcp[j + 1]], i)] = values[p]
    # the library's value gather map (step a5) places the same values
    gs = d["gsrc"]
    assert gs.size == fri.size
    assert np.array_equal(np.where(gs >= 0, np.asarray(values)[np.maximum(gs, 0)], 0.0), lu)
    got, kinds = replay(fcp, fri, diag, lu, d)
    ref = oracle.Factorization(n, cp, ri, m.perm, values)
    bad, _ = factor_mismatches(ref.lu_colptr, ref.lu_rowidx, got, ref.lu_val)
    assert bad.size == 0
    return d, kinds


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("piece", [0, 16])
def test_column_schedule_replay_matches_oracle(tmp_path, monkeypatch, case, piece):
    m = CASES[case]()
    run_case(tmp_path, monkeypatch, m, m.values(1), piece_updates=piece)


def test_replay_covers_every_task_kind_and_the_dense_block(tmp_path, monkeypatch):
    m = CASES["mesh60x60_nets16"]()
    d, kinds = run_case(tmp_path, monkeypatch, m, m.values(2))
    assert d["ftail_t0"] < m.n                      # a dense trailing block
    assert (kinds > 0).all(), kinds                 # ROW, SRC and LANE tasks
    d0, _ = run_case(tmp_path, monkeypatch, m, m.values(2), factor_tail=0)
    assert d0["ftail_t0"] == m.n                    # the final normalization pass instead


@pytest.mark.parametrize("n", [64, 100])
def test_replay_fully_dense_matrix(tmp_path, monkeypatch, n):
    # degenerate: the whole matrix is the dense trailing block (it starts at
    # column 0, so no level runs before it)
    cp, ri, v = synth.random_pattern_matrix(n, 1.0, 31 + n)

    class M:
        pass
    m = M()
    m.n, m.colptr, m.rowidx, m.perm = n, cp, ri, None
    d, kinds = run_case(tmp_path, monkeypatch, m, v)
    assert d["ftail_t0"] == 0 and d["ftail_level"] == 0 and kinds.sum() == 0


def test_replay_triangular_patterns(tmp_path, monkeypatch):
    # degenerate: no U (no updates, only normalizations) and no L (one level)
    n = 80
    cp, ri, v = synth.random_pattern_matrix(n, 0.2, 77)

    class M:
        pass
    for keep in (np.greater_equal, np.less_equal):      # lower / upper triangle of A
        cols = np.repeat(np.arange(n), np.diff(cp))
        sel = keep(ri, cols)
        ncp = np.concatenate([[0], np.cumsum(np.bincount(cols[sel], minlength=n))]).astype(np.int32)
        m = M()
        m.n, m.colptr, m.rowidx, m.perm = n, ncp, ri[sel].astype(np.int32), None
        d, kinds = run_case(tmp_path, monkeypatch, m, v[sel])
        assert kinds.sum() == 0 and len(d["pairs"]) == 0


def test_replay_random_pattern_with_permutation(tmp_path, monkeypatch):
    cp, ri, v = synth.random_pattern_matrix(150, 0.04, 11)

    class M:
        pass
    m = M()
    m.n, m.colptr, m.rowidx = 150, cp, ri
    m.perm = np.random.default_rng(5).permutation(150).astype(np.int32)
    run_case(tmp_path, monkeypatch, m, v)


def _long_segment(d):
    return int(np.nonzero(d["segs"][:, 4] - d["segs"][:, 3] >= 2)[0][0])


def _drop_row(d, fcp):
    d["segs"][_long_segment(d), 4] -= 1                      # one update never applied


def _shift_map(d, fcp):
    s = _long_segment(d)
    d["segs"][s, 3:5] += 1                                   # rows shifted by one: the wrong rows and targets


def _wrong_pivot(d, fcp):
    s = _long_segment(d)
    other = int(np.nonzero(d["segs"][:, 1] != d["segs"][s, 1])[0][0])
    d["segs"][s, 1] = d["segs"][other, 1]                    # multiplier divided by another pivot


def _short_norm(d, fcp):
    q = int(np.nonzero(d["norms"][:, 2] - d["norms"][:, 1] >= 2)[0][0])
    d["norms"][q, 2] -= 1                                     # an L entry left undivided


def _swap_kind(d, fcp):
    l = int(np.nonzero(d["lane_ptr"] > d["row_ptr"])[0][0])  # a level with ROW tasks
    d["tasks"][d["row_ptr"][l], 2] = KIND_LANE


@pytest.mark.parametrize("mutate", [_drop_row, _shift_map, _wrong_pivot, _short_norm, _swap_kind])
def test_replay_detects_planted_mistakes(tmp_path, monkeypatch, mutate):
    m = CASES["mesh30x40_nets8"]()
    with pytest.raises(AssertionError):
        run_case(tmp_path, monkeypatch, m, m.values(1), mutate=mutate)


@pytest.mark.parametrize("seed", range(4))
def test_run_lookup_with_many_runs(seed):
    """The warp lookup moves its 32-run window along segments of up to
    hundreds of runs (runs of 1-3 rows, gaps between them); the walk too."""
    rng = np.random.default_rng(seed)
    lj = 700
    offsets = np.cumsum(rng.integers(1, 4, lj) * (rng.random(lj) < 0.6) + 1)
    runs = runs_of(offsets)
    assert len(runs) > 100
    for t0, t1 in [(0, lj), (1, lj - 1), (37, 400), (255, 257), (600, 700)]:
        rb, nr = segment_runs(runs, t0, t1)
        want = offsets[t0:t1]
        assert np.array_equal(offsets_warp(runs, rb, nr, t0, t1), want)
        assert np.array_equal(offsets_walk(runs, rb, nr, t0, t1), want)
