"""Host-side check of the dataflow solve schedule (no GPU).

The schedule the analysis builds for the one-launch triangular solves is
replayed on the CPU: every item must come after everything it reads (rows,
partial-sum chunks), every entry of L and U outside the dense tail must be
read exactly once (by a row's dot product, a chunk, or the triangle sweep of
a dense diagonal block), and every row before the tail must be produced once
per sweep.  The dump is the library's diagnostic copy of the schedule
(environment variables GLU_DUMP_DF and GLU_DUMP_DF_BATCHED at glu_analyze).
"""
import numpy as np
import pytest

import synth
from paper_1908_00204_gb300 import glu


def row_views(cp, ri, n):
    """Strict lower rows of L (columns ascending) and strict upper rows of U."""
    col = np.repeat(np.arange(n, dtype=np.int64), np.diff(cp))
    low = ri > col
    up = ri < col
    # L row view: entries (i = ri, j = col) with i > j, sorted by (i, j)
    li, lj = ri[low].astype(np.int64), col[low]
    o = np.lexsort((lj, li))
    lptr = np.zeros(n + 1, np.int64)
    np.add.at(lptr, li + 1, 1)
    lptr = np.cumsum(lptr)
    # U row view: entries (i = ri, k = col) with i < k, sorted by (i, k)
    ui, uk = ri[up].astype(np.int64), col[up]
    o2 = np.lexsort((uk, ui))
    uptr = np.zeros(n + 1, np.int64)
    np.add.at(uptr, ui + 1, 1)
    uptr = np.cumsum(uptr)
    return lptr, lj[o], uptr, uk[o2]


def load_dump(path):
    w = np.fromfile(path, np.int64)
    nitems, nfwd, nfc, nbc, nsf, nsb, t0 = (int(x) for x in w[:7])
    q = 7
    items = w[q:q + 8 * nitems].reshape(nitems, 8)
    q += 8 * nitems
    fch = w[q:q + 2 * nfc].reshape(nfc, 2)
    q += 2 * nfc
    bch = w[q:q + 2 * nbc].reshape(nbc, 2)
    q += 2 * nbc
    snf = w[q:q + nsf]
    q += nsf
    snb = w[q:q + nsb]
    return items, nfwd, fch, bch, snf, snb, t0


RSPLIT_B = 4   # copies of a dense diagonal block item in the batched schedule


def block_copies(items, nfwd):
    """The batched schedule lists each dense diagonal block RSPLIT_B times in
    a row, copy q (field 5) taking the right-hand sides r = q mod RSPLIT_B,
    with the block's ordinal (field 6) for its completion counter.  Checks
    that layout and returns the list with one item per block."""
    keep, k, nb, nf = [], 0, 0, 0
    while k < len(items):
        it = items[k]
        if it[4] & 4:
            group = items[k:k + RSPLIT_B]
            assert len(group) == RSPLIT_B
            assert (group[:, :5] == it[:5]).all(), "copies differ"
            assert group[:, 5].tolist() == list(range(RSPLIT_B))
            assert (group[:, 6] == nb).all(), "block ordinals not consecutive"
            nb += 1
            step = RSPLIT_B
        else:
            assert it[5] == 0 and it[6] == 0
            step = 1
        keep.append(it)
        if k < nfwd:
            nf += 1
        k += step
    return np.array(keep, dtype=items.dtype).reshape(-1, 8), nf


def replay(n, t0, items, ptr, cols, chunks, snx, backward):
    done = np.zeros(n, bool)
    if backward:
        done[t0:] = True                      # the tail is solved before
    chunk_done = np.zeros(len(chunks), bool)
    read = np.zeros(len(cols), np.int32)      # times each entry is read
    nblocks = 0
    for row, cb, ce, ch, fl, *_ in items:
        if fl & 2:                            # a chunk
            p0, p1 = chunks[ch]
            assert not chunk_done[ch]
            assert done[cols[p0:p1]].all(), "chunk before a row it reads"
            read[p0:p1] += 1
            chunk_done[ch] = True
        elif fl & 4:                          # a dense diagonal block [row, cb)
            c0, c1, off = row, cb, ce
            nblocks += 1
            assert 4 <= c1 - c0 <= 32
            for r in range(c0, c1):
                b, e = ptr[r], ptr[r + 1]
                if backward:
                    inner = np.arange(r + 1, c1)
                    assert np.array_equal(cols[b:b + len(inner)], inner), "U block not dense"
                    b += len(inner)
                else:
                    inner = np.arange(c0, r)
                    assert np.array_equal(cols[e - len(inner):e], inner), "L block not dense"
                    e -= len(inner)
                cs, cend = snx[off + r - c0], snx[off + r - c0 + 1]
                assert chunk_done[cs:cend].all(), "block before its chunks"
                pos = b
                for c in range(cs, cend):     # the chunks tile the outside entries
                    assert chunks[c][0] == pos
                    pos = chunks[c][1]
                assert pos == e
                # entries inside the block are read by the sweep
                if backward:
                    read[ptr[r]:ptr[r] + (c1 - 1 - r)] += 1
                else:
                    read[ptr[r + 1] - (r - c0):ptr[r + 1]] += 1
            assert not done[c0:c1].any()
            done[c0:c1] = True
        else:                                 # a row
            b, e = ptr[row], ptr[row + 1]
            if ce > cb:
                assert chunk_done[cb:ce].all(), "row before its chunks"
                pos = b
                for c in range(cb, ce):
                    assert chunks[c][0] == pos
                    pos = chunks[c][1]
                assert pos == e
            else:
                assert done[cols[b:e]].all(), "row before a row it reads"
                read[b:e] += 1
            assert not done[row]
            done[row] = True
    assert done[:t0].all(), "a row is never produced"
    return read, nblocks


class _Pattern:
    def __init__(self, n, colptr, rowidx):
        self.n, self.colptr, self.rowidx, self.perm = n, colptr, rowidx, None


def _triangle(n, upper):
    cp, ri, _ = synth.random_pattern_matrix(n, 0.2, 78)
    cols = np.repeat(np.arange(n), np.diff(cp))
    sel = ri <= cols if upper else ri >= cols
    ncp = np.concatenate([[0], np.cumsum(np.bincount(cols[sel], minlength=n))]).astype(np.int32)
    return _Pattern(n, ncp, ri[sel].astype(np.int32))


@pytest.mark.parametrize("variant", ["single", "batched"])
@pytest.mark.parametrize("case", ["grid32", "mesh_nets", "mesh100x200", "dense100", "lower", "upper"])
def test_df_schedule_topological_and_complete(tmp_path, monkeypatch, case, variant):
    # "batched": the schedule of the batched solves (a dense tail of at most
    # 736 rows, each block item in RSPLIT_B copies), dumped by
    # GLU_DUMP_DF_BATCHED
    if case == "grid32":
        m = synth.make("grid32_natural", 0)
    elif case == "mesh_nets":
        m = synth.CircuitMatrix(synth.CircuitSpec(30, 40, 8, 60, 0.02, 0.05, "nd"), 3)
    elif case == "dense100":
        # degenerate: the dense tail is the whole matrix, no dataflow item
        cp, ri, _ = synth.random_pattern_matrix(100, 1.0, 5)
        m = _Pattern(100, cp, ri)
    elif case in ("lower", "upper"):
        # degenerate: one of the two sweeps has only diagonal rows
        m = _triangle(90, case == "upper")
    else:
        m = synth.make("mesh100x200_nets64", 1)
    path = tmp_path / "df.bin"
    monkeypatch.setenv("GLU_DUMP_DF" if variant == "single" else "GLU_DUMP_DF_BATCHED", str(path))
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(host_only=1))
    cp, ri = glu.glu_get_fill(h)
    glu.glu_destroy(h)
    items, nfwd, fch, bch, snf, snb, t0 = load_dump(path)
    if variant == "batched":
        items, nfwd = block_copies(items, nfwd)
    n = m.n
    lptr, lcol, uptr, ucol = row_views(np.asarray(cp, np.int64), np.asarray(ri, np.int64), n)
    fwd = [tuple(int(x) for x in r) for r in items[:nfwd]]
    bwd = [tuple(int(x) for x in r) for r in items[nfwd:]]
    assert all(not (r[4] & 1) for r in fwd) and all(r[4] & 1 for r in bwd)
    # forward: rows before the tail; the tail rows' outside entries are chunks
    fwd_rows = [r for r in fwd if not (r[4] & 2)]
    assert all(r[0] < t0 for r in fwd_rows)
    read_f, nbf = replay(n, t0, fwd, lptr, lcol, fch, snf, backward=False)
    rows_of = np.repeat(np.arange(n), np.diff(lptr))
    before_tail = (rows_of < t0) | (lcol < t0)
    assert (read_f[before_tail] == 1).all()
    assert (read_f[~before_tail] == 0).all()  # inside the tail: the tail kernel
    read_b, nbb = replay(n, t0, bwd, uptr, ucol, bch, snb, backward=True)
    urows = np.repeat(np.arange(n), np.diff(uptr))
    assert (read_b[urows < t0] == 1).all()
    assert nbf == nbb
    if case == "mesh100x200":
        assert nbf > 10                       # separators give dense blocks
    if case == "dense100":
        assert t0 == 0 and len(items) == 0


def test_df_schedule_without_blocks(tmp_path, monkeypatch):
    m = synth.CircuitMatrix(synth.CircuitSpec(30, 40, 8, 60, 0.02, 0.05, "nd"), 3)
    path = tmp_path / "df.bin"
    monkeypatch.setenv("GLU_DUMP_DF", str(path))
    h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(host_only=1, solve_blocks=0))
    glu.glu_destroy(h)
    items, nfwd, fch, bch, snf, snb, t0 = load_dump(path)
    assert len(snf) == 0 and len(snb) == 0
    assert not (items[:, 4] & 4).any()


def test_schedule_independent_of_analysis_threads(tmp_path, monkeypatch):
    """The symbolic fill, the row views, the gather map and both
    factorization schedules are built on host threads; the result must not
    depend on their number (the fill, the full column schedule with its
    gather map, the dataflow items and the supernodal schedule compared
    between 1, 2 and 7 threads)."""
    m = synth.make("mesh100x200_nets64", 1)
    out = {}
    for nth in (1, 2, 7):
        monkeypatch.setenv("GLU_ANALYZE_THREADS", str(nth))
        monkeypatch.setenv("GLU_DUMP_COLUMNS", str(tmp_path / f"c{nth}.bin"))
        monkeypatch.setenv("GLU_DUMP_DF", str(tmp_path / f"d{nth}.bin"))
        h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(host_only=1))
        cp, ri = glu.glu_get_fill(h)
        out[nth] = [np.asarray(cp).tobytes(), np.asarray(ri).tobytes(),
                    (tmp_path / f"c{nth}.bin").read_bytes(), (tmp_path / f"d{nth}.bin").read_bytes()]
        glu.glu_destroy(h)
        monkeypatch.delenv("GLU_DUMP_COLUMNS")
        monkeypatch.setenv("GLU_DUMP_BLOCKS", str(tmp_path / f"b{nth}.bin"))
        h = glu.glu_analyze(m.n, m.colptr, m.rowidx, m.perm, glu.default_options(host_only=1, factor_blocks=1))
        out[nth].append((tmp_path / f"b{nth}.bin").read_bytes())
        glu.glu_destroy(h)
        monkeypatch.delenv("GLU_DUMP_BLOCKS")
    assert out[1] == out[2] == out[7]
