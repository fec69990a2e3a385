"""The trailing-update tiles of the factorization's dense block
(paper_1908_00204_gb300/csrc/kernels_dense.cu, step C), replayed on the CPU
with the kernel's index arithmetic: the tile width of least makespan, block
0's tile over the next diagonal block, and the mapping of the remaining tiles
onto the other blocks.  Every entry of the m x m trailing block must be
updated exactly once, for any block count, and block 0's tile must hold the
whole next diagonal block (the look-ahead factorization reads nothing else)."""
import pytest

DT_TM, DT_TN, DT_NB = 32, 64, 32


def tile_width(m, g):
    """dt_tile_width: of 64, 32 and 16 columns, the fewest rounds of equal
    tiles times a tile's width, the widest among equals."""
    ntr = (m + DT_TM - 1) // DT_TM
    best, best_cost = DT_TN, None
    for tn in (64, 32, 16):
        tiles = ntr * ((m + tn - 1) // tn)
        cost = ((tiles + g - 1) // g) * tn
        if best_cost is None or cost < best_cost:
            best, best_cost = tn, cost
    return best


def tiles(m, grid):
    """(block, r0, k0, width) of every tile of one panel's update, offsets
    relative to the first trailing row and column (c1 = 0)."""
    gr = grid - 1 if grid > 1 else 1
    tn = tile_width(m, gr)
    ntr = (m + DT_TM - 1) // DT_TM
    n0 = (m - DT_NB + tn - 1) // tn if m > DT_NB else 0
    nrow = (m + tn - 1) // tn
    nreg = n0 + (ntr - 1) * nrow
    out = [(0, 0, 0, DT_NB)]                          # block 0: the next diagonal block
    for b in (range(1, grid) if grid > 1 else [0]):
        u = b - 1 if grid > 1 else 0
        while u < nreg:
            if u < n0:
                r0, k0 = 0, DT_NB + u * tn
            else:
                q = u - n0
                r0, k0 = (1 + q // nrow) * DT_TM, (q % nrow) * tn
            out.append((b, r0, k0, tn))
            u += gr
    return out


@pytest.mark.parametrize("grid", [1, 2, 7, 152])
def test_every_entry_updated_once(grid):
    for m in list(range(1, 140)) + [233, 263, 434, 465, 900, 1700]:
        seen = {}
        for b, r0, k0, w in tiles(m, grid):
            for r in range(r0, min(r0 + DT_TM, m)):
                for k in range(k0, min(k0 + w, m)):
                    assert (r, k) not in seen, (m, grid, r, k)
                    seen[(r, k)] = b
        assert len(seen) == m * m, (m, grid)
        # block 0 owns the whole next diagonal block
        nb = min(DT_NB, m)
        assert all(seen[(r, k)] == 0 for r in range(nb) for k in range(nb))
        if grid > 1:
            # and nothing else: the look-ahead starts right after its one tile
            assert sum(1 for t in tiles(m, grid) if t[0] == 0) == 1


def test_tile_width_spreads_the_work():
    # a tall trailing block on the full grid: narrow tiles fill the blocks
    assert tile_width(434, 151) == 16
    # the chosen width has the least rounds x width of the three, the widest
    # among equals
    for m in range(1, 2000, 7):
        for g in (1, 7, 151):
            ntr = (m + 31) // 32
            cost = {w: ((ntr * ((m + w - 1) // w) + g - 1) // g) * w for w in (64, 32, 16)}
            tn = tile_width(m, g)
            assert cost[tn] == min(cost.values())
            assert tn == max(w for w in cost if cost[w] == cost[tn])
