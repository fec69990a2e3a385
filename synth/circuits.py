"""Seeded synthetic circuit-like matrices (the workload stand-ins).

This module only builds inputs: a nodal conductance matrix of a 2-D resistive
mesh with optional supply nets and local controlled sources, its fill-reducing
ordering, right-hand sides and value re-draws for a fixed pattern.  It holds
none of the factorization's arithmetic and is imported by both the oracle side
(tests, bench CPU leg) and the GPU side (tests, bench), which is the only code
the two sides share.

The paper measures on SuiteSparse circuit matrices (Section IV, Table I); those
are not used here.  The generator stands in for them with the same character:
symmetric-pattern conductance stamps, a few unsymmetric entries, a handful of
high-fanout nets, nnz/n of 5-7 before fill.

Recipe (all draws from ``numpy.random.default_rng(seed)``):

* mesh ``rows x cols``, node id ``r*cols + c``; every horizontal and vertical
  edge stamps a conductance g ~ U[1e-3, 1] as ``-g`` at (u,v) and (v,u);
  a fraction ``unsym_frac`` of the edges has one side (chosen at random)
  scaled by U[0.5, 1.5], so the values are unsymmetric, the pattern is not;
* ``n_nets`` supply nets are extra unknowns numbered after the mesh; each net
  couples to ``net_fanout`` distinct random mesh nodes with a symmetric stamp
  ``-g``, g ~ U[1e-3, 1];
* a fraction ``ctrl_frac`` of mesh nodes i each get one controlled-source entry
  (i, m) with m a different node at Manhattan distance <= 2, value
  +-U[1e-3, 1] with a random sign; only (i, m) is stamped, so the pattern
  becomes unsymmetric;
* the diagonal is the row's absolute off-diagonal sum plus 1e-3;
* ordering: ``natural`` (identity) or ``nd``: geometric nested dissection of
  the grid (split the longer side at its middle line, recurse into both halves,
  then the separator line; leaves of at most ``leaf x leaf`` nodes in
  row-major order); a controlled source that straddles a separator line puts
  its far endpoint into that separator, so the order dissects the matrix
  graph; the nets come after every mesh node.

The pattern (which edges, couplings and source positions exist) depends on the
pattern seed only; ``values(seed)`` redraws every value on the fixed pattern.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, Optional

import numpy as np


@dataclasses.dataclass(frozen=True)
class CircuitSpec:
    rows: int
    cols: int
    n_nets: int = 0
    net_fanout: int = 0
    ctrl_frac: float = 0.0
    unsym_frac: float = 0.05
    order: str = "nd"          # "nd" or "natural"
    leaf: int = 8

    @property
    def n_mesh(self) -> int:
        return self.rows * self.cols

    @property
    def n(self) -> int:
        return self.n_mesh + self.n_nets


def _serving_spec(n_target: int) -> CircuitSpec:
    # grid aspect 4:5, 64 nets coupling to 0.5% of the nodes, 2% sources
    r = max(8, int(round(np.sqrt(0.8 * n_target))))
    c = max(8, int(round(n_target / r)))
    return CircuitSpec(r, c, 64, max(1, int(round(0.005 * r * c))), 0.02)


#: The workloads, named by what they are.
WORKLOADS: Dict[str, CircuitSpec] = {
    # 32x32 grid, natural order, no nets or sources: n = 1024
    "grid32_natural": CircuitSpec(32, 32, 0, 0, 0.0, 0.05, "natural"),
    # 400x500 power-grid mesh + 64 nets (0.5% fanout each) + 2% sources, ND
    "mesh400x500_nets64": CircuitSpec(400, 500, 64, 1000, 0.02, 0.05, "nd"),
    # the same generator at 100x200 (batched workload)
    "mesh100x200_nets64": CircuitSpec(100, 200, 64, 100, 0.02, 0.05, "nd"),
    # 1000x1000 mesh + 256 nets of fanout 5000 + 2% sources, ND
    "mesh1000x1000_nets256": CircuitSpec(1000, 1000, 256, 5000, 0.02, 0.05, "nd"),
}
for _n in (5_000, 20_000, 50_000, 100_000, 200_000, 500_000):
    WORKLOADS[f"serve{_n // 1000}k"] = _serving_spec(_n)


def nd_order(rows: int, cols: int, leaf: int = 8,
             couplings: Optional[tuple] = None) -> np.ndarray:
    """Geometric nested dissection of a rows x cols grid (node id r*cols+c).

    ``couplings`` = (u, v) arrays of extra mesh-to-mesh entries (controlled
    sources).  A coupling whose endpoints lie on both sides of a separator
    line would join the two halves, so its endpoint right of (or below) the
    line joins the separator; the order is then a true dissection of the
    matrix graph.
    """
    n = rows * cols
    placed = np.zeros(n, bool)
    if couplings is not None and len(couplings[0]):
        cu = np.asarray(couplings[0], np.int64)
        cv = np.asarray(couplings[1], np.int64)
        # orient every coupling so that the second endpoint is the larger id
        a, b = np.minimum(cu, cv), np.maximum(cu, cv)
        keep = a != b
        a, b = a[keep], b[keep]
    else:
        a = b = np.zeros(0, np.int64)
    ar, ac = a // cols, a % cols
    br, bc = b // cols, b % cols
    out = []
    stack = [("rect", 0, rows, 0, cols)]
    while stack:
        item = stack.pop()
        if item[0] == "emit":
            sep = item[1]
            out.append(sep)
            continue
        _, r0, r1, c0, c1 = item
        h, w = r1 - r0, c1 - c0
        if h <= 0 or w <= 0:
            continue
        rr, cc = np.meshgrid(np.arange(r0, r1), np.arange(c0, c1), indexing="ij")
        ids = (rr * cols + cc).ravel()
        if h <= leaf and w <= leaf:
            out.append(ids[~placed[ids]])
            placed[ids] = True
            continue
        inside = ((ar >= r0) & (ar < r1) & (ac >= c0) & (ac < c1) &
                  (br >= r0) & (br < r1) & (bc >= c0) & (bc < c1))
        inside &= ~placed[a] & ~placed[b]
        if w >= h:
            m = c0 + w // 2
            line = np.arange(r0, r1) * cols + m
            cross = inside & (np.minimum(ac, bc) < m) & (np.maximum(ac, bc) > m)
            far = np.where(ac > m, a, b)[cross]
            sub = [("rect", r0, r1, c0, m), ("rect", r0, r1, m + 1, c1)]
        else:
            m = r0 + h // 2
            line = m * cols + np.arange(c0, c1)
            cross = inside & (np.minimum(ar, br) < m) & (np.maximum(ar, br) > m)
            far = np.where(ar > m, a, b)[cross]
            sub = [("rect", r0, m, c0, c1), ("rect", m + 1, r1, c0, c1)]
        sep = np.concatenate([line[~placed[line]], np.unique(far[~placed[far]])])
        sep = sep[np.sort(np.unique(sep, return_index=True)[1])]
        placed[sep] = True
        # pushed in reverse: first half, second half, then the separator
        stack.append(("emit", sep))
        stack.append(sub[1])
        stack.append(sub[0])
    order = np.concatenate(out) if out else np.zeros(0, np.int64)
    assert order.size == n and np.unique(order).size == n
    return order


class CircuitMatrix:
    """A fixed sparsity pattern with value re-draws.

    Attributes (old = generator numbering, CSC with sorted unique rows):
      n, colptr[int32 n+1], rowidx[int32 nnz], perm[int32 n] (new -> old)
    """

    def __init__(self, spec: CircuitSpec, seed: int = 0):
        self.spec = spec
        self.seed = seed
        rng = np.random.default_rng(seed)
        R, C, nm = spec.rows, spec.cols, spec.n_mesh
        n = spec.n
        ids = np.arange(nm).reshape(R, C)
        eu = np.concatenate([ids[:, :-1].ravel(), ids[:-1, :].ravel()])
        ev = np.concatenate([ids[:, 1:].ravel(), ids[1:, :].ravel()])
        # net couplings: net t -> distinct random mesh nodes
        nu, nv = [], []
        for t in range(spec.n_nets):
            nodes = rng.choice(nm, size=spec.net_fanout, replace=False)
            nu.append(np.full(spec.net_fanout, nm + t, np.int64))
            nv.append(nodes.astype(np.int64))
        nu = np.concatenate(nu) if nu else np.zeros(0, np.int64)
        nv = np.concatenate(nv) if nv else np.zeros(0, np.int64)
        # controlled sources: (i, m) with 0 < |dr|+|dc| <= 2, inside the grid
        n_src = int(round(spec.ctrl_frac * nm))
        si = np.sort(rng.choice(nm, size=n_src, replace=False)) if n_src else np.zeros(0, np.int64)
        offs = np.array([(dr, dc) for dr in range(-2, 3) for dc in range(-2, 3)
                         if 0 < abs(dr) + abs(dc) <= 2])
        sm = np.empty(n_src, np.int64)
        for t, i in enumerate(si):
            r, c = divmod(int(i), C)
            while True:
                dr, dc = offs[rng.integers(len(offs))]
                if 0 <= r + dr < R and 0 <= c + dc < C:
                    sm[t] = (r + dr) * C + (c + dc)
                    break
        self._edges = (eu.astype(np.int64), ev.astype(np.int64))
        self._nets = (nu, nv)
        self._srcs = (si.astype(np.int64), sm)
        # COO of every stamp: edges both ways, nets both ways, sources one way,
        # then the diagonal
        coo_r = np.concatenate([eu, ev, nu, nv, si, np.arange(n)])
        coo_c = np.concatenate([ev, eu, nv, nu, sm, np.arange(n)])
        key = coo_c.astype(np.int64) * n + coo_r
        ukey, inv = np.unique(key, return_inverse=True)
        self.n = n
        self.nnz = int(ukey.size)
        cols = (ukey // n).astype(np.int64)
        self.rowidx = (ukey % n).astype(np.int32)
        self.colptr = np.zeros(n + 1, np.int64)
        np.add.at(self.colptr, cols + 1, 1)
        self.colptr = np.cumsum(self.colptr).astype(np.int32)
        self._inv = inv
        self._pos_row = self.rowidx.astype(np.int64)
        self._is_diag = (self._pos_row == cols)
        self._n_offdiag_coo = coo_r.size - n
        if spec.order == "natural":
            self.perm = np.arange(n, dtype=np.int32)
        else:
            self.perm = np.concatenate(
                [nd_order(R, C, spec.leaf, self._srcs), np.arange(nm, n)]).astype(np.int32)

    # ------------------------------------------------------------------ values
    def values(self, seed: int, sigma: float = 0.0, base_seed: Optional[int] = None) -> np.ndarray:
        """Values in CSC order.

        ``sigma == 0``: every stamp drawn from ``seed``.  ``sigma > 0``: stamps
        drawn from ``base_seed`` then every conductance multiplied by
        exp(N(0, sigma)) drawn from ``seed`` (a Monte-Carlo corner); the
        diagonal is recomputed either way.
        """
        spec = self.spec
        ne = self._edges[0].size
        nn = self._nets[0].size
        ns = self._srcs[0].size
        rng = np.random.default_rng(seed if sigma == 0.0 else base_seed)
        g = rng.uniform(1e-3, 1.0, ne)
        scale = np.ones(ne)
        pick = rng.random(ne) < spec.unsym_frac
        side = rng.random(ne) < 0.5
        s = rng.uniform(0.5, 1.5, ne)
        gn = rng.uniform(1e-3, 1.0, nn)
        gs = rng.uniform(1e-3, 1.0, ns) * np.where(rng.random(ns) < 0.5, -1.0, 1.0)
        if sigma > 0.0:
            r2 = np.random.default_rng(seed)
            g = g * np.exp(r2.normal(0.0, sigma, ne))
            gn = gn * np.exp(r2.normal(0.0, sigma, nn))
            gs = gs * np.exp(r2.normal(0.0, sigma, ns))
        guv = -g * np.where(pick & side, s, scale)      # entry (u, v)
        gvu = -g * np.where(pick & ~side, s, scale)     # entry (v, u)
        off = np.concatenate([guv, gvu, -gn, -gn, gs])
        vals = np.bincount(self._inv[: off.size], weights=off, minlength=self.nnz)
        absrow = np.bincount(self._pos_row, weights=np.abs(vals) * ~self._is_diag,
                             minlength=self.n)
        vals[self._is_diag] = absrow[self._pos_row[self._is_diag]] + 1e-3
        return vals

    def stats(self) -> dict:
        return {"n": self.n, "nnzA": self.nnz, "rows": self.spec.rows,
                "cols": self.spec.cols, "nets": self.spec.n_nets,
                "net_fanout": self.spec.net_fanout,
                "ctrl_sources": int(self._srcs[0].size), "order": self.spec.order}


def rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """Right-hand sides U[-1, 1], column-major (nrhs, n) as a C array."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, (nrhs, n))


def make(name: str, seed: int = 0) -> CircuitMatrix:
    return CircuitMatrix(WORKLOADS[name], seed)


def random_pattern_matrix(n: int, density: float, seed: int, *, dominant: bool = True,
                          extra: int = 0) -> tuple:
    """Small random square CSC with a full diagonal (test inputs).

    Off-diagonal entries present with probability ``density``; values
    U[-1, 1]; with ``dominant`` the diagonal is 1 + the larger of the row and
    column absolute sums, so no-pivot elimination is stable and partial
    pivoting would not swap rows.  Returns (colptr, rowidx, values) int32/f64.
    """
    rng = np.random.default_rng(seed)
    M = (rng.random((n, n)) < density) * rng.uniform(-1.0, 1.0, (n, n))
    np.fill_diagonal(M, 0.0)
    mask = (M != 0.0)
    for _ in range(extra):  # a few explicit structural zeros
        i, j = rng.integers(n, size=2)
        if i != j:
            mask[i, j] = True
            M[i, j] = 0.0
    d = 1.0 + np.maximum(np.abs(M).sum(0), np.abs(M).sum(1))
    if not dominant:
        d = rng.uniform(0.5, 1.5, n) * np.where(rng.random(n) < 0.5, -1, 1)
    np.fill_diagonal(M, d)
    np.fill_diagonal(mask, True)
    colptr = np.zeros(n + 1, np.int32)
    rows, vals = [], []
    for j in range(n):
        r = np.nonzero(mask[:, j])[0]
        rows.append(r)
        vals.append(M[r, j])
        colptr[j + 1] = colptr[j] + r.size
    return colptr, np.concatenate(rows).astype(np.int32), np.concatenate(vals)
