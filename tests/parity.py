"""Comparison helpers for GPU-vs-oracle parity (test infrastructure)."""
import numpy as np

FACTOR_RTOL = 1e-10      # per entry, relative
BERR_TOL = 1e-12         # normwise backward error of a solve
U32 = 2.0 ** -24         # unit roundoff of FP32


def _factor_parts(lu_colptr, lu_rowidx, vals):
    """Unit lower L and upper U (scipy CSC, float64) of A_s = L + U - I."""
    import scipy.sparse as sp
    n = lu_colptr.size - 1
    col = np.repeat(np.arange(n), np.diff(lu_colptr))
    row = np.asarray(lu_rowidx)
    vals = np.asarray(vals, np.float64)
    low = row > col
    L = sp.csc_matrix((vals[low], (row[low], col[low])), shape=(n, n)) + sp.identity(n, format="csc")
    U = sp.csc_matrix((vals[~low], (row[~low], col[~low])), shape=(n, n))
    return L.tocsc(), U.tocsc()


def update_counts(lu_colptr, lu_rowidx):
    """Per entry (i, j) of the pattern, a bound on the number of updates
    l_ik u_kj it takes: min(#U entries of column j, #L entries of row i)."""
    n = lu_colptr.size - 1
    col = np.repeat(np.arange(n), np.diff(lu_colptr))
    row = np.asarray(lu_rowidx)
    ucnt = np.bincount(col[row < col], minlength=n)
    lrow = np.bincount(row[row > col], minlength=n)
    return np.minimum(ucnt[col], lrow[row])


def _values_on(P, i, jc, n):
    """P[i, jc] for pattern entries (i, jc) that lie in P's structure (CSC,
    any order): one sorted-key search, no scipy fancy indexing."""
    P = P.tocsc()
    P.sort_indices()
    pc = np.repeat(np.arange(P.shape[1]), np.diff(P.indptr)).astype(np.int64)
    keys = pc * n + P.indices
    want = jc.astype(np.int64) * n + i
    at = np.searchsorted(keys, want)
    at = np.minimum(at, max(keys.size - 1, 0))
    hit = keys.size > 0
    out = np.where(hit & (keys[at] == want), P.data[at] if keys.size else 0.0, 0.0)
    return out


def fp32_factor_check(n, colptr, rowidx, values, perm, lu_colptr, lu_rowidx, got32, ref64, cols=None,
                      no_cancel=0.5, fwd_safety=8.0):
    """FP32 factors (got32) of B = P A P^T against rounding-error theory and
    the FP64 oracle's factors (ref64), on the columns ``cols`` (sorted; all
    if None).

    The model of FP32 arithmetic: fl(x op y) = (x op y)(1 + d) + e, |d| <= u
    = 2^-24, |e| <= 2^-126: the level kernels add into the target entries
    with FP32 reductions in L2, which flush subnormal inputs and results to
    zero (PTX red.add.f32), so underflow is not gradual there.
    1. Componentwise backward error, the theorem for LU in floating point
       (Higham, Accuracy and Stability of Numerical Algorithms, Thm 9.3):
       the computed factors of the FP32-rounded matrix B32 satisfy
       |B32 - L U| <= gamma_m |L||U| entrywise, gamma_m = m u / (1 - m u), m
       the number of rounded operations along the entry's recurrence (its
       c_ij updates, the subtraction from b_ij and, for L, the division),
       m = c_ij + 2, whatever the summation order; the underflow terms add at
       most m 2^-126 max(1, |U|max).  With |B - B32| <= u |B|:
       |B - L U|_ij <= u |b_ij| + gamma_m (|L||U|)_ij + m 2^-126 max(1, |U|max).
    2. Forward error against the FP64 factors, on the entries whose FP64 value
       is not the result of cancellation (|x_ref| >= no_cancel *
       (|L_ref||U_ref|)_ij, for L divided by |u_jj|): the entry's own rounding
       contributes m u relative; errors its operands inherited from
       cancellation elsewhere can add more, which no per-entry bound from the
       pattern alone covers, so this part is a statistic: the share of clean
       entries with |x - x_ref| <= fwd_safety * m (u |x_ref| + 2^-126
       max(1, |U|max)) (the last term: FP32's subnormal range, where relative
       accuracy ends) and the largest relative difference among them.
    Returns a dict: backward_worst (<= 1 passes), forward_within (share),
    forward_worst_rel, counts."""
    import scipy.sparse as sp
    cp, ri, v = np.asarray(colptr), np.asarray(rowidx), np.asarray(values, np.float64)
    A = sp.csc_matrix((v, ri, cp), shape=(n, n))
    p = np.arange(n) if perm is None else np.asarray(perm)
    B = A[p, :][:, p].tocsc()
    Lh, Uh = _factor_parts(lu_colptr, lu_rowidx, got32)
    Lr, Ur = _factor_parts(lu_colptr, lu_rowidx, ref64)
    cols = np.arange(n) if cols is None else np.asarray(cols)
    c = update_counts(lu_colptr, lu_rowidx)
    col_of = np.repeat(np.arange(n), np.diff(lu_colptr))
    q = np.nonzero(np.isin(col_of, cols))[0]
    i, j = np.asarray(lu_rowidx)[q].astype(np.int64), col_of[q]
    pos = np.searchsorted(cols, j)
    Us, Urs = Uh[:, cols], Ur[:, cols]
    LUv = _values_on(Lh @ Us, i, pos, n)
    Mv = _values_on(abs(Lh) @ abs(Us), i, pos, n)
    Bv = _values_on(B[:, cols], i, pos, n)
    Mr = _values_on(abs(Lr) @ abs(Urs), i, pos, n)
    m = c[q] + 2.0
    gamma = m * U32 / (1.0 - m * U32)
    umax = max(1.0, float(np.abs(Uh.diagonal()).max()) if n else 1.0)
    bound = U32 * np.abs(Bv) + gamma * Mv + m * 2.0 ** -126 * umax
    back = np.abs(Bv - LUv) / bound
    x, xr = np.asarray(got32, np.float64)[q], np.asarray(ref64)[q]
    low = i > j
    dj = np.abs(np.asarray(Ur.diagonal()))[j]
    scale = np.where(low, Mr / np.where(dj > 0, dj, 1.0), Mr)
    clean = np.abs(xr) >= no_cancel * scale
    fbound = fwd_safety * m * (U32 * np.abs(xr) + 2.0 ** -126 * umax)
    fwd = np.abs(x - xr) / fbound
    tiny = np.abs(xr) < 2.0 ** -100            # relative differences mean nothing down there
    rel = np.abs(x - xr) / np.maximum(np.abs(xr), 1e-300)
    return {"backward_worst": float(back.max()) if back.size else 0.0,
            "forward_within": float((fwd[clean] <= 1.0).mean()) if clean.any() else 1.0,
            "forward_worst_rel": float(rel[clean & ~tiny].max()) if (clean & ~tiny).any() else 0.0,
            "entries": int(q.size), "clean_entries": int(clean.sum()),
            "max_rel_err": float((np.abs(x - xr) / np.maximum(np.abs(xr), 1e-30)).max())}


def factor_mismatches(lu_colptr, lu_rowidx, got, ref, rtol=FACTOR_RTOL):
    """Entries of the factor that miss the per-entry bound (rtol: a scalar or
    one value per entry).

    An entry passes if |got - ref| <= rtol * |ref|.  An entry whose reference
    value is small against the magnitudes that produced it (cancellation)
    passes if |got - ref| <= rtol * (|L| |U|)_ij, evaluated from the
    reference factor for that entry alone.  Returns (bad_indices,
    n_cancellation_entries).
    """
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref)
    rtol = np.broadcast_to(np.asarray(rtol, np.float64), ref.shape)
    err = np.abs(got - ref)
    bad = np.nonzero(~(err <= rtol * np.abs(ref)))[0]
    if bad.size == 0:
        return bad, 0
    col_of = np.searchsorted(lu_colptr, bad, side="right") - 1
    still = []
    canc = 0
    for q, j in zip(bad, col_of):
        i = lu_rowidx[q]
        # (|L||U|)_ij = sum_k |L(i,k)| |U(k,j)|, k <= min(i,j), L(i,i) = 1
        cb, ce = lu_colptr[j], lu_colptr[j + 1]
        rows_j = lu_rowidx[cb:ce]
        vals_j = np.abs(ref[cb:ce])
        kmax = min(i, j)
        s = 0.0
        for kk in range(rows_j.size):
            k = rows_j[kk]
            if k > kmax:
                break
            if k == i:
                s += vals_j[kk]          # L(i,i) = 1 times U(i,j)
                continue
            kb, ke = lu_colptr[k], lu_colptr[k + 1]
            pos = kb + np.searchsorted(lu_rowidx[kb:ke], i)
            if pos < ke and lu_rowidx[pos] == i:
                s += abs(ref[pos]) * vals_j[kk]
        if i > j:  # L(i,j) = value / U(j,j): scale by the pivot
            d = abs(ref[cb + np.searchsorted(rows_j, j)])
            s = s / d if d > 0 else np.inf
        canc += 1
        if not (err[q] <= rtol[q] * s):
            still.append(q)
    return np.asarray(still, np.int64), canc


def backward_error(n, colptr, rowidx, aval, b, x):
    """max over right-hand sides of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    import oracle
    b = np.atleast_2d(b)
    x = np.atleast_2d(x)
    r = oracle.residual(n, colptr, rowidx, aval, b, x)
    absA = np.zeros(n)
    np.add.at(absA, rowidx, np.abs(aval))
    anorm = absA.max() if n else 0.0
    out = 0.0
    for k in range(b.shape[0]):
        den = anorm * np.abs(x[k]).max() + np.abs(b[k]).max()
        out = max(out, np.abs(r[k]).max() / den if den > 0 else 0.0)
    return out
