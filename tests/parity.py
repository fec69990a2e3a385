"""Comparison helpers for GPU-vs-oracle parity (test infrastructure)."""
import numpy as np

FACTOR_RTOL = 1e-10      # per entry, relative
BERR_TOL = 1e-12         # normwise backward error of a solve


def factor_mismatches(lu_colptr, lu_rowidx, got, ref, rtol=FACTOR_RTOL):
    """Entries of the FP64 factor that miss the per-entry bound.

    An entry passes if |got - ref| <= rtol * |ref|.  An entry whose reference
    value is small against the magnitudes that produced it (cancellation)
    passes if |got - ref| <= rtol * (|L| |U|)_ij, evaluated from the
    reference factor for that entry alone.  Returns (bad_indices,
    n_cancellation_entries).
    """
    got = np.asarray(got)
    ref = np.asarray(ref)
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
        if not (err[q] <= rtol * s):
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
