/*
 * glu_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of what the GLU3.0 method
 * computes (Peng & Tan, "GLU3.0: Fast GPU-based Parallel Sparse LU
 * Factorization for Circuit Simulation"), used to check the CUDA library.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it; the library never does.  It shares no code with the library.
 *
 * Compiled with -O2 -ffp-contract=off: every multiply and subtract is rounded
 * separately, in IEEE double precision.
 *
 * Conventions: 0-based indices; CSC with sorted, duplicate-free row indices;
 * B = P A P^T with B(i,j) = A(perm[i], perm[j]) (perm maps new -> old).
 * The factor is stored as one CSC array A_s = L + U - I over the filled
 * pattern (Section II-A): strict lower part = L (unit diagonal implied),
 * upper part including the diagonal = U.
 *
 * Functions that produce variable-size output malloc it; the caller frees it
 * with oracle_free().  Error codes: 0 ok, -1 invalid input, -2 structurally
 * singular (missing diagonal), -3 zero pivot, -4 non-finite pivot or value,
 * -5 out of memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_INVALID -1
#define OR_STRUCT_SINGULAR -2
#define OR_ZERO_PIVOT -3
#define OR_NONFINITE -4
#define OR_OOM -5

void oracle_free(void *p) { free(p); }

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* ---------------------------------------------------------------------------
 * Input check and symmetric permutation (the preprocessing step of the flow
 * in Section II-C; the permutation is supplied by the caller).
 * bsrc[p] = index in A's arrays of B's entry p.
 * ------------------------------------------------------------------------- */
int oracle_permute(int32_t n, const int32_t *colptr, const int32_t *rowidx,
                   const int32_t *perm, int32_t *bcolptr, int32_t *browidx,
                   int64_t *bsrc) {
    if (n < 0) return OR_INVALID;
    if (colptr[0] != 0) return OR_INVALID;
    for (int32_t j = 0; j < n; j++) {
        if (colptr[j + 1] < colptr[j]) return OR_INVALID;
        for (int32_t p = colptr[j]; p < colptr[j + 1]; p++) {
            if (rowidx[p] < 0 || rowidx[p] >= n) return OR_INVALID;
            if (p > colptr[j] && rowidx[p] <= rowidx[p - 1]) return OR_INVALID;
        }
    }
    int32_t *iperm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!iperm) return OR_OOM;
    for (int32_t i = 0; i < n; i++) iperm[i] = -1;
    for (int32_t i = 0; i < n; i++) {
        if (perm[i] < 0 || perm[i] >= n || iperm[perm[i]] != -1) { free(iperm); return OR_INVALID; }
        iperm[perm[i]] = i;
    }
    bcolptr[0] = 0;
    for (int32_t j = 0; j < n; j++) {
        int32_t oj = perm[j];
        int32_t len = colptr[oj + 1] - colptr[oj];
        int32_t base = bcolptr[j];
        bcolptr[j + 1] = base + len;
        /* insertion sort of the mapped rows, carrying the source index */
        for (int32_t t = 0; t < len; t++) {
            int32_t p = colptr[oj] + t;
            int32_t r = iperm[rowidx[p]];
            int32_t u = t;
            while (u > 0 && browidx[base + u - 1] > r) {
                browidx[base + u] = browidx[base + u - 1];
                bsrc[base + u] = bsrc[base + u - 1];
                u--;
            }
            browidx[base + u] = r;
            bsrc[base + u] = p;
        }
    }
    free(iperm);
    /* every column of B must hold its diagonal */
    for (int32_t j = 0; j < n; j++) {
        int found = 0;
        for (int32_t p = bcolptr[j]; p < bcolptr[j + 1]; p++) if (browidx[p] == j) found = 1;
        if (!found) return OR_STRUCT_SINGULAR;
    }
    return OR_OK;
}

/* ---------------------------------------------------------------------------
 * Symbolic fill-in (Section II-A: the left-looking method allows the fill of
 * L and U to be found before the numeric work).  Column j of A_s is the set
 * of rows reached from struct(B(:,j)) in the graph with an edge k -> i for
 * every L(i,k) != 0, k < j; only nodes k < j are expanded (Gilbert & Peierls).
 * Plain depth-first search, no pruning.  Rows are returned sorted.
 * ------------------------------------------------------------------------- */
int oracle_symbolic(int32_t n, const int32_t *bcolptr, const int32_t *browidx,
                    int64_t **out_colptr, int32_t **out_rowidx, int64_t *out_nnz) {
    int64_t cap = (int64_t)bcolptr[n] * 2 + 16;
    int64_t *cp = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t *ri = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    /* L pattern (strict lower) of finished columns: lptr[k]..lend[k] in ri */
    int64_t *lbeg = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int64_t *spos = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t *found = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!cp || !ri || !lbeg || !mark || !stack || !spos || !found) {
        free(cp); free(ri); free(lbeg); free(mark); free(stack); free(spos); free(found);
        return OR_OOM;
    }
    for (int32_t i = 0; i < n; i++) mark[i] = -1;
    cp[0] = 0;
    for (int32_t j = 0; j < n; j++) {
        int32_t nf = 0;
        for (int32_t p = bcolptr[j]; p < bcolptr[j + 1]; p++) {
            int32_t s = browidx[p];
            if (mark[s] == j) continue;
            /* iterative DFS from s */
            int32_t top = 0;
            stack[0] = s;
            mark[s] = j;
            found[nf++] = s;
            spos[0] = (s < j) ? lbeg[s] : 0;
            while (top >= 0) {
                int32_t v = stack[top];
                if (v >= j) { top--; continue; }           /* not expanded */
                int64_t end = cp[v + 1];
                int64_t q = spos[top];
                int pushed = 0;
                while (q < end) {
                    int32_t w = ri[q++];
                    if (mark[w] != j) {
                        spos[top] = q;
                        mark[w] = j;
                        found[nf++] = w;
                        top++;
                        stack[top] = w;
                        spos[top] = (w < j) ? lbeg[w] : 0;
                        pushed = 1;
                        break;
                    }
                }
                if (!pushed) top--;
            }
        }
        qsort(found, (size_t)nf, sizeof(int32_t), cmp_i32);
        if (cp[j] + nf > cap) {
            while (cp[j] + nf > cap) cap *= 2;
            int32_t *nri = (int32_t *)realloc(ri, sizeof(int32_t) * (size_t)cap);
            if (!nri) { free(cp); free(ri); free(lbeg); free(mark); free(stack); free(spos); free(found); return OR_OOM; }
            ri = nri;
        }
        int64_t base = cp[j];
        int64_t lb = -1;
        for (int32_t t = 0; t < nf; t++) {
            ri[base + t] = found[t];
            if (lb < 0 && found[t] > j) lb = base + t;
        }
        cp[j + 1] = base + nf;
        lbeg[j] = (lb < 0) ? cp[j + 1] : lb;
        /* the diagonal must be in the pattern: it always is, since B has it */
    }
    free(lbeg); free(mark); free(stack); free(spos); free(found);
    *out_colptr = cp;
    *out_rowidx = ri;
    *out_nnz = cp[n];
    return OR_OK;
}

/* ---------------------------------------------------------------------------
 * Relaxed column dependency detection, Algorithm 4 (Section III-A):
 * column k depends on i < k if (a) A_s(i,k) != 0 (an entry of U above the
 * diagonal) and column i of L is not empty ("looking up"), or (b)
 * A_s(k,i) != 0 (an entry of L left of the diagonal, "looking left").
 * The list of each k is a set, returned in ascending order.
 * ------------------------------------------------------------------------- */
int oracle_deps(int32_t n, const int64_t *cp, const int32_t *ri,
                int64_t **out_ptr, int32_t **out_idx) {
    /* has_l[i]: column i of L holds an entry below the diagonal */
    char *has_l = (char *)calloc((size_t)n + 1, 1);
    /* row view of L: for each row k, the columns i < k with A_s(k,i) != 0 */
    int64_t *rp = (int64_t *)calloc((size_t)n + 2, sizeof(int64_t));
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!has_l || !rp || !mark || !tmp) { free(has_l); free(rp); free(mark); free(tmp); return OR_OOM; }
    int64_t nl = 0;
    for (int32_t i = 0; i < n; i++)
        for (int64_t p = cp[i]; p < cp[i + 1]; p++)
            if (ri[p] > i) { has_l[i] = 1; rp[ri[p] + 1]++; nl++; }
    for (int32_t k = 0; k < n; k++) rp[k + 1] += rp[k];
    int32_t *rc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nl > 0 ? nl : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!rc || !fill) { free(has_l); free(rp); free(mark); free(tmp); free(rc); free(fill); return OR_OOM; }
    for (int32_t k = 0; k < n; k++) fill[k] = rp[k];
    for (int32_t i = 0; i < n; i++)
        for (int64_t p = cp[i]; p < cp[i + 1]; p++)
            if (ri[p] > i) rc[fill[ri[p]]++] = i;
    free(fill);

    int64_t cap = nl * 2 + 16, cnt = 0;
    int64_t *dp = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t *di = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    if (!dp || !di) { free(has_l); free(rp); free(mark); free(tmp); free(rc); free(dp); free(di); return OR_OOM; }
    for (int32_t i = 0; i < n; i++) mark[i] = -1;
    dp[0] = 0;
    for (int32_t k = 0; k < n; k++) {
        int32_t m = 0;
        /* look up: rows i < k of column k of U whose L column is not empty */
        for (int64_t p = cp[k]; p < cp[k + 1]; p++) {
            int32_t i = ri[p];
            if (i < k && has_l[i] && mark[i] != k) { mark[i] = k; tmp[m++] = i; }
        }
        /* look left: columns i < k with an entry in row k of L */
        for (int64_t p = rp[k]; p < rp[k + 1]; p++) {
            int32_t i = rc[p];
            if (mark[i] != k) { mark[i] = k; tmp[m++] = i; }
        }
        qsort(tmp, (size_t)m, sizeof(int32_t), cmp_i32);
        if (cnt + m > cap) {
            while (cnt + m > cap) cap *= 2;
            int32_t *nd = (int32_t *)realloc(di, sizeof(int32_t) * (size_t)cap);
            if (!nd) { free(has_l); free(rp); free(mark); free(tmp); free(rc); free(dp); free(di); return OR_OOM; }
            di = nd;
        }
        memcpy(di + cnt, tmp, sizeof(int32_t) * (size_t)m);
        cnt += m;
        dp[k + 1] = cnt;
    }
    free(has_l); free(rp); free(mark); free(tmp); free(rc);
    *out_ptr = dp;
    *out_idx = di;
    return OR_OK;
}

/* ---------------------------------------------------------------------------
 * Levelization (Section II-C: columns grouped into levels of mutually
 * independent columns).  The paper names no rule; the one used is the
 * longest-path depth: level(k) = 0 without dependencies, else
 * 1 + max level of its dependencies.  Within a level, columns ascend.
 * level_of has n entries; level_ptr has nlevels+1; level_cols has n.
 * ------------------------------------------------------------------------- */
int oracle_levels(int32_t n, const int64_t *dp, const int32_t *di,
                  int32_t *level_of, int32_t *out_nlevels,
                  int32_t **out_level_ptr, int32_t **out_level_cols) {
    int32_t nlev = 0;
    for (int32_t k = 0; k < n; k++) {
        int32_t lv = 0;
        for (int64_t p = dp[k]; p < dp[k + 1]; p++) {
            if (di[p] >= k) return OR_INVALID;
            if (level_of[di[p]] + 1 > lv) lv = level_of[di[p]] + 1;
        }
        level_of[k] = lv;
        if (lv + 1 > nlev) nlev = lv + 1;
    }
    int32_t *lp = (int32_t *)calloc((size_t)nlev + 1, sizeof(int32_t));
    int32_t *lc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!lp || !lc) { free(lp); free(lc); return OR_OOM; }
    for (int32_t k = 0; k < n; k++) lp[level_of[k] + 1]++;
    for (int32_t l = 0; l < nlev; l++) lp[l + 1] += lp[l];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nlev + 1));
    if (!fill) { free(lp); free(lc); return OR_OOM; }
    for (int32_t l = 0; l <= nlev; l++) fill[l] = lp[l];
    for (int32_t k = 0; k < n; k++) lc[fill[level_of[k]]++] = k;
    free(fill);
    *out_nlevels = nlev;
    *out_level_ptr = lp;
    *out_level_cols = lc;
    return OR_OK;
}

/* ---------------------------------------------------------------------------
 * Numeric factorization, Algorithm 1 (Gilbert-Peierls left-looking,
 * Section II-A).  For each column j: load B(:,j) into a dense work vector x;
 * for every k < j with A_s(k,j) != 0, in ascending k, do the vector
 * multiply-and-subtract x(i) -= A_s(i,k) * x(k) over the rows i > k of
 * column k of L; the rows <= j of x are column j of U; x(j) is the pivot;
 * the rows > j divided by the pivot are column j of L.
 * lu_val is in the order of the filled pattern (cp, ri).  bval is B's values
 * in B's CSC order.  On a zero or non-finite pivot the function stops and
 * stores the column in *bad_col.
 * ------------------------------------------------------------------------- */
int oracle_numeric(int32_t n, const int32_t *bcolptr, const int32_t *browidx,
                   const double *bval, const int64_t *cp, const int32_t *ri,
                   double *lu_val, int32_t *bad_col) {
    double *x = (double *)calloc((size_t)n + 1, sizeof(double));
    int64_t *dpos = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!x || !dpos) { free(x); free(dpos); return OR_OOM; }
    *bad_col = -1;
    for (int32_t j = 0; j < n; j++) {
        dpos[j] = -1;
        for (int64_t p = cp[j]; p < cp[j + 1]; p++) if (ri[p] == j) dpos[j] = p;
        if (dpos[j] < 0) { free(x); free(dpos); *bad_col = j; return OR_STRUCT_SINGULAR; }
    }
    for (int32_t j = 0; j < n; j++) {
        for (int64_t p = cp[j]; p < cp[j + 1]; p++) x[ri[p]] = 0.0;
        for (int32_t p = bcolptr[j]; p < bcolptr[j + 1]; p++) x[browidx[p]] = bval[p];
        /* triangular solve: rows of column j above the diagonal, ascending */
        for (int64_t p = cp[j]; p < dpos[j]; p++) {
            int32_t k = ri[p];
            double xk = x[k];
            for (int64_t q = dpos[k] + 1; q < cp[k + 1]; q++) {
                double prod = lu_val[q] * xk;
                x[ri[q]] = x[ri[q]] - prod;
            }
        }
        double piv = x[j];
        if (!isfinite(piv)) { *bad_col = j; free(x); free(dpos); return OR_NONFINITE; }
        if (piv == 0.0) { *bad_col = j; free(x); free(dpos); return OR_ZERO_PIVOT; }
        for (int64_t p = cp[j]; p <= dpos[j]; p++) lu_val[p] = x[ri[p]];
        for (int64_t p = dpos[j] + 1; p < cp[j + 1]; p++) lu_val[p] = x[ri[p]] / piv;
    }
    free(x); free(dpos);
    return OR_OK;
}

/* ---------------------------------------------------------------------------
 * Triangular solves (Section I: x follows from solving the two triangular
 * systems in turn).  Solves B z = c with c = P b, then x = P^T z, i.e.
 * x(perm[i]) = z(i) and c(i) = b(perm[i]); nrhs columns, each of length n,
 * stored one after the other.  Forward substitution with unit L, column by
 * column; backward substitution with U, column by column from the last.
 * ------------------------------------------------------------------------- */
int oracle_solve(int32_t n, const int64_t *cp, const int32_t *ri, const double *lu_val,
                 const int32_t *perm, const double *b, double *x, int32_t nrhs) {
    double *z = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    int64_t *dpos = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!z || !dpos) { free(z); free(dpos); return OR_OOM; }
    for (int32_t j = 0; j < n; j++) {
        dpos[j] = -1;
        for (int64_t p = cp[j]; p < cp[j + 1]; p++) if (ri[p] == j) dpos[j] = p;
        if (dpos[j] < 0) { free(z); free(dpos); return OR_STRUCT_SINGULAR; }
    }
    for (int32_t r = 0; r < nrhs; r++) {
        const double *br = b + (size_t)r * n;
        double *xr = x + (size_t)r * n;
        for (int32_t i = 0; i < n; i++) z[i] = br[perm[i]];
        for (int32_t j = 0; j < n; j++) {
            double zj = z[j];
            for (int64_t p = dpos[j] + 1; p < cp[j + 1]; p++) z[ri[p]] = z[ri[p]] - lu_val[p] * zj;
        }
        for (int32_t j = n - 1; j >= 0; j--) {
            z[j] = z[j] / lu_val[dpos[j]];
            double zj = z[j];
            for (int64_t p = cp[j]; p < dpos[j]; p++) z[ri[p]] = z[ri[p]] - lu_val[p] * zj;
        }
        for (int32_t i = 0; i < n; i++) xr[perm[i]] = z[i];
    }
    free(z); free(dpos);
    return OR_OK;
}

/* ---------------------------------------------------------------------------
 * Solve levels (not in the paper; defined for the level-scheduled solves):
 * forward: lf(i) = 0 if row i of L has no entry left of the diagonal, else
 * 1 + max lf(j) over L(i,j) != 0; backward, for i from the last row down:
 * lb(i) = 0 if row i of U has no entry right of the diagonal, else
 * 1 + max lb(k) over U(i,k) != 0, k > i.
 * ------------------------------------------------------------------------- */
int oracle_solve_levels(int32_t n, const int64_t *cp, const int32_t *ri,
                        int32_t *lev_fwd, int32_t *lev_bwd) {
    for (int32_t i = 0; i < n; i++) { lev_fwd[i] = 0; lev_bwd[i] = 0; }
    /* column sweep ascending: an entry L(i,j) raises lf(i) once lf(j) is final */
    for (int32_t j = 0; j < n; j++)
        for (int64_t p = cp[j]; p < cp[j + 1]; p++) {
            int32_t i = ri[p];
            if (i > j && lev_fwd[j] + 1 > lev_fwd[i]) lev_fwd[i] = lev_fwd[j] + 1;
        }
    /* column sweep descending: an entry U(i,k), i < k, raises lb(i) */
    for (int32_t k = n - 1; k >= 0; k--)
        for (int64_t p = cp[k]; p < cp[k + 1]; p++) {
            int32_t i = ri[p];
            if (i < k && lev_bwd[k] + 1 > lev_bwd[i]) lev_bwd[i] = lev_bwd[k] + 1;
        }
    return OR_OK;
}

/* Flop count of one factorization on the pattern: sum over columns j of
 * l_j divisions plus 2 * l_j * u_j multiply-subtracts, where l_j counts the
 * rows below the diagonal in column j and u_j the columns right of the
 * diagonal in row j (Algorithm 2, normalization and submatrix update). */
double oracle_flops(int32_t n, const int64_t *cp, const int32_t *ri) {
    int64_t *l = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *u = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int32_t j = 0; j < n; j++)
        for (int64_t p = cp[j]; p < cp[j + 1]; p++) {
            if (ri[p] > j) l[j]++;
            else if (ri[p] < j) u[ri[p]]++;
        }
    double f = 0.0;
    for (int32_t j = 0; j < n; j++) f += (double)l[j] + 2.0 * (double)l[j] * (double)u[j];
    free(l); free(u);
    return f;
}

/* FP64 residual r = b - A x on A's own CSC (used for the solve's backward
 * error); nrhs columns stored one after the other. */
void oracle_residual(int32_t n, const int32_t *colptr, const int32_t *rowidx,
                     const double *aval, const double *b, const double *x,
                     double *r, int32_t nrhs) {
    for (int32_t c = 0; c < nrhs; c++) {
        const double *xc = x + (size_t)c * n;
        double *rc = r + (size_t)c * n;
        for (int32_t i = 0; i < n; i++) rc[i] = b[(size_t)c * n + i];
        for (int32_t j = 0; j < n; j++)
            for (int32_t p = colptr[j]; p < colptr[j + 1]; p++)
                rc[rowidx[p]] = rc[rowidx[p]] - aval[p] * xc[j];
    }
}
