/* abi_host.c -- the C ABI used from plain C99, host analysis only (no GPU).
 *
 * Two matrices with closed-form results:
 *   a tridiagonal n = 5: nnz(L+U) = 3n - 2 = 13, levels = n = 5 (a chain);
 *   an arrow n = 6 with a dense last row and column: no fill-in,
 *     nnz(L+U) = 3n - 2 = 16, levels = 2 (columns 0..4, then column 5).
 * Also: a malformed input is rejected with GLU_ERR_INVALID and a handle is
 * not returned; glu_order_nd returns a permutation; glu_static_pivot puts a
 * matrix's large anti-diagonal on the diagonal.  Prints "ok" on success,
 * else the first failed check, and exits non-zero. */
#include <stdio.h>
#include <stdlib.h>

#include "glu.h"

#define CHECK(c)                                                    \
    do {                                                            \
        if (!(c)) {                                                 \
            printf("check failed at line %d: %s\n", __LINE__, #c); \
            return 1;                                               \
        }                                                           \
    } while (0)

static int analyze(int32_t n, const int32_t *cp, const int32_t *ri, int64_t want_nnz, int32_t want_levels) {
    glu_options o;
    glu_handle *h = NULL;
    const int64_t *lcp = NULL;
    const int32_t *lri = NULL, *lp = NULL, *lc = NULL;
    int64_t nnz = -1;
    int32_t nl = -1, j;
    glu_stats st;
    glu_default_options(&o);
    o.host_only = 1;
    CHECK(glu_analyze_opts(n, cp, ri, NULL, &o, &h) == GLU_OK && h != NULL);
    CHECK(glu_get_fill(h, &lcp, &lri, &nnz) == GLU_OK);
    CHECK(nnz == want_nnz && lcp[0] == 0 && lcp[n] == nnz);
    for (j = 0; j < n; j++) CHECK(lcp[j + 1] > lcp[j]);
    CHECK(glu_get_levels(h, &nl, &lp, &lc) == GLU_OK);
    CHECK(nl == want_levels && lp[0] == 0 && lp[nl] == n);
    CHECK(glu_get_stats(h, &st) == GLU_OK && st.n == n && st.nnz_lu == want_nnz && st.nlevels == want_levels);
    glu_destroy(h);
    return 0;
}

int main(void) {
    /* tridiagonal, n = 5 */
    const int32_t tcp[6] = {0, 2, 5, 8, 11, 13};
    const int32_t tri[13] = {0, 1, 0, 1, 2, 1, 2, 3, 2, 3, 4, 3, 4};
    /* arrow, n = 6: diagonal, last row and last column */
    const int32_t acp[7] = {0, 2, 4, 6, 8, 10, 16};
    const int32_t ari[16] = {0, 5, 1, 5, 2, 5, 3, 5, 4, 5, 0, 1, 2, 3, 4, 5};
    /* rows out of order in column 1 */
    const int32_t bcp[3] = {0, 1, 3};
    const int32_t bri[3] = {0, 1, 0};
    int32_t perm[6], seen[6] = {0, 0, 0, 0, 0, 0}, i;
    glu_handle *h = (glu_handle *)&seen;   /* must be cleared on failure */
    glu_options o;

    if (analyze(5, tcp, tri, 13, 5)) return 1;
    if (analyze(6, acp, ari, 16, 2)) return 1;
    glu_default_options(&o);
    o.host_only = 1;
    CHECK(glu_analyze_opts(2, bcp, bri, NULL, &o, &h) == GLU_ERR_INVALID && h == NULL);
    CHECK(glu_strerror(GLU_ERR_INVALID) != NULL);
    CHECK(glu_order_nd(6, acp, ari, perm) == GLU_OK);
    for (i = 0; i < 6; i++) {
        CHECK(perm[i] >= 0 && perm[i] < 6 && !seen[perm[i]]);
        seen[perm[i]] = 1;
    }
    {
        /* static pivoting: a full 3 x 3 matrix whose large entries sit on the
         * anti-diagonal, so the matching reverses the rows */
        const int32_t fcp[4] = {0, 3, 6, 9};
        const int32_t fri[9] = {0, 1, 2, 0, 1, 2, 0, 1, 2};
        const double fv[9] = {1.0, 2.0, 100.0, 3.0, 50.0, 1.0, 20.0, 1.0, 2.0};
        int32_t rp[3];
        double rs[3], cs[3];
        CHECK(glu_static_pivot(3, fcp, fri, fv, rp, rs, cs) == GLU_OK);
        CHECK(rp[0] == 2 && rp[1] == 1 && rp[2] == 0);
        for (i = 0; i < 3; i++) {
            const double d = rs[rp[i]] * fv[3 * i + rp[i]] * cs[i];
            CHECK(d > 1.0 - 1e-12 && d < 1.0 + 1e-12);
        }
    }
    printf("ok\n");
    return 0;
}
