// match.cpp -- static pivoting with scaling for callers without one.
//
// The factorization flow of the paper starts from a matrix whose rows were
// permuted and scaled so that the diagonal is large (MC64, Section II-C,
// Fig. 5), then ordered to reduce fill.  This file gives the first step: a
// row permutation that maximizes the product of the diagonal magnitudes,
// with row and column scalings after which every matched entry has
// magnitude 1 and no entry exceeds 1.
//
// The product is maximized as a minimum-cost perfect matching of columns to
// rows with cost c(i,j) = log(max_k |a_kj|) - log|a_ij| >= 0 over the
// nonzero entries, solved by successive shortest augmenting paths (Dijkstra
// on reduced costs c(i,j) - u_i - v_j >= 0, row and column potentials kept
// feasible after every augmentation).  At the end every matched edge has
// reduced cost 0, so with r_i = exp(u_i) and s_j = exp(v_j) / max_k |a_kj|
// the scaled entry |r_i a_ij s_j| = exp(-(reduced cost)) is 1 on the
// matching and at most 1 elsewhere.  Deterministic.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <limits>
#include <queue>
#include <utility>
#include <vector>

#include "glu_internal.h"

namespace glu {

int static_pivot(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *values, int32_t *row_perm,
                 double *row_scale, double *col_scale) {
    if (n < 0 || (n > 0 && (!colptr || !rowidx || !values || !row_perm || !row_scale || !col_scale)))
        return GLU_ERR_INVALID;
    if (n == 0) return GLU_OK;
    if (colptr[0] != 0) return GLU_ERR_INVALID;
    for (int32_t j = 0; j < n; j++) {
        if (colptr[j + 1] < colptr[j]) return GLU_ERR_INVALID;
        for (int32_t p = colptr[j]; p < colptr[j + 1]; p++)
            if (rowidx[p] < 0 || rowidx[p] >= n || !std::isfinite(values[p])) return GLU_ERR_INVALID;
    }
    const double INF = std::numeric_limits<double>::infinity();
    // costs of the nonzero entries (explicit zeros are not edges)
    std::vector<double> cost((size_t)colptr[n], INF);
    std::vector<double> lmax((size_t)n, -INF);   // log of each column's largest magnitude
    for (int32_t j = 0; j < n; j++) {
        for (int32_t p = colptr[j]; p < colptr[j + 1]; p++)
            if (values[p] != 0.0) lmax[j] = std::max(lmax[j], std::log(std::fabs(values[p])));
        if (lmax[j] == -INF) return GLU_ERR_STRUCT_SINGULAR;   // an empty column
        for (int32_t p = colptr[j]; p < colptr[j + 1]; p++)
            if (values[p] != 0.0) cost[p] = lmax[j] - std::log(std::fabs(values[p]));
    }
    // feasible start: u_i = the smallest cost in row i, v_j = the smallest
    // c(i,j) - u_i in column j (reduced costs >= 0, each column with a zero)
    std::vector<double> u((size_t)n, INF), v((size_t)n, INF);
    for (int32_t j = 0; j < n; j++)
        for (int32_t p = colptr[j]; p < colptr[j + 1]; p++) u[rowidx[p]] = std::min(u[rowidx[p]], cost[p]);
    for (int32_t i = 0; i < n; i++)
        if (u[i] == INF) return GLU_ERR_STRUCT_SINGULAR;   // a row without a nonzero
    for (int32_t j = 0; j < n; j++)
        for (int32_t p = colptr[j]; p < colptr[j + 1]; p++)
            if (cost[p] != INF) v[j] = std::min(v[j], cost[p] - u[rowidx[p]]);
    std::vector<int32_t> mate_row((size_t)n, -1);   // column matched to each row
    std::vector<int32_t> mate_col((size_t)n, -1);   // row matched to each column
    // greedy start: a column takes a free row along an edge of reduced cost 0
    for (int32_t j = 0; j < n; j++)
        for (int32_t p = colptr[j]; p < colptr[j + 1]; p++) {
            const int32_t i = rowidx[p];
            if (cost[p] != INF && cost[p] - u[i] - v[j] == 0.0 && mate_row[i] < 0) {
                mate_row[i] = j;
                mate_col[j] = i;
                break;
            }
        }
    // one shortest augmenting path per column left free
    std::vector<double> dist((size_t)n, INF);
    std::vector<int32_t> pred((size_t)n, -1);      // column from which each row was reached
    std::vector<uint8_t> done((size_t)n, 0);
    std::vector<int32_t> touched, settled;
    using Item = std::pair<double, int32_t>;
    for (int32_t j0 = 0; j0 < n; j0++) {
        if (mate_col[j0] >= 0) continue;
        std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
        touched.clear();
        settled.clear();
        auto relax = [&](int32_t j, double dj) {
            for (int32_t p = colptr[j]; p < colptr[j + 1]; p++) {
                if (cost[p] == INF) continue;
                const int32_t i = rowidx[p];
                if (done[i]) continue;
                const double nd = dj + (cost[p] - u[i] - v[j]);
                if (nd < dist[i] || (nd == dist[i] && pred[i] > j)) {
                    if (dist[i] == INF) touched.push_back(i);
                    dist[i] = nd;
                    pred[i] = j;
                    heap.push(Item(nd, i));
                }
            }
        };
        relax(j0, 0.0);
        int32_t free_row = -1;
        double D = 0.0;
        while (!heap.empty()) {
            const Item it = heap.top();
            heap.pop();
            const int32_t i = it.second;
            if (done[i] || it.first != dist[i]) continue;
            done[i] = 1;
            settled.push_back(i);
            if (mate_row[i] < 0) {
                free_row = i;
                D = dist[i];
                break;
            }
            relax(mate_row[i], dist[i]);
        }
        if (free_row < 0) {
            for (int32_t i : touched) {
                dist[i] = INF;
                pred[i] = -1;
                done[i] = 0;
            }
            return GLU_ERR_STRUCT_SINGULAR;
        }
        // potentials: each column of the search tree rises by D minus the
        // distance at which it was reached, each settled row falls likewise
        v[j0] += D;
        for (int32_t i : settled) {
            if (i == free_row) continue;
            v[mate_row[i]] += D - dist[i];
            u[i] -= D - dist[i];
        }
        // augment along the path back to j0
        for (int32_t i = free_row; i >= 0;) {
            const int32_t j = pred[i];
            const int32_t prev = mate_col[j];
            mate_col[j] = i;
            mate_row[i] = j;
            i = j == j0 ? -1 : prev;
        }
        for (int32_t i : touched) {
            dist[i] = INF;
            pred[i] = -1;
            done[i] = 0;
        }
    }
    // The potentials were updated in floating point over many augmentations:
    // take each v_j again as the smallest c_ij - u_i of its column, so every
    // reduced cost computed from the final u and v is >= 0 (the scaled
    // entries are then <= 1 up to the rounding of exp and the products).
    for (int32_t j = 0; j < n; j++) {
        double vj = INF;
        for (int32_t p = colptr[j]; p < colptr[j + 1]; p++) {
            if (values[p] == 0.0) continue;
            vj = std::min(vj, (lmax[j] - std::log(std::fabs(values[p]))) - u[rowidx[p]]);
        }
        row_perm[j] = mate_col[j];
        col_scale[j] = std::exp(vj - lmax[j]);
    }
    for (int32_t i = 0; i < n; i++) row_scale[i] = std::exp(u[i]);
    return GLU_OK;
}

int apply_static_pivot(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *values,
                       const int32_t *row_perm, const double *row_scale, const double *col_scale,
                       int32_t *out_rowidx, double *out_values) {
    if (n < 0 || (n > 0 && (!colptr || !rowidx || !values || !row_perm || !out_rowidx || !out_values)))
        return GLU_ERR_INVALID;
    if (n == 0) return GLU_OK;
    if (colptr[0] != 0) return GLU_ERR_INVALID;
    // new_row[row_perm[k]] = k: row_perm must be a permutation
    std::vector<int32_t> new_row((size_t)n, -1);
    for (int32_t k = 0; k < n; k++) {
        const int32_t r = row_perm[k];
        if (r < 0 || r >= n || new_row[r] >= 0) return GLU_ERR_INVALID;
        new_row[r] = k;
    }
    std::vector<std::pair<int32_t, double>> col;
    for (int32_t j = 0; j < n; j++) {
        const int32_t b = colptr[j], e = colptr[j + 1];
        if (e < b) return GLU_ERR_INVALID;
        col.clear();
        const double cs = col_scale ? col_scale[j] : 1.0;
        for (int32_t p = b; p < e; p++) {
            const int32_t r = rowidx[p];
            if (r < 0 || r >= n) return GLU_ERR_INVALID;
            const double rs = row_scale ? row_scale[r] : 1.0;
            col.emplace_back(new_row[r], rs * values[p] * cs);
        }
        std::sort(col.begin(), col.end(),
                  [](const std::pair<int32_t, double> &x, const std::pair<int32_t, double> &y) {
                      return x.first < y.first;
                  });
        for (size_t q = 0; q < col.size(); q++) {
            if (q > 0 && col[q].first == col[q - 1].first) return GLU_ERR_INVALID;   // duplicate row
            out_rowidx[b + (int32_t)q] = col[q].first;
            out_values[b + (int32_t)q] = col[q].second;
        }
    }
    return GLU_OK;
}

}  // namespace glu
