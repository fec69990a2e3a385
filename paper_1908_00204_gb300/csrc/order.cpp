// order.cpp -- a fill-reducing symmetric ordering for callers without one.
//
// The factorization flow of the paper starts from a fill-reducing order
// (Section II-C, Fig. 5); the analysis takes it as `perm`.  This file gives a
// graph nested dissection of the pattern of A + A^T for callers that have
// none.  Vertices of much higher degree than the typical one (supply nets,
// coupled to many nodes, would shrink every level structure to a few huge
// levels) are set aside and ordered last, by degree.  Of the rest, a subgraph
// larger than a leaf is split by a level structure rooted at a
// pseudo-peripheral vertex -- the smallest level near the middle is the
// separator, thinned of vertices with neighbours on one side only, and ordered
// last -- and each side is ordered recursively; a leaf is
// ordered by minimum degree on its own elimination graph.  Deterministic:
// ties go to the smaller original index.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "glu_internal.h"

namespace glu {
namespace {

constexpr int32_t ND_LEAF = 32;

struct Graph {
    std::vector<int64_t> ptr;
    std::vector<int32_t> adj;
};

// Symmetric adjacency of A + A^T without the diagonal, neighbours ascending.
Graph symmetric_graph(int32_t n, const int32_t *colptr, const int32_t *rowidx) {
    std::vector<int64_t> deg((size_t)n + 1, 0);
    for (int32_t j = 0; j < n; j++)
        for (int32_t p = colptr[j]; p < colptr[j + 1]; p++) {
            const int32_t i = rowidx[p];
            if (i == j) continue;
            deg[i + 1]++;
            deg[j + 1]++;
        }
    for (int32_t i = 0; i < n; i++) deg[i + 1] += deg[i];
    std::vector<int32_t> adj((size_t)deg[n]);
    std::vector<int64_t> f(deg.begin(), deg.end() - 1);
    for (int32_t j = 0; j < n; j++)
        for (int32_t p = colptr[j]; p < colptr[j + 1]; p++) {
            const int32_t i = rowidx[p];
            if (i == j) continue;
            adj[f[i]++] = j;
            adj[f[j]++] = i;
        }
    Graph g;
    g.ptr.assign(1, 0);
    for (int32_t i = 0; i < n; i++) {
        auto b = adj.begin() + deg[i], e = adj.begin() + deg[i + 1];
        std::sort(b, e);
        e = std::unique(b, e);
        g.adj.insert(g.adj.end(), b, e);
        g.ptr.push_back((int64_t)g.adj.size());
    }
    return g;
}

class Dissector {
public:
    Dissector(const Graph &g, int32_t n) : g_(g), mark_((size_t)n, -1), level_((size_t)n, -1) {}

    // Orders the vertices of `set` (all with mark_ == tag) into out.
    void order(std::vector<int32_t> set, std::vector<int32_t> &out) {
        if ((int32_t)set.size() <= ND_LEAF) {
            leaf(set, out);
            return;
        }
        const int32_t tag = next_tag_++;
        for (int32_t v : set) mark_[v] = tag;
        // the component of the smallest vertex; the rest is ordered on its own
        std::sort(set.begin(), set.end());
        std::vector<std::vector<int32_t>> levels = bfs(pseudo_peripheral(set[0], tag), tag);
        std::vector<int32_t> comp;
        for (const auto &lv : levels) comp.insert(comp.end(), lv.begin(), lv.end());
        if (comp.size() < set.size()) {
            const int32_t done = next_tag_++;
            for (int32_t v : comp) mark_[v] = done;
            std::vector<int32_t> rest;
            for (int32_t v : set)
                if (mark_[v] == tag) rest.push_back(v);
            order(comp, out);
            order(rest, out);
            return;
        }
        if (levels.size() < 3) {
            leaf(set, out);
            return;
        }
        // separator: the smallest level among those around the middle
        const int64_t half = (int64_t)set.size() / 2;
        int64_t cum = 0;
        size_t mid = 0;
        for (size_t l = 0; l < levels.size(); l++) {
            cum += (int64_t)levels[l].size();
            if (cum >= half) {
                mid = l;
                break;
            }
        }
        const size_t lo = std::max<size_t>(1, mid - std::min(mid, levels.size() / 8));
        const size_t hi = std::min(levels.size() - 2, mid + levels.size() / 8);
        size_t best = std::min(std::max(mid, lo), hi);
        for (size_t l = lo; l <= hi; l++)
            if (levels[l].size() < levels[best].size()) best = l;
        std::vector<int32_t> a, b;
        for (size_t l = 0; l < best; l++) a.insert(a.end(), levels[l].begin(), levels[l].end());
        for (size_t l = best + 1; l < levels.size(); l++) b.insert(b.end(), levels[l].begin(), levels[l].end());
        // thin the separator: a vertex with no neighbour beyond it joins the
        // near side, one with no neighbour before it the far side
        for (size_t l = 0; l < levels.size(); l++)
            for (int32_t v : levels[l]) level_[v] = (int32_t)l;
        std::vector<int32_t> sep;
        for (int32_t v : levels[best]) {
            bool before = false, after = false;
            for (int64_t p = g_.ptr[v]; p < g_.ptr[v + 1]; p++) {
                const int32_t w = g_.adj[p];
                if (mark_[w] != tag) continue;
                before |= level_[w] < (int32_t)best;
                after |= level_[w] > (int32_t)best;
            }
            if (!after) a.push_back(v);
            else if (!before) b.push_back(v);
            else sep.push_back(v);
        }
        order(a, out);
        order(b, out);
        std::sort(sep.begin(), sep.end());
        out.insert(out.end(), sep.begin(), sep.end());
    }

private:
    std::vector<std::vector<int32_t>> bfs(int32_t root, int32_t tag) {
        std::vector<std::vector<int32_t>> levels;
        std::vector<int32_t> cur(1, root);
        const int32_t seen = next_tag_++;
        mark_[root] = seen;
        while (!cur.empty()) {
            levels.push_back(cur);
            std::vector<int32_t> nxt;
            for (int32_t v : cur)
                for (int64_t p = g_.ptr[v]; p < g_.ptr[v + 1]; p++) {
                    const int32_t w = g_.adj[p];
                    if (mark_[w] == tag) {
                        mark_[w] = seen;
                        nxt.push_back(w);
                    }
                }
            std::sort(nxt.begin(), nxt.end());
            cur.swap(nxt);
        }
        // restore the set's tag for the caller
        for (const auto &lv : levels)
            for (int32_t v : lv) mark_[v] = tag;
        return levels;
    }

    // A vertex of (nearly) maximal eccentricity: repeat BFS from a vertex of
    // minimum degree in the last level while the depth grows.
    int32_t pseudo_peripheral(int32_t start, int32_t tag) {
        int32_t v = start;
        size_t depth = 0;
        for (int it = 0; it < 8; it++) {
            auto levels = bfs(v, tag);
            if (levels.size() <= depth) break;
            depth = levels.size();
            int32_t best = levels.back()[0];
            for (int32_t w : levels.back())
                if (degree(w, tag) < degree(best, tag)) best = w;
            v = best;
        }
        return v;
    }

    int64_t degree(int32_t v, int32_t tag) const {
        int64_t d = 0;
        for (int64_t p = g_.ptr[v]; p < g_.ptr[v + 1]; p++) d += mark_[g_.adj[p]] == tag;
        return d;
    }

    // Minimum degree on the leaf's own graph (eliminating a vertex joins its
    // remaining neighbours).
    void leaf(std::vector<int32_t> set, std::vector<int32_t> &out) {
        std::sort(set.begin(), set.end());
        const int32_t k = (int32_t)set.size();
        std::vector<std::vector<char>> adj((size_t)k, std::vector<char>((size_t)k, 0));
        const int32_t tag = next_tag_++;
        for (int32_t q = 0; q < k; q++) {
            mark_[set[q]] = tag;
            level_[set[q]] = q;
        }
        for (int32_t q = 0; q < k; q++)
            for (int64_t p = g_.ptr[set[q]]; p < g_.ptr[set[q] + 1]; p++) {
                const int32_t w = g_.adj[p];
                if (mark_[w] == tag) adj[q][level_[w]] = 1;
            }
        std::vector<char> gone((size_t)k, 0);
        for (int32_t step = 0; step < k; step++) {
            int32_t best = -1, bd = 0;
            for (int32_t q = 0; q < k; q++) {
                if (gone[q]) continue;
                int32_t d = 0;
                for (int32_t r = 0; r < k; r++) d += !gone[r] && adj[q][r];
                if (best < 0 || d < bd) {
                    best = q;
                    bd = d;
                }
            }
            gone[best] = 1;
            out.push_back(set[best]);
            for (int32_t r = 0; r < k; r++)
                if (!gone[r] && adj[best][r])
                    for (int32_t s = 0; s < k; s++)
                        if (s != r && !gone[s] && adj[best][s]) adj[r][s] = 1;
        }
        const int32_t done = next_tag_++;
        for (int32_t v : set) mark_[v] = done;
    }

    const Graph &g_;
    std::vector<int32_t> mark_;
    std::vector<int32_t> level_;
    int32_t next_tag_ = 0;
};

}  // namespace

int order_nested_dissection(int32_t n, const int32_t *colptr, const int32_t *rowidx, int32_t *perm) {
    if (n < 0 || (n > 0 && (!colptr || !rowidx || !perm))) return GLU_ERR_INVALID;
    if (n == 0) return GLU_OK;
    if (colptr[0] != 0) return GLU_ERR_INVALID;
    for (int32_t j = 0; j < n; j++) {
        if (colptr[j + 1] < colptr[j]) return GLU_ERR_INVALID;
        for (int32_t p = colptr[j]; p < colptr[j + 1]; p++)
            if (rowidx[p] < 0 || rowidx[p] >= n) return GLU_ERR_INVALID;
    }
    const Graph g = symmetric_graph(n, colptr, rowidx);
    // dense vertices: degree above max(16, 8 x the median degree)
    std::vector<int64_t> deg((size_t)n);
    for (int32_t i = 0; i < n; i++) deg[i] = g.ptr[i + 1] - g.ptr[i];
    std::vector<int64_t> sorted_deg(deg);
    std::nth_element(sorted_deg.begin(), sorted_deg.begin() + n / 2, sorted_deg.end());
    const int64_t limit = std::max<int64_t>(16, 8 * sorted_deg[n / 2]);
    std::vector<int32_t> keep, dense;
    for (int32_t i = 0; i < n; i++) (deg[i] > limit ? dense : keep).push_back(i);
    std::vector<int32_t> out;
    out.reserve((size_t)n);
    Dissector d(g, n);
    d.order(keep, out);
    std::stable_sort(dense.begin(), dense.end(), [&](int32_t a, int32_t b) { return deg[a] < deg[b]; });
    out.insert(out.end(), dense.begin(), dense.end());
    if ((int32_t)out.size() != n) return GLU_ERR_INTERNAL;
    std::copy(out.begin(), out.end(), perm);
    return GLU_OK;
}

}  // namespace glu
