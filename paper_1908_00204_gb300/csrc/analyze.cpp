// analyze.cpp -- host half of glu_analyze (the CPU part of the flow, Fig. 5).
//
// Steps: input checks and B = P A P^T; symbolic fill-in of L+U with a
// depth-first reachability search pruned by symmetric pruning (Eisenstat &
// Liu), which returns the same pattern as the plain search of Section II-A in
// less time; the relaxed dependencies of Algorithm 4 by merging two sorted
// lists per column; levels by longest path (Section II-C); the per-level
// update schedule of Algorithm 2 / Algorithm 5 (sources of a level, their
// target columns, the warp tasks); the row views and levels of the two
// triangular solves.
#include <algorithm>
#include <array>
#include <atomic>
#include <condition_variable>
#include <mutex>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <system_error>
#include <thread>

#include "glu_internal.h"

namespace glu {
namespace {

// Starts fn on a new thread (th must have room reserved), or runs it here
// when no thread can be created: the analysis's results never depend on how
// many threads ran it.
template <class F>
void spawn_or_run(std::vector<std::thread> &th, F fn) {
    try {
        th.emplace_back(fn);
    } catch (const std::system_error &) {
        fn();
    }
}

// Host threads of the analysis: the machine's, at most 16, or
// GLU_ANALYZE_THREADS (1..64).
int analysis_threads() {
    int nth = std::max(1, std::min<int>(16, (int)std::thread::hardware_concurrency()));
    if (const char *e = std::getenv("GLU_ANALYZE_THREADS")) nth = std::max(1, std::min(64, std::atoi(e)));
    return nth;
}

// Cuts the columns [0, n) into nth consecutive ranges of about equal weight
// (ptr[n+1] a prefix sum of the columns' weights); returns nth + 1 bounds.
template <class I>
std::vector<int32_t> column_ranges(int32_t n, const I *ptr, int nth) {
    std::vector<int32_t> cut(1, 0);
    const int64_t total = (int64_t)ptr[n];
    for (int t = 1; t < nth; t++) {
        const int64_t want = total * t / nth;
        const int32_t j = (int32_t)(std::lower_bound(ptr, ptr + n + 1, (I)want) - ptr);
        cut.push_back(std::max(cut.back(), std::min(j, n)));
    }
    cut.push_back(n);
    return cut;
}

// Runs fn(t) for t in [0, nth) on nth threads (this one included).  An
// allocation failure on any of them is rethrown here once all have joined.
template <class F>
void run_threads(int nth, F fn) {
    std::atomic<bool> failed{false};
    auto job = [&](int t) {
        try {
            fn(t);
        } catch (const std::bad_alloc &) {
            failed = true;
        }
    };
    std::vector<std::thread> th;
    th.reserve((size_t)nth);
    for (int t = 1; t < nth; t++) spawn_or_run(th, [&job, t] { job(t); });
    job(0);
    for (std::thread &x : th) x.join();
    if (failed) throw std::bad_alloc();
}

// std::lower_bound for a value expected near the start of [first, last):
// an exponential search from first, then a binary search inside the bracket
// (everything before lo is known to be < v).
template <class T>
const T *gallop_lower_bound(const T *first, const T *last, T v) {
    const T *lo = first;
    ptrdiff_t step = 1;
    for (;;) {
        if (last - lo <= step) return std::lower_bound(lo, last, v);
        if (!(lo[step - 1] < v)) return std::lower_bound(lo, lo + step, v);
        lo += step;
        step *= 2;
    }
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------
// Input checks and the symmetric permutation.  Two stable counting sorts
// (by new row, then by new column) give B's columns with sorted rows.
int permute_input(HostPlan &P, std::vector<int64_t> &bptr, std::vector<int32_t> &brow,
                  std::vector<int32_t> &bsrc, std::string &why) {
    const int32_t n = P.n;
    const int64_t nnz = P.nnz_a;
    std::vector<int32_t> cnt((size_t)n + 1, 0);
    std::vector<int32_t> order1((size_t)nnz);
    for (int64_t p = 0; p < nnz; p++) cnt[P.iperm[P.a_rowidx[p]] + 1]++;
    for (int32_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    for (int32_t c = 0; c < n; c++)
        for (int32_t p = P.a_colptr[c]; p < P.a_colptr[c + 1]; p++)
            order1[cnt[P.iperm[P.a_rowidx[p]]]++] = p;
    // column of each A entry in the new numbering
    std::vector<int32_t> colof((size_t)nnz);
    for (int32_t c = 0; c < n; c++)
        for (int32_t p = P.a_colptr[c]; p < P.a_colptr[c + 1]; p++) colof[p] = P.iperm[c];
    bptr.assign((size_t)n + 1, 0);
    for (int64_t p = 0; p < nnz; p++) bptr[colof[p] + 1]++;
    for (int32_t j = 0; j < n; j++) bptr[j + 1] += bptr[j];
    std::vector<int64_t> fill(bptr.begin(), bptr.end() - 1);
    brow.resize((size_t)nnz);
    bsrc.resize((size_t)nnz);
    for (int64_t q = 0; q < nnz; q++) {
        int32_t p = order1[q];
        int64_t dst = fill[colof[p]]++;
        brow[dst] = P.iperm[P.a_rowidx[p]];
        bsrc[dst] = p;
    }
    for (int32_t j = 0; j < n; j++) {
        bool diag = false;
        for (int64_t q = bptr[j]; q < bptr[j + 1]; q++) diag |= (brow[q] == j);
        if (!diag) {
            why = "column " + std::to_string(j) + " of P A P^T has no diagonal entry";
            return GLU_ERR_STRUCT_SINGULAR;
        }
    }
    return GLU_OK;
}

// ---------------------------------------------------------------------------
// Symbolic fill-in.  Column j of A_s is the set reached from struct(B(:,j))
// through the edges k -> i of L(i,k) != 0 with k < j.  After column j is
// known, every k < j with U(k,j) != 0 and L(j,k) != 0 can drop from its
// search list the rows of L(:,k) below j: they are reached through j
// (symmetric pruning); the result is unchanged.
//
// In parallel by subtrees.  struct(L+U) lies inside the Cholesky pattern of
// B + B^T, so every k < j with U(k,j) != 0 is a descendant of j in the
// elimination tree of B + B^T: column j reads, and prunes, only columns of
// its own subtree.  Small disjoint subtrees are computed at once on threads,
// each into its own row buffer.  The tree above them is cut into chains
// (paths along which every node has one child in that part of the tree); a
// chain runs, bottom up, once the chains below it are done, several at once.
// The buffers are finally copied into column order.  The result is the same
// for any thread count.

// Elimination tree of B + B^T (Liu's algorithm with path compression):
// parent[j] > j, or -1 for a root.
std::vector<int32_t> etree_of_symmetric(int32_t n, const std::vector<int64_t> &bptr,
                                        const std::vector<int32_t> &brow) {
    // B's strictly lower entries B(r, i), r > i, listed by row r
    std::vector<int64_t> lp((size_t)n + 1, 0);
    for (int32_t i = 0; i < n; i++)
        for (int64_t q = bptr[i]; q < bptr[i + 1]; q++)
            if (brow[q] > i) lp[brow[q] + 1]++;
    for (int32_t r = 0; r < n; r++) lp[r + 1] += lp[r];
    std::vector<int32_t> lc((size_t)lp[n]);
    {
        std::vector<int64_t> f(lp.begin(), lp.end() - 1);
        for (int32_t i = 0; i < n; i++)
            for (int64_t q = bptr[i]; q < bptr[i + 1]; q++)
                if (brow[q] > i) lc[f[brow[q]]++] = i;
    }
    std::vector<int32_t> parent((size_t)n, -1), anc((size_t)n, -1);
    auto link = [&](int32_t i, int32_t j) {
        int32_t r = i;
        while (anc[r] != -1 && anc[r] != j) {
            const int32_t t = anc[r];
            anc[r] = j;
            r = t;
        }
        if (anc[r] == -1) {
            anc[r] = j;
            parent[r] = j;
        }
    };
    for (int32_t j = 0; j < n; j++) {
        for (int64_t q = bptr[j]; q < bptr[j + 1]; q++)
            if (brow[q] < j) link(brow[q], j);
        for (int64_t q = lp[j]; q < lp[j + 1]; q++) link(lc[q], j);
    }
    return parent;
}

int symbolic(HostPlan &P, const std::vector<int64_t> &bptr, const std::vector<int32_t> &brow) {
    const int32_t n = P.n;
    const int nth = analysis_threads();
    // ---- the subtrees computed in parallel (none with one thread)
    const std::vector<int32_t> parent = etree_of_symmetric(n, bptr, brow);
    std::vector<int64_t> size((size_t)n, 1);
    for (int32_t j = 0; j < n; j++)
        if (parent[j] >= 0) size[parent[j]] += size[j];
    std::vector<int32_t> comp((size_t)n, -1);   // subtree task of each column, -1: above them
    int32_t ntask = 0;
    if (nth > 1) {
        const int64_t target = std::max<int64_t>(1, n / ((int64_t)nth * 4));
        std::vector<int64_t> cptr((size_t)n + 1, 0);
        for (int32_t j = 0; j < n; j++)
            if (parent[j] >= 0) cptr[parent[j] + 1]++;
        for (int32_t j = 0; j < n; j++) cptr[j + 1] += cptr[j];
        std::vector<int32_t> child((size_t)cptr[n]);
        {
            std::vector<int64_t> f(cptr.begin(), cptr.end() - 1);
            for (int32_t j = 0; j < n; j++)
                if (parent[j] >= 0) child[f[parent[j]]++] = j;
        }
        std::vector<int32_t> stack;
        for (int32_t j = 0; j < n; j++)
            if (parent[j] < 0) stack.push_back(j);
        while (!stack.empty()) {
            const int32_t v = stack.back();
            stack.pop_back();
            if (size[v] <= target) {
                comp[v] = ntask++;
            } else {
                for (int64_t q = cptr[v]; q < cptr[v + 1]; q++) stack.push_back(child[q]);
            }
        }
        for (int32_t j = n - 1; j >= 0; j--)
            if (comp[j] < 0 && parent[j] >= 0 && comp[parent[j]] >= 0) comp[j] = comp[parent[j]];
    }
    std::vector<std::vector<int32_t>> cols((size_t)ntask + 1);   // last: the columns above
    for (int32_t j = 0; j < n; j++) cols[comp[j] >= 0 ? comp[j] : ntask].push_back(j);
    // ---- per column: buffer, start in it, length, diagonal and pruned end
    // (offsets relative to the column's start)
    std::vector<int32_t> cb((size_t)n);
    std::vector<int64_t> cs((size_t)n), cl((size_t)n), cd((size_t)n), ce((size_t)n);
    std::vector<uint8_t> pruned((size_t)n, 0);
    std::vector<std::vector<int32_t>> bufs((size_t)ntask + 1);
    struct Scratch {
        std::vector<int32_t> mark, stk, found;
        std::vector<int64_t> nxt;
    };
    auto column = [&](int32_t j, int32_t bid, Scratch &sc) {
        std::vector<int32_t> &mark = sc.mark, &stk = sc.stk, &found = sc.found;
        std::vector<int64_t> &nxt = sc.nxt;
        found.clear();
        int32_t lo = n;   // smallest row found
        for (int64_t q = bptr[j]; q < bptr[j + 1]; q++) {
            const int32_t s = brow[q];
            if (mark[s] == j) continue;
            mark[s] = j;
            found.push_back(s);
            lo = std::min(lo, s);
            if (s >= j) continue;
            int32_t top = 0;
            stk[0] = s;
            nxt[0] = cd[s] + 1;
            while (top >= 0) {
                const int32_t v = stk[top];
                const int32_t *rv = bufs[cb[v]].data() + cs[v];
                const int64_t e = ce[v];
                int64_t t = nxt[top];
                while (t < e && mark[rv[t]] == j) t++;
                if (t == e) {
                    top--;
                    continue;
                }
                const int32_t w = rv[t];
                nxt[top] = t + 1;
                mark[w] = j;
                found.push_back(w);
                lo = std::min(lo, w);
                if (w < j) {
                    top++;
                    stk[top] = w;
                    nxt[top] = cd[w] + 1;
                }
            }
        }
        // ascending order: a set that fills at least 1/8 of its range [lo, n)
        // (the dense trailing columns) by a scan of the marks, else a sort
        const int64_t f = (int64_t)found.size();
        if (f >= 256 && (int64_t)(n - lo) <= 8 * f) {
            found.clear();
            for (int32_t i = lo; i < n; i++)
                if (mark[i] == j) found.push_back(i);
        } else {
            std::sort(found.begin(), found.end());
        }
        std::vector<int32_t> &out = bufs[bid];
        cb[j] = bid;
        cs[j] = (int64_t)out.size();
        out.insert(out.end(), found.begin(), found.end());
        const int64_t d = std::lower_bound(found.begin(), found.end(), j) - found.begin();
        cl[j] = (int64_t)found.size();
        cd[j] = d;
        ce[j] = (int64_t)found.size();
        // symmetric pruning of the columns k with U(k,j) != 0
        for (int64_t q = 0; q < d; q++) {
            const int32_t k = found[q];
            if (pruned[k]) continue;
            const int32_t *rk = bufs[cb[k]].data() + cs[k];
            const int32_t *lb = rk + cd[k] + 1;
            const int32_t *le = rk + cl[k];
            const int32_t *it = std::lower_bound(lb, le, j);
            if (it != le && *it == j) {
                ce[k] = (it - rk) + 1;
                pruned[k] = 1;
            }
        }
    };
    auto scratch = [n](Scratch &sc) {
        sc.mark.assign((size_t)n, -1);
        sc.stk.resize((size_t)n + 1);
        sc.nxt.resize((size_t)n + 1);
        sc.found.reserve(1024);
    };
    // subtrees, largest first, taken by threads as they finish
    std::vector<int32_t> order((size_t)ntask);
    for (int32_t t = 0; t < ntask; t++) order[t] = t;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return cols[a].size() > cols[b].size(); });
    // the columns above the subtrees: chains, each continuing the chain of
    // its node's only child there
    const std::vector<int32_t> &top = cols[ntask];
    std::vector<int32_t> ntop((size_t)n, 0), only((size_t)n, -1), chain_of((size_t)n, -1);
    for (int32_t j : top)
        if (parent[j] >= 0) {
            ntop[parent[j]]++;
            only[parent[j]] = j;
        }
    std::vector<std::vector<int32_t>> chains;
    for (int32_t j : top) {
        if (ntop[j] == 1) {
            chain_of[j] = chain_of[only[j]];
        } else {
            chain_of[j] = (int32_t)chains.size();
            chains.emplace_back();
        }
        chains[chain_of[j]].push_back(j);
    }
    const int32_t nchain = (int32_t)chains.size();
    std::vector<int32_t> pending((size_t)nchain);
    for (int32_t c = 0; c < nchain; c++) pending[c] = ntop[chains[c][0]];
    // The chain that ends the matrix -- its columns are [c0, n) -- runs last,
    // in two phases (top_chain below) when it is long: the dense trailing
    // block and the nets' columns, whose reach sets cover much of the matrix,
    // would otherwise be one thread's sequential work.
    int32_t tc = -1;
    if (nth > 1 && n > 0 && comp[n - 1] < 0) {
        const std::vector<int32_t> &cc = chains[chain_of[n - 1]];
        const int32_t c0 = n - (int32_t)cc.size();
        bool tail = cc.size() >= 32;
        for (size_t i = 0; tail && i < cc.size(); i++) tail = cc[i] == c0 + (int32_t)i;
        if (tail) tc = chain_of[n - 1];
    }
    bufs.resize((size_t)ntask + nchain);
    std::vector<Scratch> scr((size_t)nth);
    // The final chain [c0, n): every row of L(:,j) for j >= c0 lies in the
    // chain, so the rows below c0 that column j reaches are reached through
    // columns below c0 only, whose structures are final once the other
    // chains are done.  Phase 1 (columns in parallel): those rows, sorted,
    // and the rows of the chain met on the way.  Phase 2 (in column order):
    // the closure of the latter through the chain's own columns, and the
    // column is the two lists one after the other.  The reach sets are those
    // of column(); only the columns of the chain are pruned (the others are
    // searched no more), which changes no set.
    auto top_chain = [&](const std::vector<int32_t> &cc, int32_t bid) {
        const int32_t c0 = cc.front();
        const int32_t len = (int32_t)cc.size();
        std::vector<std::vector<int32_t>> below((size_t)len), entry((size_t)len);
        std::atomic<int32_t> nextc{0};
        run_threads(nth, [&](int t) {
            Scratch &sc = scr[t];
            if (sc.mark.empty()) scratch(sc);
            std::vector<int32_t> &mark = sc.mark, &stk = sc.stk;
            std::vector<int64_t> &nxt = sc.nxt;
            for (int32_t i; (i = nextc.fetch_add(1)) < len;) {
                const int32_t j = c0 + i;
                std::vector<int32_t> &out = below[(size_t)i], &ent = entry[(size_t)i];
                int32_t lo = c0;
                for (int64_t q = bptr[j]; q < bptr[j + 1]; q++) {
                    const int32_t s = brow[q];
                    if (mark[s] == j) continue;
                    mark[s] = j;
                    if (s >= c0) {
                        ent.push_back(s);
                        continue;
                    }
                    out.push_back(s);
                    lo = std::min(lo, s);
                    int32_t top = 0;
                    stk[0] = s;
                    nxt[0] = cd[s] + 1;
                    while (top >= 0) {
                        const int32_t v = stk[top];
                        const int32_t *rv = bufs[cb[v]].data() + cs[v];
                        const int64_t e = ce[v];
                        int64_t t2 = nxt[top];
                        while (t2 < e && mark[rv[t2]] == j) t2++;
                        if (t2 == e) {
                            top--;
                            continue;
                        }
                        const int32_t w = rv[t2];
                        nxt[top] = t2 + 1;
                        mark[w] = j;
                        if (w >= c0) {
                            ent.push_back(w);
                            continue;
                        }
                        out.push_back(w);
                        lo = std::min(lo, w);
                        top++;
                        stk[top] = w;
                        nxt[top] = cd[w] + 1;
                    }
                }
                const int64_t f = (int64_t)out.size();
                if (f >= 256 && (int64_t)(c0 - lo) <= 8 * f) {
                    out.clear();
                    for (int32_t r = lo; r < c0; r++)
                        if (mark[r] == j) out.push_back(r);
                } else {
                    std::sort(out.begin(), out.end());
                }
            }
        });
        std::vector<int32_t> cm((size_t)len, -1), cstk, cfound;
        std::vector<int64_t> cnx;
        std::vector<int32_t> &buf = bufs[(size_t)bid];
        for (int32_t i = 0; i < len; i++) {
            const int32_t j = c0 + i;
            cfound.clear();
            for (const int32_t e0 : entry[(size_t)i]) {
                if (cm[(size_t)(e0 - c0)] == j) continue;
                cm[(size_t)(e0 - c0)] = j;
                cfound.push_back(e0);
                if (e0 >= j) continue;
                cstk.assign(1, e0);
                cnx.assign(1, cd[e0] + 1);
                while (!cstk.empty()) {
                    const int32_t v = cstk.back();
                    const int32_t *rv = bufs[cb[v]].data() + cs[v];
                    const int64_t e = ce[v];
                    int64_t t2 = cnx.back();
                    while (t2 < e && cm[(size_t)(rv[t2] - c0)] == j) t2++;
                    if (t2 == e) {
                        cstk.pop_back();
                        cnx.pop_back();
                        continue;
                    }
                    const int32_t w = rv[t2];
                    cnx.back() = t2 + 1;
                    cm[(size_t)(w - c0)] = j;
                    cfound.push_back(w);
                    if (w < j) {
                        cstk.push_back(w);
                        cnx.push_back(cd[w] + 1);
                    }
                }
            }
            std::sort(cfound.begin(), cfound.end());
            const std::vector<int32_t> &out = below[(size_t)i];
            cb[j] = bid;
            cs[j] = (int64_t)buf.size();
            buf.insert(buf.end(), out.begin(), out.end());
            buf.insert(buf.end(), cfound.begin(), cfound.end());
            const int64_t dc = std::lower_bound(cfound.begin(), cfound.end(), j) - cfound.begin();
            cl[j] = (int64_t)(out.size() + cfound.size());
            cd[j] = (int64_t)out.size() + dc;
            ce[j] = cl[j];
            // symmetric pruning of the chain's columns k with U(k,j) != 0
            for (int64_t q = 0; q < dc; q++) {
                const int32_t k = cfound[(size_t)q];
                if (pruned[k]) continue;
                const int32_t *rk = bufs[cb[k]].data() + cs[k];
                const int32_t *lb = rk + cd[k] + 1;
                const int32_t *le = rk + cl[k];
                const int32_t *it = std::lower_bound(lb, le, j);
                if (it != le && *it == j) {
                    ce[k] = (it - rk) + 1;
                    pruned[k] = 1;
                }
            }
            std::vector<int32_t>().swap(below[(size_t)i]);
            std::vector<int32_t>().swap(entry[(size_t)i]);
        }
    };
    // subtrees first, taken by threads as they finish
    std::atomic<int32_t> next{0};
    run_threads(ntask > 0 ? nth : 1, [&](int t) {
        scratch(scr[t]);
        for (int32_t i; (i = next.fetch_add(1)) < ntask;)
            for (int32_t j : cols[order[i]]) column(j, order[i], scr[t]);
    });
    // then the chains, each once the chains below it are done
    std::mutex mu;
    std::condition_variable cv;
    std::vector<int32_t> ready;
    for (int32_t c = 0; c < nchain; c++)
        if (pending[c] == 0 && c != tc) ready.push_back(c);
    int32_t remaining = nchain - (tc >= 0 ? 1 : 0);
    bool aborted = false;
    run_threads(nchain > 0 ? nth : 1, [&](int t) {
        if (scr[t].mark.empty()) scratch(scr[t]);
        try {
            for (;;) {
                int32_t c;
                {
                    std::unique_lock<std::mutex> lk(mu);
                    cv.wait(lk, [&] { return !ready.empty() || remaining == 0 || aborted; });
                    if (ready.empty()) return;
                    c = ready.back();
                    ready.pop_back();
                }
                for (int32_t j : chains[c]) column(j, ntask + c, scr[t]);
                {
                    std::lock_guard<std::mutex> lk(mu);
                    remaining--;
                    const int32_t p = parent[chains[c].back()];
                    if (p >= 0 && --pending[chain_of[p]] == 0 && chain_of[p] != tc) ready.push_back(chain_of[p]);
                }
                cv.notify_all();
            }
        } catch (...) {
            {
                std::lock_guard<std::mutex> lk(mu);
                aborted = true;
            }
            cv.notify_all();
            throw;
        }
    });
    if (tc >= 0) top_chain(chains[tc], ntask + tc);
    scr.clear();
    // ---- column order
    P.lu_colptr.assign((size_t)n + 1, 0);
    P.diag_pos.assign((size_t)n, 0);
    for (int32_t j = 0; j < n; j++) P.lu_colptr[j + 1] = P.lu_colptr[j] + cl[j];
    P.lu_rowidx.resize((size_t)P.lu_colptr[n]);
    const std::vector<int32_t> cut = column_ranges(n, P.lu_colptr.data(), nth);
    run_threads(nth, [&](int t) {
        for (int32_t j = cut[t]; j < cut[t + 1]; j++) {
            std::copy_n(bufs[cb[j]].data() + cs[j], cl[j], P.lu_rowidx.data() + P.lu_colptr[j]);
            P.diag_pos[j] = P.lu_colptr[j] + cd[j];
        }
    });
    return GLU_OK;
}

// Compressed-row views of the strict lower and strict upper parts.
// Each thread counts, then places, the entries of one range of columns;
// a row's entries from an earlier range come first, so every row lists its
// columns in ascending order.
void row_views(HostPlan &P) {
    const int32_t n = P.n;
    const int nth = analysis_threads();
    const std::vector<int32_t> cut = column_ranges(n, P.lu_colptr.data(), nth);
    // per thread, per row: entries of the thread's columns (then its offsets)
    std::vector<std::vector<int64_t>> lc((size_t)nth), uc((size_t)nth);
    run_threads(nth, [&](int t) {
        lc[t].assign((size_t)n, 0);
        uc[t].assign((size_t)n, 0);
        for (int32_t j = cut[t]; j < cut[t + 1]; j++) {
            for (int64_t p = P.lu_colptr[j]; p < P.diag_pos[j]; p++) uc[t][P.lu_rowidx[p]]++;
            for (int64_t p = P.diag_pos[j] + 1; p < P.lu_colptr[j + 1]; p++) lc[t][P.lu_rowidx[p]]++;
        }
    });
    P.lrow_ptr.assign((size_t)n + 1, 0);
    P.urow_ptr.assign((size_t)n + 1, 0);
    int64_t la = 0, ua = 0;
    for (int32_t i = 0; i < n; i++) {
        P.lrow_ptr[i] = la;
        P.urow_ptr[i] = ua;
        for (int t = 0; t < nth; t++) {
            const int64_t l = lc[t][i], u = uc[t][i];
            lc[t][i] = la;
            uc[t][i] = ua;
            la += l;
            ua += u;
        }
    }
    P.lrow_ptr[n] = la;
    P.urow_ptr[n] = ua;
    P.nnz_l = la;
    P.nnz_u = ua + n;
    P.lrow_col.resize((size_t)la);
    P.lrow_pos.resize((size_t)la);
    P.urow_col.resize((size_t)ua);
    P.urow_pos.resize((size_t)ua);
    run_threads(nth, [&](int t) {
        std::vector<int64_t> &lf = lc[t], &uf = uc[t];
        for (int32_t j = cut[t]; j < cut[t + 1]; j++) {
            for (int64_t p = P.lu_colptr[j]; p < P.diag_pos[j]; p++) {
                const int64_t q = uf[P.lu_rowidx[p]]++;
                P.urow_col[q] = j;
                P.urow_pos[q] = p;
            }
            for (int64_t p = P.diag_pos[j] + 1; p < P.lu_colptr[j + 1]; p++) {
                const int64_t q = lf[P.lu_rowidx[p]]++;
                P.lrow_col[q] = j;
                P.lrow_pos[q] = p;
            }
        }
    });
}

// ---------------------------------------------------------------------------
// Algorithm 4: deps(k) = { i < k : U(i,k) != 0 and L(:,i) not empty }
//                      u { i < k : L(k,i) != 0 }.
// Both lists are ascending (the rows of column k above the diagonal, and
// row k of the L view), so one merge gives the sorted, duplicate-free set.
void dependencies(HostPlan &P) {
    const int32_t n = P.n;
    P.dep_ptr.assign((size_t)n + 1, 0);
    P.dep_idx.clear();
    P.dep_idx.reserve((size_t)(P.nnz_l + P.nnz_u));
    auto has_l = [&](int32_t i) { return P.lu_colptr[i + 1] - 1 > P.diag_pos[i]; };
    for (int32_t k = 0; k < n; k++) {
        int64_t a = P.lu_colptr[k], ae = P.diag_pos[k];
        int64_t b = P.lrow_ptr[k], be = P.lrow_ptr[k + 1];
        while (a < ae || b < be) {
            // skip up-looking candidates whose L column is empty
            while (a < ae && !has_l(P.lu_rowidx[a])) a++;
            int32_t va = a < ae ? P.lu_rowidx[a] : INT32_MAX;
            int32_t vb = b < be ? P.lrow_col[b] : INT32_MAX;
            if (va == INT32_MAX && vb == INT32_MAX) break;
            if (va <= vb) {
                P.dep_idx.push_back(va);
                a++;
                if (va == vb) b++;
            } else {
                P.dep_idx.push_back(vb);
                b++;
            }
        }
        P.dep_ptr[k + 1] = (int64_t)P.dep_idx.size();
    }
}

// The levels' column lists from level_of: columns of a level ascending.
void group_levels(HostPlan &P) {
    const int32_t n = P.n;
    int32_t nl = n > 0 ? 1 : 0;
    for (int32_t k = 0; k < n; k++) nl = std::max(nl, P.level_of[k] + 1);
    P.level_ptr.assign((size_t)nl + 1, 0);
    for (int32_t k = 0; k < n; k++) P.level_ptr[P.level_of[k] + 1]++;
    for (int32_t l = 0; l < nl; l++) P.level_ptr[l + 1] += P.level_ptr[l];
    P.level_cols.resize((size_t)n);
    std::vector<int32_t> f(P.level_ptr.begin(), P.level_ptr.end() - 1);
    for (int32_t k = 0; k < n; k++) P.level_cols[f[P.level_of[k]]++] = k;
    P.max_level_width = 0;
    for (int32_t l = 0; l < nl; l++)
        P.max_level_width = std::max(P.max_level_width, P.level_ptr[l + 1] - P.level_ptr[l]);
}

// Longest-path levels; columns of a level ascending.
void levelize(HostPlan &P) {
    const int32_t n = P.n;
    P.level_of.assign((size_t)n, 0);
    for (int32_t k = 0; k < n; k++) {
        int32_t lv = 0;
        for (int64_t p = P.dep_ptr[k]; p < P.dep_ptr[k + 1]; p++)
            lv = std::max(lv, P.level_of[P.dep_idx[p]] + 1);
        P.level_of[k] = lv;
    }
    group_levels(P);
}

// ---------------------------------------------------------------------------
// The update schedule.  Level l's sources are its columns j with a non-empty
// L(:,j); each source updates every target k with U(j,k) != 0 (Algorithm 5).
// The pairs (j,k) of a level are grouped by target; a group with few sources
// becomes KIND_ROW tasks (split by row ranges when large), a group with many
// sources becomes one KIND_SRC task per touched 32-position chunk of column
// k.  Each level's kernel also normalizes the previous level's L columns.
int schedule(HostPlan &P, const glu_options &opt, int num_sms) {
    const int32_t n = P.n;
    const int32_t nl = (int32_t)P.level_ptr.size() - 1;
    const int64_t piece = opt.piece_updates > 0 ? opt.piece_updates : 1024;
    // task-size thresholds; the environment overrides them for sweeps (every
    // value gives a valid schedule)
    auto env_int = [](const char *name, int64_t dflt, int64_t lo, int64_t hi) {
        const char *e = std::getenv(name);
        return e ? std::max(lo, std::min(hi, (int64_t)std::atoll(e))) : dflt;
    };
    // groups with at least this many sources use KIND_SRC chunk tasks
    const int32_t src_min = opt.src_min > 0 ? std::max<int32_t>(2, opt.src_min)
                                            : (int32_t)env_int("GLU_SRC_MIN", 5, 2, 1 << 20);
    auto lstart = [&](int32_t j) { return P.diag_pos[j] + 1; };
    auto lcount = [&](int32_t j) { return (int32_t)(P.lu_colptr[j + 1] - P.diag_pos[j] - 1); };

    // pairs, bucketed by the source's level; scanning targets k ascending
    // (and rows j ascending inside column k) leaves every bucket sorted by
    // (k, j).
    // (a counting sort by level over ranges of target columns, one per
    // thread; a thread's columns precede the next thread's, so the order
    // within a bucket is the same as a sequential scan's)
    const int nth = analysis_threads();
    const std::vector<int32_t> kcut = column_ranges(n, P.lu_colptr.data(), nth);
    std::vector<std::vector<int64_t>> lcnt((size_t)nth);
    run_threads(nth, [&](int t) {
        lcnt[t].assign((size_t)nl, 0);
        for (int32_t k = kcut[t]; k < kcut[t + 1]; k++)
            for (int64_t p = P.lu_colptr[k]; p < P.diag_pos[k]; p++) {
                const int32_t j = P.lu_rowidx[p];
                if (lcount(j) > 0) lcnt[t][P.level_of[j]]++;
            }
    });
    std::vector<int64_t> lvl_pair_ptr((size_t)nl + 1, 0);
    for (int32_t l = 0; l < nl; l++) {
        int64_t at = lvl_pair_ptr[l];
        for (int t = 0; t < nth; t++) {
            const int64_t c = lcnt[t][l];
            lcnt[t][l] = at;     // now this thread's first slot in bucket l
            at += c;
        }
        lvl_pair_ptr[l + 1] = at;
    }
    const int64_t npairs = lvl_pair_ptr[nl];
    P.pair_j.resize((size_t)npairs);
    P.pair_k.resize((size_t)npairs);
    P.pair_pos.resize((size_t)npairs);
    P.pair_map.resize((size_t)npairs + 1);
    run_threads(nth, [&](int t) {
        std::vector<int64_t> &f = lcnt[t];
        for (int32_t k = kcut[t]; k < kcut[t + 1]; k++)
            for (int64_t p = P.lu_colptr[k]; p < P.diag_pos[k]; p++) {
                const int32_t j = P.lu_rowidx[p];
                if (lcount(j) == 0) continue;
                const int64_t q = f[P.level_of[j]]++;
                P.pair_j[q] = j;
                P.pair_k[q] = k;
                P.pair_pos[q] = p;
            }
    });
    // pair_map: exclusive prefix sum of the sources' L counts, by chunks
    std::vector<int64_t> csum((size_t)nth + 1, 0);
    auto chunk = [&](int t) { return npairs * t / nth; };
    run_threads(nth, [&](int t) {
        int64_t s = 0;
        for (int64_t q = chunk(t); q < chunk(t + 1); q++) s += lcount(P.pair_j[q]);
        csum[t + 1] = s;
    });
    for (int t = 0; t < nth; t++) csum[t + 1] += csum[t];
    run_threads(nth, [&](int t) {
        int64_t a = csum[t];
        for (int64_t q = chunk(t); q < chunk(t + 1); q++) {
            P.pair_map[q] = a;
            a += lcount(P.pair_j[q]);
        }
    });
    const int64_t acc = csum[nth];
    P.pair_map[npairs] = acc;
    P.n_updates = acc;
    const double ts_pairs = now_ms();
    if (opt.verbose)
        std::fprintf(stderr, "glu_analyze: column schedule: %lld pairs, %lld updates\n", (long long)npairs,
                     (long long)acc);
    if (npairs > INT32_MAX) return GLU_ERR_TOO_LARGE;   // PSeg.pair is 32-bit

    P.tasks.clear();
    P.lvl_task_ptr.assign((size_t)nl + 1, 0);
    P.lvl_row_ptr.assign((size_t)nl, 0);
    P.lvl_lane_ptr.assign((size_t)nl, 0);
    // tasks up to this many updates (and lane_segs segments) run on one lane
    // (32 and 2 measured best on the 200k-unknown mesh: 22.5 ms per FP64
    // refactorization against 23.5 ms with 64 and 4, factors bitwise equal)
    const int64_t lane_max = opt.lane_max > 0 ? opt.lane_max : env_int("GLU_LANE_MAX", 32, 1, 1 << 20);
    const int32_t lane_segs = opt.lane_segs > 0 ? std::min<int32_t>(64, opt.lane_segs)
                                                : (int32_t)env_int("GLU_LANE_SEGS", 2, 1, 64);
    P.level_mode.assign((size_t)nl, 0);
    (void)num_sms;
    // Levels are scheduled independently: contiguous ranges of levels run on
    // host threads, each into its own segment and task lists (task segment
    // indices and level task offsets relative to them), concatenated in level
    // order afterwards -- the result does not depend on the thread count.
    struct Part {
        std::vector<PSeg> psegs;
        std::vector<Task> tasks;
        std::vector<int32_t> tend, rowp, lanep;   // per level, relative to tasks
        std::vector<int8_t> mode;
    };
    // host-side fault injection for tests: GLU_TEST_FAIL_LEVEL=<l> makes the
    // scheduling of level l fail as an allocation would
    const char *fail_env = std::getenv("GLU_TEST_FAIL_LEVEL");
    const int32_t fail_level = fail_env ? std::atoi(fail_env) : -1;
    auto run_levels = [&](int32_t l0, int32_t l1, Part &pt) {
    std::vector<PSeg> &psegs = pt.psegs;
    std::vector<Task> lvl_tasks;
    // per-chunk scratch for splitting one group
    std::vector<int64_t> chunk_work;
    // a group's segments per chunk: routed in (source, chunk) order into one
    // list, then placed chunk by chunk keeping that order (a stable counting
    // sort); chunk ch's are routed[cstart[ch] - ccount[ch], cstart[ch])
    std::vector<int32_t> ccount;
    std::vector<int64_t> cstart;
    std::vector<std::pair<int32_t, PSeg>> flat;
    std::vector<PSeg> routed;
    struct SegSpan {
        const PSeg *b;
        size_t n;
        size_t size() const { return n; }
        const PSeg &operator[](size_t i) const { return b[i]; }
        const PSeg *begin() const { return b; }
        const PSeg *end() const { return b + n; }
    };
    auto chunk_segs = [&](int32_t ch) {
        return SegSpan{routed.data() + cstart[(size_t)ch] - ccount[(size_t)ch], (size_t)ccount[(size_t)ch]};
    };
    std::vector<int32_t> touched;
    std::vector<int32_t> cuts;   // a heavily shared chunk's segment cuts
    std::vector<PSeg> sub;
    for (int32_t l = l0; l < l1; l++) {
        if (l == fail_level) throw std::bad_alloc();
        lvl_tasks.clear();
        int64_t g = lvl_pair_ptr[l];
        const int64_t ge_l = lvl_pair_ptr[l + 1];
        const int64_t piece_l = piece;
        while (g < ge_l) {
            const int32_t k = P.pair_k[g];
            int64_t ge = g;
            int64_t work = 0;
            while (ge < ge_l && P.pair_k[ge] == k) { work += lcount(P.pair_j[ge]); ge++; }
            const int64_t nsrc = ge - g;
            if (nsrc < src_min && work <= piece_l) {
                Task t{(int32_t)0, 0, KIND_ROW, 0, 0, work};
                t.seg_begin = (int32_t)psegs.size();
                for (int64_t q = g; q < ge; q++)
                    psegs.push_back(PSeg{(int32_t)q, 0, lcount(P.pair_j[q]), 0});
                t.seg_end = (int32_t)psegs.size();
                lvl_tasks.push_back(t);
                g = ge;
                continue;
            }
            // Split column k into 32-position chunks; route every source's
            // rows to the chunks they fall in.
            const int64_t c0 = P.lu_colptr[k];
            const int64_t clen = P.lu_colptr[k + 1] - c0;
            const int64_t nchunks = (clen + SRC_SLOTS - 1) / SRC_SLOTS;
            if ((int64_t)chunk_work.size() < nchunks) {
                chunk_work.resize((size_t)nchunks, 0);
                ccount.resize((size_t)nchunks, 0);
                cstart.resize((size_t)nchunks, 0);
            }
            touched.clear();
            const int32_t *krows = P.lu_rowidx.data() + c0;
            for (int64_t q = g; q < ge; q++) {
                const int32_t j = P.pair_j[q];
                const int32_t *L = P.lu_rowidx.data() + lstart(j);
                const int32_t lj = lcount(j);
                int32_t t = 0;
                // rows of L(:,j) lie below row j, which sits at pair_pos in column k;
                // both lists ascend, so each search starts where the last one ended
                int64_t pos = P.pair_pos[q] - c0 + 1;
                while (t < lj) {
                    // position of row L[t] inside column k
                    pos = gallop_lower_bound(krows + pos, krows + clen, L[t]) - krows;
                    int64_t ch = pos / SRC_SLOTS;
                    int64_t chend = std::min<int64_t>((ch + 1) * SRC_SLOTS, clen);
                    int32_t t1;
                    if (chend >= clen) {
                        t1 = lj;
                    } else {
                        int32_t endrow = krows[chend];
                        t1 = (int32_t)(gallop_lower_bound(L + t, L + lj, endrow) - L);
                    }
                    if (ccount[(size_t)ch]++ == 0) touched.push_back((int32_t)ch);
                    flat.emplace_back((int32_t)ch, PSeg{(int32_t)q, t, t1, 0});
                    chunk_work[ch] += t1 - t;
                    t = t1;
                }
            }
            std::sort(touched.begin(), touched.end());
            {
                int64_t at = 0;
                for (int32_t ch : touched) {
                    cstart[(size_t)ch] = at;
                    at += ccount[(size_t)ch];
                }
                routed.resize((size_t)at);
                for (const auto &e : flat) routed[(size_t)cstart[(size_t)e.first]++] = e.second;
                flat.clear();
            }
            if (nsrc >= src_min) {
                // Chunks reached by two or more segments become KIND_SRC
                // tasks.  A chunk reached by one segment holds rows that no
                // other source of this group updates: those segments need no
                // ordering, so consecutive ones of a source merge (up to
                // piece_l rows) and are packed into small tasks.
                std::vector<PSeg> priv;
                auto add_priv = [&](const PSeg &sg) {
                    if (!priv.empty() && priv.back().pair == sg.pair && priv.back().t1 == sg.t0 &&
                        priv.back().t1 - priv.back().t0 + (sg.t1 - sg.t0) <= piece_l)
                        priv.back().t1 = sg.t1;
                    else
                        priv.push_back(sg);
                };
                for (int32_t ch : touched) {
                    const SegSpan cs = chunk_segs(ch);
                    const int64_t cb = (int64_t)ch * SRC_SLOTS;
                    const int64_t cl = std::min<int64_t>(SRC_SLOTS, clen - cb);
                    if (cs.size() < 2) {
                        add_priv(cs[0]);
                    } else if (chunk_work[ch] <= piece_l) {
                        Task t{(int32_t)psegs.size(), 0, KIND_SRC, (int32_t)cl, c0 + cb, chunk_work[ch]};
                        psegs.insert(psegs.end(), cs.begin(), cs.end());
                        t.seg_end = (int32_t)psegs.size();
                        lvl_tasks.push_back(t);
                    } else {
                        // A heavily shared chunk: a task's time is its lanes'
                        // serial work, so split the chunk's positions into
                        // equal parts (16, 8, ... positions) until each part
                        // holds at most piece_l updates.  A segment's rows
                        // split at the parts' first rows.
                        // a part's updates are the rows of the chunk's segments
                        // that sit on its positions: count them per position once
                        // (each segment's rows and the column's rows both ascend)
                        std::array<int64_t, SRC_SLOTS> at{};
                        for (const PSeg &sg : cs) {
                            const int32_t *L = P.lu_rowidx.data() + lstart(P.pair_j[sg.pair]);
                            int64_t p = cb;
                            for (int32_t t = sg.t0; t < sg.t1; t++) {
                                while (krows[p] < L[t]) p++;
                                at[(size_t)(p - cb)]++;
                            }
                        }
                        int64_t part = SRC_SLOTS;
                        while (part > 1) {
                            int64_t worst = 0;
                            for (int64_t p0 = 0; p0 < cl; p0 += part) {
                                int64_t w = 0;
                                for (int64_t q = p0; q < std::min(p0 + part, cl); q++) w += at[(size_t)q];
                                worst = std::max(worst, w);
                            }
                            if (worst <= piece_l) break;
                            part /= 2;
                        }
                        // each segment cut at the parts' first positions: cut[i] is
                        // its first row on a position of part i or later
                        const int64_t nparts = (cl + part - 1) / part;
                        cuts.resize(cs.size() * (size_t)(nparts + 1));
                        for (size_t si = 0; si < cs.size(); si++) {
                            const PSeg &sg = cs[si];
                            const int32_t *L = P.lu_rowidx.data() + lstart(P.pair_j[sg.pair]);
                            int32_t *cut = cuts.data() + si * (size_t)(nparts + 1);
                            int32_t t = sg.t0;
                            int64_t p = cb;
                            cut[0] = sg.t0;
                            for (int64_t i = 1; i < nparts; i++) {
                                while (t < sg.t1) {
                                    while (krows[p] < L[t]) p++;
                                    if (p >= cb + i * part) break;
                                    t++;
                                }
                                cut[i] = t;
                            }
                            cut[nparts] = sg.t1;
                        }
                        for (int64_t i = 0; i < nparts; i++) {
                            const int64_t p0 = cb + i * part, p1 = std::min(p0 + part, cb + cl);
                            sub.clear();
                            int64_t w = 0;
                            for (size_t si = 0; si < cs.size(); si++) {
                                const int32_t *cut = cuts.data() + si * (size_t)(nparts + 1);
                                if (cut[i + 1] > cut[i]) {
                                    sub.push_back(PSeg{cs[si].pair, cut[i], cut[i + 1], 0});
                                    w += cut[i + 1] - cut[i];
                                }
                            }
                            if (sub.empty()) continue;
                            if (sub.size() == 1) { add_priv(sub[0]); continue; }
                            Task t{(int32_t)psegs.size(), 0, KIND_SRC, (int32_t)(p1 - p0), c0 + p0, w};
                            psegs.insert(psegs.end(), sub.begin(), sub.end());
                            t.seg_end = (int32_t)psegs.size();
                            lvl_tasks.push_back(t);
                        }
                    }
                    ccount[(size_t)ch] = 0;
                    chunk_work[ch] = 0;
                }
                // (private segments are independent: small packs run on one
                // lane each, a large segment alone on a warp)
                size_t a = 0;
                while (a < priv.size()) {
                    Task t{(int32_t)psegs.size(), 0, KIND_ROW, 0, 0, 0};
                    while (a < priv.size() &&
                           (t.work == 0 || (t.work + (priv[a].t1 - priv[a].t0) <= lane_max &&
                                            (int32_t)psegs.size() - t.seg_begin < 2))) {
                        t.work += priv[a].t1 - priv[a].t0;
                        psegs.push_back(priv[a]);
                        a++;
                    }
                    t.seg_end = (int32_t)psegs.size();
                    lvl_tasks.push_back(t);
                }
            } else {                // few sources, much work: consecutive chunks merged into
                // KIND_ROW pieces of about `piece_l` updates; inside a piece
                // the segments of one source are contiguous in t, so they
                // merge into one, kept in ascending source order.
                size_t a = 0;
                while (a < touched.size()) {
                    size_t b = a;
                    int64_t w = 0;
                    while (b < touched.size() && (b == a || w + chunk_work[touched[b]] <= piece_l)) {
                        w += chunk_work[touched[b]];
                        b++;
                    }
                    Task t{(int32_t)psegs.size(), 0, KIND_ROW, 0, 0, w};
                    for (int64_t q = g; q < ge; q++) {
                        int32_t lo = INT32_MAX, hi = -1;
                        for (size_t c = a; c < b; c++)
                            for (const PSeg &s : chunk_segs(touched[c]))
                                if (s.pair == (int32_t)q) { lo = std::min(lo, s.t0); hi = std::max(hi, s.t1); }
                        if (hi > lo) psegs.push_back(PSeg{(int32_t)q, lo, hi, 0});
                    }
                    t.seg_end = (int32_t)psegs.size();
                    lvl_tasks.push_back(t);
                    a = b;
                }
                for (int32_t ch : touched) { ccount[(size_t)ch] = 0; chunk_work[ch] = 0; }
            }
            g = ge;
        }
        // kinds: small tasks run on one lane; a chunk task with short
        // segments keeps lanes over segments; the rest lanes over rows
        // (a chunk task's segments hold at most 32 rows each, so lanes over
        // rows would leave most lanes idle and pay one round trip per segment)
        // The level's time is the longest serial chain of one work item, and
        // every segment applied in sequence adds a few dependent memory round
        // trips, so a lane task holds at most lane_segs (2) segments.
        for (Task &t : lvl_tasks) {
            const int32_t ns = t.seg_end - t.seg_begin;
            if (t.kind == KIND_SRC && ns >= 4) continue;
            t.kind = (t.work <= lane_max && ns <= lane_segs) ? KIND_LANE : KIND_ROW;
        }
        // grouped by kind, largest first inside a kind: warps take tasks in order
        std::stable_sort(lvl_tasks.begin(), lvl_tasks.end(), [](const Task &a, const Task &b) {
            const int ka = a.kind == KIND_SRC ? 0 : (a.kind == KIND_ROW ? 1 : 2);
            const int kb = b.kind == KIND_SRC ? 0 : (b.kind == KIND_ROW ? 1 : 2);
            if (ka != kb) return ka < kb;
            return a.work > b.work;
        });
        const int32_t tb = (int32_t)pt.tasks.size();
        pt.tasks.insert(pt.tasks.end(), lvl_tasks.begin(), lvl_tasks.end());
        const int32_t te = (int32_t)pt.tasks.size();
        int32_t r = tb, ln = tb;
        for (int32_t q = tb; q < te; q++) {
            if (pt.tasks[q].kind == KIND_SRC) { r = q + 1; ln = q + 1; }
            else if (pt.tasks[q].kind == KIND_ROW) ln = q + 1;
        }
        pt.tend.push_back(te);
        pt.rowp.push_back(r);
        pt.lanep.push_back(ln);
        const int32_t width = P.level_ptr[l + 1] - P.level_ptr[l];
        const int32_t tail = opt.tail_threshold > 0 ? opt.tail_threshold : 0;
        const int32_t wide = opt.wide_threshold > 0 ? opt.wide_threshold : 256;
        int8_t mode = width <= tail ? 2 : (width > wide ? 0 : 1);
        if (opt.mode_force >= 0 && opt.mode_force <= 2) mode = (int8_t)opt.mode_force;
        pt.mode.push_back(mode);
    }
    };
    // Ranges of levels ("parts") with about equal numbers of pairs, several
    // per thread: threads take the next part as they finish (a pair's work
    // varies a lot), and the parts are concatenated in level order
    // afterwards -- the result depends on neither the thread count nor the
    // cut.
    const int32_t nparts = std::max(1, std::min(nl, nth * 8));
    std::vector<int32_t> cut(1, 0);
    for (int32_t t = 1; t < nparts; t++) {
        const int64_t want = npairs * t / nparts;
        const int32_t l = (int32_t)(std::lower_bound(lvl_pair_ptr.begin(), lvl_pair_ptr.end(), want) -
                                    lvl_pair_ptr.begin());
        cut.push_back(std::max(cut.back(), std::min(l, nl)));
    }
    cut.push_back(nl);
    std::vector<Part> parts(cut.size() - 1);
    // runs fn(t) for every part t on nth threads (this one included); an
    // allocation failure on any of them is rethrown here after all joined
    auto for_parts = [&](auto fn) {
        std::atomic<size_t> next{0};
        std::atomic<bool> failed{false};
        auto worker = [&] {
            try {
                for (size_t t; !failed && (t = next.fetch_add(1)) < parts.size();) fn(t);
            } catch (const std::bad_alloc &) {
                failed = true;
            }
        };
        std::vector<std::thread> th;
        th.reserve((size_t)nth);
        for (int t = 1; t < nth; t++) spawn_or_run(th, worker);
        worker();
        for (std::thread &x : th) x.join();
        if (failed) throw std::bad_alloc();
    };
    for_parts([&](size_t t) { run_levels(cut[t], cut[t + 1], parts[t]); });
    const double ts_tasks = now_ms();
    // concatenate: each part's tasks and segments go to their offsets (the
    // segments flattened into self-contained records), in parallel
    std::vector<int64_t> sbase(parts.size() + 1, 0), tbase(parts.size() + 1, 0);
    for (size_t t = 0; t < parts.size(); t++) {
        sbase[t + 1] = sbase[t] + (int64_t)parts[t].psegs.size();
        tbase[t + 1] = tbase[t] + (int64_t)parts[t].tasks.size();
    }
    // segment and task indices are 32-bit in the device records
    if (sbase[parts.size()] > INT32_MAX || tbase[parts.size()] > INT32_MAX) return GLU_ERR_TOO_LARGE;
    P.tasks.resize((size_t)tbase[parts.size()]);
    P.segs.resize((size_t)sbase[parts.size()]);
    auto place = [&](size_t t) {
        const Part &pt = parts[t];
        const int32_t sb = (int32_t)sbase[t];
        for (size_t q = 0; q < pt.tasks.size(); q++) {
            Task tk = pt.tasks[q];
            tk.seg_begin += sb;
            tk.seg_end += sb;
            P.tasks[(size_t)tbase[t] + q] = tk;
        }
        for (size_t q = 0; q < pt.psegs.size(); q++) {
            const PSeg &ps = pt.psegs[q];
            Seg &sg = P.segs[(size_t)sbase[t] + q];
            sg.pos = P.pair_pos[ps.pair];
            sg.dj = P.diag_pos[P.pair_j[ps.pair]];
            sg.rb = ps.pair;          // the device replaces it with the segment's runs
            sg.t0 = ps.t0;
            sg.t1 = ps.t1;
        }
    };
    for_parts(place);
    for (size_t t = 0; t < parts.size(); t++) {
        const Part &pt = parts[t];
        const int32_t tb = (int32_t)tbase[t];
        for (int32_t q = 0; q < cut[t + 1] - cut[t]; q++) {
            const int32_t l = cut[t] + q;
            P.lvl_task_ptr[l + 1] = tb + pt.tend[q];
            P.lvl_row_ptr[l] = tb + pt.rowp[q];
            P.lvl_lane_ptr[l] = tb + pt.lanep[q];
            P.level_mode[l] = pt.mode[q];
            P.levels_by_mode[pt.mode[q]]++;
        }
    }
    parts.clear();
    const double ts_flat = now_ms();

    // normalization items: level l's columns run in level l+1's kernel; the
    // last level's columns in the final pass
    const int32_t nchunk = 256;   // rows per item: 8 divisions per lane
    P.norms.clear();
    P.lvl_norm_ptr.assign((size_t)nl + 2, 0);
    for (int32_t l = 0; l <= nl; l++) {
        if (l >= 1) {
            for (int32_t c = P.level_ptr[l - 1]; c < P.level_ptr[l]; c++) {
                int32_t j = P.level_cols[c];
                int32_t lj = lcount(j);
                for (int32_t t = 0; t < lj; t += nchunk)
                    P.norms.push_back(NormItem{j, t, std::min(lj, t + nchunk), 0});
            }
        }
        P.lvl_norm_ptr[l + 1] = (int32_t)P.norms.size();
    }
    if (opt.verbose)
        std::fprintf(stderr, "glu_analyze: schedule phases: tasks %.0f ms (%d threads), flatten %.0f ms, "
                     "normalization items %.0f ms; %zu segments, %zu tasks\n", ts_tasks - ts_pairs, nth,
                     ts_flat - ts_tasks, now_ms() - ts_flat, P.segs.size(), P.tasks.size());
    P.has_schedule = true;
    return GLU_OK;
}

// Dense diagonal blocks ("supernodes") of the solve among the rows [0, t0):
// maximal runs [c0, c1) in which L(B, B) is dense lower and U(B, B) dense
// upper, cut into pieces of at most sn_max rows; pieces of at least SN_MIN
// rows are kept.
std::vector<std::pair<int32_t, int32_t>> solve_blocks(const HostPlan &P, int32_t t0, int32_t sn_max) {
    std::vector<std::pair<int32_t, int32_t>> out;
    auto flush = [&](int32_t c0, int32_t c1) {
        for (int32_t a = c0; a < c1; a += sn_max) {
            const int32_t b = std::min(c1, a + sn_max);
            if (b - a >= SN_MIN) out.emplace_back(a, b);
        }
    };
    int32_t c0 = 0;
    for (int32_t i = 1; i <= t0; i++) {
        bool ext = i < t0;
        if (ext) {
            // L row i holds columns c0..i-1 iff i - c0 of its entries are >= c0
            const int32_t *lc = P.lrow_col.data();
            const int64_t lb = P.lrow_ptr[i], le = P.lrow_ptr[i + 1];
            const int64_t nl = le - (std::lower_bound(lc + lb, lc + le, c0) - lc);
            // U column i holds rows c0..i-1 iff i - c0 of its rows above the diagonal are >= c0
            const int32_t *ur = P.lu_rowidx.data();
            const int64_t ub = P.lu_colptr[i], ue = P.diag_pos[i];
            const int64_t nu = ue - (std::lower_bound(ur + ub, ur + ue, c0) - ur);
            ext = nl == i - c0 && nu == i - c0;
        }
        if (!ext) {
            flush(c0, i);
            c0 = i;
        }
    }
    return out;
}

// Dataflow schedule of the solve for a chunk size and a dense tail [t0, n).
// Items: a row (its dot product, or the sum of its chunks' partials when it
// has more than `chunk` entries), a chunk (a partial dot product of at most
// `chunk` entries), and -- when `blocks` > 0 -- a dense diagonal block of
// the solve (at most `blocks` rows), whose rows' entries outside the block are always chunks and whose
// own triangle one warp sweeps.  Forward items cover the rows before the tail
// and the tail rows' partial sums over the columns before it (forward chunks
// tail_cb[i]..tail_ce[i]-1); backward items the rows before the tail.  Each
// item comes after everything it reads: levels are longest paths with every
// block contracted to one node, a chunk sits at 1 + the highest level it
// reads and before the rows of its level.  snx lists, per block, the first
// chunk of each of its rows and the end (offset in the item's third field).
void build_df(const HostPlan &P, int64_t chunk, int32_t t0, int32_t blocks, std::vector<int32_t> &out,
              std::vector<SolveChunk> &dff, std::vector<SolveChunk> &dfb, std::vector<int32_t> &tcb,
              std::vector<int32_t> &tce, int32_t &nfwd, std::vector<int32_t> &snx_f, std::vector<int32_t> &snx_b) {
    const int32_t n = P.n;
    const auto bl = blocks > 0 ? solve_blocks(P, t0, blocks) : std::vector<std::pair<int32_t, int32_t>>();
    std::vector<int32_t> bof((size_t)n, -1);
    for (size_t q = 0; q < bl.size(); q++)
        for (int32_t i = bl[q].first; i < bl[q].second; i++) bof[i] = (int32_t)q;
    dff.clear();
    dfb.clear();
    snx_f.clear();
    snx_b.clear();
    tcb.assign((size_t)(n - t0), 0);
    tce.assign((size_t)(n - t0), 0);
    struct Rec { int32_t level, type, seq; std::array<int32_t, 8> item; };
    auto add_chunks = [&](std::vector<SolveChunk> &ch, int64_t b, int64_t e) {
        for (int64_t p = b; p < e; p += chunk) ch.push_back(SolveChunk{p, std::min(e, p + chunk)});
    };
    // a record per chunk from c_begin on, at 1 + the highest level its
    // entries read; returns the highest of those (the level of a row made of
    // these chunks), 0 without chunks
    auto chunk_recs = [&](bool bwd, const std::vector<SolveChunk> &ch, int32_t c_begin, const std::vector<int32_t> &lv,
                          const int32_t *colv, int32_t row, std::vector<Rec> &recs) {
        int32_t top = 0;
        for (int32_t c = c_begin; c < (int32_t)ch.size(); c++) {
            int32_t m = 0;
            for (int64_t p = ch[c].p0; p < ch[c].p1; p++) m = std::max(m, lv[colv[p]] + 1);
            recs.push_back(Rec{m, 0, (int32_t)recs.size(), {row, 0, 0, c, (bwd ? 1 : 0) | 2, 0, 0, 0}});
            top = std::max(top, m);
        }
        return top;
    };
    // records in (level, type) order, each key's records in the order they
    // were made: a stable counting sort on 2 * level + type
    auto finish = [](std::vector<Rec> &recs) {
        int32_t maxl = 0;
        for (const Rec &r : recs) maxl = std::max(maxl, r.level);
        std::vector<int64_t> at((size_t)2 * ((size_t)maxl + 1) + 1, 0);
        for (const Rec &r : recs) at[(size_t)(2 * r.level + r.type) + 1]++;
        for (size_t k = 1; k < at.size(); k++) at[k] += at[k - 1];
        std::vector<Rec> sorted(recs.size());
        for (const Rec &r : recs) sorted[(size_t)at[(size_t)(2 * r.level + r.type)]++] = r;
        recs.swap(sorted);
    };
    // ---- forward (unit L), rows ascending
    std::vector<int32_t> lf((size_t)n, 0);
    std::vector<Rec> frec;
    for (int32_t i = 0; i < t0;) {
        if (bof[i] >= 0) {
            const int32_t c0 = bl[bof[i]].first, c1 = bl[bof[i]].second;
            int32_t lev = 0;
            const int32_t off = (int32_t)snx_f.size();
            for (int32_t r = c0; r < c1; r++) {
                // entries before the block: all but the last r - c0 (all in chunks)
                const int64_t b = P.lrow_ptr[r], e = P.lrow_ptr[r + 1] - (r - c0);
                const int32_t cb = (int32_t)dff.size();
                snx_f.push_back(cb);
                add_chunks(dff, b, e);
                lev = std::max(lev, chunk_recs(false, dff, cb, lf, P.lrow_col.data(), r, frec));
            }
            snx_f.push_back((int32_t)dff.size());
            for (int32_t r = c0; r < c1; r++) lf[r] = lev;
            frec.push_back(Rec{lev, 1, (int32_t)frec.size(), {c0, c1, off, -1, 4, 0, 0, 0}});
            i = c1;
            continue;
        }
        const int64_t b = P.lrow_ptr[i], e = P.lrow_ptr[i + 1];
        int32_t lev = 0;
        int32_t cb = (int32_t)dff.size(), ce = cb;
        if (e - b > chunk) {   // the row's level from its chunks' (its entries read columns < i)
            add_chunks(dff, b, e);
            ce = (int32_t)dff.size();
            lev = chunk_recs(false, dff, cb, lf, P.lrow_col.data(), i, frec);
        } else {
            for (int64_t p = b; p < e; p++) lev = std::max(lev, lf[P.lrow_col[p]] + 1);
        }
        lf[i] = lev;
        frec.push_back(Rec{lev, 1, (int32_t)frec.size(), {i, cb, ce, -1, 0, 0, 0, 0}});
        i++;
    }
    for (int32_t i = t0; i < n; i++) {
        // entries of tail row i in columns < t0 form a prefix (columns ascend)
        const int64_t b = P.lrow_ptr[i];
        int64_t e = b;
        while (e < P.lrow_ptr[i + 1] && P.lrow_col[e] < t0) e++;
        const int32_t cb = (int32_t)dff.size();
        add_chunks(dff, b, e);
        tcb[i - t0] = cb;
        tce[i - t0] = (int32_t)dff.size();
        chunk_recs(false, dff, cb, lf, P.lrow_col.data(), i, frec);
    }
    finish(frec);
    // ---- backward (U), rows descending; the tail is solved before
    std::vector<int32_t> lb((size_t)n, -1);
    std::vector<Rec> brec;
    for (int32_t i = t0 - 1; i >= 0;) {
        if (bof[i] >= 0) {
            const int32_t c0 = bl[bof[i]].first, c1 = bl[bof[i]].second;
            int32_t lev = 0;
            const int32_t off = (int32_t)snx_b.size();
            for (int32_t r = c0; r < c1; r++) {
                // U row r's entries after the block: all but the first c1 - 1 - r (all in chunks)
                const int64_t b = P.urow_ptr[r] + (c1 - 1 - r), e = P.urow_ptr[r + 1];
                const int32_t cb = (int32_t)dfb.size();
                snx_b.push_back(cb);
                add_chunks(dfb, b, e);
                lev = std::max(lev, chunk_recs(true, dfb, cb, lb, P.urow_col.data(), r, brec));
            }
            snx_b.push_back((int32_t)dfb.size());
            for (int32_t r = c0; r < c1; r++) lb[r] = lev;
            brec.push_back(Rec{lev, 1, (int32_t)brec.size(), {c0, c1, off, -1, 1 | 4, 0, 0, 0}});
            i = c0 - 1;
            continue;
        }
        const int64_t b = P.urow_ptr[i], e = P.urow_ptr[i + 1];
        int32_t lev = 0;
        int32_t cb = (int32_t)dfb.size(), ce = cb;
        if (e - b > chunk) {   // the row's level from its chunks' (its entries read columns > i)
            add_chunks(dfb, b, e);
            ce = (int32_t)dfb.size();
            lev = chunk_recs(true, dfb, cb, lb, P.urow_col.data(), i, brec);
        } else {
            for (int64_t p = b; p < e; p++) lev = std::max(lev, lb[P.urow_col[p]] + 1);
        }
        lb[i] = lev;
        brec.push_back(Rec{lev, 1, (int32_t)brec.size(), {i, cb, ce, -1, 1, 0, 0, 0}});
        i--;
    }
    finish(brec);
    out.clear();
    for (const Rec &r : frec) out.insert(out.end(), r.item.begin(), r.item.end());
    nfwd = (int32_t)(out.size() / 8);
    for (const Rec &r : brec) out.insert(out.end(), r.item.begin(), r.item.end());
}

// ---------------------------------------------------------------------------
// The supernodal schedule.  Supernodes: maximal runs of at most BSN_MAX
// columns whose diagonal block is dense and whose columns have the same rows
// below the run.  Block levels: longest paths of the dependency graph
// (Algorithm 4) with each supernode contracted to one node.  Pairs: for each
// supernode B, every column k past B with U(j, k) != 0 for some j in B; by
// the fill theorem the rows of B present in column k form a suffix of B and
// column k holds every row of R_B.
void block_schedule(HostPlan &P) {
    const int32_t n = P.n;
    std::vector<int32_t> &c0v = P.sn_c0;
    c0v.assign(1, 0);
    auto below = [&](int32_t j) { return P.lu_colptr[j + 1] - P.diag_pos[j] - 1; };
    for (int32_t i = 1; i <= n; i++) {
        const int32_t c0 = c0v.back();
        bool ext = i < n && i - c0 < BSN_MAX;
        if (ext) {
            // U part of column i holds rows c0..i-1 (they are its last i - c0 rows above the diagonal)
            const int64_t ub = P.lu_colptr[i], ue = P.diag_pos[i];
            ext = ue - ub >= i - c0 && (i == c0 || (P.lu_rowidx[ue - (i - c0)] == c0));
            // column i-1 continues with row i right below its diagonal, then exactly the rows
            // column i has below its diagonal
            if (ext) ext = below(i - 1) == below(i) + 1 && P.lu_rowidx[P.diag_pos[i - 1] + 1] == i;
            if (ext) {
                const int32_t *a = P.lu_rowidx.data() + P.diag_pos[i - 1] + 2;
                const int32_t *b = P.lu_rowidx.data() + P.diag_pos[i] + 1;
                ext = std::equal(a, a + below(i), b);
            }
        }
        if (!ext) c0v.push_back(i);
    }
    if (n == 0) c0v.assign(1, 0);
    const int32_t nsn = (int32_t)c0v.size() - 1;
    std::vector<int32_t> sof((size_t)n);
    P.sn_r.assign((size_t)nsn, 0);
    for (int32_t q = 0; q < nsn; q++) {
        for (int32_t j = c0v[q]; j < c0v[q + 1]; j++) sof[j] = q;
        P.sn_r[q] = (int32_t)below(c0v[q + 1] - 1);
    }
    // block levels
    std::vector<int32_t> blev((size_t)nsn, 0);
    int32_t nbl = nsn > 0 ? 1 : 0;
    for (int32_t q = 0; q < nsn; q++) {
        int32_t lv = 0;
        for (int32_t j = c0v[q]; j < c0v[q + 1]; j++)
            for (int64_t p = P.dep_ptr[j]; p < P.dep_ptr[j + 1]; p++) {
                const int32_t d = P.dep_idx[p];
                if (d < c0v[q]) lv = std::max(lv, blev[sof[d]] + 1);
            }
        blev[q] = lv;
        nbl = std::max(nbl, lv + 1);
    }
    P.nblev = nbl;
    // pairs, bucketed by level, each bucket sorted by (k, sn): scanning
    // columns k ascending and their U rows ascending gives that order.  On
    // threads, one range of columns each: count per level, then place; a
    // thread's columns precede the next thread's, so every bucket comes out
    // in the order of one sequential scan.
    const int nth = analysis_threads();
    const std::vector<int32_t> kc = column_ranges(n, P.lu_colptr.data(), nth);
    std::vector<std::vector<int64_t>> lcnt((size_t)nth);
    // a column's pairs: the supernodes of its U rows that end before it, each
    // once, with its first such row
    auto column_pairs = [&](int32_t k, std::vector<int32_t> &last, auto emit) {
        for (int64_t p = P.lu_colptr[k]; p < P.diag_pos[k]; p++) {
            const int32_t j = P.lu_rowidx[p];
            const int32_t q = sof[j];
            if (c0v[q + 1] > k || last[q] == k) continue;
            last[q] = k;
            emit(q, j, p);
        }
    };
    run_threads(nth, [&](int t) {
        std::vector<int64_t> &cnt = lcnt[t];
        cnt.assign((size_t)nbl, 0);
        std::vector<int32_t> last((size_t)nsn, -1);   // last column that recorded a pair for sn
        for (int32_t k = kc[t]; k < kc[t + 1]; k++)
            column_pairs(k, last, [&](int32_t q, int32_t, int64_t) { cnt[blev[q]]++; });
    });
    std::vector<int64_t> lcount((size_t)nbl + 1, 0);
    for (int32_t l = 0; l < nbl; l++) {
        int64_t at = lcount[l];
        for (int t = 0; t < nth; t++) {
            const int64_t c = lcnt[t][l];
            lcnt[t][l] = at;     // now this thread's first slot in bucket l
            at += c;
        }
        lcount[l + 1] = at;
    }
    P.bpairs.resize((size_t)lcount[nbl]);
    run_threads(nth, [&](int t) {
        std::vector<int64_t> &f = lcnt[t];
        std::vector<int32_t> last((size_t)nsn, -1);
        for (int32_t k = kc[t]; k < kc[t + 1]; k++)
            column_pairs(k, last, [&](int32_t q, int32_t j, int64_t p) {
                P.bpairs[f[blev[q]]++] = BPair{q, k, j - c0v[q], 0, p, 0};
            });
    });
    // map bases: exclusive prefix sum of the pairs' R_B sizes, by chunks
    const int64_t npr = lcount[nbl];
    std::vector<int64_t> msum((size_t)nth + 1, 0);
    auto pch = [&](int t) { return npr * t / nth; };
    run_threads(nth, [&](int t) {
        int64_t s = 0;
        for (int64_t q = pch(t); q < pch(t + 1); q++) s += P.sn_r[P.bpairs[q].sn];
        msum[t + 1] = s;
    });
    for (int t = 0; t < nth; t++) msum[t + 1] += msum[t];
    run_threads(nth, [&](int t) {
        int64_t mb = msum[t];
        for (int64_t q = pch(t); q < pch(t + 1); q++) {
            P.bpairs[q].mb = mb;
            mb += P.sn_r[P.bpairs[q].sn];
        }
    });
    P.bmap_size = msum[nth];
    // per level: diagonal blocks, panel items, update tasks
    P.bdiag.clear();
    P.bdiag_ptr.assign((size_t)nbl + 1, 0);
    P.bitems.clear();
    P.bitem_ptr.assign((size_t)nbl + 1, 0);
    P.bsegs.clear();
    P.btasks.clear();
    P.btask_ptr.assign((size_t)nbl + 1, 0);
    std::vector<std::vector<int32_t>> by_level((size_t)nbl);
    for (int32_t q = 0; q < nsn; q++) by_level[blev[q]].push_back(q);
    for (int32_t l = 0; l < nbl; l++) {
        for (int32_t q : by_level[l])
            if (c0v[q + 1] - c0v[q] >= 2) P.bdiag.push_back(q);
        P.bdiag_ptr[l + 1] = (int32_t)P.bdiag.size();
        for (int32_t q : by_level[l])
            for (int32_t t = 0; t < P.sn_r[q]; t += 32)
                P.bitems.push_back(BItem{q, 0, t, std::min(P.sn_r[q], t + 32)});
        for (int64_t p = lcount[l]; p < lcount[l + 1]; p++) {
            const BPair &bp = P.bpairs[p];
            if (c0v[bp.sn + 1] - c0v[bp.sn] - bp.f >= 2) P.bitems.push_back(BItem{bp.sn, 1, (int32_t)p, 0});
        }
        P.bitem_ptr[l + 1] = (int32_t)P.bitems.size();
    }
    // Update tasks, level ranges on threads (each into its own lists, task
    // segment indices relative to them), concatenated in level order: the
    // result does not depend on the thread count.
    struct BPart {
        std::vector<BSeg> segs;
        std::vector<BTask> tasks;
        std::vector<int32_t> tend;   // per level, relative to tasks
    };
    const int32_t nparts = std::max(1, std::min(nbl, nth * 8));
    std::vector<int32_t> cut(1, 0);
    for (int32_t t = 1; t < nparts; t++) {
        const int64_t want = lcount[nbl] * t / nparts;
        const int32_t l = (int32_t)(std::lower_bound(lcount.begin(), lcount.end(), want) - lcount.begin());
        cut.push_back(std::max(cut.back(), std::min(l, nbl)));
    }
    cut.push_back(nbl);
    std::vector<BPart> parts(cut.size() - 1);
    std::atomic<size_t> next{0};
    run_threads(nth, [&](int) {
        std::vector<std::vector<BSeg>> cbucket;   // per chunk of the current target column
        std::vector<int32_t> touched;
        for (size_t pi; (pi = next.fetch_add(1)) < parts.size();) {
            std::vector<BSeg> &segs = parts[pi].segs;
            std::vector<BTask> &tasks = parts[pi].tasks;
            for (int32_t l = cut[pi]; l < cut[pi + 1]; l++) {
                // update tasks: the level's pairs grouped by target column; each
                // BCHUNK-position chunk of the column touched by some R_B is a task,
                // its segments the pairs' rows inside the chunk, in supernode order.
                // Each pair's rows are routed to their chunks in one pass (rows and
                // positions both ascend, so every search starts where the last ended).
                int64_t g = lcount[l];
                while (g < lcount[l + 1]) {
                    const int32_t k = P.bpairs[g].k;
                    int64_t ge = g;
                    while (ge < lcount[l + 1] && P.bpairs[ge].k == k) ge++;
                    const int64_t cb = P.lu_colptr[k], clen = P.lu_colptr[k + 1] - cb;
                    const int32_t *kr = P.lu_rowidx.data() + cb;
                    const int64_t nch = (clen + BCHUNK - 1) / BCHUNK;
                    if ((int64_t)cbucket.size() < nch) cbucket.resize((size_t)nch);
                    touched.clear();
                    for (int64_t p = g; p < ge; p++) {
                        const int32_t q = P.bpairs[p].sn;
                        const int32_t r = P.sn_r[q];
                        const int32_t *R = P.lu_rowidx.data() + P.lu_colptr[c0v[q + 1]] - r;
                        int64_t pos = 0;
                        for (int32_t t = 0; t < r;) {
                            pos = gallop_lower_bound(kr + pos, kr + clen, R[t]) - kr;
                            const int64_t ch = pos / BCHUNK;
                            const int64_t chend = (ch + 1) * BCHUNK;
                            const int32_t t1 =
                                chend >= clen ? r : (int32_t)(gallop_lower_bound(R + t, R + r, kr[chend]) - R);
                            if (cbucket[ch].empty()) touched.push_back((int32_t)ch);
                            cbucket[ch].push_back(BSeg{(int32_t)p, t, t1, 0});
                            t = t1;
                        }
                    }
                    std::sort(touched.begin(), touched.end());
                    for (int32_t ch : touched) {
                        BTask t{(int32_t)segs.size(), 0};
                        segs.insert(segs.end(), cbucket[ch].begin(), cbucket[ch].end());
                        t.seg_end = (int32_t)segs.size();
                        tasks.push_back(t);
                        cbucket[ch].clear();
                    }
                    g = ge;
                }
                parts[pi].tend.push_back((int32_t)tasks.size());
            }
        }
    });
    // concatenation: each part's segments and tasks to their offsets, on threads
    std::vector<int64_t> sbase(parts.size() + 1, 0), tbase(parts.size() + 1, 0);
    for (size_t pi = 0; pi < parts.size(); pi++) {
        for (int32_t q = 0; q < cut[pi + 1] - cut[pi]; q++)
            P.btask_ptr[cut[pi] + q + 1] = (int32_t)(tbase[pi] + parts[pi].tend[q]);
        sbase[pi + 1] = sbase[pi] + (int64_t)parts[pi].segs.size();
        tbase[pi + 1] = tbase[pi] + (int64_t)parts[pi].tasks.size();
    }
    P.bsegs.resize((size_t)sbase[parts.size()]);
    P.btasks.resize((size_t)tbase[parts.size()]);
    std::atomic<size_t> nextp{0};
    run_threads(nth, [&](int) {
        for (size_t pi; (pi = nextp.fetch_add(1)) < parts.size();) {
            BPart &pt = parts[pi];
            const int32_t sb = (int32_t)sbase[pi];
            std::copy(pt.segs.begin(), pt.segs.end(), P.bsegs.begin() + sbase[pi]);
            for (size_t q = 0; q < pt.tasks.size(); q++)
                P.btasks[(size_t)tbase[pi] + q] = BTask{pt.tasks[q].seg_begin + sb, pt.tasks[q].seg_end + sb};
            pt = BPart();
        }
    });
}

// Start of the largest trailing block [t0, n), n - t0 <= tmax, in which every
// entry of L+U is present (n: none).
int32_t dense_trailing_block(const HostPlan &P, int32_t tmax) {
    const int32_t n = P.n;
    tmax = std::min(n, tmax);
    int32_t best = n;
    for (int32_t T = 1; T <= tmax; T++) {
        const int32_t t0 = n - T;
        // adding row/column t0: column t0 needs rows t0..n-1, row t0 needs
        // columns t0..n-1 (the columns > t0 hold row t0 iff their count of
        // rows >= t0 reaches n - t0)
        bool ok = P.lu_colptr[t0 + 1] - P.diag_pos[t0] == T;
        for (int32_t j = t0 + 1; ok && j < n; j++) {
            const int64_t q = P.lu_colptr[j + 1] - T;
            ok = q >= P.lu_colptr[j] && P.lu_rowidx[q] == t0;
        }
        if (!ok) break;
        best = t0;
    }
    return best;
}

// Dense trailing block of the factorization: the largest dense [t0, n),
// FTAIL_MIN <= n - t0 <= FTAIL_MAX, whose columns are the last levels, one
// column per level, with every column before t0 in an earlier level.  The
// level sweep then stops before level(t0): by then every update from
// outside the block has been applied, and the block is factored as a dense
// matrix (no pivoting) instead of one level per column.
void factor_tail(HostPlan &P, const glu_options &opt) {
    const int32_t n = P.n, nl = (int32_t)P.level_ptr.size() - 1;
    P.ftail_t0 = n;
    P.ftail_level = nl;
    if (opt.factor_tail == 0 || n < FTAIL_MIN) return;
    const int32_t d0 = dense_trailing_block(P, FTAIL_MAX);
    if (n - d0 < FTAIL_MIN) return;
    std::vector<int32_t> pm(n + 1, -1);   // pm[t] = max level of the columns before t
    for (int32_t j = 0; j < n; j++) pm[j + 1] = std::max(pm[j], P.level_of[j]);
    int32_t best = n;
    for (int32_t t = n - 1; t >= d0; t--) {
        if (P.level_of[t] != nl - (n - t) || pm[t] >= P.level_of[t]) break;
        best = t;
    }
    if (n - best >= FTAIL_MIN) {
        P.ftail_t0 = best;
        P.ftail_level = P.level_of[best];
    }
}

// Solve levels: forward lf(i) = 1 + max lf(j) over L(i,j) != 0 (0 if none);
// backward lb(i) = 1 + max lb(k) over U(i,k) != 0, k > i (0 if none).
void solve_levels(HostPlan &P, const glu_options &opt) {
    // host-side fault injection for tests (as GLU_TEST_FAIL_LEVEL)
    if (std::getenv("GLU_TEST_FAIL_SOLVE")) throw std::bad_alloc();
    const int32_t n = P.n;
    std::vector<int32_t> lf((size_t)n, 0), lb((size_t)n, 0);
    int32_t nf = n ? 1 : 0, nb = n ? 1 : 0;
    for (int32_t i = 0; i < n; i++) {
        int32_t v = 0;
        for (int64_t p = P.lrow_ptr[i]; p < P.lrow_ptr[i + 1]; p++) v = std::max(v, lf[P.lrow_col[p]] + 1);
        lf[i] = v;
        nf = std::max(nf, v + 1);
    }
    for (int32_t i = n - 1; i >= 0; i--) {
        int32_t v = 0;
        for (int64_t p = P.urow_ptr[i]; p < P.urow_ptr[i + 1]; p++) v = std::max(v, lb[P.urow_col[p]] + 1);
        lb[i] = v;
        nb = std::max(nb, v + 1);
    }
    auto group = [n](const std::vector<int32_t> &lv, int32_t nlev, std::vector<int32_t> &ptr,
                     std::vector<int32_t> &rows) {
        ptr.assign((size_t)nlev + 1, 0);
        for (int32_t i = 0; i < n; i++) ptr[lv[i] + 1]++;
        for (int32_t l = 0; l < nlev; l++) ptr[l + 1] += ptr[l];
        rows.resize((size_t)n);
        std::vector<int32_t> f(ptr.begin(), ptr.end() - 1);
        for (int32_t i = 0; i < n; i++) rows[f[lv[i]]++] = i;
    };
    group(lf, nf, P.fwd_ptr, P.fwd_rows);
    group(lb, nb, P.bwd_ptr, P.bwd_rows);
    // rows with more than `chunk` entries: their dot products are split
    // into chunks, summed later in chunk order
    auto items = [](const std::vector<int32_t> &ptr, const std::vector<int32_t> &rows,
                    const std::vector<int64_t> &rptr, int64_t chunk, std::vector<SolveRow> &it,
                    std::vector<SolveChunk> &ch, std::vector<int32_t> &chp) {
        const size_t nlev = ptr.size() - 1;
        it.clear();
        ch.clear();
        chp.assign(nlev + 1, 0);
        for (size_t l = 0; l < nlev; l++) {
            for (int32_t q = ptr[l]; q < ptr[l + 1]; q++) {
                const int32_t i = rows[q];
                const int64_t b = rptr[i], e = rptr[i + 1];
                SolveRow r{i, (int32_t)ch.size(), (int32_t)ch.size(), 0};
                if (e - b > chunk) {
                    for (int64_t p = b; p < e; p += chunk) ch.push_back(SolveChunk{p, std::min(e, p + chunk)});
                    r.ce = (int32_t)ch.size();
                }
                it.push_back(r);
            }
            chp[l + 1] = (int32_t)ch.size();
        }
    };
    items(P.fwd_ptr, P.fwd_rows, P.lrow_ptr, SOLVE_CHUNK, P.fwd_items, P.fwd_chunks, P.fwd_chunk_ptr);
    items(P.bwd_ptr, P.bwd_rows, P.urow_ptr, SOLVE_CHUNK, P.bwd_items, P.bwd_chunks, P.bwd_chunk_ptr);
    // Dense tail: the largest trailing block [t0, n), TAIL_MIN <= n - t0 <=
    // TAIL_MAX, in which every entry of L+U is present.
    P.tail_t0 = n;
    if (opt.solve_tail != 0) {
        const int32_t best = dense_trailing_block(P, TAIL_MAX);
        if (n - best >= TAIL_MIN) P.tail_t0 = best;
    }
    build_df(P, SOLVE_CHUNK, P.tail_t0, opt.solve_blocks != 0 ? SN_MAX : 0, P.df_items, P.df_fchunks, P.df_bchunks,
             P.tail_cb, P.tail_ce, P.df_nfwd, P.df_snx_f, P.df_snx_b);
    items(P.fwd_ptr, P.fwd_rows, P.lrow_ptr, SOLVE_CHUNK_B, P.bfwd_items, P.bfwd_chunks, P.bfwd_chunk_ptr);
    items(P.bwd_ptr, P.bwd_rows, P.urow_ptr, SOLVE_CHUNK_B, P.bbwd_items, P.bbwd_chunks, P.bbwd_chunk_ptr);
    // batched: the tail's values for 32 sets sit in shared memory, so at most
    // TAIL_MAX_B rows of the dense block (a trailing part of it is dense too)
    P.btail_t0 = (P.tail_t0 < n) ? std::max<int32_t>(P.tail_t0, n - TAIL_MAX_B) : n;
    build_df(P, SOLVE_CHUNK_B, P.btail_t0, opt.solve_blocks != 0 ? SN_MAX_B : 0, P.df_items_b, P.bdf_fchunks,
             P.bdf_bchunks, P.btail_cb, P.btail_ce, P.bdf_nfwd, P.bdf_snx_f, P.bdf_snx_b);
    // batched: a dense diagonal block item becomes RSPLIT_B adjacent copies,
    // copy q taking the right-hand sides r = q (mod RSPLIT_B), so that the
    // block's column sweeps for different right-hand sides run side by side;
    // the last copy to finish publishes the block's rows
    std::vector<int32_t> ex;
    ex.reserve(P.df_items_b.size());
    int32_t nfwd = 0, nblk = 0;
    for (size_t k = 0; k < P.df_items_b.size() / 8; k++) {
        const int32_t *it = &P.df_items_b[8 * k];
        const int32_t copies = (it[4] & 4) ? RSPLIT_B : 1;
        for (int32_t q = 0; q < copies; q++) {
            ex.insert(ex.end(), it, it + 8);
            if (copies > 1) {
                ex[ex.size() - 3] = q;
                ex[ex.size() - 2] = nblk;
            }
        }
        if (copies > 1) nblk++;
        if ((int64_t)k < P.bdf_nfwd) nfwd += copies;
    }
    P.df_items_b.swap(ex);
    P.bdf_nfwd = nfwd;
    P.bdf_nblocks = nblk;
}

}  // namespace

// Dataflow runs: maximal runs of consecutive mode-2 levels before the dense
// trailing block (the last run also takes the final normalization pass when
// there is no dense block) run as one launch whose work items wait on
// counters instead of level barriers.  A task of level l in a run needs
// (a) the columns of level l final -- every task of the run that targets
// them done -- and (b) every task of an earlier level of the run that
// targets its own column done (U(j,k) final, and the additions into the
// column in level order).  Tasks before the run are complete when it starts.
void dataflow_tables(HostPlan &P) {
    const int32_t nl = (int32_t)P.level_ptr.size() - 1;
    const int64_t ntask = (int64_t)P.tasks.size();
    P.task_col.assign((size_t)ntask, 0);
    P.task_before.assign((size_t)ntask, 0);
    P.lvl_total.assign((size_t)nl + 1, 0);
    P.lvl_ntasks.assign((size_t)nl + 1, 0);
    P.lvl_item_ptr.assign((size_t)nl + 2, 0);
    for (int64_t t = 0; t < ntask; t++) {
        const Task &tk = P.tasks[(size_t)t];
        P.task_col[(size_t)t] = tk.seg_end > tk.seg_begin ? P.pair_k[(size_t)P.segs[(size_t)tk.seg_begin].rb] : 0;
    }
    for (int32_t l = 0; l <= nl; l++) {
        const int64_t nn = P.lvl_norm_ptr[l + 1] - P.lvl_norm_ptr[l];
        int64_t nsrc = 0, nrow = 0, nlane = 0;
        if (l < nl) {
            nsrc = P.lvl_row_ptr[l] - P.lvl_task_ptr[l];
            nrow = P.lvl_lane_ptr[l] - P.lvl_row_ptr[l];
            nlane = P.lvl_task_ptr[l + 1] - P.lvl_lane_ptr[l];
            P.lvl_ntasks[l] = P.lvl_task_ptr[l + 1] - P.lvl_task_ptr[l];
        }
        P.lvl_item_ptr[l + 1] = P.lvl_item_ptr[l] + (int32_t)(nn + nsrc + nrow + (nlane + 31) / 32);
    }
    const bool dense = P.ftail_t0 < P.n;
    const int32_t lend = dense ? P.ftail_level : nl;
    std::vector<int32_t> cnt((size_t)P.n, 0);
    std::vector<int32_t> touched;
    int32_t l = 0;
    while (l < lend) {
        if (P.level_mode[l] != 2) {
            l++;
            continue;
        }
        int32_t e = l;
        while (e < lend && P.level_mode[e] == 2) e++;
        for (int32_t q = l; q < e; q++) {
            // before-counts from the earlier levels of the run, then this level's
            for (int32_t t = P.lvl_task_ptr[q]; t < P.lvl_task_ptr[q + 1]; t++)
                P.task_before[(size_t)t] = cnt[(size_t)P.task_col[(size_t)t]];
            for (int32_t t = P.lvl_task_ptr[q]; t < P.lvl_task_ptr[q + 1]; t++) {
                const int32_t k = P.task_col[(size_t)t];
                if (cnt[(size_t)k]++ == 0) touched.push_back(k);
                // only targets inside the run: a later run starts with its
                // counters at zero, everything before it being complete
                if (P.level_of[(size_t)k] < e) P.lvl_total[(size_t)P.level_of[(size_t)k]]++;
            }
        }
        for (int32_t k : touched) cnt[(size_t)k] = 0;
        touched.clear();
        l = e;
    }
}

int column_schedule(HostPlan &P, const glu_options &opt, int num_sms) {
    return P.has_schedule ? GLU_OK : schedule(P, opt, num_sms);
}

int analyze_host(int32_t n, const int32_t *colptr, const int32_t *rowidx, const int32_t *perm,
                 const glu_options &opt, int num_sms, HostPlan &P, std::string &why) {
    if (n < 0 || (n > 0 && (!colptr || !rowidx))) { why = "bad arguments"; return GLU_ERR_INVALID; }
    P.n = n;
    if (n == 0) {
        P.lu_colptr.assign(1, 0);
        P.dep_ptr.assign(1, 0);
        P.level_ptr.assign(1, 0);
        P.lvl_task_ptr.assign(1, 0);
        P.lvl_norm_ptr.assign(2, 0);
        P.pair_map.assign(1, 0);
        P.lrow_ptr.assign(1, 0);
        P.urow_ptr.assign(1, 0);
        P.fwd_ptr.assign(1, 0);
        P.bwd_ptr.assign(1, 0);
        P.fwd_chunk_ptr.assign(1, 0);
        P.bwd_chunk_ptr.assign(1, 0);
        P.bfwd_chunk_ptr.assign(1, 0);
        P.bbwd_chunk_ptr.assign(1, 0);
        P.tail_t0 = 0;
        P.acsr_ptr.assign(1, 0);
        return GLU_OK;
    }
    if (colptr[0] != 0) { why = "colptr[0] != 0"; return GLU_ERR_INVALID; }
    for (int32_t j = 0; j < n; j++) {
        if (colptr[j + 1] < colptr[j]) { why = "colptr decreases at column " + std::to_string(j); return GLU_ERR_INVALID; }
        for (int32_t p = colptr[j]; p < colptr[j + 1]; p++) {
            if (rowidx[p] < 0 || rowidx[p] >= n) { why = "row index out of range in column " + std::to_string(j); return GLU_ERR_INVALID; }
            if (p > colptr[j] && rowidx[p] <= rowidx[p - 1]) { why = "rows not strictly ascending in column " + std::to_string(j); return GLU_ERR_INVALID; }
        }
    }
    P.nnz_a = colptr[n];
    P.a_colptr.assign(colptr, colptr + n + 1);
    P.a_rowidx.assign(rowidx, rowidx + P.nnz_a);
    P.perm.resize((size_t)n);
    P.iperm.assign((size_t)n, -1);
    for (int32_t i = 0; i < n; i++) {
        int32_t o = perm ? perm[i] : i;
        if (o < 0 || o >= n || P.iperm[o] != -1) { why = "perm is not a permutation"; return GLU_ERR_INVALID; }
        P.perm[i] = o;
        P.iperm[o] = i;
    }
    double t0 = now_ms();
    std::vector<int64_t> bptr;
    std::vector<int32_t> brow, bsrc;
    int rc = permute_input(P, bptr, brow, bsrc, why);
    if (rc != GLU_OK) return rc;
    rc = symbolic(P, bptr, brow);
    if (rc != GLU_OK) return rc;
    if (opt.verbose)
        std::fprintf(stderr, "glu_analyze: symbolic fill %.0f ms, nnz(L+U) = %lld\n", now_ms() - t0,
                     (long long)P.lu_colptr[n]);
    // value gather map: each B entry's position in its LU column
    const int64_t nnz = P.lu_colptr[n];
    P.gsrc.assign((size_t)nnz, -1);
    P.max_col_len = 0;
    {
        const int nth = analysis_threads();
        const std::vector<int32_t> cut = column_ranges(n, P.lu_colptr.data(), nth);
        std::vector<int64_t> longest((size_t)nth, 0);
        run_threads(nth, [&](int t) {
            for (int32_t j = cut[t]; j < cut[t + 1]; j++) {
                const int32_t *cb = P.lu_rowidx.data() + P.lu_colptr[j];
                const int32_t *ce = P.lu_rowidx.data() + P.lu_colptr[j + 1];
                longest[t] = std::max<int64_t>(longest[t], ce - cb);
                for (int64_t q = bptr[j]; q < bptr[j + 1]; q++) {
                    const int32_t *it = std::lower_bound(cb, ce, brow[q]);
                    P.gsrc[it - P.lu_rowidx.data()] = bsrc[q];
                }
            }
        });
        for (int64_t v : longest) P.max_col_len = std::max(P.max_col_len, v);
    }
    row_views(P);
    double t1 = now_ms();
    double t2 = t1;
    if (opt.gpu_analysis != 0 && !opt.host_only) {
        // Algorithm 4 and the levels on the GPU (bit-identical results)
        const int rc = gpu_dependencies_levels(P, opt.spin_limit_us, why);
        if (rc != GLU_OK) return rc;
        t2 = now_ms();
        group_levels(P);
    } else {
        dependencies(P);
        t2 = now_ms();
        levelize(P);
    }
    double t3 = now_ms();
    if (opt.verbose)
        std::fprintf(stderr, "glu_analyze: row views %.0f ms, deps %.0f ms (%lld), levels %.0f ms (%d)\n",
                     t1 - t0, t2 - t1, (long long)P.dep_ptr[n], t3 - t2, (int)P.level_ptr.size() - 1);
    // the column schedule (and its position map) is only built here for the
    // column-level factorization; the supernodal one builds it on demand
    // (the batched path runs column levels)
    // the solve's schedule reads only the fill and its row views: it is built
    // on its own thread while the factorization's schedule is built
    // (an allocation failure on either thread is rethrown here once both
    // have finished)
    std::atomic<bool> solve_failed{false};
    double t_solve = 0.0;
    auto solve_job = [&P, &opt, &solve_failed, &t_solve] {
        const double ts = now_ms();
        try {
            solve_levels(P, opt);
        } catch (const std::bad_alloc &) {
            solve_failed = true;
        }
        t_solve = now_ms() - ts;
    };
    std::thread solve_thread;
    try {
        solve_thread = std::thread(solve_job);
    } catch (const std::system_error &) {
    }
    rc = GLU_OK;
    bool failed = false;
    try {
        if (opt.factor_blocks == 0) rc = schedule(P, opt, num_sms);
        if (rc == GLU_OK) {
            factor_tail(P, opt);
            if (opt.factor_blocks != 0) block_schedule(P);
        }
    } catch (const std::bad_alloc &) {
        failed = true;
    }
    const double t_sched = now_ms() - t3;
    if (solve_thread.joinable())
        solve_thread.join();
    else if (!failed)
        solve_job();   // no thread could be started: the solve schedule on this one
    if (opt.verbose)
        std::fprintf(stderr, "glu_analyze: factorization schedule %.0f ms, solve schedule %.0f ms (concurrent)\n",
                     t_sched, t_solve);
    if (failed || solve_failed) throw std::bad_alloc();
    if (rc != GLU_OK) {
        why = "the column schedule has more than 2^31 segments, tasks or pairs";
        return rc;
    }
    // A in compressed rows (original numbering), for residuals
    P.acsr_ptr.assign((size_t)n + 1, 0);
    for (int64_t p = 0; p < P.nnz_a; p++) P.acsr_ptr[P.a_rowidx[p] + 1]++;
    for (int32_t i = 0; i < n; i++) P.acsr_ptr[i + 1] += P.acsr_ptr[i];
    P.acsr_col.resize((size_t)P.nnz_a);
    P.acsr_src.resize((size_t)P.nnz_a);
    {
        std::vector<int64_t> f(P.acsr_ptr.begin(), P.acsr_ptr.end() - 1);
        for (int32_t c = 0; c < n; c++)
            for (int32_t p = colptr[c]; p < colptr[c + 1]; p++) {
                int64_t q = f[rowidx[p]]++;
                P.acsr_col[q] = c;
                P.acsr_src[q] = p;
            }
    }
    double t4 = now_ms();
    P.flops = 0.0;
    int64_t npairs = 0, nupd = 0;
    for (int32_t j = 0; j < n; j++) {
        const int64_t lj = P.lu_colptr[j + 1] - P.diag_pos[j] - 1;
        const int64_t uj = P.urow_ptr[j + 1] - P.urow_ptr[j];
        P.flops += (double)lj + 2.0 * (double)lj * (double)uj;
        if (lj > 0) {
            npairs += uj;
            nupd += lj * uj;
        }
    }
    P.n_pairs = npairs;
    P.n_updates = nupd;
    P.ms_symbolic = t1 - t0;
    P.ms_deps = t2 - t1;
    P.ms_levels = t3 - t2;
    P.ms_schedule = t4 - t3;
    return GLU_OK;
}

}  // namespace glu
