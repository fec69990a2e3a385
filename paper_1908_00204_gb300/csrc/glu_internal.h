// glu_internal.h -- shared declarations of the library (not part of the ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <memory>
#include <new>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/glu.h"

namespace glu {

// An allocator that default-initializes: resize() leaves trivially
// constructible elements unwritten, so large host arrays that are filled
// right after sizing are not zeroed first (and their pages are first touched
// by the threads that fill them).
template <class T>
struct NoInitAllocator : std::allocator<T> {
    using value_type = T;
    template <class U>
    struct rebind {
        using other = NoInitAllocator<U>;
    };
    NoInitAllocator() noexcept = default;
    template <class U>
    NoInitAllocator(const NoInitAllocator<U> &) noexcept {}
    template <class U>
    void construct(U *p) noexcept(std::is_nothrow_default_constructible<U>::value) {
        ::new ((void *)p) U;
    }
    template <class U, class... Args>
    void construct(U *p, Args &&...args) {
        ::new ((void *)p) U(std::forward<Args>(args)...);
    }
};

// Task kinds of a level's work list.
//   KIND_SRC:  many short segments on one 32-position chunk: lanes over
//              segments, shared-memory accumulators, fixed-order reduction;
//   KIND_ROW:  a warp applies the segments in order, lanes over rows;
//   KIND_LANE: a small task run start to finish by a single lane.
enum : int32_t { KIND_ROW = 0, KIND_SRC = 1, KIND_LANE = 2 };

// A segment of one (source j, target k) column pair: rows t0..t1-1 of L(:,j)
// (t counts from the first row below the diagonal), with everything needed
// to apply it in one record: pos = position of U(j,k), dj = position of the
// pivot of j, and rb.  On the host rb is the pair's index; on the device it
// locates the segment's runs (see Run): the first run overlapping t0..t1-1 in
// bits 0..43, the number of runs overlapping them in bits 44..63.
struct alignas(16) Seg {
    int64_t pos;
    int64_t dj;
    int64_t rb;
    int32_t t0;
    int32_t t1;
};
constexpr int RUN_BASE_BITS = 44;

// Where the rows of L(:,j) sit in target column k.  By the fill theorem
// every row of L(:,j) is a row of column k below U(j,k); the rows of L(:,j)
// fall on runs of consecutive positions of column k.  A run is stored as
// (ts, off): rows t = ts, ts+1, ... of L(:,j) (up to the next run's ts) are
// at positions pos(U(j,k)) + 1 + off + (t - ts).  A pair's runs are
// consecutive in one table, ts ascending, the first with ts = 0; the
// level kernels locate a row's run by warp ballots and shuffles over them.
struct Run {
    int32_t ts;
    int32_t off;
};

// Scheduling-time segment (pair index + row range).
struct PSeg {
    int32_t pair;
    int32_t t0;
    int32_t t1;
    int32_t spare;
};

// Normalization item: rows t0..t1-1 of L(:,j) divided by the pivot.
struct NormItem {
    int32_t col;
    int32_t t0;
    int32_t t1;
    int32_t spare;
};

// A task of a level: segments [seg_begin, seg_end).
//   KIND_ROW: one warp applies the segments one after the other (ascending
//             source), lanes over the rows of each segment.
//   KIND_SRC: one warp, lanes over segments; the products land in per-lane
//             shared-memory accumulators for the 32 target positions
//             base .. base+nslots-1, reduced in a fixed order at the end.
struct Task {
    int32_t seg_begin;
    int32_t seg_end;
    int32_t kind;
    int32_t nslots;
    int64_t base;
    int64_t work;   // host only: number of updates (for ordering)
};

constexpr int SRC_SLOTS = 32;

// Supernodal ("block") factorization.  A supernode B = columns [c0, c1),
// at most BSN_MAX of them, has a dense diagonal block and the same rows R_B
// below it in every column.  Per block level: the diagonal blocks are
// factored (warp per supernode), then the panel rows L21 = A21 U11^-1 and the
// target rows U12 = L11^-1 A12 (warp items), then every target column takes
// A(R_B, k) -= L21 U12(:, k) from the level's supernodes (warp tasks owning
// BCHUNK positions of the column).
constexpr int32_t BSN_MAX = 32;
constexpr int32_t BCHUNK = 128;

struct BPair {          // supernode sn updates target column k
    int32_t sn;
    int32_t k;
    int32_t f;          // first column offset in B with U(c0 + f, k) != 0 (a suffix of B)
    int32_t spare;
    int64_t upos;       // position of U(c0 + f, k) in the CSC values
    int64_t mb;         // first map entry: offsets in column k of the rows R_B
};

struct BSeg {           // rows t0..t1-1 of R_B applied to the pair's target column
    int32_t pair, t0, t1, spare;
};

struct BTask {
    int32_t seg_begin, seg_end;
};

struct BItem {          // panel work: kind 0 rows [a, b) of R_B, kind 1 the pair a
    int32_t sn, kind, a, b;
};

// Triangular-solve work: a row of a solve level; rows with many entries get
// their dot product split into chunks computed first (partials cb..ce-1).
struct SolveRow {
    int32_t row;
    int32_t cb;
    int32_t ce;
    int32_t spare;
};
struct SolveChunk {
    int64_t p0;
    int64_t p1;
};
#ifndef GLU_SOLVE_CHUNK
#define GLU_SOLVE_CHUNK 128
#endif
constexpr int64_t SOLVE_CHUNK = GLU_SOLVE_CHUNK;   // single matrix: lanes over a row's entries (<= 128)
constexpr int64_t SOLVE_CHUNK_B = 32;   // batched: lanes over the sets, entries in sequence
constexpr int32_t TAIL_MIN = 32, TAIL_MAX = 1024;   // dense-tail solve size range
constexpr int32_t TAIL_MAX_B = 736;                 // batched: tail rows x 32 sets in shared memory
constexpr int32_t FTAIL_MIN = 64, FTAIL_MAX = 3200;  // dense-tail factorization size range
#ifndef GLU_SN_MAX
#define GLU_SN_MAX 32
#endif
constexpr int32_t SN_MIN = 4, SN_MAX = GLU_SN_MAX;   // dense diagonal blocks of the dataflow solve
                                                     // (a multiple of 32, <= 128; 32 measured best)
constexpr int32_t RSPLIT_B = 4;                     // batched: copies of a dense diagonal block item
constexpr int32_t SN_MAX_B = 32;                     // the same in the batched solve (rows in registers)

// Everything glu_analyze computes on the host.
struct HostPlan {
    int32_t n = 0;
    int64_t nnz_a = 0;
    // input copy (original numbering) and permutation
    std::vector<int32_t> a_colptr, a_rowidx, perm, iperm;
    // filled pattern of A_s = L + U - I (new numbering)
    std::vector<int64_t> lu_colptr;
    std::vector<int32_t> lu_rowidx;
    std::vector<int64_t> diag_pos;
    std::vector<int32_t> gsrc;          // per LU position: index into A's values, -1 = fill
    int64_t max_col_len = 0;
    // dependencies (Algorithm 4) and levels
    std::vector<int64_t> dep_ptr;
    std::vector<int32_t> dep_idx;
    std::vector<int32_t> level_of, level_ptr, level_cols;
    // update schedule
    std::vector<int32_t> pair_j, pair_k;
    std::vector<int64_t> pair_pos, pair_map;
    int64_t n_updates = 0, n_pairs = 0;
    bool has_schedule = false;           // the column-level schedule is built
    std::vector<Seg, NoInitAllocator<Seg>> segs;
    std::vector<Task, NoInitAllocator<Task>> tasks;
    std::vector<int32_t> lvl_task_ptr;  // nlevels + 1
    // inside level l: [lvl_task_ptr[l], lvl_row_ptr[l]) KIND_SRC,
    // [lvl_row_ptr[l], lvl_lane_ptr[l]) KIND_ROW, [lvl_lane_ptr[l], lvl_task_ptr[l+1]) KIND_LANE
    std::vector<int32_t> lvl_row_ptr, lvl_lane_ptr;
    std::vector<NormItem> norms;
    std::vector<int32_t> lvl_norm_ptr;  // nlevels + 2: level l's kernel runs [l, l+1); [L, L+1) is the final pass
    std::vector<int8_t> level_mode;
    // dataflow runs (consecutive mode-2 levels in one launch, see
    // dataflow_tables): per task its target column and how many tasks of
    // earlier levels of its run target that column; per level (nlevels + 1)
    // the run's tasks that target the level's columns, the level's own tasks,
    // and the global prefix of work items (warp items) per level
    std::vector<int32_t> task_col, task_before;
    std::vector<int32_t> lvl_total, lvl_ntasks, lvl_item_ptr;
    // solve schedule (row views of L and U, levels)
    std::vector<int64_t> lrow_ptr, urow_ptr;
    std::vector<int32_t, NoInitAllocator<int32_t>> lrow_col, urow_col;
    std::vector<int64_t, NoInitAllocator<int64_t>> lrow_pos, urow_pos;
    std::vector<int32_t> fwd_ptr, fwd_rows, bwd_ptr, bwd_rows;
    // per solve level: rows (with their chunk ranges) and chunks
    std::vector<SolveRow> fwd_items, bwd_items;
    std::vector<SolveChunk> fwd_chunks, bwd_chunks;
    std::vector<int32_t> fwd_chunk_ptr, bwd_chunk_ptr;   // nlevels + 1
    // dataflow solve: items in topological order, packed as int32 x 8
    // {row, cb, ce, chunk, flags, 0, 0, 0}; forward items first
    std::vector<int32_t> df_items;
    int32_t df_nfwd = 0;                       // number of forward items
    std::vector<SolveChunk> df_fchunks, df_bchunks;
    // dense tail [tail_t0, n) solved by one block (tail_t0 == n: none); the
    // partial sums of each tail row over the columns before the tail are
    // forward chunks tail_cb[i]..tail_ce[i]-1
    int32_t tail_t0 = 0;
    std::vector<int32_t> tail_cb, tail_ce;
    // dense diagonal blocks of the dataflow solve: per block, the first chunk
    // of each row's entries outside the block, then the end
    std::vector<int32_t> df_snx_f, df_snx_b;
    // the same for the batched solve, with shorter chunks
    std::vector<SolveRow> bfwd_items, bbwd_items;
    std::vector<SolveChunk> bfwd_chunks, bbwd_chunks;
    std::vector<int32_t> bfwd_chunk_ptr, bbwd_chunk_ptr;
    std::vector<int32_t> df_items_b;
    int32_t bdf_nfwd = 0, btail_t0 = 0, bdf_nblocks = 0;
    std::vector<SolveChunk> bdf_fchunks, bdf_bchunks;
    std::vector<int32_t> btail_cb, btail_ce;
    std::vector<int32_t> bdf_snx_f, bdf_snx_b;
    // supernodal factorization (built when the block mode is selected)
    std::vector<int32_t> sn_c0;          // nsn + 1 column boundaries
    std::vector<int32_t> sn_r;           // |R_B|
    std::vector<int32_t> bdiag, bdiag_ptr;   // supernodes of >= 2 columns, by block level
    std::vector<BItem> bitems;
    std::vector<int32_t> bitem_ptr;
    std::vector<BPair, NoInitAllocator<BPair>> bpairs;
    std::vector<BSeg, NoInitAllocator<BSeg>> bsegs;
    std::vector<BTask, NoInitAllocator<BTask>> btasks;
    std::vector<int32_t> btask_ptr;
    int64_t bmap_size = 0;
    int32_t nblev = 0;
    // dense trailing block of the factorization [ftail_t0, n) (ftail_t0 == n:
    // none); the level sweep runs levels [0, ftail_level) and the
    // normalizations of level ftail_level, then the block is factored dense
    int32_t ftail_t0 = 0, ftail_level = 0;
    // A in compressed rows (original numbering) for residuals
    std::vector<int64_t> acsr_ptr;
    std::vector<int32_t> acsr_col;
    std::vector<int64_t> acsr_src;
    // statistics
    int64_t nnz_l = 0, nnz_u = 0;
    double flops = 0.0;
    int32_t max_level_width = 0;
    int32_t levels_by_mode[3] = {0, 0, 0};
    double ms_symbolic = 0, ms_deps = 0, ms_levels = 0, ms_schedule = 0;
};

// Runs every host step of glu_analyze.  Returns a GLU_ code.
int analyze_host(int32_t n, const int32_t *colptr, const int32_t *rowidx, const int32_t *perm,
                 const glu_options &opt, int num_sms, HostPlan &P, std::string &why);

// Nested-dissection ordering of the pattern of A + A^T (order.cpp): perm[new]
// = old.  Returns a GLU_ code.
int order_nested_dissection(int32_t n, const int32_t *colptr, const int32_t *rowidx, int32_t *perm);
int static_pivot(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *values, int32_t *row_perm,
                 double *row_scale, double *col_scale);
int apply_static_pivot(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *values,
                       const int32_t *row_perm, const double *row_scale, const double *col_scale,
                       int32_t *out_rowidx, double *out_values);

// Algorithm 4 and the longest-path levels on the GPU (analyze_gpu.cu): fills
// P.dep_ptr, P.dep_idx and P.level_of from the fill and the row views of L.
int gpu_dependencies_levels(HostPlan &P, int32_t spin_limit_us, std::string &why);

// The tables of the dataflow level runs (task_col, task_before, lvl_total,
// lvl_ntasks, lvl_item_ptr) for the column-level schedule.
void dataflow_tables(HostPlan &P);

// The column-level update schedule (pairs, segments, tasks, normalization
// items) if analyze_host skipped it.  GLU_OK, or GLU_ERR_TOO_LARGE when a
// 32-bit index of the device records would overflow; throws std::bad_alloc.
int column_schedule(HostPlan &P, const glu_options &opt, int num_sms);

}  // namespace glu
