// capi.cu -- the C ABI declared in include/glu.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "glu_device.cuh"
#include "glu_internal.h"

using namespace glu;

struct glu_handle {
    HostPlan P;
    glu_options opt{};
    int device = 0;
    int num_sms = 152;
    cudaStream_t stream = nullptr;
    // device memory: one arena for the schedule, the row lookup apart
    char *arena = nullptr;
    size_t arena_bytes = 0;
    Run *d_runs = nullptr;        // run table (lookup 0)
    void *d_map = nullptr;        // position map (lookup 2 or 4 bytes per update)
    size_t map_total = 0;         // bytes of the row lookup
    int64_t n_runs = 0;
    int lookup = 0;
    char *carena = nullptr;      // the column-level schedule (built on first use in block mode)
    size_t carena_bytes = 0;
    bool col_ready = false;
    // supernodal factorization tables and map
    int32_t *d_lu_rowidx = nullptr;
    int32_t *d_sn_c0 = nullptr, *d_sn_r = nullptr, *d_bdiag = nullptr;
    BItem *d_bitems = nullptr;
    BPair *d_bpairs = nullptr;
    BSeg *d_bsegs = nullptr;
    BTask *d_btasks = nullptr;
    void *bmap = nullptr;
    size_t bmap_total = 0;
    int map_bytes = 2;
    double *d_lu = nullptr;
    double *d_aval = nullptr;
    int32_t *d_gsrc = nullptr;
    int64_t *d_diag = nullptr;
    int32_t *d_pair_j = nullptr;
    int64_t *d_pair_pos = nullptr;
    int64_t *d_pair_runs = nullptr;
    int64_t *d_pair_map = nullptr;
    Seg *d_segs = nullptr;
    Task *d_tasks = nullptr;
    NormItem *d_norms = nullptr;
    unsigned long long *d_err = nullptr;
    int64_t *d_lrow_ptr = nullptr, *d_lrow_pos = nullptr, *d_urow_ptr = nullptr, *d_urow_pos = nullptr;
    int32_t *d_lrow_col = nullptr, *d_urow_col = nullptr;
    int32_t *d_fwd_rows = nullptr, *d_bwd_rows = nullptr, *d_perm = nullptr;
    SolveRow *d_fwd_items = nullptr, *d_bwd_items = nullptr;
    SolveChunk *d_fwd_chunks = nullptr, *d_bwd_chunks = nullptr;
    // dataflow solve: items, ready flags (forward rows, backward rows, forward
    // chunks, backward chunks, contiguous), ticket, abort word, error word
    DFItem *d_df_items = nullptr;
    int64_t *d_lu_colptr = nullptr;
    SolveChunk *d_df_fchunks = nullptr, *d_df_bchunks = nullptr;
    int32_t *d_tail_cb = nullptr, *d_tail_ce = nullptr;
    int32_t *d_snx_f = nullptr, *d_snx_b = nullptr;   // dense diagonal blocks of the solve
    int32_t *d_flags = nullptr;
    int64_t n_flags = 0;
    unsigned *d_ticket = nullptr;
    unsigned *d_abort = nullptr;
    unsigned long long *d_serr = nullptr;
    long long spin_cycles = 0;
    // level ranges on the device (persistent multi-level launches) and the
    // grid-barrier words
    LevelRange *d_ranges = nullptr;
    unsigned *d_gbar = nullptr;          // count, abort
    // dataflow level runs (the pipelined mode): tables and counters
    char *dfarena = nullptr;
    size_t dfarena_bytes = 0;
    int32_t *d_task_col = nullptr, *d_task_before = nullptr, *d_lvl_total = nullptr, *d_lvl_ntasks = nullptr;
    int32_t *d_item_ptr = nullptr, *d_level_of = nullptr;
    int32_t *d_dfcnt = nullptr;          // cdone (n), ldone (nlevels + 1), tdone (nlevels + 1)
    unsigned *d_dfword = nullptr;        // ticket, abort
    // FP32 factors and the refinement path
    float *d_lu32 = nullptr;
    cudaGraphExec_t fgraph32 = nullptr;
    int64_t fgraph32_launches = 0;
    bool factored32 = false;
    double *d_aval_csr = nullptr;        // FP64 values in compressed-row order
    int64_t *d_acsr_ptr = nullptr;
    int32_t *d_acsr_col = nullptr;
    int64_t *d_acsr_src = nullptr;
    double *d_ir = nullptr;              // r and d, n * nrhs each
    unsigned long long *d_irnorm = nullptr;  // anorm, then rmax, xmax, bmax (nrhs each)
    int32_t *d_done = nullptr;           // nrhs flags, then the count
    double *d_berr = nullptr;
    int32_t ir_nrhs = 0;
    // batched value sets (interleaved, stride bS = batch rounded up to 32)
    int32_t bB = 0, bS = 0;            // factorized batch and its stride
    int32_t bcap = 0;                  // stride the buffers were sized for
    int bprec = 0;                     // 64 or 32: which factors are valid (0: none)
    double *d_vstage = nullptr;        // the caller's values, set-major, ld = nnz_a
    double *d_aT = nullptr;            // values interleaved
    double *d_avb = nullptr;           // values interleaved, compressed-row order
    double *d_lub = nullptr;           // FP64 factors
    float *d_lub32 = nullptr;          // FP32 factors
    int32_t *d_bflags = nullptr;
    int64_t n_bflags = 0;
    std::vector<std::pair<int, cudaGraphExec_t>> bgraphs;   // key: prec
    std::vector<int64_t> bgraph_launches;
    // batched solve buffers
    int32_t bwork_nrhs = 0;
    double *d_bwork = nullptr;         // y, z (as T), in, out, r, d, x: n*nrhs*bS each
    double *d_bpartial = nullptr;
    unsigned long long *d_bnorm = nullptr;
    int32_t *d_bdone = nullptr;
    double *d_bberr = nullptr;
    DFItem *d_bdf_items = nullptr;     // batched solve schedule (shorter chunks, smaller tail)
    SolveChunk *d_bfwd_chunks = nullptr, *d_bbwd_chunks = nullptr;
    int32_t *d_btail_cb = nullptr, *d_btail_ce = nullptr;
    int32_t *d_bsnx_f = nullptr, *d_bsnx_b = nullptr;
    // solve scratch (grown on demand): permuted vector, staging, partials
    double *d_work = nullptr;
    double *d_bstage = nullptr;
    double *d_xstage = nullptr;
    double *d_partial = nullptr;
    int64_t work_elems = 0;
    int32_t work_nrhs = 0;
    // CUDA graphs of the factor and solve sequences (captured on cap_stream)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t fgraph = nullptr;
    int64_t fgraph_launches = 0;
    std::vector<std::pair<int32_t, cudaGraphExec_t>> sgraphs;
    std::vector<std::pair<int32_t, cudaGraphExec_t>> rgraphs;   // refinement iteration per nrhs
    std::vector<int64_t> rgraph_launches;
    std::vector<double> rgraph_tol;
    std::vector<int64_t> sgraph_launches;
    // per-level timing diagnostic (GLU_LEVEL_TIMES=path)
    std::string level_times_path;
    bool factored = false;
    int32_t err_col = -1;
    double analyze_ms = 0.0;
    int64_t launches = 0;
    std::string why;
};

namespace {

int cuda_fail(glu_handle *h, cudaError_t e, const char *what) {
    if (h) h->why = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return GLU_ERR_OOM;
    return GLU_ERR_CUDA;
}

#define CK(call)                                                         \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);           \
    } while (0)

// a kernel launch through one of the launch_* helpers (counted)
#define CKL(n_launched, call)                                            \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);           \
        h->launches += (n_launched);                                     \
    } while (0)

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Arena carving: every sub-buffer 256-byte aligned.
struct Carve {
    size_t off = 0;
    template <typename T>
    size_t take(size_t count) {
        size_t o = (off + 255) & ~size_t(255);
        off = o + count * sizeof(T) + 1;
        return o;
    }
};

template <typename T>
T *at(char *base, size_t off) { return reinterpret_cast<T *>(base + off); }

template <typename T, typename A>
cudaError_t upload(T *dst, const std::vector<T, A> &src) {
    if (src.empty()) return cudaSuccess;
    return cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

FactorArgs<double> fargs(glu_handle *h);
SolveArgs<double> sargs(glu_handle *h);
int setup_column_plan(glu_handle *h);

// Work list of level l (l == nlevels: the final normalization pass).
LevelRange level_range(const HostPlan &P, int32_t l) {
    const int32_t nl = (int32_t)P.level_ptr.size() - 1;
    LevelRange r;
    r.t_begin = l < nl ? P.lvl_task_ptr[l] : 0;
    r.row_begin = l < nl ? P.lvl_row_ptr[l] : 0;
    r.lane_begin = l < nl ? P.lvl_lane_ptr[l] : 0;
    r.t_end = l < nl ? P.lvl_task_ptr[l + 1] : 0;
    r.n_begin = P.lvl_norm_ptr[l];
    r.n_end = P.lvl_norm_ptr[l + 1];
    return r;
}

// Launch the levels of one factorization: a run of consecutive pipelined
// (mode 2) levels, and the final normalization pass after them, goes into
// one persistent launch; every other level is one launch.  With a dense
// trailing block the sweep stops before the block's first level: that
// level's normalizations run alone, then the block is factored densely.
template <typename T>
BlockArgs<T> bargs_t(glu_handle *h, T *lu);

template <typename T>
int enqueue_levels(glu_handle *h, const FactorArgs<T> &a, cudaStream_t st) {
    HostPlan &P = h->P;
    if (h->opt.factor_blocks != 0) {
        // the supernodal sweep: per block level, diagonal blocks, panels, updates
        const BlockArgs<T> ba = bargs_t<T>(h, a.lu);
        for (int32_t l = 0; l < P.nblev; l++) {
            int launched = 0;
            CK(launch_block_level<T>(ba, h->map_bytes, P.bdiag_ptr[l], P.bdiag_ptr[l + 1], P.bitem_ptr[l],
                                     P.bitem_ptr[l + 1], P.btask_ptr[l], P.btask_ptr[l + 1], h->num_sms, st,
                                     &launched));
            h->launches += launched;
        }
        return GLU_OK;
    }
    const int32_t nl = (int32_t)P.level_ptr.size() - 1;
    const bool dense = P.ftail_t0 < P.n;
    const int32_t lend = dense ? P.ftail_level : nl;   // levels [0, lend) run here
    GridBarrier bar{h->d_gbar, h->d_gbar + 1, h->d_err, h->spin_cycles};
    int32_t l = 0;
    while (l < lend || (!dense && l == nl)) {
        const bool pipelined = l == nl ? (nl > 0 && P.level_mode[nl - 1] == 2) : P.level_mode[l] == 2;
        if (!pipelined) {
            const LevelRange r = level_range(P, l);
            CKL((r.t_end - r.t_begin) + (r.n_end - r.n_begin) > 0, launch_level<T>(a, h->lookup, r, h->num_sms, st));
            l++;
            continue;
        }
        int32_t e = l;
        while (e < lend && P.level_mode[e] == 2) e++;
        if (!dense && e == nl) e = nl + 1;   // include the final pass
        if (e - l == 1) {
            const LevelRange r = level_range(P, l);
            CKL((r.t_end - r.t_begin) + (r.n_end - r.n_begin) > 0, launch_level<T>(a, h->lookup, r, h->num_sms, st));
        } else {
            // one dataflow launch for the run, its counters zeroed first
            CK(cudaMemsetAsync(h->d_dfcnt, 0, ((size_t)P.n + 2 * ((size_t)nl + 1)) * sizeof(int32_t), st));
            CK(cudaMemsetAsync(h->d_dfword, 0, 2 * sizeof(unsigned), st));
            DFFactorArgs d;
            d.ranges = h->d_ranges;
            d.item_ptr = h->d_item_ptr;
            d.l0 = l;
            d.l1 = e;
            d.task_col = h->d_task_col;
            d.task_before = h->d_task_before;
            d.lvl_total = h->d_lvl_total;
            d.lvl_ntasks = h->d_lvl_ntasks;
            d.level_of = h->d_level_of;
            d.cdone = h->d_dfcnt;
            d.ldone = h->d_dfcnt + P.n;
            d.tdone = d.ldone + nl + 1;
            d.ticket = h->d_dfword;
            d.abort = h->d_dfword + 1;
            d.err = h->d_err;
            d.spin_limit_cycles = h->spin_cycles;
            d.fault_col = h->opt.fault_row;
            d.max_items = 0;
            for (int32_t q = l; q < e; q++)
                d.max_items = std::max(d.max_items, P.lvl_item_ptr[q + 1] - P.lvl_item_ptr[q]);
            CKL(1, launch_levels_df<T>(a, h->lookup, d, h->num_sms, st));
        }
        l = e;
    }
    if (dense) {
        LevelRange r = level_range(P, lend);
        r.t_begin = r.row_begin = r.lane_begin = r.t_end = 0;   // normalizations only
        CKL(r.n_end > r.n_begin, launch_level<T>(a, h->lookup, r, h->num_sms, st));
        DenseTailArgs d{P.ftail_t0, P.n - P.ftail_t0, h->d_lu_colptr};
        CKL(1, launch_dense_tail<T>(a.lu, d, bar, h->num_sms, st));
    }
    return GLU_OK;
}

// Refinement graphs hold the work and refinement buffers; they go when
// either is reallocated.
void drop_rgraphs(glu_handle *h) {
    for (auto &g : h->rgraphs) cudaGraphExecDestroy(g.second);
    h->rgraphs.clear();
    h->rgraph_launches.clear();
    h->rgraph_tol.clear();
}

int ensure_work(glu_handle *h, int32_t nrhs) {
    if (nrhs <= h->work_nrhs) return GLU_OK;
    const int64_t elems = (int64_t)h->P.n * nrhs;
    const int64_t nch = (int64_t)std::max(h->P.fwd_chunks.size() + h->P.bwd_chunks.size(),
                                          h->P.df_fchunks.size() + h->P.df_bchunks.size()) * nrhs;
    // graphs captured with the old buffers are stale
    for (auto &g : h->sgraphs) cudaGraphExecDestroy(g.second);
    h->sgraphs.clear();
    h->sgraph_launches.clear();
    drop_rgraphs(h);
    cudaFree(h->d_work);
    cudaFree(h->d_bstage);
    cudaFree(h->d_xstage);
    cudaFree(h->d_partial);
    h->d_work = h->d_bstage = h->d_xstage = h->d_partial = nullptr;
    h->work_elems = 0;
    h->work_nrhs = 0;
    CK(cudaMalloc(&h->d_work, 2 * elems * sizeof(double)));   // y, and z of the dataflow solve
    CK(cudaMalloc(&h->d_bstage, elems * sizeof(double)));
    CK(cudaMalloc(&h->d_xstage, elems * sizeof(double)));
    CK(cudaMalloc(&h->d_partial, std::max<int64_t>(nch, 1) * sizeof(double)));
    h->work_elems = elems;
    h->work_nrhs = nrhs;
    return GLU_OK;
}

// The factor sequence: error reset, value gather, one kernel per level (the
// last one only normalizes), pivot check.
int enqueue_factor(glu_handle *h, const double *av, cudaStream_t st, std::vector<cudaEvent_t> *lev_events) {
    HostPlan &P = h->P;
    CKL(1, launch_reset_err(h->d_err, st));
    CKL(P.lu_colptr[P.n] > 0, launch_gather<double>(h->d_lu, av, h->d_gsrc, P.lu_colptr[P.n], st));
    FactorArgs<double> a = fargs(h);
    const int32_t nl = (int32_t)P.level_ptr.size() - 1;
    if (lev_events && h->opt.factor_blocks != 0) {
        // per-level timing diagnostic of the supernodal sweep: events around
        // each block level's launches
        const BlockArgs<double> ba = bargs_t<double>(h, h->d_lu);
        CK(cudaEventRecord((*lev_events)[0], st));
        for (int32_t l = 0; l < P.nblev; l++) {
            int launched = 0;
            CK(launch_block_level<double>(ba, h->map_bytes, P.bdiag_ptr[l], P.bdiag_ptr[l + 1], P.bitem_ptr[l],
                                          P.bitem_ptr[l + 1], P.btask_ptr[l], P.btask_ptr[l + 1], h->num_sms, st,
                                          &launched));
            h->launches += launched;
            CK(cudaEventRecord((*lev_events)[l + 1], st));
        }
    } else if (lev_events) {
        // per-level timing diagnostic: one launch per level (column levels)
        const int rc0 = setup_column_plan(h);
        if (rc0 != GLU_OK) return rc0;
        a = fargs(h);
        CK(cudaEventRecord((*lev_events)[0], st));
        for (int32_t l = 0; l <= nl; l++) {
            const LevelRange r = level_range(P, l);
            CKL((r.t_end - r.t_begin) + (r.n_end - r.n_begin) > 0,
                launch_level<double>(a, h->lookup, r, h->num_sms, st));
            CK(cudaEventRecord((*lev_events)[l + 1], st));
        }
    } else {
        int rc = enqueue_levels<double>(h, a, st);
        if (rc != GLU_OK) return rc;
    }
    CKL(P.n > 0, launch_pivot_check<double>(h->d_lu, h->d_diag, P.n, h->d_err, st));
    return GLU_OK;
}

// The dataflow solve of y (already permuted) into z: forward items, the dense
// tail on one block, backward items.
template <typename T>
int enqueue_df(glu_handle *h, const SolveArgs<T> &a, T *y, T *z, T *partial, int32_t nrhs, cudaStream_t st) {
    HostPlan &P = h->P;
    const int32_t n = P.n;
    CK(cudaMemsetAsync(h->d_flags, 0, h->n_flags * sizeof(int32_t), st));
    CK(cudaMemsetAsync(h->d_serr, 0xff, sizeof(unsigned long long), st));
    DFSolveArgs d;
    d.blk_done = nullptr;
    d.epoch = 1;
    d.fault_row = h->opt.fault_row;
    d.fchunks = h->d_df_fchunks;
    d.bchunks = h->d_df_bchunks;
    d.fpartial_v = partial;
    d.bpartial_v = partial + (int64_t)P.df_fchunks.size() * nrhs;
    d.fready = h->d_flags;
    d.bready = h->d_flags + n;
    d.fchunk_ready = h->d_flags + 2 * (int64_t)n;
    d.bchunk_ready = d.fchunk_ready + P.df_fchunks.size();
    d.ticket = h->d_ticket;
    d.abort = h->d_abort;
    d.err = h->d_serr;
    d.spin_limit_cycles = h->spin_cycles;
    d.fsnx = h->d_snx_f;
    d.bsnx = h->d_snx_b;
    const int32_t nall = (int32_t)(P.df_items.size() / 8);
    d.items = h->d_df_items;
    d.nitems = P.df_nfwd;
    CKL(d.nitems > 0, launch_solve_df<T>(a, d, y, z, nrhs, h->num_sms, st));
    if (P.tail_t0 < n) {
        TailArgs ta{P.tail_t0, h->d_tail_cb, h->d_tail_ce, d.bready, d.epoch};
        CKL(1, launch_solve_tail<T>(a, h->d_lu_colptr, ta, partial, y, z, nrhs, st));
    }
    d.items = h->d_df_items + P.df_nfwd;
    d.nitems = nall - P.df_nfwd;
    CKL(d.nitems > 0, launch_solve_df<T>(a, d, y, z, nrhs, h->num_sms, st));
    return GLU_OK;
}

// The solve sequence from device b to device x.
int enqueue_solve(glu_handle *h, const double *db, double *dx, int32_t nrhs, cudaStream_t st) {
    HostPlan &P = h->P;
    const int32_t n = P.n;
    double *y = h->d_work;
    CKL(1, launch_permute_in<double>(y, db, h->d_perm, n, nrhs, st));
    SolveArgs<double> a = sargs(h);
    if (h->opt.solve_mode == 1) {
        double *z = y + (int64_t)n * nrhs;
        int rc = enqueue_df<double>(h, a, y, z, h->d_partial, nrhs, st);
        if (rc != GLU_OK) return rc;
        CKL(1, launch_permute_out<double>(dx, z, h->d_perm, n, nrhs, st));
        return GLU_OK;
    }
    int launched = 0;
    for (size_t l = 0; l + 1 < P.fwd_ptr.size(); l++) {
        CK(launch_solve_level<double>(a, false, y, nrhs, h->d_fwd_items + P.fwd_ptr[l], P.fwd_ptr[l + 1] - P.fwd_ptr[l],
                                      h->d_fwd_chunks, P.fwd_chunk_ptr[l], P.fwd_chunk_ptr[l + 1], h->d_partial, st,
                                      &launched));
        h->launches += launched;
    }
    for (size_t l = 0; l + 1 < P.bwd_ptr.size(); l++) {
        CK(launch_solve_level<double>(a, true, y, nrhs, h->d_bwd_items + P.bwd_ptr[l], P.bwd_ptr[l + 1] - P.bwd_ptr[l],
                                      h->d_bwd_chunks, P.bwd_chunk_ptr[l], P.bwd_chunk_ptr[l + 1], h->d_partial, st,
                                      &launched));
        h->launches += launched;
    }
    CKL(1, launch_permute_out<double>(dx, y, h->d_perm, n, nrhs, st));
    return GLU_OK;
}

template <typename T>
BlockArgs<T> bargs_t(glu_handle *h, T *lu) {
    BlockArgs<T> a;
    a.lu = lu;
    a.colptr = h->d_lu_colptr;
    a.rowidx = h->d_lu_rowidx;
    a.diag_pos = h->d_diag;
    a.sn_c0 = h->d_sn_c0;
    a.sn_r = h->d_sn_r;
    a.bdiag = h->d_bdiag;
    a.bitems = h->d_bitems;
    a.bpairs = h->d_bpairs;
    a.bsegs = h->d_bsegs;
    a.btasks = h->d_btasks;
    a.map = h->bmap;
    a.err = h->d_err;
    return a;
}

template <typename T>
FactorArgs<T> fargs_t(glu_handle *h, T *lu) {
    FactorArgs<T> a;
    a.lu = lu;
    a.diag_pos = h->d_diag;
    a.map = h->d_map;
    a.runs = h->d_runs;
    a.segs = h->d_segs;
    a.tasks = h->d_tasks;
    a.norms = h->d_norms;
    a.err = h->d_err;
    return a;
}

template <typename T>
SolveArgs<T> sargs_t(glu_handle *h, const T *lu) {
    SolveArgs<T> a;
    a.lu = lu;
    a.diag_pos = h->d_diag;
    a.lrow_ptr = h->d_lrow_ptr;
    a.lrow_col = h->d_lrow_col;
    a.lrow_pos = h->d_lrow_pos;
    a.urow_ptr = h->d_urow_ptr;
    a.urow_col = h->d_urow_col;
    a.urow_pos = h->d_urow_pos;
    a.n = h->P.n;
    return a;
}

// The FP32 factor sequence (same schedule as the FP64 one).
int enqueue_factor_f32(glu_handle *h, cudaStream_t st) {
    HostPlan &P = h->P;
    CKL(1, launch_reset_err(h->d_err, st));
    CKL(P.lu_colptr[P.n] > 0, launch_gather<float>(h->d_lu32, h->d_aval, h->d_gsrc, P.lu_colptr[P.n], st));
    FactorArgs<float> a = fargs_t<float>(h, h->d_lu32);
    int rc = enqueue_levels<float>(h, a, st);
    if (rc != GLU_OK) return rc;
    CKL(P.n > 0, launch_pivot_check<float>(h->d_lu32, h->d_diag, P.n, h->d_err, st));
    // FP64 values in row order for the residuals
    CKL(P.nnz_a > 0, launch_csr_values(h->d_aval_csr, h->d_aval, h->d_acsr_src, P.nnz_a, st));
    return GLU_OK;
}

// FP32 dataflow solve of db (FP64) into dx (FP64): rounding to FP32 on the
// way in, FP32 sweeps, widening on the way out.
int enqueue_solve_f32(glu_handle *h, const double *db, double *dx, int32_t nrhs, cudaStream_t st) {
    HostPlan &P = h->P;
    const int32_t n = P.n;
    float *y = reinterpret_cast<float *>(h->d_work);
    float *z = y + (int64_t)n * nrhs;
    CKL(1, launch_permute_in<float>(y, db, h->d_perm, n, nrhs, st));
    SolveArgs<float> a = sargs_t<float>(h, h->d_lu32);
    int rc = enqueue_df<float>(h, a, y, z, reinterpret_cast<float *>(h->d_partial), nrhs, st);
    if (rc != GLU_OK) return rc;
    CKL(1, launch_permute_out<float>(dx, z, h->d_perm, n, nrhs, st));
    return GLU_OK;
}

int ensure_ir(glu_handle *h, int32_t nrhs) {
    if (nrhs <= h->ir_nrhs) return GLU_OK;
    drop_rgraphs(h);
    cudaFree(h->d_ir);
    cudaFree(h->d_irnorm);
    cudaFree(h->d_done);
    cudaFree(h->d_berr);
    h->d_ir = nullptr;
    h->d_irnorm = nullptr;
    h->d_done = nullptr;
    h->d_berr = nullptr;
    h->ir_nrhs = 0;
    const int64_t elems = (int64_t)h->P.n * nrhs;
    CK(cudaMalloc(&h->d_ir, 2 * std::max<int64_t>(elems, 1) * sizeof(double)));
    CK(cudaMalloc(&h->d_irnorm, (1 + 3 * (size_t)nrhs) * sizeof(unsigned long long)));
    CK(cudaMalloc(&h->d_done, (1 + (size_t)nrhs) * sizeof(int32_t)));
    CK(cudaMalloc(&h->d_berr, (size_t)nrhs * sizeof(double)));
    h->ir_nrhs = nrhs;
    return GLU_OK;
}

// Capture `fn` (which enqueues on the given stream) into an executable graph.
template <typename F>
int capture(glu_handle *h, F &&fn, cudaGraphExec_t *exec, int64_t *launches) {
    cudaGraph_t g = nullptr;
    const int64_t before = h->launches;
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = fn(h->cap_stream);
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (rc != GLU_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    *launches = h->launches - before;
    h->launches = before;
    return GLU_OK;
}

int decode_err(glu_handle *h, unsigned long long w) {
    if (w == ERR_NONE) return GLU_OK;
    h->err_col = (int32_t)(w >> 8);
    switch ((unsigned)(w & 0xff)) {
        case DEVERR_ZERO_PIVOT: return GLU_ERR_ZERO_PIVOT;
        case DEVERR_NONFINITE: return GLU_ERR_NONFINITE;
        case DEVERR_TIMEOUT: return GLU_ERR_TIMEOUT;
        default: return GLU_ERR_INTERNAL;
    }
}

int read_err(glu_handle *h) {
    unsigned long long w = ERR_NONE, ws = ERR_NONE;
    CK(cudaMemcpyAsync(&w, h->d_err, sizeof(w), cudaMemcpyDeviceToHost, h->stream));
    if (h->d_serr) CK(cudaMemcpyAsync(&ws, h->d_serr, sizeof(ws), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    int rc = decode_err(h, w);          // a factorization error takes precedence
    return rc != GLU_OK ? rc : decode_err(h, ws);
}

FactorArgs<double> fargs(glu_handle *h) {
    FactorArgs<double> a;
    a.lu = h->d_lu;
    a.diag_pos = h->d_diag;
    a.map = h->d_map;
    a.runs = h->d_runs;
    a.segs = h->d_segs;
    a.tasks = h->d_tasks;
    a.norms = h->d_norms;
    a.err = h->d_err;
    return a;
}

SolveArgs<double> sargs(glu_handle *h) {
    SolveArgs<double> a;
    a.lu = h->d_lu;
    a.diag_pos = h->d_diag;
    a.lrow_ptr = h->d_lrow_ptr;
    a.lrow_col = h->d_lrow_col;
    a.lrow_pos = h->d_lrow_pos;
    a.urow_ptr = h->d_urow_ptr;
    a.urow_col = h->d_urow_col;
    a.urow_pos = h->d_urow_pos;
    a.n = h->P.n;
    return a;
}

// The column-level schedule on the device: pair tables, segments, tasks,
// normalization items, per-level ranges and the run table (built by k_runs
// and k_seg_runs).  Run by glu_analyze for the column-level factorization and
// on first use otherwise (the batched path runs column levels).
int setup_column_plan(glu_handle *h) {
    if (h->col_ready) return GLU_OK;
    HostPlan &P = h->P;
    try {
        const int rc = column_schedule(P, h->opt, h->num_sms);
        if (rc != GLU_OK) return rc;
    } catch (const std::bad_alloc &) {
        return GLU_ERR_OOM;
    }
    const int64_t npairs = (int64_t)P.pair_j.size();
    // the row lookup: the position map unless it would exceed the budget
    const int64_t map_need = std::max<int64_t>(P.n_updates, 1) * h->map_bytes;
    const int want = h->opt.row_lookup;
    h->lookup = (want == 1 || (want != 2 && map_need <= (int64_t)GLU_MAP_BUDGET_BYTES)) ? h->map_bytes : 0;
    Carve c;
    const size_t o_pj = c.take<int32_t>(P.pair_j.size()), o_ppos = c.take<int64_t>(P.pair_pos.size()),
                 o_pruns = c.take<int64_t>((size_t)npairs + 1), o_pmap = c.take<int64_t>((size_t)npairs + 1),
                 o_segs = c.take<Seg>(P.segs.size()), o_tasks = c.take<Task>(P.tasks.size()),
                 o_norms = c.take<NormItem>(P.norms.size()), o_pk = c.take<int32_t>(P.pair_k.size()),
                 o_rng = c.take<LevelRange>(P.level_ptr.size()),
                 o_cnt = c.take<int32_t>((size_t)std::max<int64_t>(npairs, 1));
    h->carena_bytes = c.off + 256;
    CK(cudaMalloc(&h->carena, h->carena_bytes));
    char *A = h->carena;
    h->d_pair_j = at<int32_t>(A, o_pj);
    h->d_pair_pos = at<int64_t>(A, o_ppos);
    h->d_pair_runs = at<int64_t>(A, o_pruns);
    h->d_pair_map = at<int64_t>(A, o_pmap);
    h->d_segs = at<Seg>(A, o_segs);
    h->d_tasks = at<Task>(A, o_tasks);
    h->d_norms = at<NormItem>(A, o_norms);
    h->d_ranges = at<LevelRange>(A, o_rng);
    int32_t *d_pair_k = at<int32_t>(A, o_pk);
    int32_t *d_counts = at<int32_t>(A, o_cnt);
    CK(upload(h->d_pair_j, P.pair_j));
    CK(upload(h->d_pair_pos, P.pair_pos));
    CK(upload(h->d_segs, P.segs));          // rb: the pair index until the passes below
    CK(upload(h->d_tasks, P.tasks));
    CK(upload(h->d_norms, P.norms));
    CK(upload(d_pair_k, P.pair_k));
    {
        std::vector<LevelRange> rg(P.level_ptr.size());
        for (size_t l = 0; l < rg.size(); l++) rg[l] = level_range(P, (int32_t)l);
        CK(upload(h->d_ranges, rg));
    }
    RunBuildArgs rb;
    rb.lu_colptr = h->d_lu_colptr;
    rb.lu_rowidx = h->d_lu_rowidx;
    rb.diag_pos = h->d_diag;
    rb.pair_j = h->d_pair_j;
    rb.pair_k = d_pair_k;
    rb.pair_pos = h->d_pair_pos;
    rb.pair_runs = h->d_pair_runs;
    rb.pair_map = h->d_pair_map;
    rb.counts = d_counts;
    rb.runs = nullptr;
    rb.map = nullptr;
    rb.segs = h->d_segs;
    rb.npairs = npairs;
    rb.nsegs = (int64_t)P.segs.size();
    rb.err = h->d_err;
    if (h->lookup != 0) {
        // position map: every pair's offsets at pair_map[pair], then every
        // segment's first entry
        CK(upload(h->d_pair_map, P.pair_map));
        h->map_total = (size_t)map_need;
        CK(cudaMalloc(&h->d_map, h->map_total));
        rb.map = h->d_map;
        CK(launch_run_build(rb, 3, h->map_bytes, h->stream));
        CK(launch_run_build(rb, 4, h->map_bytes, h->stream));
    } else {
        // run table: count each pair's runs, lay them out (prefix sum on the
        // host), write them, then point every segment at its runs
        CK(launch_run_build(rb, 0, 0, h->stream));
        std::vector<int64_t> pr((size_t)npairs + 1, 0);
        {
            std::vector<int32_t> cnt((size_t)npairs);
            if (npairs > 0)
                CK(cudaMemcpyAsync(cnt.data(), d_counts, npairs * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                   h->stream));
            CK(cudaStreamSynchronize(h->stream));
            for (int64_t q = 0; q < npairs; q++) pr[(size_t)q + 1] = pr[(size_t)q] + cnt[(size_t)q];
        }
        h->n_runs = pr[(size_t)npairs];
        CK(upload(h->d_pair_runs, pr));
        h->map_total = (size_t)std::max<int64_t>(h->n_runs, 1) * sizeof(Run);
        CK(cudaMalloc(&h->d_runs, h->map_total));
        rb.runs = h->d_runs;
        CK(launch_run_build(rb, 1, 0, h->stream));
        CK(launch_run_build(rb, 2, 0, h->stream));
    }
    // the dataflow runs' tables, when some level runs in the pipelined mode
    bool any_df = false;
    for (int8_t md : P.level_mode) any_df = any_df || md == 2;
    if (any_df) {
        dataflow_tables(P);
        const size_t nlev1 = P.level_ptr.size();
        Carve c2;
        const size_t o_tc = c2.take<int32_t>(P.task_col.size()), o_tb = c2.take<int32_t>(P.task_before.size()),
                     o_lt = c2.take<int32_t>(nlev1), o_ln = c2.take<int32_t>(nlev1),
                     o_ip = c2.take<int32_t>(nlev1 + 1), o_lo = c2.take<int32_t>((size_t)P.n),
                     o_cn = c2.take<int32_t>((size_t)P.n + 2 * nlev1), o_w = c2.take<unsigned>(2);
        h->dfarena_bytes = c2.off + 256;
        CK(cudaMalloc(&h->dfarena, h->dfarena_bytes));
        char *D = h->dfarena;
        h->d_task_col = at<int32_t>(D, o_tc);
        h->d_task_before = at<int32_t>(D, o_tb);
        h->d_lvl_total = at<int32_t>(D, o_lt);
        h->d_lvl_ntasks = at<int32_t>(D, o_ln);
        h->d_item_ptr = at<int32_t>(D, o_ip);
        h->d_level_of = at<int32_t>(D, o_lo);
        h->d_dfcnt = at<int32_t>(D, o_cn);
        h->d_dfword = at<unsigned>(D, o_w);
        CK(upload(h->d_task_col, P.task_col));
        CK(upload(h->d_task_before, P.task_before));
        CK(upload(h->d_lvl_total, P.lvl_total));
        CK(upload(h->d_lvl_ntasks, P.lvl_ntasks));
        CK(upload(h->d_item_ptr, P.lvl_item_ptr));
        CK(upload(h->d_level_of, P.level_of));
    }
    h->col_ready = true;
    return GLU_OK;
}

int upload_plan(glu_handle *h) {
    HostPlan &P = h->P;
    const int32_t n = P.n;
    const int64_t nnz = P.lu_colptr[n];
    Carve c;
    size_t o_lu = c.take<double>(nnz), o_aval = c.take<double>(P.nnz_a), o_gsrc = c.take<int32_t>(nnz),
           o_diag = c.take<int64_t>(n), o_err = c.take<unsigned long long>(1),
           o_lrp = c.take<int64_t>(n + 1), o_lrc = c.take<int32_t>(P.lrow_col.size()),
           o_lrpos = c.take<int64_t>(P.lrow_pos.size()), o_urp = c.take<int64_t>(n + 1),
           o_urc = c.take<int32_t>(P.urow_col.size()), o_urpos = c.take<int64_t>(P.urow_pos.size()),
           o_fwd = c.take<int32_t>(P.fwd_rows.size()), o_bwd = c.take<int32_t>(P.bwd_rows.size()),
           o_perm = c.take<int32_t>(n), o_lcp = c.take<int64_t>(n + 1), o_lri = c.take<int32_t>(nnz),
           o_fi = c.take<SolveRow>(P.fwd_items.size()), o_bi = c.take<SolveRow>(P.bwd_items.size()),
           o_fc = c.take<SolveChunk>(P.fwd_chunks.size()), o_bc = c.take<SolveChunk>(P.bwd_chunks.size()),
           o_dfi = c.take<int32_t>(P.df_items.size()),
           o_flags = c.take<int32_t>(2 * (size_t)n + P.df_fchunks.size() + P.df_bchunks.size()),
           o_dffc = c.take<SolveChunk>(P.df_fchunks.size()), o_dfbc = c.take<SolveChunk>(P.df_bchunks.size()),
           o_tcb = c.take<int32_t>(P.tail_cb.size()), o_tce = c.take<int32_t>(P.tail_ce.size()),
           o_snf = c.take<int32_t>(P.df_snx_f.size()), o_snb = c.take<int32_t>(P.df_snx_b.size()),
           o_ticket = c.take<unsigned>(1), o_abort = c.take<unsigned>(1), o_serr = c.take<unsigned long long>(1),
           o_acp = c.take<int64_t>(n + 1), o_acc = c.take<int32_t>(P.acsr_col.size()),
           o_acs = c.take<int64_t>(P.acsr_src.size()), o_acv = c.take<double>(P.acsr_src.size()),
           o_bdfi = c.take<int32_t>(P.df_items_b.size()), o_bfc = c.take<SolveChunk>(P.bdf_fchunks.size()),
           o_bbc = c.take<SolveChunk>(P.bdf_bchunks.size()), o_btcb = c.take<int32_t>(P.btail_cb.size()),
           o_btce = c.take<int32_t>(P.btail_ce.size()), o_bsnf = c.take<int32_t>(P.bdf_snx_f.size()),
           o_bsnb = c.take<int32_t>(P.bdf_snx_b.size()),
           o_gbar = c.take<unsigned>(2),
           o_snc0 = c.take<int32_t>(P.sn_c0.size()), o_snr = c.take<int32_t>(P.sn_r.size()),
           o_bdg = c.take<int32_t>(P.bdiag.size()), o_bit = c.take<BItem>(P.bitems.size()),
           o_bpr = c.take<BPair>(P.bpairs.size()), o_bsg = c.take<BSeg>(P.bsegs.size()),
           o_btk = c.take<BTask>(P.btasks.size());
    h->arena_bytes = c.off + 256;
    CK(cudaMalloc(&h->arena, h->arena_bytes));
    char *A = h->arena;
    h->d_lu = at<double>(A, o_lu);
    h->d_aval = at<double>(A, o_aval);
    h->d_gsrc = at<int32_t>(A, o_gsrc);
    h->d_diag = at<int64_t>(A, o_diag);
    h->d_err = at<unsigned long long>(A, o_err);
    h->d_lrow_ptr = at<int64_t>(A, o_lrp);
    h->d_lrow_col = at<int32_t>(A, o_lrc);
    h->d_lrow_pos = at<int64_t>(A, o_lrpos);
    h->d_urow_ptr = at<int64_t>(A, o_urp);
    h->d_urow_col = at<int32_t>(A, o_urc);
    h->d_urow_pos = at<int64_t>(A, o_urpos);
    h->d_fwd_rows = at<int32_t>(A, o_fwd);
    h->d_bwd_rows = at<int32_t>(A, o_bwd);
    h->d_perm = at<int32_t>(A, o_perm);
    h->d_fwd_items = at<SolveRow>(A, o_fi);
    h->d_bwd_items = at<SolveRow>(A, o_bi);
    h->d_fwd_chunks = at<SolveChunk>(A, o_fc);
    h->d_bwd_chunks = at<SolveChunk>(A, o_bc);
    h->d_df_items = at<DFItem>(A, o_dfi);
    h->d_flags = at<int32_t>(A, o_flags);
    h->n_flags = 2 * (int64_t)n + (int64_t)P.df_fchunks.size() + (int64_t)P.df_bchunks.size();
    h->d_df_fchunks = at<SolveChunk>(A, o_dffc);
    h->d_df_bchunks = at<SolveChunk>(A, o_dfbc);
    h->d_tail_cb = at<int32_t>(A, o_tcb);
    h->d_tail_ce = at<int32_t>(A, o_tce);
    h->d_snx_f = at<int32_t>(A, o_snf);
    h->d_snx_b = at<int32_t>(A, o_snb);
    h->d_ticket = at<unsigned>(A, o_ticket);
    h->d_abort = at<unsigned>(A, o_abort);
    h->d_serr = at<unsigned long long>(A, o_serr);
    h->d_acsr_ptr = at<int64_t>(A, o_acp);
    h->d_acsr_col = at<int32_t>(A, o_acc);
    h->d_acsr_src = at<int64_t>(A, o_acs);
    h->d_aval_csr = at<double>(A, o_acv);
    h->d_bdf_items = at<DFItem>(A, o_bdfi);
    h->d_bfwd_chunks = at<SolveChunk>(A, o_bfc);
    h->d_bbwd_chunks = at<SolveChunk>(A, o_bbc);
    h->d_btail_cb = at<int32_t>(A, o_btcb);
    h->d_btail_ce = at<int32_t>(A, o_btce);
    h->d_bsnx_f = at<int32_t>(A, o_bsnf);
    h->d_bsnx_b = at<int32_t>(A, o_bsnb);
    h->d_gbar = at<unsigned>(A, o_gbar);
    int64_t *d_lcp = at<int64_t>(A, o_lcp);
    h->d_lu_colptr = d_lcp;
    int32_t *d_lri = at<int32_t>(A, o_lri);
    h->d_lu_rowidx = d_lri;
    h->d_sn_c0 = at<int32_t>(A, o_snc0);
    h->d_sn_r = at<int32_t>(A, o_snr);
    h->d_bdiag = at<int32_t>(A, o_bdg);
    h->d_bitems = at<BItem>(A, o_bit);
    h->d_bpairs = at<BPair>(A, o_bpr);
    h->d_bsegs = at<BSeg>(A, o_bsg);
    h->d_btasks = at<BTask>(A, o_btk);
    CK(upload(h->d_gsrc, P.gsrc));
    CK(upload(h->d_diag, P.diag_pos));
    CK(upload(h->d_lrow_ptr, P.lrow_ptr));
    CK(upload(h->d_lrow_col, P.lrow_col));
    CK(upload(h->d_lrow_pos, P.lrow_pos));
    CK(upload(h->d_urow_ptr, P.urow_ptr));
    CK(upload(h->d_urow_col, P.urow_col));
    CK(upload(h->d_urow_pos, P.urow_pos));
    CK(upload(h->d_fwd_rows, P.fwd_rows));
    CK(upload(h->d_bwd_rows, P.bwd_rows));
    CK(upload(h->d_perm, P.perm));
    CK(upload(h->d_fwd_items, P.fwd_items));
    CK(upload(h->d_bwd_items, P.bwd_items));
    CK(upload(h->d_fwd_chunks, P.fwd_chunks));
    CK(upload(h->d_bwd_chunks, P.bwd_chunks));
    CK(upload(reinterpret_cast<int32_t *>(h->d_df_items), P.df_items));
    CK(upload(h->d_df_fchunks, P.df_fchunks));
    CK(upload(h->d_df_bchunks, P.df_bchunks));
    CK(upload(h->d_tail_cb, P.tail_cb));
    CK(upload(h->d_snx_f, P.df_snx_f));
    CK(upload(h->d_snx_b, P.df_snx_b));
    CK(upload(h->d_tail_ce, P.tail_ce));
    CK(upload(h->d_acsr_ptr, P.acsr_ptr));
    CK(upload(h->d_acsr_col, P.acsr_col));
    CK(upload(h->d_acsr_src, P.acsr_src));
    CK(upload(reinterpret_cast<int32_t *>(h->d_bdf_items), P.df_items_b));
    CK(upload(h->d_bfwd_chunks, P.bdf_fchunks));
    CK(upload(h->d_bbwd_chunks, P.bdf_bchunks));
    CK(upload(h->d_btail_cb, P.btail_cb));
    CK(upload(h->d_btail_ce, P.btail_ce));
    CK(upload(h->d_bsnx_f, P.bdf_snx_f));
    CK(upload(h->d_bsnx_b, P.bdf_snx_b));
    CK(cudaMemset(h->d_flags, 0, std::max<int64_t>(h->n_flags, 1) * sizeof(int32_t)));
    CK(cudaMemset(h->d_serr, 0xff, sizeof(unsigned long long)));
    {
        int khz = 0;
        CK(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, h->device));
        const long long us = h->opt.spin_limit_us > 0 ? h->opt.spin_limit_us : 2000000;
        h->spin_cycles = us * (long long)(khz > 0 ? khz : 2000000) / 1000;
    }
    CK(upload(d_lcp, P.lu_colptr));
    CK(upload(d_lri, P.lu_rowidx));
    CK(upload(h->d_sn_c0, P.sn_c0));
    CK(upload(h->d_sn_r, P.sn_r));
    CK(upload(h->d_bdiag, P.bdiag));
    CK(upload(h->d_bitems, P.bitems));
    CK(upload(h->d_bpairs, P.bpairs));
    CK(upload(h->d_bsegs, P.bsegs));
    CK(upload(h->d_btasks, P.btasks));
    h->map_bytes = (P.max_col_len <= 65536) ? 2 : 4;
    CK(launch_reset_err(h->d_err, h->stream));
    if (P.has_schedule) {
        const int rc0 = setup_column_plan(h);
        if (rc0 != GLU_OK) return rc0;
    }
    if (h->opt.factor_blocks != 0) {
        h->bmap_total = (size_t)std::max<int64_t>(P.bmap_size, 1) * h->map_bytes;
        CK(cudaMalloc(&h->bmap, h->bmap_total));
        BlockArgs<double> ba = bargs_t<double>(h, h->d_lu);
        CK(launch_bmap_build(ba, h->map_bytes, (int64_t)P.bpairs.size(), h->num_sms, h->stream));
    }
    int rc = read_err(h);
    if (rc != GLU_OK) {
        h->why = "run table build found a row outside its target column";
        return GLU_ERR_INTERNAL;
    }
    return GLU_OK;
}

}  // namespace

extern "C" {

void glu_default_options(glu_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->struct_size = (int32_t)sizeof(glu_options);
    o->mode_force = -1;
    o->tail_threshold = 0;
    o->piece_updates = 1024;
    o->wide_threshold = 256;
    o->use_graph = 1;
    o->verbose = 0;
    o->solve_mode = 1;
    o->spin_limit_us = 2000000;
    o->fault_row = -1;
    o->solve_tail = 1;
    o->factor_tail = 1;
    o->solve_blocks = 1;
    o->gpu_analysis = 1;
}

int glu_analyze_opts(int32_t n, const int32_t *colptr, const int32_t *rowidx, const int32_t *perm,
                     const glu_options *opts, glu_handle **out) {
    if (!out) return GLU_ERR_INVALID;
    *out = nullptr;
    auto t0 = std::chrono::steady_clock::now();
    glu_handle *h = new (std::nothrow) glu_handle();
    if (!h) return GLU_ERR_OOM;
    glu_default_options(&h->opt);
    if (opts) {
        if (opts->struct_size != (int32_t)sizeof(glu_options)) { delete h; return GLU_ERR_INVALID; }
        h->opt = *opts;
    }
    int rc;
    int sms = 152;
    if (!h->opt.host_only) {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaGetLastError();
    }
    try {
        rc = analyze_host(n, colptr, rowidx, perm, h->opt, sms, h->P, h->why);
    } catch (const std::bad_alloc &) {
        h->why = "a host allocation failed";
        rc = GLU_ERR_OOM;
    }
    if (rc != GLU_OK) {
        if (h->opt.verbose) std::fprintf(stderr, "glu_analyze: %s\n", h->why.c_str());
        delete h;
        return rc;
    }
    if (h->opt.verbose && h->opt.factor_blocks) {
        const HostPlan &P = h->P;
        std::fprintf(stderr,
                     "glu_analyze: supernodal schedule: %zu supernodes, %d block levels, %zu pairs, %lld map "
                     "entries, %zu update segments, %zu update tasks\n",
                     P.sn_r.size(), (int)P.nblev, P.bpairs.size(), (long long)P.bmap_size, P.bsegs.size(),
                     P.btasks.size());
    }
    if (h->opt.verbose) {
        const HostPlan &P = h->P;
        int64_t cnt[3] = {0, 0, 0}, sg[3] = {0, 0, 0}, wk[3] = {0, 0, 0};
        for (const Task &t : P.tasks) { cnt[t.kind]++; sg[t.kind] += t.seg_end - t.seg_begin; wk[t.kind] += t.work; }
        std::fprintf(stderr, "glu_analyze: ROW tasks %lld segs %lld updates %lld | SRC tasks %lld segs %lld updates %lld"
                     " | LANE tasks %lld segs %lld updates %lld\n",
                     (long long)cnt[0], (long long)sg[0], (long long)wk[0], (long long)cnt[1], (long long)sg[1],
                     (long long)wk[1], (long long)cnt[2], (long long)sg[2], (long long)wk[2]);
        std::fprintf(stderr,
                     "glu_analyze: n=%d nnzA=%lld nnzLU=%lld levels=%d pairs=%zu updates=%lld tasks=%zu segs=%zu "
                     "flops=%.4g map=%dB  ms: symbolic %.1f deps %.1f levels %.1f schedule %.1f total %.1f\n",
                     P.n, (long long)P.nnz_a, (long long)P.lu_colptr[P.n], (int)P.level_ptr.size() - 1,
                     P.pair_j.size(), (long long)P.n_updates, P.tasks.size(), P.segs.size(), P.flops,
                     (P.max_col_len <= 65536) ? 2 : 4, P.ms_symbolic, P.ms_deps, P.ms_levels, P.ms_schedule, std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
    }
    if (const char *dump = std::getenv("GLU_DUMP_SCHEDULE")) {
        // per level: width, ROW tasks/segs/updates, SRC tasks/segs/updates,
        // largest task (updates, segments)
        if (FILE *fp = std::fopen(dump, "w")) {
            const HostPlan &P = h->P;
            for (size_t l = 0; l + 1 < P.level_ptr.size(); l++) {
                int64_t c[3] = {0, 0, 0}, sg[3] = {0, 0, 0}, wk[3] = {0, 0, 0}, mw = 0, ms = 0;
                int64_t mseg[3] = {0, 0, 0};
                for (int32_t t = P.lvl_task_ptr[l]; t < P.lvl_task_ptr[l + 1]; t++) {
                    const Task &tk = P.tasks[t];
                    mseg[tk.kind] = std::max<int64_t>(mseg[tk.kind], tk.seg_end - tk.seg_begin);
                    c[tk.kind]++;
                    sg[tk.kind] += tk.seg_end - tk.seg_begin;
                    wk[tk.kind] += tk.work;
                    mw = std::max<int64_t>(mw, tk.work);
                    ms = std::max<int64_t>(ms, tk.seg_end - tk.seg_begin);
                }
                std::fprintf(fp, "%zu %d %lld %lld %lld %lld %lld %lld %lld %lld %lld %lld %lld %lld %lld %lld\n", l,
                             P.level_ptr[l + 1] - P.level_ptr[l], (long long)c[0], (long long)sg[0],
                             (long long)wk[0], (long long)c[1], (long long)sg[1], (long long)wk[1], (long long)c[2],
                             (long long)sg[2], (long long)wk[2], (long long)mw, (long long)ms, (long long)mseg[0],
                             (long long)mseg[1], (long long)mseg[2]);
            }
            std::fclose(fp);
        }
    }
    if (const char *dump = std::getenv("GLU_DUMP_COLUMNS")) {
        // the column-level schedule as int64 words: counts (levels, pairs,
        // segments, tasks, normalization items), the dense block (ftail_t0,
        // ftail_level), then lvl_task_ptr, lvl_row_ptr, lvl_lane_ptr,
        // lvl_norm_ptr, pairs (j, k, pos, first update), segments (pos, dj,
        // pair, t0, t1), tasks (seg_begin, seg_end, kind, nslots, base),
        // normalization items (col, t0, t1), the value gather map (one A
        // index or -1 per entry of L+U)
        if (FILE *fp = std::fopen(dump, "wb")) {
            const HostPlan &P = h->P;
            std::vector<int64_t> w = {(int64_t)P.level_ptr.size() - 1, (int64_t)P.pair_j.size(),
                                      (int64_t)P.segs.size(), (int64_t)P.tasks.size(), (int64_t)P.norms.size(),
                                      P.ftail_t0, P.ftail_level};
            for (int32_t v : P.lvl_task_ptr) w.push_back(v);
            for (int32_t v : P.lvl_row_ptr) w.push_back(v);
            for (int32_t v : P.lvl_lane_ptr) w.push_back(v);
            for (int32_t v : P.lvl_norm_ptr) w.push_back(v);
            for (size_t q = 0; q < P.pair_j.size(); q++)
                w.insert(w.end(), {P.pair_j[q], P.pair_k[q], P.pair_pos[q], P.pair_map[q]});
            for (const Seg &g : P.segs) w.insert(w.end(), {g.pos, g.dj, g.rb, g.t0, g.t1});
            for (const Task &t : P.tasks) w.insert(w.end(), {t.seg_begin, t.seg_end, t.kind, t.nslots, t.base});
            for (const NormItem &it : P.norms) w.insert(w.end(), {it.col, it.t0, it.t1});
            w.insert(w.end(), P.gsrc.begin(), P.gsrc.end());
            std::fwrite(w.data(), sizeof(int64_t), w.size(), fp);
            std::fclose(fp);
        }
    }
    if (const char *dump = std::getenv("GLU_DUMP_BLOCKS")) {
        // the supernodal schedule as int64 words: counts (supernodes, block
        // levels, diagonal list, panel items, pairs, segments, tasks), then
        // sn_c0, sn_r, bdiag_ptr, bdiag, bitem_ptr, bitems (4 each),
        // bpairs (sn, k, f, upos, mb), bsegs (pair, t0, t1), btask_ptr,
        // btasks (2 each)
        if (FILE *fp = std::fopen(dump, "wb")) {
            const HostPlan &P = h->P;
            std::vector<int64_t> w = {(int64_t)P.sn_r.size(), P.nblev, (int64_t)P.bdiag.size(),
                                      (int64_t)P.bitems.size(), (int64_t)P.bpairs.size(), (int64_t)P.bsegs.size(),
                                      (int64_t)P.btasks.size()};
            for (int32_t v : P.sn_c0) w.push_back(v);
            for (int32_t v : P.sn_r) w.push_back(v);
            for (int32_t v : P.bdiag_ptr) w.push_back(v);
            for (int32_t v : P.bdiag) w.push_back(v);
            for (int32_t v : P.bitem_ptr) w.push_back(v);
            for (const BItem &b : P.bitems) w.insert(w.end(), {b.sn, b.kind, b.a, b.b});
            for (const BPair &b : P.bpairs) w.insert(w.end(), {b.sn, b.k, b.f, b.upos, b.mb});
            for (const BSeg &b : P.bsegs) w.insert(w.end(), {b.pair, b.t0, b.t1});
            for (int32_t v : P.btask_ptr) w.push_back(v);
            for (const BTask &b : P.btasks) w.insert(w.end(), {b.seg_begin, b.seg_end});
            std::fwrite(w.data(), sizeof(int64_t), w.size(), fp);
            std::fclose(fp);
        }
    }
    // the dataflow solve schedules (single and batched) as int64 words:
    // counts (items, forward items, forward chunks, backward chunks, block
    // tables f / b, tail start), then items (8 each), chunks (p0, p1), block
    // tables
    auto dump_df = [](const char *path, const std::vector<int32_t> &items, int64_t nfwd,
                      const std::vector<SolveChunk> &fch, const std::vector<SolveChunk> &bch,
                      const std::vector<int32_t> &snf, const std::vector<int32_t> &snb, int64_t t0) {
        if (FILE *fp = std::fopen(path, "wb")) {
            std::vector<int64_t> w = {(int64_t)items.size() / 8, nfwd, (int64_t)fch.size(), (int64_t)bch.size(),
                                      (int64_t)snf.size(), (int64_t)snb.size(), t0};
            for (int32_t v : items) w.push_back(v);
            for (const SolveChunk &c : fch) { w.push_back(c.p0); w.push_back(c.p1); }
            for (const SolveChunk &c : bch) { w.push_back(c.p0); w.push_back(c.p1); }
            for (int32_t v : snf) w.push_back(v);
            for (int32_t v : snb) w.push_back(v);
            std::fwrite(w.data(), sizeof(int64_t), w.size(), fp);
            std::fclose(fp);
        }
    };
    if (const char *dump = std::getenv("GLU_DUMP_DF")) {
        const HostPlan &P = h->P;
        dump_df(dump, P.df_items, P.df_nfwd, P.df_fchunks, P.df_bchunks, P.df_snx_f, P.df_snx_b, P.tail_t0);
    }
    if (const char *dump = std::getenv("GLU_DUMP_DF_BATCHED")) {
        const HostPlan &P = h->P;
        dump_df(dump, P.df_items_b, P.bdf_nfwd, P.bdf_fchunks, P.bdf_bchunks, P.bdf_snx_f, P.bdf_snx_b,
                P.btail_t0);
    }
    if (h->opt.host_only) {
        h->analyze_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        *out = h;
        return GLU_OK;
    }
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) { glu_destroy(h); return e == cudaErrorMemoryAllocation ? GLU_ERR_OOM : GLU_ERR_CUDA; }
    e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { glu_destroy(h); return GLU_ERR_CUDA; }
    if (const char *lt = std::getenv("GLU_LEVEL_TIMES")) h->level_times_path = lt;
    rc = upload_plan(h);
    if (rc != GLU_OK) {
        if (h->opt.verbose) std::fprintf(stderr, "glu_analyze: %s\n", h->why.c_str());
        glu_destroy(h);
        return rc;
    }
    h->analyze_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return GLU_OK;
}

int glu_analyze(int32_t n, const int32_t *colptr, const int32_t *rowidx, const int32_t *perm, glu_handle **out) {
    return glu_analyze_opts(n, colptr, rowidx, perm, nullptr, out);
}

int glu_set_stream(glu_handle *h, void *s) {
    if (!h) return GLU_ERR_INVALID;
    h->stream = static_cast<cudaStream_t>(s);
    return GLU_OK;
}

int glu_factor(glu_handle *h, const double *values) {
    if (!h || h->opt.host_only) return GLU_ERR_INVALID;
    HostPlan &P = h->P;
    if (P.nnz_a > 0 && !values) return GLU_ERR_INVALID;
    CK(cudaSetDevice(h->device));
    h->err_col = -1;
    const bool dev = P.nnz_a > 0 && is_device_ptr(values);
    if (h->opt.use_graph) {
        // the graph reads the values from the handle's staging buffer
        if (P.nnz_a > 0)
            CK(cudaMemcpyAsync(h->d_aval, values, P.nnz_a * sizeof(double),
                               dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
        if (!h->fgraph) {
            int rc = capture(h, [&](cudaStream_t st) { return enqueue_factor(h, h->d_aval, st, nullptr); },
                             &h->fgraph, &h->fgraph_launches);
            if (rc != GLU_OK) return rc;
        }
        CK(cudaGraphLaunch(h->fgraph, h->stream));
        h->launches += h->fgraph_launches;
    } else {
        const double *av = values;
        if (P.nnz_a > 0 && !dev) {
            CK(cudaMemcpyAsync(h->d_aval, values, P.nnz_a * sizeof(double), cudaMemcpyHostToDevice, h->stream));
            av = h->d_aval;
        }
        if (!h->level_times_path.empty()) {
            const size_t nev = h->opt.factor_blocks != 0 ? (size_t)P.nblev + 1 : P.level_ptr.size() + 1;
            std::vector<cudaEvent_t> ev(nev);
            for (auto &e : ev) CK(cudaEventCreate(&e));
            int rc = enqueue_factor(h, av, h->stream, &ev);
            if (rc != GLU_OK) return rc;
            CK(cudaEventSynchronize(ev.back()));
            if (FILE *fp = std::fopen(h->level_times_path.c_str(), "w")) {
                for (size_t l = 0; l + 1 < nev; l++) {
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, ev[l], ev[l + 1]);
                    std::fprintf(fp, "%zu %.6f\n", l, ms);
                }
                std::fclose(fp);
            }
            for (auto &e : ev) cudaEventDestroy(e);
        } else {
            int rc = enqueue_factor(h, av, h->stream, nullptr);
            if (rc != GLU_OK) return rc;
        }
    }
    h->factored = true;
    if (P.nnz_a > 0 && !dev) return glu_sync(h);   // host input: report errors now
    return GLU_OK;
}

int glu_sync(glu_handle *h) {
    if (!h) return GLU_ERR_INVALID;
    if (h->opt.host_only) return GLU_OK;
    CK(cudaSetDevice(h->device));
    int rc = read_err(h);
    if (rc == GLU_ERR_ZERO_PIVOT || rc == GLU_ERR_NONFINITE) {
        h->factored = h->factored32 = false;
        h->bprec = 0;
    }
    return rc;
}

int glu_solve(glu_handle *h, const double *b, double *x, int32_t nrhs) {
    if (!h || nrhs < 0 || h->opt.host_only) return GLU_ERR_INVALID;
    if (!h->factored) return GLU_ERR_NOT_FACTORED;
    HostPlan &P = h->P;
    const int32_t n = P.n;
    const int64_t elems = (int64_t)n * nrhs;
    if (elems == 0) return GLU_OK;
    if (!b || !x) return GLU_ERR_INVALID;
    CK(cudaSetDevice(h->device));
    int rc = ensure_work(h, nrhs);
    if (rc != GLU_OK) return rc;
    const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
    if (h->opt.use_graph) {
        CK(cudaMemcpyAsync(h->d_bstage, b, elems * sizeof(double),
                           bdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
        size_t gi = 0;
        while (gi < h->sgraphs.size() && h->sgraphs[gi].first != nrhs) gi++;
        if (gi == h->sgraphs.size()) {
            cudaGraphExec_t ex = nullptr;
            int64_t nl = 0;
            rc = capture(h, [&](cudaStream_t st) { return enqueue_solve(h, h->d_bstage, h->d_xstage, nrhs, st); },
                         &ex, &nl);
            if (rc != GLU_OK) return rc;
            h->sgraphs.emplace_back(nrhs, ex);
            h->sgraph_launches.push_back(nl);
        }
        CK(cudaGraphLaunch(h->sgraphs[gi].second, h->stream));
        h->launches += h->sgraph_launches[gi];
        CK(cudaMemcpyAsync(x, h->d_xstage, elems * sizeof(double),
                           xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
        if (!xdev) return glu_sync(h);
        return GLU_OK;
    }
    const double *db = b;
    if (!bdev) {
        CK(cudaMemcpyAsync(h->d_bstage, b, elems * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        db = h->d_bstage;
    }
    double *dx = xdev ? x : h->d_xstage;
    rc = enqueue_solve(h, db, dx, nrhs, h->stream);
    if (rc != GLU_OK) return rc;
    if (!xdev) {
        CK(cudaMemcpyAsync(x, dx, elems * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        return glu_sync(h);
    }
    return GLU_OK;
}

int glu_factor_f32(glu_handle *h, const double *values) {
    if (!h || h->opt.host_only) return GLU_ERR_INVALID;
    HostPlan &P = h->P;
    if (P.nnz_a > 0 && !values) return GLU_ERR_INVALID;
    CK(cudaSetDevice(h->device));
    if (!h->d_lu32) CK(cudaMalloc(&h->d_lu32, std::max<int64_t>(P.lu_colptr[P.n], 1) * sizeof(float)));
    h->err_col = -1;
    const bool dev = P.nnz_a > 0 && is_device_ptr(values);
    // the FP64 values stay in the handle: the residuals of the refinement use them
    if (P.nnz_a > 0)
        CK(cudaMemcpyAsync(h->d_aval, values, P.nnz_a * sizeof(double),
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    if (h->opt.use_graph) {
        if (!h->fgraph32) {
            int rc = capture(h, [&](cudaStream_t st) { return enqueue_factor_f32(h, st); }, &h->fgraph32,
                             &h->fgraph32_launches);
            if (rc != GLU_OK) return rc;
        }
        CK(cudaGraphLaunch(h->fgraph32, h->stream));
        h->launches += h->fgraph32_launches;
    } else {
        int rc = enqueue_factor_f32(h, h->stream);
        if (rc != GLU_OK) return rc;
    }
    h->factored32 = true;
    if (P.nnz_a > 0 && !dev) return glu_sync(h);
    return GLU_OK;
}

int glu_solve_refine(glu_handle *h, const double *b, double *x, int32_t nrhs, double tol, int32_t maxit,
                     glu_refine_info *info) {
    if (!h || nrhs < 0 || maxit < 0 || !(tol >= 0.0) || h->opt.host_only) return GLU_ERR_INVALID;
    if (!h->factored32) return GLU_ERR_NOT_FACTORED;
    glu_refine_info inf{0, 1, 0.0, 0.0};
    HostPlan &P = h->P;
    const int32_t n = P.n;
    const int64_t elems = (int64_t)n * nrhs;
    if (elems == 0) {
        if (info) *info = inf;
        return GLU_OK;
    }
    if (!b || !x) return GLU_ERR_INVALID;
    CK(cudaSetDevice(h->device));
    int rc = ensure_work(h, nrhs);
    if (rc != GLU_OK) return rc;
    rc = ensure_ir(h, nrhs);
    if (rc != GLU_OK) return rc;
    cudaStream_t st = h->stream;
    // b, the iterate x and the residual r live in the handle's buffers, so
    // that one iteration (FP32 solve of r, x += d on the sides not done,
    // r = b - A x with its norms, the check) is the same graph every time.
    // x starts at 0, so the first residual is b itself.
    double *db = h->d_bstage, *dx = h->d_xstage;
    double *r = h->d_ir, *d = h->d_ir + elems;
    CK(cudaMemcpyAsync(db, b, elems * sizeof(double),
                       is_device_ptr(b) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    unsigned long long *anorm = h->d_irnorm, *rmax = anorm + 1, *xmax = rmax + nrhs, *bmax = xmax + nrhs;
    int32_t *done = h->d_done, *ndone = h->d_done + nrhs;
    CK(cudaMemsetAsync(h->d_irnorm, 0, (1 + 3 * (size_t)nrhs) * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(done, 0, (size_t)nrhs * sizeof(int32_t), st));
    CKL(1, launch_anorm(h->d_acsr_ptr, h->d_aval_csr, n, anorm, st));
    CKL(1, launch_absmax(db, n, nrhs, bmax, st));
    CK(cudaMemsetAsync(dx, 0, elems * sizeof(double), st));
    CK(cudaMemcpyAsync(r, db, elems * sizeof(double), cudaMemcpyDeviceToDevice, st));
    auto step = [&](cudaStream_t cs) -> int {
        int rc2 = enqueue_solve_f32(h, r, d, nrhs, cs);
        if (rc2 != GLU_OK) return rc2;
        CKL(1, launch_update(dx, d, done, n, nrhs, cs));
        CK(cudaMemsetAsync(rmax, 0, 2 * (size_t)nrhs * sizeof(unsigned long long), cs));
        CK(cudaMemsetAsync(ndone, 0, sizeof(int32_t), cs));
        CKL(1, launch_residual(h->d_acsr_ptr, h->d_acsr_col, h->d_aval_csr, db, dx, r, n, nrhs, rmax, xmax, cs));
        CKL(1, launch_check(rmax, xmax, bmax, anorm, nrhs, tol, done, h->d_berr, ndone, cs));
        return GLU_OK;
    };
    size_t gi = 0;
    if (h->opt.use_graph) {
        // the check's tolerance is a kernel argument: one graph per (nrhs, tol)
        while (gi < h->rgraphs.size() && !(h->rgraphs[gi].first == nrhs && h->rgraph_tol[gi] == tol)) gi++;
        if (gi == h->rgraphs.size()) {
            cudaGraphExec_t ex = nullptr;
            int64_t nl = 0;
            rc = capture(h, step, &ex, &nl);
            if (rc != GLU_OK) return rc;
            h->rgraphs.emplace_back(nrhs, ex);
            h->rgraph_launches.push_back(nl);
            h->rgraph_tol.push_back(tol);
        }
    }
    std::vector<double> berr((size_t)nrhs);
    int32_t solves = 0;
    while (true) {
        if (solves >= 1 + maxit) {
            inf.converged = 0;
            break;
        }
        if (h->opt.use_graph) {
            CK(cudaGraphLaunch(h->rgraphs[gi].second, st));
            h->launches += h->rgraph_launches[gi];
        } else {
            rc = step(st);
            if (rc != GLU_OK) return rc;
        }
        solves++;
        int32_t nd = 0;
        CK(cudaMemcpyAsync(&nd, ndone, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(berr.data(), h->d_berr, (size_t)nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        double mx = 0.0;
        for (double e : berr) mx = std::max(mx, e);
        inf.berr = mx;
        if (solves == 1) inf.berr_first = mx;
        if (nd == nrhs) {
            inf.converged = 1;
            break;
        }
    }
    inf.iterations = std::max(0, solves - 1);
    if (info) *info = inf;
    CK(cudaMemcpyAsync(x, dx, elems * sizeof(double), is_device_ptr(x) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       st));
    return glu_sync(h);
}

int glu_get_fill(const glu_handle *h, const int64_t **cp, const int32_t **ri, int64_t *nnz) {
    if (!h) return GLU_ERR_INVALID;
    if (cp) *cp = h->P.lu_colptr.data();
    if (ri) *ri = h->P.lu_rowidx.data();
    if (nnz) *nnz = h->P.lu_colptr.empty() ? 0 : h->P.lu_colptr.back();
    return GLU_OK;
}

int glu_get_deps(const glu_handle *h, const int64_t **dp, const int32_t **di) {
    if (!h) return GLU_ERR_INVALID;
    if (dp) *dp = h->P.dep_ptr.data();
    if (di) *di = h->P.dep_idx.data();
    return GLU_OK;
}

int glu_get_levels(const glu_handle *h, int32_t *nlevels, const int32_t **lp, const int32_t **lc) {
    if (!h) return GLU_ERR_INVALID;
    if (nlevels) *nlevels = (int32_t)h->P.level_ptr.size() - 1;
    if (lp) *lp = h->P.level_ptr.data();
    if (lc) *lc = h->P.level_cols.data();
    return GLU_OK;
}

int glu_get_factors(glu_handle *h, double *out) {
    if (!h || !out) return GLU_ERR_INVALID;
    if (!h->factored) return GLU_ERR_NOT_FACTORED;
    const int64_t nnz = h->P.lu_colptr[h->P.n];
    if (nnz == 0) return GLU_OK;
    CK(cudaSetDevice(h->device));
    CK(cudaMemcpyAsync(out, h->d_lu, nnz * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return glu_sync(h);
}

int glu_get_factors_f32(glu_handle *h, float *out) {
    if (!h || !out || h->opt.host_only) return GLU_ERR_INVALID;
    if (!h->factored32) return GLU_ERR_NOT_FACTORED;
    const int64_t nnz = h->P.lu_colptr[h->P.n];
    if (nnz == 0) return GLU_OK;
    CK(cudaSetDevice(h->device));
    CK(cudaMemcpyAsync(out, h->d_lu32, nnz * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    return glu_sync(h);
}

int glu_get_stats(const glu_handle *h, glu_stats *s) {
    if (!h || !s) return GLU_ERR_INVALID;
    const HostPlan &P = h->P;
    std::memset(s, 0, sizeof(*s));
    s->n = P.n;
    s->nlevels = (int32_t)P.level_ptr.size() - 1;
    s->nnz_a = P.nnz_a;
    s->nnz_lu = P.lu_colptr[P.n];
    s->nnz_l = P.nnz_l;
    s->nnz_u = P.nnz_u;
    s->n_deps = P.dep_ptr[P.n];
    s->n_pairs = P.n_pairs;
    s->n_updates = P.n_updates;
    s->flops = P.flops;
    for (int i = 0; i < 3; i++) s->levels_by_mode[i] = P.levels_by_mode[i];
    s->solve_levels_fwd = (int32_t)P.fwd_ptr.size() - 1;
    s->solve_levels_bwd = (int32_t)P.bwd_ptr.size() - 1;
    s->max_level_width = P.max_level_width;
    s->device_bytes = (int64_t)(h->arena_bytes + h->carena_bytes + h->map_total + h->bmap_total + h->dfarena_bytes +
                                4 * h->work_elems * sizeof(double) +
                                (int64_t)std::max(P.fwd_chunks.size(), P.bwd_chunks.size()) * h->work_nrhs *
                                    sizeof(double));
    s->analyze_ms = h->analyze_ms;
    s->kernel_launches = h->launches;
    s->tail_rows = P.n - P.tail_t0;
    s->factor_tail_cols = P.n - P.ftail_t0;
    s->row_lookup = !h->col_ready ? 0 : (h->lookup != 0 ? 1 : 2);
    s->lookup_bytes = (int64_t)h->map_total;
    s->n_runs = h->n_runs;
    return GLU_OK;
}

int glu_last_error_info(const glu_handle *h, int32_t *column) {
    if (!h || !column) return GLU_ERR_INVALID;
    *column = h->err_col;
    return GLU_OK;
}

void glu_destroy(glu_handle *h) {
    if (!h) return;
    if (h->opt.host_only) {
        delete h;
        return;
    }
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    if (h->fgraph) cudaGraphExecDestroy(h->fgraph);
    if (h->fgraph32) cudaGraphExecDestroy(h->fgraph32);
    for (auto &g : h->bgraphs) cudaGraphExecDestroy(g.second);
    cudaFree(h->d_vstage);
    cudaFree(h->d_aT);
    cudaFree(h->d_avb);
    cudaFree(h->d_lub);
    cudaFree(h->d_lub32);
    cudaFree(h->d_bflags);
    cudaFree(h->d_bwork);
    cudaFree(h->d_bpartial);
    cudaFree(h->d_bnorm);
    cudaFree(h->d_bdone);
    cudaFree(h->d_bberr);
    cudaFree(h->d_lu32);
    cudaFree(h->d_ir);
    cudaFree(h->d_irnorm);
    cudaFree(h->d_done);
    cudaFree(h->d_berr);
    drop_rgraphs(h);
    for (auto &g : h->sgraphs) cudaGraphExecDestroy(g.second);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    cudaFree(h->arena);
    cudaFree(h->d_runs);
    cudaFree(h->d_map);
    cudaFree(h->dfarena);
    cudaFree(h->bmap);
    cudaFree(h->carena);
    cudaFree(h->d_work);
    cudaFree(h->d_bstage);
    cudaFree(h->d_xstage);
    cudaFree(h->d_partial);
    delete h;
}

int glu_order_nd(int32_t n, const int32_t *colptr, const int32_t *rowidx, int32_t *perm) {
    try {
        return order_nested_dissection(n, colptr, rowidx, perm);
    } catch (const std::bad_alloc &) {
        return GLU_ERR_OOM;
    }
}

int glu_static_pivot(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *values,
                     int32_t *row_perm, double *row_scale, double *col_scale) {
    try {
        return static_pivot(n, colptr, rowidx, values, row_perm, row_scale, col_scale);
    } catch (const std::bad_alloc &) {
        return GLU_ERR_OOM;
    }
}

int glu_apply_static_pivot(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *values,
                           const int32_t *row_perm, const double *row_scale, const double *col_scale,
                           int32_t *out_rowidx, double *out_values) {
    try {
        return apply_static_pivot(n, colptr, rowidx, values, row_perm, row_scale, col_scale, out_rowidx,
                                  out_values);
    } catch (const std::bad_alloc &) {
        return GLU_ERR_OOM;
    }
}

const char *glu_strerror(int code) {
    switch (code) {
        case GLU_OK: return "ok";
        case GLU_ERR_INVALID: return "invalid argument or malformed input";
        case GLU_ERR_STRUCT_SINGULAR: return "structurally singular: a column of P A P^T lacks its diagonal";
        case GLU_ERR_ZERO_PIVOT: return "zero pivot";
        case GLU_ERR_NONFINITE: return "non-finite pivot";
        case GLU_ERR_OOM: return "out of memory";
        case GLU_ERR_CUDA: return "CUDA runtime error";
        case GLU_ERR_TIMEOUT: return "bounded device wait timed out";
        case GLU_ERR_NOT_FACTORED: return "no successful factorization to solve with";
        case GLU_ERR_INTERNAL: return "internal consistency check failed";
        case GLU_ERR_TOO_LARGE: return "problem exceeds a fixed limit (glu_solve_noalloc's scratch, or 2^31 schedule records)";
        default: return "unknown error code";
    }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// glu_solve_noalloc: the solve with its scratch in a fixed file-scope device
// array instead of handle-owned allocations.  In host code the array's name
// is only a stand-in for the symbol; its device address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.
namespace {

__device__ __align__(256) double g_noalloc_scratch[GLU_NOALLOC_SCRATCH_DOUBLES];

std::mutex g_noalloc_mu;
std::vector<double *> g_noalloc_addr;   // per device; nullptr until looked up

cudaError_t noalloc_scratch_address(int device, double **out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if ((int)g_noalloc_addr.size() <= device) g_noalloc_addr.resize((size_t)device + 1, nullptr);
    if (!g_noalloc_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[device] = static_cast<double *>(p);
    }
    *out = g_noalloc_addr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" int glu_solve_noalloc(glu_handle *h, const double *b, double *x, int32_t nrhs) {
    if (!h || nrhs < 0 || h->opt.host_only) return GLU_ERR_INVALID;
    if (!h->factored) return GLU_ERR_NOT_FACTORED;
    HostPlan &P = h->P;
    const int32_t n = P.n;
    const int64_t elems = (int64_t)n * nrhs;
    if (elems == 0) return GLU_OK;
    if (!b || !x || !is_device_ptr(b) || !is_device_ptr(x)) return GLU_ERR_INVALID;
    // The handle's own solve schedule: the dataflow solve needs y and z (n *
    // nrhs values each) and its chunk partial sums; the per-level solve
    // (solve_mode 0) needs y and its level chunks.  Each part 32-value aligned.
    const bool df = h->opt.solve_mode == 1;
    const int64_t yelems = (elems + 31) / 32 * 32;
    const int64_t nch = df ? (int64_t)(P.df_fchunks.size() + P.df_bchunks.size()) * nrhs
                           : (int64_t)std::max(P.fwd_chunks.size(), P.bwd_chunks.size()) * nrhs;
    const int64_t need = (df ? 2 : 1) * yelems + nch;
    if (need > (int64_t)GLU_NOALLOC_SCRATCH_DOUBLES) {
        h->why = "glu_solve_noalloc: needs " + std::to_string(need) + " doubles of scratch, the array holds " +
                 std::to_string((long long)GLU_NOALLOC_SCRATCH_DOUBLES);
        return GLU_ERR_TOO_LARGE;
    }
    CK(cudaSetDevice(h->device));
    double *scratch = nullptr;
    CK(noalloc_scratch_address(h->device, &scratch));
    double *y = scratch;
    cudaStream_t st = h->stream;
    CKL(1, launch_permute_in<double>(y, b, h->d_perm, n, nrhs, st));
    SolveArgs<double> a = sargs(h);
    if (df) {
        // the same launches as glu_solve's dataflow solve (its ready flags,
        // ticket and error word belong to the handle, allocated by glu_analyze)
        double *z = y + yelems;
        int rc = enqueue_df<double>(h, a, y, z, z + yelems, nrhs, st);
        if (rc != GLU_OK) return rc;
        CKL(1, launch_permute_out<double>(x, z, h->d_perm, n, nrhs, st));
        return GLU_OK;
    }
    double *partial = scratch + yelems;
    int launched = 0;
    for (size_t l = 0; l + 1 < P.fwd_ptr.size(); l++) {
        CK(launch_solve_level<double>(a, false, y, nrhs, h->d_fwd_items + P.fwd_ptr[l], P.fwd_ptr[l + 1] - P.fwd_ptr[l],
                                      h->d_fwd_chunks, P.fwd_chunk_ptr[l], P.fwd_chunk_ptr[l + 1], partial, st,
                                      &launched));
        h->launches += launched;
    }
    for (size_t l = 0; l + 1 < P.bwd_ptr.size(); l++) {
        CK(launch_solve_level<double>(a, true, y, nrhs, h->d_bwd_items + P.bwd_ptr[l], P.bwd_ptr[l + 1] - P.bwd_ptr[l],
                                      h->d_bwd_chunks, P.bwd_chunk_ptr[l], P.bwd_chunk_ptr[l + 1], partial, st,
                                      &launched));
        h->launches += launched;
    }
    CKL(1, launch_permute_out<double>(x, y, h->d_perm, n, nrhs, st));
    return GLU_OK;
}

// ---------------------------------------------------------------------------
// Batched value sets.
namespace {

int ensure_batch(glu_handle *h, int32_t S, bool f32) {
    HostPlan &P = h->P;
    const int64_t nnz = P.lu_colptr[P.n];
    if (S != h->bcap) {
        for (auto &g : h->bgraphs) cudaGraphExecDestroy(g.second);
        h->bgraphs.clear();
        h->bgraph_launches.clear();
        cudaFree(h->d_vstage);
        cudaFree(h->d_aT);
        cudaFree(h->d_avb);
        cudaFree(h->d_lub);
        cudaFree(h->d_lub32);
        cudaFree(h->d_bflags);
        h->d_vstage = h->d_aT = h->d_avb = h->d_lub = nullptr;
        h->d_lub32 = nullptr;
        h->d_bflags = nullptr;
        h->bcap = 0;
        h->bwork_nrhs = 0;   // solve buffers depend on the stride too
        const int32_t G = S / 32;
        const int64_t na = std::max<int64_t>(P.nnz_a, 1);
        CK(cudaMalloc(&h->d_vstage, na * S * sizeof(double)));
        CK(cudaMalloc(&h->d_aT, na * S * sizeof(double)));
        CK(cudaMalloc(&h->d_avb, na * S * sizeof(double)));
        h->n_bflags =
            (2 * (int64_t)P.n + (int64_t)P.bdf_fchunks.size() + (int64_t)P.bdf_bchunks.size() + P.bdf_nblocks) * G;
        CK(cudaMalloc(&h->d_bflags, std::max<int64_t>(h->n_bflags, 1) * sizeof(int32_t)));
        h->bcap = S;
    }
    if (f32 && !h->d_lub32) CK(cudaMalloc(&h->d_lub32, std::max<int64_t>(nnz, 1) * S * sizeof(float)));
    if (!f32 && !h->d_lub) CK(cudaMalloc(&h->d_lub, std::max<int64_t>(nnz, 1) * S * sizeof(double)));
    return GLU_OK;
}

template <typename T>
int enqueue_factor_b(glu_handle *h, T *lu, int32_t B, int32_t S, cudaStream_t st) {
    HostPlan &P = h->P;
    CKL(1, launch_reset_err(h->d_err, st));
    CKL(P.nnz_a > 0, launch_values_in(h->d_aT, h->d_vstage, P.nnz_a, B, P.nnz_a, S, st));
    CKL(P.lu_colptr[P.n] > 0, launch_gather_b<T>(lu, h->d_aT, h->d_gsrc, P.lu_colptr[P.n], S, st));
    FactorArgs<T> a = fargs_t<T>(h, lu);
    const int32_t nl = (int32_t)P.level_ptr.size() - 1;
    for (int32_t l = 0; l <= nl; l++) {
        LevelRange r;
        r.t_begin = l < nl ? P.lvl_task_ptr[l] : 0;
        r.row_begin = l < nl ? P.lvl_row_ptr[l] : 0;
        r.lane_begin = l < nl ? P.lvl_lane_ptr[l] : 0;
        r.t_end = l < nl ? P.lvl_task_ptr[l + 1] : 0;
            r.n_begin = P.lvl_norm_ptr[l];
        r.n_end = P.lvl_norm_ptr[l + 1];
        CKL((r.t_end - r.t_begin) + (r.n_end - r.n_begin) > 0, launch_level_b<T>(a, h->lookup, r, S, h->num_sms, st));
    }
    CKL(P.n > 0, launch_pivot_b<T>(lu, h->d_diag, P.n, B, S, h->d_err, st));
    return GLU_OK;
}

int factor_batched(glu_handle *h, const double *values, int32_t batch, int64_t ld, bool f32) {
    if (!h || h->opt.host_only || batch <= 0) return GLU_ERR_INVALID;
    HostPlan &P = h->P;
    if (P.nnz_a > 0 && (!values || ld < P.nnz_a)) return GLU_ERR_INVALID;
    CK(cudaSetDevice(h->device));
    int rc = setup_column_plan(h);   // batches run the column-level schedule
    if (rc != GLU_OK) return rc;
    const int32_t S = (batch + 31) / 32 * 32;
    h->bprec = 0;
    rc = ensure_batch(h, S, f32);
    if (rc != GLU_OK) return rc;
    h->err_col = -1;
    cudaStream_t st = h->stream;
    const bool dev = P.nnz_a > 0 && is_device_ptr(values);
    if (P.nnz_a > 0)
        CK(cudaMemcpy2DAsync(h->d_vstage, P.nnz_a * sizeof(double), values, ld * sizeof(double),
                             P.nnz_a * sizeof(double), batch, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             st));
    // the graph depends on the batch through the padding lanes: key on both
    const int key = (f32 ? 1 : 0) | (batch << 1);
    size_t gi = 0;
    while (gi < h->bgraphs.size() && h->bgraphs[gi].first != key) gi++;
    if (gi == h->bgraphs.size()) {
        cudaGraphExec_t ex = nullptr;
        int64_t nlaunch = 0;
        if (f32)
            rc = capture(h, [&](cudaStream_t cs) { return enqueue_factor_b<float>(h, h->d_lub32, batch, S, cs); }, &ex,
                         &nlaunch);
        else
            rc = capture(h, [&](cudaStream_t cs) { return enqueue_factor_b<double>(h, h->d_lub, batch, S, cs); }, &ex,
                         &nlaunch);
        if (rc != GLU_OK) return rc;
        h->bgraphs.emplace_back(key, ex);
        h->bgraph_launches.push_back(nlaunch);
    }
    CK(cudaGraphLaunch(h->bgraphs[gi].second, st));
    h->launches += h->bgraph_launches[gi];
    h->bB = batch;
    h->bS = S;
    h->bprec = f32 ? 32 : 64;
    if (P.nnz_a > 0 && !dev) return glu_sync(h);
    return GLU_OK;
}

int ensure_bwork(glu_handle *h, int32_t nrhs) {
    if (nrhs <= h->bwork_nrhs) return GLU_OK;
    cudaFree(h->d_bwork);
    cudaFree(h->d_bpartial);
    cudaFree(h->d_bnorm);
    cudaFree(h->d_bdone);
    cudaFree(h->d_bberr);
    h->d_bwork = h->d_bpartial = h->d_bberr = nullptr;
    h->d_bnorm = nullptr;
    h->d_bdone = nullptr;
    h->bwork_nrhs = 0;
    const int64_t S = h->bcap;
    const int64_t e = std::max<int64_t>((int64_t)h->P.n * nrhs * S, 1);
    const int64_t nch = std::max<int64_t>((int64_t)(h->P.bdf_fchunks.size() + h->P.bdf_bchunks.size()) * nrhs * S, 1);
    CK(cudaMalloc(&h->d_bwork, 7 * e * sizeof(double)));
    CK(cudaMalloc(&h->d_bpartial, nch * sizeof(double)));
    CK(cudaMalloc(&h->d_bnorm, (S + 3 * (size_t)nrhs * S) * sizeof(unsigned long long)));
    CK(cudaMalloc(&h->d_bdone, (1 + (size_t)nrhs * S) * sizeof(int32_t)));
    CK(cudaMalloc(&h->d_bberr, (size_t)nrhs * S * sizeof(double)));
    h->bwork_nrhs = nrhs;
    return GLU_OK;
}

template <typename T>
int enqueue_solve_b(glu_handle *h, const T *lu, const double *in, double *out, int32_t nrhs, cudaStream_t st) {
    HostPlan &P = h->P;
    const int32_t n = P.n, S = h->bS, G = S / 32;
    const int64_t e = (int64_t)n * nrhs * S;
    T *y = reinterpret_cast<T *>(h->d_bwork);
    T *z = y + e;
    CK(cudaMemsetAsync(h->d_bflags, 0, h->n_bflags * sizeof(int32_t), st));
    CK(cudaMemsetAsync(h->d_serr, 0xff, sizeof(unsigned long long), st));
    SolveArgs<T> sa = sargs_t<T>(h, lu);
    DFSolveArgs d;
    d.items = h->d_bdf_items;
    d.nitems = (int32_t)(P.df_items_b.size() / 8);
    d.epoch = 1;
    d.fault_row = -1;
    d.fchunks = h->d_bfwd_chunks;
    d.bchunks = h->d_bbwd_chunks;
    T *part = reinterpret_cast<T *>(h->d_bpartial);
    d.fpartial_v = part;
    d.bpartial_v = part + (int64_t)P.bdf_fchunks.size() * nrhs * S;
    d.fready = h->d_bflags;
    d.bready = h->d_bflags + (int64_t)n * G;
    d.fchunk_ready = h->d_bflags + 2 * (int64_t)n * G;
    d.bchunk_ready = d.fchunk_ready + (int64_t)P.bdf_fchunks.size() * G;
    d.blk_done = d.bchunk_ready + (int64_t)P.bdf_bchunks.size() * G;
    d.ticket = h->d_ticket;
    d.abort = h->d_abort;
    d.err = h->d_serr;
    d.spin_limit_cycles = h->spin_cycles;
    d.fsnx = h->d_bsnx_f;
    d.bsnx = h->d_bsnx_b;
    TailArgs ta{P.btail_t0, h->d_btail_cb, h->d_btail_ce, d.bready, d.epoch};
    CKL(4 + (P.btail_t0 < n), launch_solve_b<T>(sa, d, P.bdf_nfwd, ta, in, out, y, z, h->d_perm, nrhs, S,
                                                h->num_sms, st));
    return GLU_OK;
}

}  // namespace

extern "C" int glu_factor_batched(glu_handle *h, const double *values, int32_t batch, int64_t ld) {
    return factor_batched(h, values, batch, ld, false);
}

extern "C" int glu_factor_batched_f32(glu_handle *h, const double *values, int32_t batch, int64_t ld) {
    return factor_batched(h, values, batch, ld, true);
}

extern "C" int glu_solve_batched(glu_handle *h, const double *b, double *x, int32_t nrhs, int32_t batch) {
    if (!h || h->opt.host_only || nrhs < 0 || batch <= 0) return GLU_ERR_INVALID;
    if (h->bprec != 64) return GLU_ERR_NOT_FACTORED;
    if (batch != h->bB) return GLU_ERR_INVALID;
    HostPlan &P = h->P;
    const int32_t n = P.n, S = h->bS;
    const int64_t elems = (int64_t)n * nrhs * batch;
    if (elems == 0) return GLU_OK;
    if (!b || !x) return GLU_ERR_INVALID;
    CK(cudaSetDevice(h->device));
    int rc = ensure_bwork(h, nrhs);
    if (rc != GLU_OK) return rc;
    cudaStream_t st = h->stream;
    const int64_t e = (int64_t)n * nrhs * S;
    double *bin = h->d_bwork + 2 * e, *bout = h->d_bwork + 3 * e, *stage = h->d_bwork + 4 * e;
    const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
    const double *src = b;
    if (!bdev) {
        CK(cudaMemcpyAsync(stage, b, elems * sizeof(double), cudaMemcpyHostToDevice, st));
        src = stage;
    }
    CKL(1, launch_rhs_in(bin, src, n, nrhs, batch, S, st));
    rc = enqueue_solve_b<double>(h, h->d_lub, bin, bout, nrhs, st);
    if (rc != GLU_OK) return rc;
    double *dst = xdev ? x : stage;
    CKL(1, launch_rhs_out(dst, bout, n, nrhs, batch, S, st));
    if (!xdev) {
        CK(cudaMemcpyAsync(x, stage, elems * sizeof(double), cudaMemcpyDeviceToHost, st));
        return glu_sync(h);
    }
    return GLU_OK;
}

extern "C" int glu_solve_batched_refine(glu_handle *h, const double *b, double *x, int32_t nrhs, int32_t batch,
                                        double tol, int32_t maxit, glu_refine_info *info) {
    if (!h || h->opt.host_only || nrhs < 0 || batch <= 0 || maxit < 0 || !(tol >= 0.0)) return GLU_ERR_INVALID;
    if (h->bprec != 32) return GLU_ERR_NOT_FACTORED;
    if (batch != h->bB) return GLU_ERR_INVALID;
    glu_refine_info inf{0, 1, 0.0, 0.0};
    HostPlan &P = h->P;
    const int32_t n = P.n, S = h->bS;
    const int64_t elems = (int64_t)n * nrhs * batch;
    if (elems == 0) {
        if (info) *info = inf;
        return GLU_OK;
    }
    if (!b || !x) return GLU_ERR_INVALID;
    CK(cudaSetDevice(h->device));
    int rc = ensure_bwork(h, nrhs);
    if (rc != GLU_OK) return rc;
    cudaStream_t st = h->stream;
    const int64_t e = (int64_t)n * nrhs * S;
    double *bin = h->d_bwork + 2 * e, *stage = h->d_bwork + 3 * e, *r = h->d_bwork + 4 * e, *d = h->d_bwork + 5 * e,
           *xi = h->d_bwork + 6 * e;
    unsigned long long *anorm = h->d_bnorm, *rmax = anorm + S, *xmax = rmax + (int64_t)nrhs * S,
                       *bmax = xmax + (int64_t)nrhs * S;
    int32_t *done = h->d_bdone, *ndone = h->d_bdone + (int64_t)nrhs * S;
    const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
    const double *src = b;
    if (!bdev) {
        CK(cudaMemcpyAsync(stage, b, elems * sizeof(double), cudaMemcpyHostToDevice, st));
        src = stage;
    }
    CKL(1, launch_rhs_in(bin, src, n, nrhs, batch, S, st));
    CK(cudaMemsetAsync(h->d_bnorm, 0, (S + 3 * (size_t)nrhs * S) * sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(done, 0, (size_t)nrhs * S * sizeof(int32_t), st));
    CKL(3, launch_ir_b(0, h->d_acsr_ptr, h->d_acsr_col, h->d_avb, h->d_aT, h->d_acsr_src, P.nnz_a, bin, xi, r, d, n,
                       nrhs, batch, S, anorm, rmax, xmax, bmax, tol, done, h->d_bberr, ndone, st));
    // x starts at 0, so the first residual is b itself
    CK(cudaMemsetAsync(xi, 0, e * sizeof(double), st));
    CK(cudaMemcpyAsync(r, bin, e * sizeof(double), cudaMemcpyDeviceToDevice, st));
    std::vector<double> berr((size_t)nrhs * S);
    int32_t solves = 0;
    while (true) {
        if (solves >= 1 + maxit) {
            inf.converged = 0;
            break;
        }
        rc = enqueue_solve_b<float>(h, h->d_lub32, r, d, nrhs, st);
        if (rc != GLU_OK) return rc;
        CKL(1, launch_ir_b(2, h->d_acsr_ptr, h->d_acsr_col, h->d_avb, h->d_aT, h->d_acsr_src, P.nnz_a, bin, xi, r, d, n,
                           nrhs, batch, S, anorm, rmax, xmax, bmax, tol, done, h->d_bberr, ndone, st));
        solves++;
        CK(cudaMemsetAsync(rmax, 0, 2 * (size_t)nrhs * S * sizeof(unsigned long long), st));
        CK(cudaMemsetAsync(ndone, 0, sizeof(int32_t), st));
        CKL(2, launch_ir_b(1, h->d_acsr_ptr, h->d_acsr_col, h->d_avb, h->d_aT, h->d_acsr_src, P.nnz_a, bin, xi, r, d,
                           n, nrhs, batch, S, anorm, rmax, xmax, bmax, tol, done, h->d_bberr, ndone, st));
        int32_t nd = 0;
        CK(cudaMemcpyAsync(&nd, ndone, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(berr.data(), h->d_bberr, berr.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        double mx = 0.0;
        for (double v : berr) mx = std::max(mx, v);
        inf.berr = mx;
        if (solves == 1) inf.berr_first = mx;
        if (nd == nrhs * batch) {
            inf.converged = 1;
            break;
        }
    }
    inf.iterations = std::max(0, solves - 1);
    if (info) *info = inf;
    double *dst = xdev ? x : stage;
    CKL(1, launch_rhs_out(dst, xi, n, nrhs, batch, S, st));
    if (!xdev) CK(cudaMemcpyAsync(x, stage, elems * sizeof(double), cudaMemcpyDeviceToHost, st));
    return glu_sync(h);
}

extern "C" int glu_get_factors_batched_f32(glu_handle *h, int32_t set, float *out) {
    if (!h || !out || h->opt.host_only) return GLU_ERR_INVALID;
    if (h->bprec != 32) return GLU_ERR_NOT_FACTORED;
    if (set < 0 || set >= h->bB) return GLU_ERR_INVALID;
    const int64_t nnz = h->P.lu_colptr[h->P.n];
    if (nnz == 0) return GLU_OK;
    CK(cudaSetDevice(h->device));
    CK(cudaMemcpy2DAsync(out, sizeof(float), h->d_lub32 + set, (size_t)h->bS * sizeof(float), sizeof(float), nnz,
                         cudaMemcpyDeviceToHost, h->stream));
    return glu_sync(h);
}

extern "C" int glu_get_factors_batched(glu_handle *h, int32_t set, double *out) {
    if (!h || !out || h->opt.host_only) return GLU_ERR_INVALID;
    if (h->bprec != 64) return GLU_ERR_NOT_FACTORED;
    if (set < 0 || set >= h->bB) return GLU_ERR_INVALID;
    const int64_t nnz = h->P.lu_colptr[h->P.n];
    if (nnz == 0) return GLU_OK;
    CK(cudaSetDevice(h->device));
    CK(cudaMemcpy2DAsync(out, sizeof(double), h->d_lub + set, (size_t)h->bS * sizeof(double), sizeof(double), nnz,
                         cudaMemcpyDeviceToHost, h->stream));
    return glu_sync(h);
}
