// glu_device.cuh -- device-side argument blocks and launch helpers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "glu_internal.h"

namespace glu {

// Pending device error: the smallest (column << 8 | code) wins.
constexpr unsigned long long ERR_NONE = ~0ull;
enum : unsigned { DEVERR_ZERO_PIVOT = 1, DEVERR_NONFINITE = 2, DEVERR_TIMEOUT = 3, DEVERR_INTERNAL = 4 };

// The work list of one level (indices into tasks / norms).
struct LevelRange {
    int32_t t_begin, row_begin, lane_begin, t_end;
    int32_t n_begin, n_end;
};

// Grid barrier state of the cooperative kernels (a monotone arrival count
// and an abort word, both zeroed before the launch).
struct GridBarrier {
    unsigned *count;
    unsigned *abort;
    unsigned long long *err;
    long long spin_limit_cycles;
};

#ifdef __CUDACC__
// Grid barrier of a cooperative launch: the block's first thread fences,
// arrives and waits until `target` blocks have arrived, then fences again;
// the block barriers on both sides order the other threads' accesses (the
// scheme of a cooperative-groups grid sync).  The wait is bounded: past the
// limit the block records GLU_ERR_TIMEOUT and raises the abort word; a block
// that sees the abort word stops waiting.  Returns false (in every thread of
// the block) when the launch must end.
__device__ __forceinline__ bool grid_sync(const GridBarrier &bar, unsigned target, int *s_stop) {
    __syncthreads();
    if (threadIdx.x == 0) {
        *s_stop = 0;
        __threadfence();
        atomicAdd(bar.count, 1u);
        if (*(volatile const unsigned *)bar.count < target) {
            const long long t0 = clock64();
            int spins = 0;
            while (*(volatile const unsigned *)bar.count < target) {
                __nanosleep(20);
                if ((++spins & 63) == 0) {
                    if (*(volatile const unsigned *)bar.abort) {
                        *s_stop = 1;
                        break;
                    }
                    if (clock64() - t0 > bar.spin_limit_cycles) {
                        atomicOr(bar.abort, 1u);
                        atomicMin(bar.err, (0xffffffull << 8) | DEVERR_TIMEOUT);
                        *s_stop = 1;
                        break;
                    }
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int *)s_stop == 0;
}
#endif

// The supernodal factorization's tables (see kernels_blocks.cu).
template <typename T>
struct BlockArgs {
    T *lu;
    const int64_t *colptr;
    const int32_t *rowidx;
    const int64_t *diag_pos;
    const int32_t *sn_c0, *sn_r, *bdiag;
    const BItem *bitems;
    const BPair *bpairs;
    const BSeg *bsegs;
    const BTask *btasks;
    const void *map;             // per pair, offsets in column k of the rows R_B
    unsigned long long *err;
};

// The dense trailing block [t0, t0 + nt) of the factorization: column t0 + k
// keeps rows t0 .. t0+nt-1 as its last nt entries.
struct DenseTailArgs {
    int32_t t0, nt;
    const int64_t *colptr;       // lu_colptr
};

template <typename T>
struct FactorArgs {
    T *lu;                       // values over the filled pattern
    const int64_t *diag_pos;     // n
    const void *map;             // position map (2 or 4 bytes per update), or null
    const Run *runs;             // run table, or null
    const Seg *segs;
    const Task *tasks;
    const NormItem *norms;
    unsigned long long *err;
};

// Building the row lookup of the level kernels.  Position map: per pair (j,
// k) with U(j,k) at pair_pos, the offset of every row of L(:,j) in column k
// past U(j,k), at pair_map[pair] + t.  Run table: the runs of L(:,j)'s rows in
// column k (counted first, then written at pair_runs[pair]).  Then every
// segment, which carries its pair's index, gets its map base or run range.
struct RunBuildArgs {
    const int64_t *lu_colptr;
    const int32_t *lu_rowidx;
    const int64_t *diag_pos;
    const int32_t *pair_j;
    const int32_t *pair_k;
    const int64_t *pair_pos;
    const int64_t *pair_runs;    // npairs + 1 (fill pass and segment pass)
    const int64_t *pair_map;     // npairs + 1 (position map)
    int32_t *counts;             // npairs (count pass)
    Run *runs;
    void *map;
    Seg *segs;
    int64_t npairs, nsegs;
    unsigned long long *err;
};

template <typename T>
struct SolveArgs {
    const T *lu;
    const int64_t *diag_pos;
    const int64_t *lrow_ptr;
    const int32_t *lrow_col;
    const int64_t *lrow_pos;
    const int64_t *urow_ptr;
    const int32_t *urow_col;
    const int64_t *urow_pos;
    int32_t n;
};

// Dataflow solve: one work item per row or long-row chunk, in topological
// order (forward items, then backward items).
enum : int32_t { DF_BACKWARD = 1, DF_CHUNK = 2, DF_BLOCK = 4 };
struct DFItem {
    int32_t row;
    int32_t cb;      // row item: its chunks cb..ce-1 (none if equal)
    int32_t ce;
    int32_t chunk;   // chunk item: index into the chunk list
    int32_t flags;
    int32_t sub;     // batched block copy: right-hand sides r = sub (mod RSPLIT_B)
    int32_t blk;     // batched block copy: the block's ordinal (completion counter)
    int32_t spare;
};

struct DFSolveArgs {
    const DFItem *items;      // this launch's items (a sub-range of the list)
    int32_t nitems;
    int32_t epoch;
    int32_t fault_row;            // test hook: this row never publishes (-1: none)
    const SolveChunk *fchunks, *bchunks;
    void *fpartial_v, *bpartial_v;
    int32_t *fready, *bready, *fchunk_ready, *bchunk_ready;
    unsigned *ticket;
    unsigned *abort;
    unsigned long long *err;
    long long spin_limit_cycles;
    const int32_t *fsnx, *bsnx;   // dense diagonal blocks: per row, its first outside chunk
    int32_t *blk_done;            // batched: per (block, lane group), copies finished
};

// launchers (kernels_factor.cu)
template <typename T>
cudaError_t launch_gather(T *lu, const double *aval, const int32_t *gsrc, int64_t nnz, cudaStream_t s);
// A dataflow run of levels [l0, l1) (see k_levels_df): the per-level work
// ranges and item prefix (global level indices), the per-task and per-level
// tables of dataflow_tables, and the counters (zeroed before the launch).
struct DFFactorArgs {
    const LevelRange *ranges;     // nlevels + 1
    const int32_t *item_ptr;      // nlevels + 2
    int32_t l0, l1;
    const int32_t *task_col, *task_before, *lvl_total, *lvl_ntasks, *level_of;
    int32_t *cdone;               // per column: tasks of the run done that target it
    int32_t *ldone;               // per level: tasks of the run done that target its columns
    int32_t *tdone;               // per level: its tasks done
    unsigned *ticket;
    unsigned *abort;
    unsigned long long *err;
    long long spin_limit_cycles;
    int32_t fault_col;            // test hook: tasks targeting this column never publish (-1: none)
    int32_t max_items;            // the most work items of one level of the run (sizes the grid)
};

// lookup: 2 or 4 = position map of that many bytes per update, 0 = run table
template <typename T>
cudaError_t launch_level(const FactorArgs<T> &a, int lookup, const LevelRange &r, int num_sms, cudaStream_t s);
template <typename T>
cudaError_t launch_levels_df(const FactorArgs<T> &a, int lookup, const DFFactorArgs &d, int num_sms, cudaStream_t s);
// One level of the supernodal factorization: diagonal blocks d0..d1-1,
// panel items i0..i1-1, update tasks k0..k1-1 (kernels_blocks.cu); *launched
// counts the kernels launched.
template <typename T>
cudaError_t launch_block_level(const BlockArgs<T> &a, int map_bytes, int32_t d0, int32_t d1, int32_t i0,
                               int32_t i1, int32_t k0, int32_t k1, int num_sms, cudaStream_t s, int *launched);
cudaError_t launch_bmap_build(const BlockArgs<double> &a, int map_bytes, int64_t npairs, int num_sms, cudaStream_t s);
// Dense LU of the trailing block (one cooperative launch, grid barriers).
template <typename T>
cudaError_t launch_dense_tail(T *lu, const DenseTailArgs &d, const GridBarrier &bar, int num_sms, cudaStream_t s);
template <typename T>
cudaError_t launch_pivot_check(const T *lu, const int64_t *diag_pos, int32_t n,
                               unsigned long long *err, cudaStream_t s);
// The run table: pass 0 counts each pair's runs, pass 1 writes them, pass 2
// points every segment at its runs.  The position map: pass 3 writes it
// (map_bytes per entry), pass 4 points every segment at its map entries.
cudaError_t launch_run_build(const RunBuildArgs &a, int pass, int map_bytes, cudaStream_t s);
cudaError_t launch_reset_err(unsigned long long *err, cudaStream_t s);

// launchers (kernels_solve.cu)
template <typename T>
cudaError_t launch_permute_in(T *y, const double *b, const int32_t *perm, int32_t n, int32_t nrhs,
                              cudaStream_t s);
template <typename T>
cudaError_t launch_permute_out(double *x, const T *y, const int32_t *perm, int32_t n, int32_t nrhs,
                               cudaStream_t s);
template <typename T>
cudaError_t launch_solve_df(const SolveArgs<T> &s, const DFSolveArgs &a, T *y, T *z, int32_t nrhs, int num_sms,
                            cudaStream_t st);
// One-block solve of the dense tail [t0, n): forward rows start from the
// partial sums over columns < t0, then both column sweeps in shared memory.
struct TailArgs {
    int32_t t0;
    const int32_t *cb, *ce;       // forward partial chunks of each tail row
    int32_t *bready;              // backward ready flags, set for the tail rows
    int32_t epoch;
};
template <typename T>
cudaError_t launch_solve_tail(const SolveArgs<T> &s, const int64_t *lu_colptr, const TailArgs &t, const T *fpartial,
                              T *y, T *z, int32_t nrhs, cudaStream_t st);
template <typename T>
cudaError_t launch_solve_level(const SolveArgs<T> &a, bool backward, T *y, int32_t nrhs, const SolveRow *items,
                               int32_t nitems, const SolveChunk *chunks, int32_t c0, int32_t c1, T *partial,
                               cudaStream_t s, int *launched);

// launchers (kernels_refine.cu): FP64 residual side of iterative refinement
cudaError_t launch_csr_values(double *out, const double *aval, const int64_t *src, int64_t nnz, cudaStream_t s);
cudaError_t launch_anorm(const int64_t *rp, const double *av, int32_t n, unsigned long long *anorm, cudaStream_t s);
cudaError_t launch_residual(const int64_t *rp, const int32_t *ci, const double *av, const double *b, const double *x,
                            double *r, int32_t n, int32_t nrhs, unsigned long long *rmax, unsigned long long *xmax,
                            cudaStream_t s);
cudaError_t launch_absmax(const double *v, int32_t n, int32_t nrhs, unsigned long long *out, cudaStream_t s);
cudaError_t launch_check(const unsigned long long *rmax, const unsigned long long *xmax,
                         const unsigned long long *bmax, const unsigned long long *anorm, int32_t nrhs, double tol,
                         int32_t *done, double *berr, int32_t *ndone, cudaStream_t s);
cudaError_t launch_update(double *x, const double *d, const int32_t *done, int32_t n, int32_t nrhs, cudaStream_t s);

// launchers (kernels_batched.cu): interleaved value sets, S lanes per entry
cudaError_t launch_values_in(double *aT, const double *v, int64_t nnz, int32_t B, int64_t ld, int32_t S,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_gather_b(T *lu, const double *aT, const int32_t *gsrc, int64_t nnz, int32_t S, cudaStream_t s);
template <typename T>
cudaError_t launch_level_b(const FactorArgs<T> &a, int lookup, const LevelRange &r, int32_t S, int num_sms,
                           cudaStream_t s);
template <typename T>
cudaError_t launch_pivot_b(const T *lu, const int64_t *diag_pos, int32_t n, int32_t B, int32_t S,
                           unsigned long long *err, cudaStream_t s);
cudaError_t launch_rhs_in(double *out, const double *in, int32_t n, int32_t nrhs, int32_t B, int32_t S,
                          cudaStream_t s);
cudaError_t launch_rhs_out(double *out, const double *in, int32_t n, int32_t nrhs, int32_t B, int32_t S,
                           cudaStream_t s);
template <typename T>
cudaError_t launch_solve_b(const SolveArgs<T> &sa, const DFSolveArgs &a, int32_t nfwd,
                           const TailArgs &ta, const double *in, double *out, T *y, T *z, const int32_t *perm,
                           int32_t nrhs, int32_t S, int num_sms, cudaStream_t s);
cudaError_t launch_ir_b(int op, const int64_t *rp, const int32_t *ci, const double *av, const double *aT,
                        const int64_t *src, int64_t nnz, const double *bb, double *x, double *r, const double *d,
                        int32_t n, int32_t nrhs, int32_t B, int32_t S, unsigned long long *anorm,
                        unsigned long long *rmax, unsigned long long *xmax, unsigned long long *bmax, double tol,
                        int32_t *done, double *berr, int32_t *ndone, cudaStream_t s);

}  // namespace glu
