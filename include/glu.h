/*
 * glu.h -- C ABI of the GB300 (sm_103a) sparse LU refactorization library.
 *
 * The method is GLU3.0 (Peng & Tan, "GLU3.0: Fast GPU-based Parallel Sparse
 * LU Factorization for Circuit Simulation"): a statically pivoted,
 * fill-reduced sparse A = LU is analysed once on the host (fill-in,
 * relaxed column dependencies, levels) and then refactorized on the GPU
 * many times with new values (Section III, first paragraph: the numeric part
 * repeats inside Newton-Raphson loops), level by level, with the hybrid
 * right-looking column update (Algorithm 2, Algorithm 5, Eqs. 1-3).  x
 * follows from the two triangular solves (Section I).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Indices are 0-based.  The input matrix is n x n in compressed sparse
 * column form: colptr[n+1] (colptr[0] = 0, non-decreasing), rowidx[nnz]
 * with rows sorted ascending and no duplicates inside a column; every
 * column of P A P^T must hold its diagonal.  perm[n] maps new to old:
 * the library factors B = P A P^T with B(i,j) = A(perm[i], perm[j]);
 * NULL means the identity.  The factor is stored as one CSC array over the
 * filled pattern, A_s = L + U - I (Section II-A): the strict lower part of
 * each column is L (unit diagonal implied), the rest is U.
 *
 * Values, right-hand sides and solutions are double arrays that may live in
 * host or device memory; the library tells them apart with
 * cudaPointerGetAttributes.  Multiple right-hand sides are stored one after
 * the other, each of length n (column-major n x nrhs).
 *
 * Execution is stream-ordered on the handle's stream (glu_set_stream,
 * default: the legacy default stream).  A call given only device pointers
 * returns once its work is enqueued; errors raised on the GPU (zero or
 * non-finite pivot, bounded-wait timeout) surface at the next call that
 * synchronizes: glu_sync, or any call with a host output.  A call with a
 * host output returns after the result is in host memory.
 *
 * Ownership: glu_analyze copies its inputs; the handle owns every array it
 * hands out, which stays valid until glu_destroy.  One handle must not be
 * used by two host threads at once; separate handles are independent.
 *
 * Return codes: GLU_OK (0) or one of the negative GLU_ERR_* codes below.
 *
 * Environment variables (read by glu_analyze unless noted; none is needed):
 *   GLU_ANALYZE_THREADS  host threads of the analysis (1..64; default: the
 *                        machine's, at most 16); the results do not depend on it.
 *   GLU_SRC_MIN, GLU_LANE_MAX, GLU_LANE_SEGS (unless set in glu_options)
 *                        task-size thresholds of the factorization schedule:
 *                        the source count from which a target column is split
 *                        into 32-position chunk tasks (default 5), and the
 *                        largest task run by one lane, in updates (32) and
 *                        segments (2).  Every value gives a valid schedule.
 *   GLU_DUMP_COLUMNS, GLU_DUMP_BLOCKS, GLU_DUMP_DF, GLU_DUMP_DF_BATCHED,
 *   GLU_DUMP_SCHEDULE    file paths: diagnostic copies of the column-level
 *                        schedule (with the value gather map), the supernodal
 *                        schedule, the single and batched solve schedules,
 *                        and a per-level summary.
 *   GLU_LEVEL_TIMES      file path: glu_factor without graph capture writes
 *                        each level's device time (CUDA events).
 *   GLU_TEST_FAIL_LEVEL, GLU_TEST_FAIL_SOLVE
 *                        test hooks: make the analysis fail as an allocation
 *                        would (a level of the column schedule, or the solve
 *                        schedule), to test the GLU_ERR_OOM path.
 */
#ifndef GLU_H_
#define GLU_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GLU_OK 0
#define GLU_ERR_INVALID -1          /* malformed CSC, bad permutation, bad argument */
#define GLU_ERR_STRUCT_SINGULAR -2  /* a column of P A P^T lacks its diagonal */
#define GLU_ERR_ZERO_PIVOT -3       /* a pivot is exactly zero (column in glu_last_error_info) */
#define GLU_ERR_NONFINITE -4        /* a pivot is NaN or infinite */
#define GLU_ERR_OOM -5              /* host or device allocation failed */
#define GLU_ERR_CUDA -6             /* a CUDA runtime call failed */
#define GLU_ERR_TIMEOUT -7          /* a bounded device-side wait gave up */
#define GLU_ERR_NOT_FACTORED -8     /* solve before a successful factorization */
#define GLU_ERR_INTERNAL -9         /* an internal consistency check failed */
#define GLU_ERR_TOO_LARGE -10       /* a fixed limit is exceeded: glu_solve_noalloc's scratch, or
                                       2^31 segments / tasks in the factorization schedule */

/* Size, in doubles, of the fixed device scratch array behind
 * glu_solve_noalloc (32 MiB). */
#define GLU_NOALLOC_SCRATCH_DOUBLES 4194304

typedef struct glu_handle glu_handle;

/* Tuning knobs.  glu_default_options fills every field; a zero or negative
 * value in a field means "choose automatically" unless stated otherwise. */
typedef struct glu_options {
    int32_t struct_size;      /* sizeof(glu_options); set by glu_default_options */
    int32_t mode_force;       /* -1 per-level choice; 0 warp-per-column,
                                 1 block-per-column, 2 pipelined tail, for every level */
    int32_t tail_threshold;   /* levels with at most this many columns run in the
                                 pipelined mode: consecutive such levels share one
                                 dataflow launch in which each work item waits only for
                                 the items it reads (per-column counters, bounded waits)
                                 instead of a barrier per level (the paper's stream-mode
                                 threshold is 16, Section III-B.2 item 3); 0: off */
    int32_t piece_updates;    /* target-column updates per warp task (work split size;
                                 default 1024) */
    int32_t wide_threshold;   /* levels with more columns than this run warp-per-column */
    int32_t use_graph;        /* 1: capture the level sequence in a CUDA graph */
    int32_t verbose;          /* 1: print analysis statistics to stderr */
    int32_t host_only;        /* 1: run the host analysis only; no device memory is
                                 touched and the handle can only report the analysis
                                 (glu_get_fill / deps / levels / stats) */
    int32_t solve_mode;       /* 1 (default): dataflow solve, a forward and a backward
                                 launch (the dense tail between them), items waiting on
                                 per-row ready flags; 0: one launch per solve level */
    int32_t spin_limit_us;    /* bound on any device-side wait, microseconds
                                 (default 2,000,000); past it GLU_ERR_TIMEOUT */
    int32_t fault_row;        /* testing only: in the dataflow solve this row never
                                 publishes its result, and in the pipelined levels of
                                 the factorization the tasks that update this column
                                 never publish theirs, so waits on them time out
                                 (-1: off) */
    int32_t solve_tail;       /* 1 (default): a trailing fully dense block of 32..1024
                                 rows is solved by one block in shared memory; 0: off */
    int32_t factor_tail;      /* 1 (default): a trailing fully dense block of 64..3200
                                 columns that forms the last levels (one column each)
                                 is factored as a dense matrix by one cooperative
                                 launch instead of one launch per level; 0: off */
    int32_t solve_blocks;     /* 1 (default): in the dataflow solve, dense diagonal blocks of
                                 4..32 rows are solved by one warp each (their rows'
                                 entries outside the block as parallel partial sums); 0: off */
    int32_t factor_blocks;    /* 1: supernodal factorization -- runs of up to 32 columns with a
                                 dense diagonal block and equal structure below are factored
                                 as dense panels and update their targets once per run
                                 (levels of the contracted Algorithm 4 graph); 0 (default):
                                 one level per Algorithm 4 level */
    int32_t row_lookup;       /* how the level kernels find a row of L(:,j) in target column
                                 k: 1 a position map (2 or 4 bytes per update, built
                                 once per pattern; the fastest); 2 a run table (one
                                 8-byte record per run of rows that sit on consecutive
                                 positions of column k, about one per 20 updates on
                                 circuit matrices; a warp finds its rows' runs by ballots
                                 and shuffles); 0 (default): the map when it takes at most
                                 GLU_MAP_BUDGET_BYTES, else the run table */
    int32_t src_min;          /* task shapes of the level schedule (0: default, or the
                                 environment variable of the same name):
                                 a target column hit by at least this many sources of
                                 one level is cut into 32-position chunk tasks
                                 (KIND_SRC; GLU_SRC_MIN, default 5) */
    int32_t lane_max;         /* tasks of at most this many updates ... (GLU_LANE_MAX, 32) */
    int32_t lane_segs;        /* ... and this many segments run on one lane (KIND_LANE;
                                 GLU_LANE_SEGS, 2) */
    int32_t gpu_analysis;     /* 1 (default): glu_analyze runs Algorithm 4 (the
                                 dependency lists) and the longest-path levels on the
                                 current GPU (the same result as the host's); 0: on the
                                 host.  A host_only analysis always runs on the host */
} glu_options;

/* Device memory the position map may take before row_lookup 0 switches to
 * the run table (8 GiB). */
#define GLU_MAP_BUDGET_BYTES (8LL << 30)

/* Analysis statistics (glu_get_stats). */
typedef struct glu_stats {
    int32_t n;
    int32_t nlevels;
    int64_t nnz_a;
    int64_t nnz_lu;           /* filled pattern including the diagonal */
    int64_t nnz_l;            /* strict lower part */
    int64_t nnz_u;            /* upper part including the diagonal */
    int64_t n_deps;           /* Algorithm 4 dependency edges */
    int64_t n_pairs;          /* (source j, target k) column pairs of the updates */
    int64_t n_updates;        /* multiply-subtract updates per factorization */
    double flops;             /* sum_j l_j + 2 l_j u_j */
    int32_t levels_by_mode[3];/* levels run warp-per-column / block-per-column / pipelined */
    int32_t solve_levels_fwd;
    int32_t solve_levels_bwd;
    int32_t max_level_width;
    int64_t device_bytes;     /* device memory held by the handle */
    double analyze_ms;        /* host wall time of glu_analyze */
    int64_t kernel_launches;  /* CUDA kernels this handle has launched so far */
    int32_t tail_rows;        /* rows of the dense tail solved by one block (0: none) */
    int32_t factor_tail_cols; /* columns of the dense block factored densely (0: none) */
    int32_t row_lookup;       /* the level kernels' row lookup: 1 position map, 2 run
                                 table, 0 none built yet (see glu_options.row_lookup) */
    int32_t spare;
    int64_t lookup_bytes;     /* device bytes of that map or table */
    int64_t n_runs;           /* runs in the run table (0 with the map) */
} glu_stats;

/* Outcome of glu_solve_refine. */
typedef struct glu_refine_info {
    int32_t iterations;       /* corrections applied (FP32 solves after the first) */
    int32_t converged;        /* 1 if every right-hand side reached tol */
    double berr;              /* final normwise backward error, max over the sides:
                                 ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) */
    double berr_first;        /* the same after the first FP32 solve */
} glu_refine_info;

/* Fill every field of *opts with its default. */
void glu_default_options(glu_options *opts);

/* Symbolic analysis on the host (Section III-A and the flow of Fig. 5):
 * validates the CSC input, forms B = P A P^T, computes the fill-in of L+U
 * (Section II-A), the relaxed column dependencies (Algorithm 4), the levels
 * (Section II-C: columns grouped into levels of mutually independent
 * columns; level(k) = 0 without dependencies, else 1 + the largest level
 * among its dependencies) and the per-level update schedule, then uploads the
 * schedule to the current CUDA device.  On success *out holds a new handle.
 * Errors: GLU_ERR_INVALID (malformed input), GLU_ERR_STRUCT_SINGULAR,
 * GLU_ERR_OOM (host or device memory, including allocations on the
 * analysis's worker threads), GLU_ERR_TOO_LARGE (the schedule's 32-bit record
 * indices would overflow), GLU_ERR_CUDA. */
int glu_analyze(int32_t n, const int32_t *colptr, const int32_t *rowidx,
                const int32_t *perm, glu_handle **out);

/* glu_analyze with explicit options (NULL = defaults). */
int glu_analyze_opts(int32_t n, const int32_t *colptr, const int32_t *rowidx,
                     const int32_t *perm, const glu_options *opts, glu_handle **out);

/* Stream for all later work of the handle (a cudaStream_t; NULL = legacy
 * default stream). */
int glu_set_stream(glu_handle *h, void *cuda_stream);

/* Numeric refactorization in FP64 (Algorithm 2 scheduled by levels,
 * Algorithm 5 / Eq. 3 for the subcolumn updates).  values[nnz_a] are A's
 * values in the input CSC order (host or device).  Errors surface as
 * described above: GLU_ERR_ZERO_PIVOT / GLU_ERR_NONFINITE with the smallest
 * failing column in glu_last_error_info. */
int glu_factor(glu_handle *h, const double *values);

/* Wait for the handle's stream and return the first pending device error. */
int glu_sync(glu_handle *h);

/* Solve A x = b with the last FP64 factorization: c = P b, L y = c (unit L,
 * forward), U z = y (backward), x = P^T z (Section I).  b and x hold nrhs
 * vectors of length n each; b and x must not overlap.
 * Errors: GLU_ERR_NOT_FACTORED, GLU_ERR_INVALID, pending factor errors. */
int glu_solve(glu_handle *h, const double *b, double *x, int32_t nrhs);

/* FP32 numeric refactorization: the same level-scheduled right-looking
 * update as glu_factor, on FP32 values with FP32 accumulation (the paper's
 * own precision, Section IV).  The FP64 values are kept for the residuals of
 * glu_solve_refine.  values: nnz_a doubles, host or device, A's CSC order.
 * Errors as glu_factor. */
int glu_factor_f32(glu_handle *h, const double *values);

/* Mixed-precision solve: FP32 triangular solves with the glu_factor_f32
 * factors, FP64 iterative refinement on the GPU (r = b - A x with the FP64
 * values, x += d in FP64), until the normwise backward error of every side is
 * <= tol or maxit corrections were applied.  The iterate starts at x = 0, so
 * the first FP32 solve is of b itself; each later solve is of the residual.
 * b, x: nrhs vectors of length n, host or device.  info may be NULL.  Not
 * converging is not an error: check info->converged.  Errors:
 * GLU_ERR_NOT_FACTORED (no FP32 factorization), GLU_ERR_INVALID, pending
 * device errors. */
int glu_solve_refine(glu_handle *h, const double *b, double *x, int32_t nrhs, double tol, int32_t maxit,
                     glu_refine_info *info);

/* Batched refactorization: `batch` value sets of the same pattern (Newton
 * iterations, transient steps, Monte-Carlo corners), value p of set b at
 * values[b * ld + p], ld >= nnz_a, host or device.  The level schedule of the
 * single factorization runs once for all sets, with the sets interleaved in
 * memory (lanes of a warp over the sets); the whole sequence is one
 * captured CUDA graph launch.  FP64 arithmetic.  The handle keeps one batch:
 * a later call replaces it.  A zero or non-finite pivot in any set raises
 * GLU_ERR_ZERO_PIVOT / GLU_ERR_NONFINITE with the smallest such column. */
int glu_factor_batched(glu_handle *h, const double *values, int32_t batch, int64_t ld);

/* As glu_factor_batched with FP32 values and FP32 accumulation; the FP64
 * values are kept for glu_solve_batched_refine. */
int glu_factor_batched_f32(glu_handle *h, const double *values, int32_t batch, int64_t ld);

/* Solves with the last glu_factor_batched factors: right-hand side r of set
 * b at b[(b * nrhs + r) * n ...], x likewise; host or device.  `batch` must
 * equal the factorized batch. */
int glu_solve_batched(glu_handle *h, const double *b, double *x, int32_t nrhs, int32_t batch);

/* FP32 solves with the glu_factor_batched_f32 factors and FP64 iterative
 * refinement per set and side, until every side of every set reaches tol or
 * maxit corrections; info summarizes over all sets (berr = the largest). */
int glu_solve_batched_refine(glu_handle *h, const double *b, double *x, int32_t nrhs, int32_t batch, double tol,
                             int32_t maxit, glu_refine_info *info);

/* Copy the FP64 factors of one set of the last glu_factor_batched to host
 * memory (pattern order, nnz_lu doubles); synchronizes. */
int glu_get_factors_batched(glu_handle *h, int32_t set, double *lu_val_host);

/* The same for the FP32 factors of one set of the last
 * glu_factor_batched_f32 (nnz_lu floats); synchronizes. */
int glu_get_factors_batched_f32(glu_handle *h, int32_t set, float *lu_val_host);

/* Pattern of the fill (Section II-A): lu_colptr[n+1], lu_rowidx[nnz]
 * (rows ascending per column), host memory owned by the handle. */
int glu_get_fill(const glu_handle *h, const int64_t **lu_colptr,
                 const int32_t **lu_rowidx, int64_t *nnz);

/* Algorithm 4's dependency lists: for column k, dep_idx[dep_ptr[k] ..
 * dep_ptr[k+1]) ascending, each entry a column i < k.  Host memory owned by
 * the handle. */
int glu_get_deps(const glu_handle *h, const int64_t **dep_ptr, const int32_t **dep_idx);

/* Levels: level_cols[level_ptr[l] .. level_ptr[l+1]) are the columns of
 * level l in ascending order; level_ptr has nlevels + 1 entries.  Host
 * memory owned by the handle. */
int glu_get_levels(const glu_handle *h, int32_t *nlevels, const int32_t **level_ptr,
                   const int32_t **level_cols);

/* Copy the FP64 factor values (pattern order, nnz_lu doubles) to host memory;
 * synchronizes and returns any pending device error. */
int glu_get_factors(glu_handle *h, double *lu_val_host);

/* Copy the FP32 factor values of the last glu_factor_f32 (pattern order,
 * nnz_lu floats) to host memory; synchronizes and returns any pending device
 * error (GLU_ERR_NOT_FACTORED before a successful glu_factor_f32). */
int glu_get_factors_f32(glu_handle *h, float *lu_val_host);

/* Analysis statistics. */
int glu_get_stats(const glu_handle *h, glu_stats *s);

/* Column of the last zero or non-finite pivot error (-1 if none). */
int glu_last_error_info(const glu_handle *h, int32_t *column);

/* glu_solve without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory
 * once they are running, for example a simulator's time-stepping loop whose
 * memory is all reserved up front under a fixed budget (where a cudaMalloc
 * could fail, or stall the device while it runs), or code that hands the
 * library memory owned by someone else's allocator.
 *
 * The same launches as glu_solve on the handle's solve schedule (the
 * dataflow solve by default, the per-level solve with solve_mode 0), so the
 * result equals glu_solve's bit for bit; only the scratch differs: a fixed,
 * file-scope device array of GLU_NOALLOC_SCRATCH_DOUBLES doubles, which
 * every GPU where the library's device code gets loaded holds until the
 * process exits.  The dataflow solve's ready flags and error word are the
 * handle's own, allocated by glu_analyze.  b and x must be device pointers
 * (no staging); the call is stream-ordered on the handle's stream and
 * returns once enqueued.
 *
 * Needs 2 * n * nrhs + (long-row chunks) * nrhs doubles for the dataflow
 * solve (n * nrhs + chunks * nrhs for the per-level one), each part rounded
 * up to 32 values; a larger problem is rejected with GLU_ERR_TOO_LARGE
 * before anything is launched.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture.  All calls share the one
 * array and it keeps the last call's contents (the solve writes every
 * scratch value before reading it, so nothing has to start at zero); calls
 * whose work overlaps on the GPU, from any handle or stream, race on the
 * array and must be serialized by the caller.
 * Errors: GLU_ERR_INVALID (host pointers, nrhs < 0), GLU_ERR_NOT_FACTORED,
 * GLU_ERR_TOO_LARGE, GLU_ERR_CUDA. */
int glu_solve_noalloc(glu_handle *h, const double *b, double *x, int32_t nrhs);

/* A fill-reducing symmetric ordering of the pattern of A + A^T, for callers
 * without one (the paper's flow takes a fill-reducing order before the
 * symbolic analysis, Section II-C and Fig. 5; it names MC64 + AMD, which are
 * not reproduced): graph nested dissection -- level structures from a
 * pseudo-peripheral vertex, the smallest level near the middle as separator,
 * ordered last, sides ordered recursively, leaves of at most 32 vertices by
 * minimum degree.  Host only.  colptr[n+1], rowidx[nnz]: A's CSC pattern
 * (0-based; rows need not be sorted; the diagonal may be absent); perm[n]
 * receives new -> old, to pass to glu_analyze.  Deterministic.  Errors:
 * GLU_ERR_INVALID (bad arguments or indices). */
int glu_order_nd(int32_t n, const int32_t *colptr, const int32_t *rowidx, int32_t *perm);

/* Static pivoting with scaling for callers without one (the step before the
 * fill-reducing order in the flow of Section II-C and Fig. 5, which names
 * MC64; this is not MC64's code): a row permutation that maximizes the
 * product of the diagonal magnitudes -- a minimum-cost perfect matching of
 * columns to rows, cost log(max_k |a_kj|) - log|a_ij|, by shortest
 * augmenting paths -- and scalings from its dual variables.  Host only.
 * colptr[n+1], rowidx[nnz], values[nnz]: A in CSC (0-based; rows need not
 * be sorted; explicit zeros are not used).  Outputs: row_perm[n] with
 * row_perm[j] = the row of A matched to column j (B(j,:) = A(row_perm[j],:)
 * puts the matching on B's diagonal); row_scale[n] (by A's row) and
 * col_scale[n] such that |row_scale[i] a_ij col_scale[j]| <= 1 for every
 * entry and = 1 on the matching, both up to rounding (within a few units in
 * the last place: the scalings are exponentials of dual variables).  Deterministic.  Errors: GLU_ERR_INVALID
 * (bad arguments, indices or non-finite values), GLU_ERR_STRUCT_SINGULAR (no
 * perfect matching exists), GLU_ERR_OOM. */
int glu_static_pivot(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *values,
                     int32_t *row_perm, double *row_scale, double *col_scale);

/* Apply glu_static_pivot's result: B = P_r D_r A D_c in CSC, with
 * B(k, j) = row_scale[r] * A(r, j) * col_scale[j] for r = row_perm[k], so the
 * matching sits on B's diagonal (the first step of the flow of Section II-C,
 * Fig. 5).  Host only.  B has A's column pointers: out_rowidx[nnz] and
 * out_values[nnz] (caller-allocated, nnz = colptr[n]) receive its rows,
 * ascending in every column, and values.  row_scale / col_scale may be NULL
 * (no scaling).  A x = b is then B y = P_r D_r b with x = D_c y.  Errors:
 * GLU_ERR_INVALID (bad arguments, row_perm not a permutation, an index out of
 * range, a row twice in one column), GLU_ERR_OOM. */
int glu_apply_static_pivot(int32_t n, const int32_t *colptr, const int32_t *rowidx, const double *values,
                           const int32_t *row_perm, const double *row_scale, const double *col_scale,
                           int32_t *out_rowidx, double *out_values);

/* Free the handle and everything it owns.  NULL is ignored. */
void glu_destroy(glu_handle *h);

/* Static description of a return code. */
const char *glu_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* GLU_H_ */
