// kernels_factor.cu -- numeric refactorization kernels (sm_103a).
//
// One launch per level runs that level's work list:
//   * normalization items of the previous level: L(i,j) = A_s(i,j) / A_s(j,j)
//     (Algorithm 2, the first inner loop), deferred by one level so that a
//     level needs a single launch: column j is read raw while it is a source
//     and divided afterwards;
//   * update tasks: the submatrix update of Algorithm 5 / Eq. 3 for every
//     (source j, target k) pair of the level, as
//     A_s(i,k) -= A_s(i,j) * (A_s(j,k) / A_s(j,j))   for i in L(:,j).
// Every target entry is updated by exactly one warp (or lane) per level,
// whose additions are L2 reductions issued in a fixed order (separated by
// warp barriers); the order of the updates of an entry depends only on the
// pattern, so a refactorization is deterministic run to run.
// A row of L(:,j) is found in target column k (the template parameter M) by
// a position map (M = uint16_t / uint32_t: one offset per update, built once
// per pattern; one load per update) or by the pair's run table (M = Run):
// rows of L(:,j) that sit on consecutive positions of column k form one run,
// about nine per pair on the power-grid workloads, so the table is small next
// to one position per update; a warp locates its 32 rows' runs with two
// ballots, an OR-reduction and two shuffles, a single lane by walking them.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "glu_device.cuh"

namespace glu {

namespace {

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }

__device__ __forceinline__ void raise_err(unsigned long long *err, int32_t col, unsigned code) {
    atomicMin(err, ((unsigned long long)(uint32_t)col << 8) | code);
}

// A factor value.  CG: from L2 (ld.global.cg), for the dataflow kernel, where
// other SMs write the values during the same launch and a line this SM's L1
// holds may be stale; otherwise an ordinary load (the level launches see
// every earlier write at the kernel boundary).
template <bool CG, typename T>
__device__ __forceinline__ T ldv(const T *p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// ----------------------------------------------------------------- gather
template <typename T>
__global__ void k_gather(T *__restrict__ lu, const double *__restrict__ aval,
                         const int32_t *__restrict__ gsrc, int64_t nnz) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < nnz; i += stride) {
        int32_t s = gsrc[i];
        lu[i] = s >= 0 ? (T)aval[s] : (T)0;
    }
}

// ------------------------------------------------------------- level work
// L(:,j) /= A_s(j,j) as products with one reciprocal per item: the FP64
// pipe of this part is narrow (a division is a dozen dependent operations
// on it), and x * (1/d) is within one rounding of x / d.
template <typename T, bool CG = false>
__device__ __forceinline__ void norm_item(const FactorArgs<T> &a, const NormItem it, int lane) {
    const int64_t dj = a.diag_pos[it.col];
    const T rd = (T)1 / ldv<CG>(a.lu + dj);
    T *L = a.lu + dj + 1;
    // all loads of the item first (at most 8 per lane), then the products
    constexpr int NU = 8;
    for (int32_t tb = it.t0; tb < it.t1; tb += 32 * NU) {
        T v[NU];
#pragma unroll
        for (int u = 0; u < NU; u++)
            if (tb + 32 * u < it.t1 && tb + 32 * u + lane < it.t1) v[u] = ldv<CG>(L + tb + 32 * u + lane);
#pragma unroll
        for (int u = 0; u < NU; u++)
            if (tb + 32 * u < it.t1) {              // the same for the whole warp
                if (tb + 32 * u + lane < it.t1) L[tb + 32 * u + lane] = v[u] * rd;
            }
    }
}

// Everything a segment needs, gathered once: the position of U(j,k), its
// runs, the first row of L(:,j) and the multiplier
// f = A_s(j,k) / A_s(j,j).  All of them are final when the level starts:
// U(j,k) and the pivot of a source are only written by earlier levels.
template <typename T>
struct SegMeta {
    int64_t pos;
    int64_t rb;       // first run of the segment, or its first map entry
    int64_t lstart;
    int32_t nr;       // runs of the segment (run table)
    int32_t t0;
    int32_t t1;
    T f;
};

template <typename M>
constexpr bool is_runs() { return std::is_same<M, Run>::value; }

template <typename T, typename M, bool CG = false>
__device__ __forceinline__ void load_meta(const FactorArgs<T> &a, int32_t s, SegMeta<T> &m) {
    const int4 *r = reinterpret_cast<const int4 *>(a.segs + s);
    const int4 v0 = r[0], v1 = r[1];
    m.pos = ((int64_t)(uint32_t)v0.y << 32) | (uint32_t)v0.x;
    const int64_t dj = ((int64_t)(uint32_t)v0.w << 32) | (uint32_t)v0.z;
    const uint64_t enc = ((uint64_t)(uint32_t)v1.y << 32) | (uint32_t)v1.x;
    if constexpr (is_runs<M>()) {
        m.rb = (int64_t)(enc & ((1ull << RUN_BASE_BITS) - 1));
        m.nr = (int32_t)(enc >> RUN_BASE_BITS);
    } else {
        m.rb = (int64_t)enc;
        m.nr = 0;
    }
    m.t0 = v1.z;
    m.t1 = v1.w;
    m.lstart = dj + 1;
    m.f = ldv<CG>(a.lu + m.pos) / ldv<CG>(a.lu + dj);
}

template <typename T>
__device__ __forceinline__ SegMeta<T> shfl_meta(const SegMeta<T> &m, int src) {
    SegMeta<T> o;
    o.pos = __shfl_sync(0xffffffffu, m.pos, src);
    o.rb = __shfl_sync(0xffffffffu, m.rb, src);
    o.lstart = __shfl_sync(0xffffffffu, m.lstart, src);
    o.nr = __shfl_sync(0xffffffffu, m.nr, src);
    o.t0 = __shfl_sync(0xffffffffu, m.t0, src);
    o.t1 = __shfl_sync(0xffffffffu, m.t1, src);
    o.f = __shfl_sync(0xffffffffu, m.f, src);
    return o;
}

__device__ __forceinline__ Run load_run(const Run *runs, int64_t r, int64_t rend) {
    if (r < rend) {
        const int2 v = *reinterpret_cast<const int2 *>(runs + r);
        return Run{v.x, v.y};
    }
    return Run{INT32_MAX, 0};
}

// One lane walking the rows of a segment in ascending order: the run holding
// the current row and the next three runs, loaded ahead so that crossing
// into a run rarely waits for its record.
struct RunWalk {
    int64_t r, rend;    // r: the index of n3
    Run cur, n1, n2, n3;
};

__device__ __forceinline__ void walk_begin(RunWalk &w, const Run *runs, int64_t rb, int32_t nr) {
    w.rend = rb + nr;
    w.cur = load_run(runs, rb, w.rend);
    w.n1 = load_run(runs, rb + 1, w.rend);
    w.n2 = load_run(runs, rb + 2, w.rend);
    w.n3 = load_run(runs, rb + 3, w.rend);
    w.r = rb + 3;
}

// offset in the target column (past U(j,k)) of row t >= every earlier t
__device__ __forceinline__ uint32_t walk_offset(RunWalk &w, const Run *runs, int32_t t) {
    while (t >= w.n1.ts) {
        w.cur = w.n1;
        w.n1 = w.n2;
        w.n2 = w.n3;
        w.n3 = load_run(runs, ++w.r, w.rend);
    }
    return (uint32_t)(w.cur.off + (t - w.cur.ts));
}

#ifndef GLU_ROW_UNROLL
#define GLU_ROW_UNROLL 8            // rows per lane batch, lanes over rows
#endif
#ifndef GLU_LANE_UNROLL
#define GLU_LANE_UNROLL 16          // rows per batch when one lane walks a segment
#endif
#ifndef GLU_SRC_UNROLL
#define GLU_SRC_UNROLL 8            // the same inside KIND_SRC tasks
#endif
constexpr int ROW_UNROLL = GLU_ROW_UNROLL;
constexpr int LANE_UNROLL = GLU_LANE_UNROLL;

// Rows t0..t1-1 of one segment, lanes over rows.  Within a segment every row
// hits a different target entry, so all loads of a batch go out at once; the
// target entries then take -L(i,j) f as reductions performed in L2
// (red.global.add: no load of the target on the warp's path).  A level's
// target entries have one owner warp, whose segments are separated by warp
// barriers, so each entry's sequence of additions is fixed: the results are
// the same from run to run.
// The rows' positions come from the segment's runs, held 32 at a time by the
// lanes (lane w: run wb + w).  For a group of 32 consecutive rows g0..g0+31:
// the run holding g0 is the last one starting at or before g0 (one ballot);
// the runs starting inside the group set one bit each at their first row (an
// OR-reduction); a lane's run is the first one's index plus the bits at or
// below its row.  The window moves on when a group could reach past it.
template <typename T, bool CG = false>
__device__ __forceinline__ void row_segment_runs(T *__restrict__ lu, const Run *__restrict__ runs,
                                                 const SegMeta<T> &m, int lane) {
    const T *__restrict__ L = lu + m.lstart;
    T *tgt = lu + m.pos + 1;
    const int64_t rend = m.rb + m.nr;
    int64_t wb = m.rb;
    Run w = load_run(runs, wb + lane, rend);
    for (int32_t tb = m.t0; tb < m.t1; tb += 32 * ROW_UNROLL) {
        uint32_t off[ROW_UNROLL];
        T lv[ROW_UNROLL];
#pragma unroll
        for (int u = 0; u < ROW_UNROLL; u++) {
            const int32_t t = tb + 32 * u + lane;
            if (t < m.t1) lv[u] = ldv<CG>(L + t);
        }
        if (wb + 32 >= rend) {
            // the window holds every remaining run: the groups are independent
#pragma unroll
            for (int u = 0; u < ROW_UNROLL; u++) {
                const int32_t g0 = tb + 32 * u;
                if (g0 < m.t1) {
                    const int32_t glast = min(g0 + 31, m.t1 - 1);
                    const int a = __popc(__ballot_sync(0xffffffffu, w.ts <= g0)) - 1;
                    const unsigned bit = (w.ts > g0 && w.ts <= glast) ? (1u << (w.ts - g0)) : 0u;
                    const unsigned starts = __reduce_or_sync(0xffffffffu, bit);
                    const int idx = a + __popc(starts & (0xffffffffu >> (31 - lane)));
                    const int32_t ts = __shfl_sync(0xffffffffu, w.ts, idx);
                    const int32_t of = __shfl_sync(0xffffffffu, w.off, idx);
                    off[u] = (uint32_t)(of + (g0 + lane - ts));
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < ROW_UNROLL; u++) {
                const int32_t g0 = tb + 32 * u;
                if (g0 < m.t1) {                   // the same for the whole warp
                    const int32_t glast = min(g0 + 31, m.t1 - 1);
                    if (wb + 32 < rend && __shfl_sync(0xffffffffu, w.ts, 31) <= glast) {
                        // the group may reach the run after the window: start the
                        // window at the run holding g0 (32 rows span <= 32 runs)
                        wb += __popc(__ballot_sync(0xffffffffu, w.ts <= g0)) - 1;
                        w = load_run(runs, wb + lane, rend);
                    }
                    const int a = __popc(__ballot_sync(0xffffffffu, w.ts <= g0)) - 1;
                    const unsigned bit = (w.ts > g0 && w.ts <= glast) ? (1u << (w.ts - g0)) : 0u;
                    const unsigned starts = __reduce_or_sync(0xffffffffu, bit);
                    const int idx = a + __popc(starts & (0xffffffffu >> (31 - lane)));
                    const int32_t ts = __shfl_sync(0xffffffffu, w.ts, idx);
                    const int32_t of = __shfl_sync(0xffffffffu, w.off, idx);
                    off[u] = (uint32_t)(of + (g0 + lane - ts));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < ROW_UNROLL; u++) {
            const int32_t t = tb + 32 * u + lane;
            if (t < m.t1) atomicAdd(&tgt[off[u]], -lv[u] * m.f);
        }
    }
}

// The same with the position map: the rows' offsets are loaded with L(:,j).
template <typename T, typename M, bool CG = false>
__device__ __forceinline__ void row_segment_map(T *__restrict__ lu, const M *__restrict__ map, const SegMeta<T> &m,
                                                int lane) {
    const M *__restrict__ mp = map + m.rb;
    const T *__restrict__ L = lu + m.lstart;
    T *tgt = lu + m.pos + 1;
    for (int32_t tb = m.t0; tb < m.t1; tb += 32 * ROW_UNROLL) {
        uint32_t off[ROW_UNROLL];
        T lv[ROW_UNROLL];
#pragma unroll
        for (int u = 0; u < ROW_UNROLL; u++) {
            const int32_t t = tb + 32 * u + lane;
            if (t < m.t1) {
                off[u] = mp[t];
                lv[u] = ldv<CG>(L + t);
            }
        }
        // a group of 32 rows past the end is skipped by the whole warp
#pragma unroll
        for (int u = 0; u < ROW_UNROLL; u++)
            if (tb + 32 * u < m.t1) {
                if (tb + 32 * u + lane < m.t1) atomicAdd(&tgt[off[u]], -lv[u] * m.f);
            }
    }
}

template <typename T, typename M, bool CG = false>
__device__ __forceinline__ void row_segment(const FactorArgs<T> &a, const SegMeta<T> &m, int lane) {
    if constexpr (is_runs<M>()) row_segment_runs<T, CG>(a.lu, a.runs, m, lane);
    else row_segment_map<T, M, CG>(a.lu, static_cast<const M *>(a.map), m, lane);
}

// Offsets of the rows of one segment for a single lane, in ascending order:
// map loads, or a walk over the runs.
template <typename M>
struct LaneRows {
    const M *mp;
    __device__ __forceinline__ void begin(const void *map, const Run *, int64_t rb, int32_t) {
        mp = static_cast<const M *>(map) + rb;
    }
    __device__ __forceinline__ uint32_t offset(const Run *, int32_t t) { return mp[t]; }
};
template <>
struct LaneRows<Run> {
    RunWalk w;
    __device__ __forceinline__ void begin(const void *, const Run *runs, int64_t rb, int32_t nr) {
        walk_begin(w, runs, rb, nr);
    }
    __device__ __forceinline__ uint32_t offset(const Run *runs, int32_t t) { return walk_offset(w, runs, t); }
};

// KIND_ROW tasks of one warp, tq0, tq0 + stride, ... (cnt of them), applied one
// after the other as row_task would, but with the metadata of up to 32
// segments -- spanning several tasks -- fetched at once, one per lane, so the
// multiplier divisions of a warp's many short tasks share instructions.
template <typename T, typename M, bool CG = false>
__device__ __forceinline__ void row_tasks(const FactorArgs<T> &a, int64_t tq0, int64_t stride, int64_t cnt,
                                          int lane) {
    int64_t i = 0;      // next task of the list
    int32_t skip = 0;   // segments of task i already applied
    while (i < cnt) {
        const bool valid = i + lane < cnt;
        int32_t sb = 0, ns = 0;
        if (valid) {
            const Task tk = a.tasks[tq0 + (i + lane) * stride];
            sb = tk.seg_begin;
            ns = tk.seg_end - tk.seg_begin;
            if (lane == 0) {
                sb += skip;
                ns -= skip;
            }
        }
        int32_t incl = ns;   // inclusive prefix sum of the segment counts
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        const int32_t take = min(tot, 32);
        // slot `lane` belongs to the first task whose prefix sum exceeds it
        int t = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1)
            if (__shfl_sync(0xffffffffu, incl, t + step - 1) <= lane) t += step;
        t = min(t, 31);
        const int32_t t_incl = __shfl_sync(0xffffffffu, incl, t);
        const int32_t t_ns = __shfl_sync(0xffffffffu, ns, t);
        const int32_t t_sb = __shfl_sync(0xffffffffu, sb, t);
        SegMeta<T> mine;
        if (lane < take) load_meta<T, M, CG>(a, t_sb + (lane - (t_incl - t_ns)), mine);
        for (int q = 0; q < take; q++) {
            const SegMeta<T> m = shfl_meta<T>(mine, q);
            row_segment<T, M, CG>(a, m, lane);
            __syncwarp();
        }
        if (tot <= 32) {
            i += (cnt - i < 32) ? cnt - i : 32;
            skip = 0;
        } else {
            // tasks wholly applied, then the one cut at slot 32
            const int tp = __popc(__ballot_sync(0xffffffffu, valid && incl <= 32));
            const int32_t p_incl = __shfl_sync(0xffffffffu, incl, tp);
            const int32_t p_ns = __shfl_sync(0xffffffffu, ns, tp);
            skip = (tp == 0 ? skip : 0) + (32 - (p_incl - p_ns));
            i += tp;
        }
    }
}

// KIND_SRC: lanes over segments; lane l accumulates its products into row l
// of a 32 x 33 shared-memory tile (slot = target position - base); then lane
// s sums column s over the lanes that had segments, in order, and applies
// it.  The next segment's metadata is fetched before the current one's rows.
template <typename T, typename M, bool CG = false>
__device__ __forceinline__ void src_task(const FactorArgs<T> &a, const Task &tk, int lane, T *__restrict__ acc) {
    T *__restrict__ row = acc + lane * (SRC_SLOTS + 1);
    const int nl = min(32, tk.seg_end - tk.seg_begin);   // lanes with segments
    if (lane < nl) {
#pragma unroll
        for (int s = 0; s < SRC_SLOTS; s++) row[s] = (T)0;
    }
    int32_t s = tk.seg_begin + lane;
    SegMeta<T> cur;
    bool have = s < tk.seg_end;
    if (have) load_meta<T, M, CG>(a, s, cur);
    while (have) {
        SegMeta<T> nxt;
        const int32_t s2 = s + 32;
        const bool have2 = s2 < tk.seg_end;
        if (have2) load_meta<T, M, CG>(a, s2, nxt);
        const T *__restrict__ L = a.lu + cur.lstart;
        const int32_t rel = (int32_t)(cur.pos + 1 - tk.base);
        LaneRows<M> wk;
        wk.begin(a.map, a.runs, cur.rb, cur.nr);
        for (int32_t tb = cur.t0; tb < cur.t1; tb += GLU_SRC_UNROLL) {
            uint32_t off[GLU_SRC_UNROLL];
            T lv[GLU_SRC_UNROLL];
#pragma unroll
            for (int u = 0; u < GLU_SRC_UNROLL; u++)
                if (tb + u < cur.t1) lv[u] = ldv<CG>(L + tb + u);
#pragma unroll
            for (int u = 0; u < GLU_SRC_UNROLL; u++)
                if (tb + u < cur.t1) off[u] = wk.offset(a.runs, tb + u);
#pragma unroll
            for (int u = 0; u < GLU_SRC_UNROLL; u++)
                if (tb + u < cur.t1) {
                    const int32_t slot = rel + (int32_t)off[u];
                    row[slot] = fma_t<T>(lv[u], cur.f, row[slot]);
                }
        }
        cur = nxt;
        s = s2;
        have = have2;
    }
    __syncwarp();
    if (lane < tk.nslots) {
        T sum = (T)0;
        for (int l = 0; l < nl; l++) sum += acc[l * (SRC_SLOTS + 1) + lane];
        a.lu[tk.base + lane] = ldv<CG>(a.lu + tk.base + lane) - sum;
    }
    __syncwarp();
}

// KIND_LANE: one lane applies the task's segments in order, rows batched;
// the next segment's metadata is fetched before the current one's rows.
template <typename T, typename M, bool CG = false>
__device__ __forceinline__ void lane_task(const FactorArgs<T> &a, const Task &tk) {
    SegMeta<T> nxt;
    load_meta<T, M, CG>(a, tk.seg_begin, nxt);
    for (int32_t s = tk.seg_begin; s < tk.seg_end; s++) {
        const SegMeta<T> m = nxt;
        if (s + 1 < tk.seg_end) load_meta<T, M, CG>(a, s + 1, nxt);
        const T *__restrict__ L = a.lu + m.lstart;
        T *tgt = a.lu + m.pos + 1;
        LaneRows<M> wk;
        wk.begin(a.map, a.runs, m.rb, m.nr);
        for (int32_t tb = m.t0; tb < m.t1; tb += LANE_UNROLL) {
            uint32_t off[LANE_UNROLL];
            T lv[LANE_UNROLL];
#pragma unroll
            for (int u = 0; u < LANE_UNROLL; u++)
                if (tb + u < m.t1) lv[u] = ldv<CG>(L + tb + u);
#pragma unroll
            for (int u = 0; u < LANE_UNROLL; u++)
                if (tb + u < m.t1) off[u] = wk.offset(a.runs, tb + u);
#pragma unroll
            for (int u = 0; u < LANE_UNROLL; u++)
                if (tb + u < m.t1) atomicAdd(&tgt[off[u]], -lv[u] * m.f);
        }
    }
}

// One warp per block: a block retires, and its slot goes to the next level's
// blocks, as soon as its own warp is done, and the block scheduler places
// each warp on its own (200k workload 21.4 -> 20.6 ms FP64, 14.5 -> 13.8 ms
// FP32 against blocks of 4 warps; 2 warps 21.1 ms, 8 warps 22.4 ms; the same
// factors bit for bit).
constexpr int LEVEL_WARPS = 1;
#ifndef GLU_LEVEL_BLOCKS_PER_SM
#define GLU_LEVEL_BLOCKS_PER_SM 16  // resident k_level blocks per SM the launch aims for
#endif
#ifndef GLU_LEVEL_BLOCKS_PER_SM_F32
#define GLU_LEVEL_BLOCKS_PER_SM_F32 24
#endif
#ifndef GLU_LEVEL_CAP_BIG_F32
#define GLU_LEVEL_CAP_BIG_F32 24
#endif
#ifndef GLU_LEVEL_BIG_ITEMS
#define GLU_LEVEL_BIG_ITEMS 8192
#endif
// By precision: the resident blocks per SM k_level is compiled for (its
// register budget), the grid cap in blocks per SM, and the cap for a level of
// at least GLU_LEVEL_BIG_ITEMS work items.  FP32 needs fewer registers: it is
// compiled for 24 warps per SM, and a wide level's grid of 24 per SM lets the
// block scheduler balance its uneven items (200k workload 16.1 -> 14.5 ms with
// blocks of 4 warps); narrower levels keep 16 per SM (a level of 2-8 k items
// lost with 24).  FP64 stays at 16 warps: 20 gained 1-2.5 % at 200k and lost
// 1-9 % on the 20k and 50k patterns.
template <typename T>
struct LevelOcc {
    static constexpr int blocks = GLU_LEVEL_BLOCKS_PER_SM;
    static constexpr int cap = GLU_LEVEL_BLOCKS_PER_SM;
    static constexpr int cap_big = GLU_LEVEL_BLOCKS_PER_SM;
};
template <>
struct LevelOcc<float> {
    static constexpr int blocks = GLU_LEVEL_BLOCKS_PER_SM_F32;
    static constexpr int cap = GLU_LEVEL_BLOCKS_PER_SM;
    static constexpr int cap_big = GLU_LEVEL_CAP_BIG_F32;
};

// One level.  Work items, in order: normalization items, KIND_SRC tasks and
// KIND_ROW tasks (one warp each), then KIND_LANE tasks, 32 per warp.
// The work items of one level: normalization items, KIND_SRC and KIND_ROW
// tasks (one warp each), KIND_LANE tasks (32 per warp); warps stride over them.
template <typename T, typename M>
__device__ __forceinline__ void run_level(const FactorArgs<T> &a, const LevelRange &r, int lane, int64_t warp,
                                          int64_t nw, T *acc) {
    const int64_t nn = r.n_end - r.n_begin;
    const int64_t nsrc = r.row_begin - r.t_begin;
    const int64_t nrow = r.lane_begin - r.row_begin;
    const int64_t nlane = r.t_end - r.lane_begin;
    const int64_t total = nn + nsrc + nrow + (nlane + 31) / 32;
    int64_t it = warp;
    for (; it < nn + nsrc; it += nw) {
        if (it < nn) norm_item<T>(a, a.norms[r.n_begin + it], lane);
        else src_task<T, M>(a, a.tasks[r.t_begin + (it - nn)], lane, acc);
    }
    if (it < nn + nsrc + nrow) {
        // this warp's KIND_ROW tasks: every nw-th from k0
        const int64_t k0 = it - nn - nsrc;
        const int64_t cnt = (nrow - k0 + nw - 1) / nw;
        row_tasks<T, M>(a, r.row_begin + k0, nw, cnt, lane);
        it += cnt * nw;
    }
    for (; it < total; it += nw) {
        const int64_t q = r.lane_begin + (it - nn - nsrc - nrow) * 32 + lane;
        if (q < r.t_end) lane_task<T, M>(a, a.tasks[q]);
        __syncwarp();
    }
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Pull into L2 the schedule records and map or run-table lines that this
// warp will read in level r (its items are warp, warp + nw, ...): they are
// static, and otherwise each is a first-touch DRAM read on the level's
// critical path.
template <typename T, typename M>
__device__ __forceinline__ void prefetch_level(const FactorArgs<T> &a, const LevelRange &r, int lane, int64_t warp,
                                               int64_t nw) {
    const int64_t nn = r.n_end - r.n_begin;
    const int64_t nsrc = r.row_begin - r.t_begin;
    const int64_t nrow = r.lane_begin - r.row_begin;
    const int64_t nlane = r.t_end - r.lane_begin;
    const int64_t total = nn + nsrc + nrow + (nlane + 31) / 32;
    for (int64_t it = warp; it < total; it += nw) {
        int64_t k = it - nn;
        if (k < 0) continue;
        int64_t tq;
        if (k < nsrc + nrow) {
            tq = r.t_begin + k;
        } else {
            tq = r.lane_begin + (k - nsrc - nrow) * 32 + lane;
            if (tq >= r.t_end) continue;
        }
        const Task tk = a.tasks[tq];
        const bool mine = k >= nsrc + nrow || lane == 0;
        if (!mine) continue;
        for (int32_t s = tk.seg_begin; s < tk.seg_end; s++) {
            const Seg sg = a.segs[s];
            if constexpr (is_runs<M>()) {
                const uint64_t enc = (uint64_t)sg.rb;
                const int64_t rb = (int64_t)(enc & ((1ull << RUN_BASE_BITS) - 1));
                const int32_t nr = (int32_t)(enc >> RUN_BASE_BITS);
                for (int32_t q = 0; q < nr; q += 128 / (int)sizeof(Run)) prefetch_l2(a.runs + rb + q);
            } else {
                const M *map = static_cast<const M *>(a.map);
                for (int32_t t = sg.t0; t < sg.t1; t += 128 / (int)sizeof(M)) prefetch_l2(map + sg.rb + t);
            }
        }
    }
}

// One level per launch, chained to the previous level's launch by a
// programmatic dependency: the prologue pulls this warp's (static) schedule
// records and run-table lines into L2 while the previous level still runs, then
// waits for it to finish (griddepcontrol.wait makes its writes visible);
// each block lets the next level start once its own items are done.
template <typename T, typename M>
__global__ void __launch_bounds__(LEVEL_WARPS * 32, LevelOcc<T>::blocks)
k_level(const FactorArgs<T> a, LevelRange r) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    T *acc = reinterpret_cast<T *>(smem_raw) + wib * (32 * (SRC_SLOTS + 1));
    const int64_t warp = (int64_t)blockIdx.x * LEVEL_WARPS + wib;
    const int64_t nw = (int64_t)gridDim.x * LEVEL_WARPS;
    // only a narrow level, a couple of items per warp, has a latency-bound
    // chain worth shortening; a wide level is throughput-bound
    const int64_t items = (r.n_end - r.n_begin) + (r.lane_begin - r.t_begin) + (r.t_end - r.lane_begin + 31) / 32;
    if (items <= 2 * nw) prefetch_level<T, M>(a, r, lane, warp, nw);
    asm volatile("griddepcontrol.wait;" ::: "memory");
    run_level<T, M>(a, r, lane, warp, nw, acc);
    __syncthreads();
    asm volatile("griddepcontrol.launch_dependents;");
}

// Consecutive levels in one launch (the pipelined mode, run by dataflow):
// the run's work items -- each level's normalization items, KIND_SRC and
// KIND_ROW tasks, groups of 32 KIND_LANE tasks, in level order -- are handed
// out by an atomic ticket, and instead of a barrier between levels each item
// waits for what it reads:
//   * a task of level l: every task of the run that targets a column of
//     level l done (its sources final), and the tasks of earlier levels of
//     the run that target its own column done (U(j,k) final, and its
//     additions after theirs: each target entry's additions keep the level
//     order, so the results equal the level launches' bit for bit);
//   * a normalization item of level l's columns (run in level l + 1): every
//     task of level l done (they read the columns raw) and the columns final.
// A finished task publishes with release semantics (fence, then the counter
// additions); a waiter acquires.  A warp only waits on items of earlier
// levels, handed out before its own, so the launch needs no co-residency.
// Factor values are read through L2 (other SMs write them meanwhile).  Every
// wait is bounded: past the limit the kernel records GLU_ERR_TIMEOUT and
// raises the abort word, which ends every other wait; the launch always ends.
__device__ __forceinline__ int ld_acquire_i32(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Lane 0 waits until *p >= target (or gives up); the warp agrees on the
// outcome and acquires.
__device__ __forceinline__ bool wait_ge(const int32_t *p, int32_t target, const DFFactorArgs &d, int lane) {
    int ok = 1;
    if (lane == 0 && target > 0 && ld_acquire_i32(p) < target) {
        const long long t0 = clock64();
        int spins = 0;
        unsigned nap = 32;             // polls back off: many warps may wait on one counter
        while (true) {
            __nanosleep(nap);
            nap = nap < 1024 ? nap * 2 : 1024;
            if (ld_acquire_i32(p) >= target) break;
            if ((++spins & 63) == 0) {
                if (*(volatile const unsigned *)d.abort) {
                    ok = 0;
                    break;
                }
                if (clock64() - t0 > d.spin_limit_cycles) {
                    atomicOr(d.abort, 1u);
                    atomicMin(d.err, (0xffffffull << 8) | DEVERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    return ok != 0;
}

// One lane's wait (KIND_LANE tasks): the same, without the warp.
__device__ __forceinline__ bool wait_ge_lane(const int32_t *p, int32_t target, const DFFactorArgs &d) {
    if (target <= 0 || ld_acquire_i32(p) >= target) return true;
    const long long t0 = clock64();
    int spins = 0;
    unsigned nap = 32;
    while (true) {
        __nanosleep(nap);
        nap = nap < 1024 ? nap * 2 : 1024;
        if (ld_acquire_i32(p) >= target) return true;
        if ((++spins & 63) == 0) {
            if (*(volatile const unsigned *)d.abort) return false;
            if (clock64() - t0 > d.spin_limit_cycles) {
                atomicOr(d.abort, 1u);
                atomicMin(d.err, (0xffffffull << 8) | DEVERR_TIMEOUT);
                return false;
            }
        }
    }
}

// A finished task: its additions, then its counters.
__device__ __forceinline__ void publish_task(const DFFactorArgs &d, int32_t task) {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    const int32_t k = d.task_col[task];
    if (k == d.fault_col) return;          // test hook: this column's tasks never publish
    atomicAdd(d.cdone + k, 1);
    atomicAdd(d.ldone + d.level_of[k], 1);
}

template <typename T, typename M>
__global__ void __launch_bounds__(LEVEL_WARPS * 32, 12 / LEVEL_WARPS)
k_levels_df(const FactorArgs<T> a, const DFFactorArgs d) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    T *acc = reinterpret_cast<T *>(smem_raw) + wib * (32 * (SRC_SLOTS + 1));
    const int32_t i0 = d.item_ptr[d.l0];
    const int32_t nitems = d.item_ptr[d.l1] - i0;
    while (true) {
        int32_t t = 0;
        if (lane == 0) t = (int32_t)atomicAdd(d.ticket, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= nitems) break;
        const int32_t g = i0 + t;
        int32_t lo = d.l0, hi = d.l1;      // the item's level: item_ptr[lo] <= g < item_ptr[lo + 1]
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (d.item_ptr[mid] <= g) lo = mid;
            else hi = mid;
        }
        const int32_t l = lo;
        const LevelRange r = d.ranges[l];
        const int64_t nn = r.n_end - r.n_begin;
        const int64_t nsrc = r.row_begin - r.t_begin;
        const int64_t nrow = r.lane_begin - r.row_begin;
        int64_t k = g - d.item_ptr[l];
        if (k < nn) {
            bool ok = true;
            if (l - 1 >= d.l0)
                ok = wait_ge(d.tdone + (l - 1), d.lvl_ntasks[l - 1], d, lane) &&
                     wait_ge(d.ldone + (l - 1), d.lvl_total[l - 1], d, lane);
            if (ok) norm_item<T, true>(a, a.norms[r.n_begin + k], lane);
            continue;
        }
        k -= nn;
        if (k < nsrc + nrow) {
            const int32_t task = (int32_t)(r.t_begin + k);
            const bool ok = wait_ge(d.ldone + l, d.lvl_total[l], d, lane) &&
                            wait_ge(d.cdone + d.task_col[task], d.task_before[task], d, lane);
            if (ok) {
                if (k < nsrc) src_task<T, M, true>(a, a.tasks[task], lane, acc);
                else row_tasks<T, M, true>(a, task, 1, 1, lane);
            }
            __syncwarp();
            if (lane == 0) {
                publish_task(d, task);
                atomicAdd(d.tdone + l, 1);
            }
            continue;
        }
        // a group of up to 32 KIND_LANE tasks, one per lane
        const int64_t q = r.lane_begin + (k - nsrc - nrow) * 32 + lane;
        const bool mine = q < r.t_end;
        if (mine) {
            const bool ok = wait_ge_lane(d.ldone + l, d.lvl_total[l], d) &&
                            wait_ge_lane(d.cdone + d.task_col[q], d.task_before[q], d);
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            if (ok) lane_task<T, M, true>(a, a.tasks[q]);
            publish_task(d, (int32_t)q);
        }
        const int cnt = __popc(__ballot_sync(0xffffffffu, mine));
        if (lane == 0) atomicAdd(d.tdone + l, cnt);
    }
}

// Final check of every pivot: zero or non-finite raises an error for the
// smallest such column.
template <typename T>
__global__ void k_pivot_check(const T *__restrict__ lu, const int64_t *__restrict__ diag_pos, int32_t n,
                              unsigned long long *err) {
    int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const T d = lu[diag_pos[j]];
    if (d == (T)0) raise_err(err, j, DEVERR_ZERO_PIVOT);
    else if (!isfinite(d)) raise_err(err, j, DEVERR_NONFINITE);
}

__global__ void k_reset_err(unsigned long long *err) { *err = ERR_NONE; }

// ---------------------------------------------------------------- run table
// Position of row r among rows[0, len) (ascending), or -1.
__device__ __forceinline__ int64_t find_row(const int32_t *rows, int64_t len, int32_t r) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (rows[mid] < r) lo = mid + 1;
        else hi = mid;
    }
    return (lo < len && rows[lo] == r) ? lo : -1;
}

// Pass 0 / 1, a warp per (j, k) pair: the position of every row of L(:,j) in
// column k past U(j,k) (binary search; the fill theorem says it is there), a
// run starting wherever a row's position is not its predecessor's plus one.
// Pass 0 stores the pair's run count, pass 1 writes the runs at
// pair_runs[pair] in order.  Built once per pattern at analysis.
__global__ void k_runs(const RunBuildArgs a, int fill) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = w; p < a.npairs; p += nw) {
        const int32_t j = a.pair_j[p];
        const int32_t k = a.pair_k[p];
        const int64_t pos = a.pair_pos[p];
        const int64_t dj = a.diag_pos[j];
        const int32_t lj = (int32_t)(a.lu_colptr[j + 1] - dj - 1);
        const int32_t *rows = a.lu_rowidx + pos + 1;
        const int64_t len = a.lu_colptr[k + 1] - pos - 1;
        int64_t base = fill ? a.pair_runs[p] : 0;
        int64_t prev = -2;
        for (int32_t t0 = 0; t0 < lj; t0 += 32) {
            const int32_t t = t0 + lane;
            int64_t q = 0;
            if (t < lj) {
                q = find_row(rows, len, a.lu_rowidx[dj + 1 + t]);
                if (q < 0) {
                    atomicMin(a.err, ((unsigned long long)(uint32_t)k << 8) | DEVERR_INTERNAL);
                    q = 0;
                }
            }
            int64_t left = __shfl_up_sync(0xffffffffu, q, 1);
            if (lane == 0) left = prev;
            const bool start = t < lj && (t == 0 || q != left + 1);
            const unsigned mask = __ballot_sync(0xffffffffu, start);
            if (fill && start) {
                Run *o = a.runs + base + __popc(mask & ((1u << lane) - 1));
                *o = Run{t, (int32_t)q};
            }
            base += __popc(mask);
            prev = __shfl_sync(0xffffffffu, q, 31);
        }
        if (!fill && lane == 0) a.counts[p] = (int32_t)base;
    }
}

// Pass 2, a thread per segment: its runs are those of its pair (whose index
// the host left in rb) that overlap rows t0..t1-1.
__global__ void k_seg_runs(const RunBuildArgs a) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.nsegs;
         s += (int64_t)gridDim.x * blockDim.x) {
        Seg &sg = a.segs[s];
        const int64_t pair = sg.rb;
        const int64_t lo = a.pair_runs[pair], hi = a.pair_runs[pair + 1];
        // first run starting after t0, and first run starting at or after t1
        int64_t x = lo, y = hi;
        while (x < y) {
            const int64_t mid = (x + y) >> 1;
            if (a.runs[mid].ts <= sg.t0) x = mid + 1;
            else y = mid;
        }
        const int64_t rb = x - 1;
        int64_t e = x, f = hi;
        while (e < f) {
            const int64_t mid = (e + f) >> 1;
            if (a.runs[mid].ts < sg.t1) e = mid + 1;
            else f = mid;
        }
        if (rb < lo || e - rb >= (int64_t(1) << (64 - RUN_BASE_BITS))) {
            atomicMin(a.err, (0xffffffull << 8) | DEVERR_INTERNAL);
            sg.rb = 0;
            continue;
        }
        sg.rb = (int64_t)((uint64_t)rb | ((uint64_t)(e - rb) << RUN_BASE_BITS));
    }
}

// Position map, a warp per (j, k) pair: the offset of every row of L(:,j) in
// column k past U(j,k), at pair_map[pair] + t.
template <typename M>
__global__ void k_map_build(const RunBuildArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    M *map = static_cast<M *>(a.map);
    for (int64_t p = w; p < a.npairs; p += nw) {
        const int32_t j = a.pair_j[p];
        const int32_t k = a.pair_k[p];
        const int64_t pos = a.pair_pos[p];
        const int64_t mb = a.pair_map[p];
        const int64_t dj = a.diag_pos[j];
        const int32_t lj = (int32_t)(a.lu_colptr[j + 1] - dj - 1);
        const int32_t *rows = a.lu_rowidx + pos + 1;
        const int64_t len = a.lu_colptr[k + 1] - pos - 1;
        for (int32_t t = lane; t < lj; t += 32) {
            int64_t q = find_row(rows, len, a.lu_rowidx[dj + 1 + t]);
            if (q < 0) {
                atomicMin(a.err, ((unsigned long long)(uint32_t)k << 8) | DEVERR_INTERNAL);
                q = 0;
            }
            map[mb + t] = (M)q;
        }
    }
}

// A thread per segment: its first map entry (its pair's, whose index the host
// left in rb, plus t0 is where the kernels index from: pair_map[pair]).
__global__ void k_seg_map(const RunBuildArgs a) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.nsegs;
         s += (int64_t)gridDim.x * blockDim.x) {
        Seg &sg = a.segs[s];
        sg.rb = a.pair_map[sg.rb];
    }
}

}  // namespace

template <typename T>
cudaError_t launch_gather(T *lu, const double *aval, const int32_t *gsrc, int64_t nnz, cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    int64_t blocks = (nnz + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_gather<T><<<(unsigned)blocks, 256, 0, s>>>(lu, aval, gsrc, nnz);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_level(const FactorArgs<T> &a, int lookup, const LevelRange &r, int num_sms, cudaStream_t s) {
    const int64_t items = (int64_t)(r.lane_begin - r.t_begin) + (r.t_end - r.lane_begin + 31) / 32 +
                          (r.n_end - r.n_begin);
    if (items <= 0) return cudaSuccess;
    int64_t blocks = (items + LEVEL_WARPS - 1) / LEVEL_WARPS;
    // at most the resident capacity (LevelOcc: 16 one-warp blocks per SM;
    // FP32 levels of many items 24): the next level's early blocks then take
    // only slots this level no longer needs
    const int64_t cap = (int64_t)num_sms * (items >= GLU_LEVEL_BIG_ITEMS ? LevelOcc<T>::cap_big : LevelOcc<T>::cap);
    if (blocks > cap) blocks = cap;
    const size_t smem = sizeof(T) * LEVEL_WARPS * 32 * (SRC_SLOTS + 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(LEVEL_WARPS * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (lookup == 2) return cudaLaunchKernelEx(&cfg, k_level<T, uint16_t>, a, r);
    if (lookup == 4) return cudaLaunchKernelEx(&cfg, k_level<T, uint32_t>, a, r);
    return cudaLaunchKernelEx(&cfg, k_level<T, Run>, a, r);
}

template <typename T>
cudaError_t launch_levels_df(const FactorArgs<T> &a, int lookup, const DFFactorArgs &d, int num_sms, cudaStream_t s) {
    if (d.l1 <= d.l0) return cudaSuccess;
    const size_t smem = sizeof(T) * LEVEL_WARPS * 32 * (SRC_SLOTS + 1);
    const void *fn = lookup == 2 ? (const void *)k_levels_df<T, uint16_t>
                   : lookup == 4 ? (const void *)k_levels_df<T, uint32_t>
                                 : (const void *)k_levels_df<T, Run>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, LEVEL_WARPS * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    // no more warps than the run's widest level has items (twice, so the next
    // level's items are fetched while one runs): idle warps would only poll
    unsigned blocks = (unsigned)(num_sms * per_sm);
    if (d.max_items > 0) {
        const int64_t want = (2 * (int64_t)d.max_items + LEVEL_WARPS - 1) / LEVEL_WARPS;
        if (want < (int64_t)blocks) blocks = (unsigned)(want < 1 ? 1 : want);
    }
    if (lookup == 2) k_levels_df<T, uint16_t><<<blocks, LEVEL_WARPS * 32, smem, s>>>(a, d);
    else if (lookup == 4) k_levels_df<T, uint32_t><<<blocks, LEVEL_WARPS * 32, smem, s>>>(a, d);
    else k_levels_df<T, Run><<<blocks, LEVEL_WARPS * 32, smem, s>>>(a, d);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pivot_check(const T *lu, const int64_t *diag_pos, int32_t n, unsigned long long *err,
                               cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_pivot_check<T><<<(n + 255) / 256, 256, 0, s>>>(lu, diag_pos, n, err);
    return cudaGetLastError();
}

cudaError_t launch_reset_err(unsigned long long *err, cudaStream_t s) {
    k_reset_err<<<1, 1, 0, s>>>(err);
    return cudaGetLastError();
}

cudaError_t launch_run_build(const RunBuildArgs &a, int pass, int map_bytes, cudaStream_t s) {
    if (pass == 0 || pass == 1 || pass == 3) {
        if (a.npairs == 0) return cudaSuccess;
        int64_t blocks = (a.npairs * 32 + 255) / 256;
        if (blocks > 152 * 32) blocks = 152 * 32;
        if (pass < 2) k_runs<<<(unsigned)blocks, 256, 0, s>>>(a, pass);
        else if (map_bytes == 2) k_map_build<uint16_t><<<(unsigned)blocks, 256, 0, s>>>(a);
        else k_map_build<uint32_t><<<(unsigned)blocks, 256, 0, s>>>(a);
    } else {
        if (a.nsegs == 0) return cudaSuccess;
        int64_t blocks = (a.nsegs + 255) / 256;
        if (blocks > 152 * 64) blocks = 152 * 64;
        if (pass == 2) k_seg_runs<<<(unsigned)blocks, 256, 0, s>>>(a);
        else k_seg_map<<<(unsigned)blocks, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template cudaError_t launch_gather<double>(double *, const double *, const int32_t *, int64_t, cudaStream_t);
template cudaError_t launch_gather<float>(float *, const double *, const int32_t *, int64_t, cudaStream_t);
template cudaError_t launch_level<double>(const FactorArgs<double> &, int, const LevelRange &, int, cudaStream_t);
template cudaError_t launch_level<float>(const FactorArgs<float> &, int, const LevelRange &, int, cudaStream_t);
template cudaError_t launch_levels_df<double>(const FactorArgs<double> &, int, const DFFactorArgs &, int,
                                             cudaStream_t);
template cudaError_t launch_levels_df<float>(const FactorArgs<float> &, int, const DFFactorArgs &, int, cudaStream_t);
template cudaError_t launch_pivot_check<double>(const double *, const int64_t *, int32_t, unsigned long long *,
                                                cudaStream_t);
template cudaError_t launch_pivot_check<float>(const float *, const int64_t *, int32_t, unsigned long long *,
                                               cudaStream_t);

}  // namespace glu
