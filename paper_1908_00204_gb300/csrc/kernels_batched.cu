// kernels_batched.cu -- many refactorizations that share one pattern.
//
// B value sets of the same matrix (Newton iterations, transient steps,
// Monte-Carlo corners; Section III: the numeric part repeats while the
// pattern stays) are stored interleaved: entry q of set b at [q * S + b],
// S = B rounded up to 32.  A warp takes one work item for 32 sets at once:
// every index (schedule, run table, pattern) is the same for all lanes and
// every value access is 32 consecutive elements.  Each lane owns its own
// matrix, so the right-looking update of a level (Algorithm 5 / Eq. 3) needs
// no ordering between lanes; a lane applies a task's segments in order, its
// additions as L2 reductions.  The dataflow solve and the FP64 refinement follow the single-
// matrix versions with lanes over the batch.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "glu_device.cuh"

namespace glu {
namespace {

constexpr int BU = 4;   // rows per batch of independent loads
constexpr int DU = 8;   // entries per batch of independent loads in the solve
constexpr int PB = 16;  // chunk partial sums per batch of independent loads

__device__ __forceinline__ void raise_err_b(unsigned long long *err, int32_t col, unsigned code) {
    atomicMin(err, ((unsigned long long)(uint32_t)col << 8) | code);
}

// values[b * ld + p] (set-major, as the caller gives them) -> aT[p * S + b],
// 32 x 32 tiles through shared memory.
__global__ void k_values_in(double *__restrict__ aT, const double *__restrict__ v, int64_t nnz, int32_t B,
                            int64_t ld, int32_t S) {
    __shared__ double tile[32][33];
    const int64_t p0 = (int64_t)blockIdx.x * 32;
    const int32_t b0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int32_t b = b0 + k;
        const int64_t p = p0 + threadIdx.x;
        tile[k][threadIdx.x] = (b < B && p < nnz) ? v[(int64_t)b * ld + p] : 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t p = p0 + k;
        const int32_t b = b0 + threadIdx.x;
        if (p < nnz && b < S) aT[p * S + b] = tile[threadIdx.x][k];
    }
}

template <typename T>
__global__ void k_gather_b(T *__restrict__ lu, const double *__restrict__ aT, const int32_t *__restrict__ gsrc,
                           int64_t nnz, int32_t S) {
    const int64_t total = nnz * S;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = i / S;
        const int32_t b = (int32_t)(i - q * S);
        const int32_t s = gsrc[q];
        lu[i] = s >= 0 ? (T)aT[(int64_t)s * S + b] : (T)0;
    }
}

// One level for all sets.  Items: normalization items and tasks, each
// repeated for the G = S / 32 lane groups.
template <typename T, typename M>
__global__ void __launch_bounds__(128) k_level_b(const FactorArgs<T> a, LevelRange r, int32_t S) {
    const int lane = threadIdx.x & 31;
    const int32_t G = S / 32;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t nn = r.n_end - r.n_begin;
    const int64_t nt = r.t_end - r.t_begin;
    const int64_t total = (nn + nt) * G;
    for (int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < total; it += nw) {
        const int64_t k = it / G;
        const int32_t b = (int32_t)(it - k * G) * 32 + lane;
        T *__restrict__ lu = a.lu;
        if (k < nn) {
            const NormItem ni = a.norms[r.n_begin + k];
            const int64_t dj = a.diag_pos[ni.col];
            const T rd = (T)1 / lu[dj * S + b];    // one division per item, as the single-matrix kernel
            // eight rows' loads in flight, then their products
            T *Lc = lu + (dj + 1) * S + b;
            for (int32_t tb = ni.t0; tb < ni.t1; tb += 8) {
                T v[8];
#pragma unroll
                for (int u = 0; u < 8; u++)
                    if (tb + u < ni.t1) v[u] = Lc[(int64_t)(tb + u) * S];
#pragma unroll
                for (int u = 0; u < 8; u++)
                    if (tb + u < ni.t1) Lc[(int64_t)(tb + u) * S] = v[u] * rd;
            }
            continue;
        }
        const Task tk = a.tasks[r.t_begin + (k - nn)];
        for (int32_t s = tk.seg_begin; s < tk.seg_end; s++) {
            const Seg sg = a.segs[s];
            const T f = lu[sg.pos * S + b] / lu[sg.dj * S + b];
            const T *__restrict__ L = lu + (sg.dj + 1) * S + b;
            T *tgt = lu + (sg.pos + 1) * S + b;
            // the rows' offsets: the position map, or the segment's runs walked
            // in step by the whole warp (every lane reads the same records)
            int64_t r = 0, rend = 0;
            Run cur{0, 0}, nxt{INT32_MAX, 0};
            const M *mp = nullptr;
            if constexpr (std::is_same<M, Run>::value) {
                const uint64_t enc = (uint64_t)sg.rb;
                r = (int64_t)(enc & ((1ull << RUN_BASE_BITS) - 1));
                rend = r + (int64_t)(enc >> RUN_BASE_BITS);
                cur = a.runs[r];
                nxt = r + 1 < rend ? a.runs[r + 1] : Run{INT32_MAX, 0};
            } else {
                mp = static_cast<const M *>(a.map) + sg.rb;
            }
            for (int32_t tb = sg.t0; tb < sg.t1; tb += BU) {
                int64_t off[BU];
                T lv[BU];
#pragma unroll
                for (int u = 0; u < BU; u++)
                    if (tb + u < sg.t1) lv[u] = L[(int64_t)(tb + u) * S];
#pragma unroll
                for (int u = 0; u < BU; u++)
                    if (tb + u < sg.t1) {
                        if constexpr (std::is_same<M, Run>::value) {
                            while (tb + u >= nxt.ts) {
                                cur = nxt;
                                r++;
                                nxt = r + 1 < rend ? a.runs[r + 1] : Run{INT32_MAX, 0};
                            }
                            off[u] = (int64_t)(cur.off + (tb + u - cur.ts)) * S;
                        } else {
                            off[u] = (int64_t)mp[tb + u] * S;
                        }
                    }
            // the targets take -L(i,j) f as reductions in L2; one lane (one
            // value set) applies a task's segments in order, so each entry's
            // additions come in a fixed order
#pragma unroll
                for (int u = 0; u < BU; u++)
                    if (tb + u < sg.t1) atomicAdd(&tgt[off[u]], -lv[u] * f);
            }
        }
    }
}

template <typename T>
__global__ void k_pivot_b(const T *__restrict__ lu, const int64_t *__restrict__ diag_pos, int32_t n, int32_t B,
                          int32_t S, unsigned long long *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * S) return;
    const int32_t j = (int32_t)(i / S);
    const int32_t b = (int32_t)(i - (int64_t)j * S);
    if (b >= B) return;
    const T d = lu[diag_pos[j] * S + b];
    if (d == (T)0) raise_err_b(err, j, DEVERR_ZERO_PIVOT);
    else if (!isfinite(d)) raise_err_b(err, j, DEVERR_NONFINITE);
}

// ---------------------------------------------------------------- solves
// caller layout b[(set * nrhs + r) * n + i] (original numbering) <->
// internal [(r * n + i) * S + set]
__global__ void k_rhs_in(double *__restrict__ out, const double *__restrict__ in, int32_t n, int32_t nrhs, int32_t B,
                         int32_t S) {
    const int64_t total = (int64_t)n * nrhs * S;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ri = t / S;
        const int32_t b = (int32_t)(t - ri * S);
        const int32_t r = (int32_t)(ri / n);
        const int32_t i = (int32_t)(ri - (int64_t)r * n);
        out[t] = b < B ? in[((int64_t)b * nrhs + r) * n + i] : 0.0;
    }
}

__global__ void k_rhs_out(double *__restrict__ out, const double *__restrict__ in, int32_t n, int32_t nrhs, int32_t B,
                          int32_t S) {
    const int64_t total = (int64_t)n * nrhs * S;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ri = t / S;
        const int32_t b = (int32_t)(t - ri * S);
        if (b >= B) continue;
        const int32_t r = (int32_t)(ri / n);
        const int32_t i = (int32_t)(ri - (int64_t)r * n);
        out[((int64_t)b * nrhs + r) * n + i] = in[t];
    }
}

// y[(r*n + inew)*S + b] = in[(r*n + perm[inew])*S + b] (and the inverse)
template <typename T>
__global__ void k_perm_in_b(T *__restrict__ y, const double *__restrict__ in, const int32_t *__restrict__ perm,
                            int32_t n, int32_t nrhs, int32_t S) {
    const int64_t total = (int64_t)n * nrhs * S;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ri = t / S;
        const int32_t b = (int32_t)(t - ri * S);
        const int32_t r = (int32_t)(ri / n);
        const int32_t i = (int32_t)(ri - (int64_t)r * n);
        y[t] = (T)in[((int64_t)r * n + perm[i]) * S + b];
    }
}

template <typename T>
__global__ void k_perm_out_b(double *__restrict__ out, const T *__restrict__ z, const int32_t *__restrict__ perm,
                             int32_t n, int32_t nrhs, int32_t S) {
    const int64_t total = (int64_t)n * nrhs * S;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ri = t / S;
        const int32_t b = (int32_t)(t - ri * S);
        const int32_t r = (int32_t)(ri / n);
        const int32_t i = (int32_t)(ri - (int64_t)r * n);
        out[((int64_t)r * n + perm[i]) * S + b] = (double)z[t];
    }
}

__device__ __forceinline__ int ld_acquire_b(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_b(int32_t *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void wait_b(const int32_t *flag, const DFSolveArgs &a) {
    if (ld_acquire_b(flag) == a.epoch) return;
    const long long t0 = clock64();
    int spins = 0;
    while (true) {
        __nanosleep(32);
        if (ld_acquire_b(flag) == a.epoch) return;
        if ((++spins & 63) == 0) {
            if (*(volatile const unsigned *)a.abort) return;
            if (clock64() - t0 > a.spin_limit_cycles) {
                atomicOr(a.abort, 1u);
                atomicMin(a.err, ((unsigned long long)0xffffffu << 8) | DEVERR_TIMEOUT);
                return;
            }
        }
    }
}

__device__ __forceinline__ int atomic_add_acq_rel_b(int32_t *p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ int ld_relaxed_b(const int32_t *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until flags[c * G] holds the epoch for every c in [c0, c1), the lanes
// splitting the range: relaxed polls, four in flight per lane, a bounded
// acquiring wait on any flag not yet set, then one acquire fence for the lot.
__device__ __forceinline__ void wait_range_b(const int32_t *flags, int32_t G, int32_t c0, int32_t c1, int lane,
                                             const DFSolveArgs &a) {
    for (int32_t c = c0 + lane; c < c1; c += 128) {
        int v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) v[u] = c + 32 * u < c1 ? ld_relaxed_b(flags + (int64_t)(c + 32 * u) * G) : a.epoch;
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (v[u] != a.epoch) wait_b(flags + (int64_t)(c + 32 * u) * G, a);
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// acc[r] += sum over entries p0..p1-1 of M[pos[p]] * v_r[col[p]] for this
// lane's set and RB right-hand sides (v_r = src + r * rs), entries in
// sequence.  The warp loads a window of 32 positions and columns once and
// broadcasts them; each value of M is read once for all RB right-hand sides
// and DU entries' loads are in flight together.
template <typename T, int RB>
__device__ __forceinline__ void dot_win_b(const T *__restrict__ lub, const int64_t *__restrict__ pos,
                                          const int32_t *__restrict__ col, const T *src, int64_t rs, int64_t p0,
                                          int64_t p1, int32_t S, int lane, T (&acc)[RB]) {
    for (int64_t pw = p0; pw < p1; pw += 32) {
        const int cnt = (int)((p1 - pw) < 32 ? (p1 - pw) : 32);
        int64_t mq = 0;
        int32_t mc = 0;
        if (lane < cnt) {
            mq = pos[pw + lane];
            mc = col[pw + lane];
        }
        for (int u0 = 0; u0 < cnt; u0 += DU) {
            T lv[DU], yv[DU][RB];
#pragma unroll
            for (int u = 0; u < DU; u++) {
                const int64_t q = __shfl_sync(0xffffffffu, mq, u0 + u);
                const int32_t c = __shfl_sync(0xffffffffu, mc, u0 + u);
                lv[u] = (T)0;
#pragma unroll
                for (int r = 0; r < RB; r++) yv[u][r] = (T)0;
                if (u0 + u < cnt) {
                    lv[u] = lub[q * S];
#pragma unroll
                    for (int r = 0; r < RB; r++) yv[u][r] = __ldcg(src + r * rs + (int64_t)c * S);
                }
            }
#pragma unroll
            for (int u = 0; u < DU; u++)
                if (u0 + u < cnt) {
#pragma unroll
                    for (int r = 0; r < RB; r++) acc[r] += lv[u] * yv[u][r];
                }
        }
    }
}

// The arithmetic of a chunk or row item for right-hand sides r0..r0+RB-1
// (the item's flags already acquired).
template <typename T, int RB>
__device__ __forceinline__ void item_rhs_b(const SolveArgs<T> &s, const DFSolveArgs &a, const DFItem &it, T *y, T *z,
                                           int32_t nrhs, int32_t S, int32_t b, int lane, int32_t r0, T d) {
    const int n = s.n;
    const bool bwd = it.flags & DF_BACKWARD;
    const int64_t *pos = bwd ? s.urow_pos : s.lrow_pos;
    const int32_t *col = bwd ? s.urow_col : s.lrow_col;
    const T *src = (bwd ? z : y) + (int64_t)r0 * n * S + b;
    const int64_t rs = (int64_t)n * S;
    const T *lub = s.lu + b;
    T acc[RB];
#pragma unroll
    for (int r = 0; r < RB; r++) acc[r] = (T)0;
    if (it.flags & DF_CHUNK) {
        const SolveChunk ch = (bwd ? a.bchunks : a.fchunks)[it.chunk];
        T *partial = static_cast<T *>(bwd ? a.bpartial_v : a.fpartial_v);
        dot_win_b<T, RB>(lub, pos, col, src, rs, ch.p0, ch.p1, S, lane, acc);
#pragma unroll
        for (int r = 0; r < RB; r++) partial[(((int64_t)it.chunk * nrhs) + r0 + r) * S + b] = acc[r];
        return;
    }
    const int32_t i = it.row;
    if (it.ce > it.cb) {
        const T *partial = static_cast<const T *>(bwd ? a.bpartial_v : a.fpartial_v);
        for (int32_t c0 = it.cb; c0 < it.ce; c0 += PB) {
            T pv[PB][RB];
#pragma unroll
            for (int u = 0; u < PB; u++)
#pragma unroll
                for (int r = 0; r < RB; r++)
                    pv[u][r] = c0 + u < it.ce ? __ldcg(partial + (((int64_t)(c0 + u) * nrhs) + r0 + r) * S + b) : (T)0;
#pragma unroll
            for (int u = 0; u < PB; u++)
                if (c0 + u < it.ce) {
#pragma unroll
                    for (int r = 0; r < RB; r++) acc[r] += pv[u][r];
                }
        }
    } else {
        const int64_t *rptr = bwd ? s.urow_ptr : s.lrow_ptr;
        dot_win_b<T, RB>(lub, pos, col, src, rs, rptr[i], rptr[i + 1], S, lane, acc);
    }
#pragma unroll
    for (int r = 0; r < RB; r++) {
        const int64_t at = ((int64_t)(r0 + r) * n + i) * S + b;
        const T v = __ldcg(y + at);
        (bwd ? z : y)[at] = bwd ? (v - acc[r]) * d : v - acc[r];
    }
}

// The sweeps of a dense diagonal block of ns <= NS rows (NS a size class),
// one column per template step so that every register index is a constant.
// Forward (unit L): rows below column JJ subtract L(i, JJ) v(JJ); rows from
// ns to NS - 1 are padding, computed on the block's last row and discarded,
// so the class runs without per-row branches.  Backward: v(JJ) is multiplied
// by the reciprocal of U(JJ, JJ) (taken as soon as it is loaded, off the
// column chain), then rows above subtract U(i, JJ) v(JJ).  mybase in lane k:
// the position of the block's first row in column k of the block.
template <typename T, int NS, int JJ>
struct BlockFwd {
    static __device__ __forceinline__ void run(T (&v)[NS], const T *lub, int64_t mybase, int32_t ns, int32_t S) {
        if (JJ + 1 < ns) {
            const int64_t base = __shfl_sync(0xffffffffu, mybase, JJ);
            T lv[NS - JJ - 1];
#pragma unroll
            for (int ii = JJ + 1; ii < NS; ii++) lv[ii - JJ - 1] = lub[(base + min(ii, ns - 1)) * S];
#pragma unroll
            for (int ii = JJ + 1; ii < NS; ii++) v[ii] = v[ii] - lv[ii - JJ - 1] * v[JJ];
            BlockFwd<T, NS, JJ + 1>::run(v, lub, mybase, ns, S);
        }
    }
};
template <typename T, int NS>
struct BlockFwd<T, NS, NS - 1> {
    static __device__ __forceinline__ void run(T (&)[NS], const T *, int64_t, int32_t, int32_t) {}
};

template <typename T, int NS, int JJ>
struct BlockBwd {
    static __device__ __forceinline__ void run(T (&v)[NS], const T *lub, int64_t mybase, int32_t ns, int32_t S) {
        if (JJ < ns) {
            const int64_t base = __shfl_sync(0xffffffffu, mybase, JJ);
            T uv[JJ + 1];
#pragma unroll
            for (int ii = 0; ii <= JJ; ii++) uv[ii] = lub[(base + ii) * S];
            v[JJ] = v[JJ] * ((T)1 / uv[JJ]);
#pragma unroll
            for (int ii = 0; ii < JJ; ii++) v[ii] = v[ii] - uv[ii] * v[JJ];
        }
        BlockBwd<T, NS, JJ - 1>::run(v, lub, mybase, ns, S);
    }
};
template <typename T, int NS>
struct BlockBwd<T, NS, -1> {
    static __device__ __forceinline__ void run(T (&)[NS], const T *, int64_t, int32_t, int32_t) {}
};

// A dense diagonal block [c0, c0 + ns) of the dataflow solve for one lane
// group (lane = set) and the right-hand sides r0, r0 + RSPLIT_B, ..., ns <= NS,
// the flags of its chunks already acquired.
// Each row's right-hand side less its chunks' partial sums (subtracted in
// chunk order, PB loads in flight) is gathered in this warp's shared rows sv,
// then swept in registers.  Lane kk holds row kk's chunk end and the block's
// first-row position in column c0 + kk, broadcast by shuffles.
template <typename T, int NS>
__device__ __forceinline__ void block_item_b(const T *lub, const T *partial, T *y, T *out_base, T *sv, bool bwd,
                                             int32_t c0, int32_t ns, int32_t cbeg, int32_t cend, int32_t myend,
                                             int64_t mybase, int32_t n, int32_t r0, int32_t nrhs, int32_t S,
                                             int32_t b) {
    for (int32_t r = r0; r < nrhs; r += RSPLIT_B) {
        T v[NS];
#pragma unroll
        for (int kk = 0; kk < NS; kk++) v[kk] = __ldcg(y + ((int64_t)r * n + c0 + min(kk, ns - 1)) * S + b);
        if (cend > cbeg) {
#pragma unroll
            for (int kk = 0; kk < NS; kk++) sv[kk * 32] = v[kk];
            int32_t cur = 0, nxt = __shfl_sync(0xffffffffu, myend, 0);
            for (int32_t c = cbeg; c < cend; c += PB) {
                T pv[PB];
#pragma unroll
                for (int u = 0; u < PB; u++)
                    pv[u] = __ldcg(partial + (((int64_t)min(c + u, cend - 1) * nrhs) + r) * S + b);
#pragma unroll
                for (int u = 0; u < PB; u++)
                    if (c + u < cend) {
                        while (c + u >= nxt) nxt = __shfl_sync(0xffffffffu, myend, ++cur);
                        sv[cur * 32] -= pv[u];
                    }
            }
#pragma unroll
            for (int kk = 0; kk < NS; kk++) v[kk] = sv[kk * 32];
        }
        if (!bwd)
            BlockFwd<T, NS, 0>::run(v, lub, mybase, ns, S);
        else
            BlockBwd<T, NS, NS - 1>::run(v, lub, mybase, ns, S);
        T *out = out_base + ((int64_t)r * n + c0) * S + b;
#pragma unroll
        for (int kk = 0; kk < NS; kk++)
            if (kk < ns) out[(int64_t)kk * S] = v[kk];
    }
}

// Dataflow solve for all sets: work item (DF item, lane group).  Flags are per
// (row, group) and per (chunk, group).  Forward writes y, backward z.  The
// lanes of a warp acquire the flags of an item's entries together, then each
// lane runs the entries in sequence for its own set.
template <typename T>
__global__ void __launch_bounds__(128, 4) k_solve_df_b(const SolveArgs<T> s, const DFSolveArgs a, T *y, T *z,
                                                    int32_t nrhs, int32_t S) {
    __shared__ __align__(16) unsigned char blk_rows[4 * SN_MAX_B * 32 * sizeof(T)];   // per warp: a block's rows
    const int lane = threadIdx.x & 31;
    const int n = s.n;
    const int32_t G = S / 32;
    const int64_t total = (int64_t)a.nitems * G;
    while (true) {
        int64_t t = 0;
        if (lane == 0) t = (int64_t)atomicAdd(a.ticket, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total) break;
        const int64_t k = t / G;
        const int32_t g = (int32_t)(t - k * G);
        const int32_t b = g * 32 + lane;
        const DFItem it = a.items[k];
        const bool bwd = it.flags & DF_BACKWARD;
        const int64_t *rptr = bwd ? s.urow_ptr : s.lrow_ptr;
        const int32_t *col = bwd ? s.urow_col : s.lrow_col;
        int32_t *ready = bwd ? a.bready : a.fready;
        if (it.flags & DF_BLOCK) {
            // a dense diagonal block [c0, c1) of at most SN_MAX_B rows, run by
            // the code of its size class for the right-hand sides r = it.sub
            // (mod RSPLIT_B); the last of the block's copies to finish (a
            // counter per block and lane group) publishes its rows
            const int32_t c0 = it.row, ns = it.cb - it.row;
            if (it.sub < nrhs) {
                const T *lub = s.lu + b;
                const int32_t *snx = (bwd ? a.bsnx : a.fsnx) + it.ce;
                const int32_t *crd = bwd ? a.bchunk_ready : a.fchunk_ready;
                const int32_t cbeg = snx[0];
                const int32_t myend = lane < ns ? snx[lane + 1] : 0;
                const int64_t mybase = lane < ns ? s.diag_pos[c0 + lane] - lane : 0;
                const int32_t cend = __shfl_sync(0xffffffffu, myend, ns - 1);
                wait_range_b(crd + g, G, cbeg, cend, lane, a);
                __syncwarp();
                const T *partial = static_cast<const T *>(bwd ? a.bpartial_v : a.fpartial_v);
                T *sv = reinterpret_cast<T *>(blk_rows) + (threadIdx.x >> 5) * (SN_MAX_B * 32) + lane;
                T *ob = bwd ? z : y;
                const int32_t q = it.sub;
                if (ns <= 8)
                    block_item_b<T, 8>(lub, partial, y, ob, sv, bwd, c0, ns, cbeg, cend, myend, mybase, n, q, nrhs, S,
                                       b);
                else if (ns <= 16)
                    block_item_b<T, 16>(lub, partial, y, ob, sv, bwd, c0, ns, cbeg, cend, myend, mybase, n, q, nrhs,
                                        S, b);
                else if (ns <= 24)
                    block_item_b<T, 24>(lub, partial, y, ob, sv, bwd, c0, ns, cbeg, cend, myend, mybase, n, q, nrhs,
                                        S, b);
                else
                    block_item_b<T, SN_MAX_B>(lub, partial, y, ob, sv, bwd, c0, ns, cbeg, cend, myend, mybase, n, q,
                                              nrhs, S, b);
            }
            __syncwarp();
            int last = 0;
            if (lane == 0) last = atomic_add_acq_rel_b(a.blk_done + (int64_t)it.blk * G + g, 1) == RSPLIT_B - 1;
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last)
                for (int32_t kk = lane; kk < ns; kk += 32) st_release_b(ready + (int64_t)(c0 + kk) * G + g, a.epoch);
            continue;
        }
        // chunk or row item: acquire the flags of its entries' columns (or of
        // its chunks), then all right-hand sides, four at a time.  A backward
        // item runs after the forward launch and the tail have completed.
        // d: the reciprocal of U(i, i) for a backward row
        const T d = (bwd && !(it.flags & DF_CHUNK)) ? (T)1 / s.lu[s.diag_pos[it.row] * S + b] : (T)1;
        if (it.flags & DF_CHUNK) {
            const SolveChunk ch = (bwd ? a.bchunks : a.fchunks)[it.chunk];
            for (int64_t p = ch.p0 + lane; p < ch.p1; p += 32) wait_b(ready + (int64_t)col[p] * G + g, a);
        } else if (it.ce > it.cb) {
            wait_range_b((bwd ? a.bchunk_ready : a.fchunk_ready) + g, G, it.cb, it.ce, lane, a);
        } else {
            for (int64_t p = rptr[it.row] + lane; p < rptr[it.row + 1]; p += 32)
                wait_b(ready + (int64_t)col[p] * G + g, a);
        }
        __syncwarp();
        int32_t r0 = 0;
        for (; r0 + 4 <= nrhs; r0 += 4) item_rhs_b<T, 4>(s, a, it, y, z, nrhs, S, b, lane, r0, d);
        if (r0 + 2 <= nrhs) {
            item_rhs_b<T, 2>(s, a, it, y, z, nrhs, S, b, lane, r0, d);
            r0 += 2;
        }
        if (r0 < nrhs) item_rhs_b<T, 1>(s, a, it, y, z, nrhs, S, b, lane, r0, d);
        __syncwarp();
        if (lane == 0) {
            if (it.flags & DF_CHUNK)
                st_release_b((bwd ? a.bchunk_ready : a.fchunk_ready) + (int64_t)it.chunk * G + g, a.epoch);
            else
                st_release_b(ready + (int64_t)it.row * G + g, a.epoch);
        }
    }
}

// The dense tail [t0, n) for one group of 32 sets and one right-hand side per
// block (lane = set), in panels of TP columns.  Forward: one warp finishes
// the panel's rows against its strictly lower triangle, then all warps
// subtract the panel's columns from the rows below, TP independent loads a
// row.  Backward likewise with the upper triangle, its diagonal and the rows
// above.  Each row takes its column updates in the same order as a column-
// at-a-time sweep.  The tail's right-hand side and the positions of its
// columns stay in shared memory; the next panel's triangle is staged there
// during the current update, so a panel costs two barriers.
constexpr int TP = 16;
constexpr int TRI_B = TP * (TP + 1) / 2;

template <typename T>
__device__ __forceinline__ void stage_tri_b(T *tri, const T *lub, const int64_t *lb, int32_t j0, int32_t kb, int32_t S,
                                            bool bwd, int w, int nwarp, int lane) {
    if (!bwd) {
        // strictly lower: (i, k), k < i, at i (i - 1) / 2 + k
        for (int i = 1 + w; i < kb; i += nwarp)
            for (int k = 0; k < i; k++) tri[(i * (i - 1) / 2 + k) * 32 + lane] = lub[(lb[j0 + k] + j0 + i) * S];
    } else {
        // upper with the diagonal: (i, j), i <= j, at j (j + 1) / 2 + i
        for (int j = w; j < kb; j += nwarp)
            for (int i = 0; i <= j; i++) tri[(j * (j + 1) / 2 + i) * 32 + lane] = lub[(lb[j0 + j] + j0 + i) * S];
    }
}

template <typename T>
__global__ void __launch_bounds__(512, 1) k_solve_tail_b(const SolveArgs<T> s, const TailArgs ta,
                                                      const T *__restrict__ fpartial, const T *y, T *z, int32_t nrhs,
                                                      int32_t S) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int32_t n = s.n, t0 = ta.t0, NT = n - t0, G = S / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int32_t g = blockIdx.x, r = blockIdx.y;
    const int32_t b = g * 32 + lane;
    int64_t *lb = reinterpret_cast<int64_t *>(smem_raw);   // [NT]: position of tail row 0 in column t0 + j
    T *yt = reinterpret_cast<T *>(lb + NT);                // [NT][32]
    T *tri = yt + (int64_t)NT * 32;                        // [TRI_B][32]
    const T *lub = s.lu + b;
    for (int32_t j = threadIdx.x; j < NT; j += blockDim.x) lb[j] = s.diag_pos[t0 + j] - j;
    for (int32_t ii = w; ii < NT; ii += nwarp) {
        T v = __ldcg(y + ((int64_t)r * n + t0 + ii) * S + b);
        for (int32_t c = ta.cb[ii]; c < ta.ce[ii]; c++) v -= __ldcg(fpartial + (((int64_t)c * nrhs) + r) * S + b);
        yt[ii * 32 + lane] = v;
    }
    __syncthreads();
    // forward, panels ascending
    stage_tri_b<T>(tri, lub, lb, 0, NT < TP ? NT : TP, S, false, w, nwarp, lane);
    __syncthreads();
    for (int32_t j0 = 0; j0 < NT; j0 += TP) {
        const int32_t kb = (NT - j0) < TP ? (NT - j0) : TP;
        if (w == 0) {
            T v[TP];
#pragma unroll
            for (int i = 0; i < TP; i++) v[i] = i < kb ? yt[(j0 + i) * 32 + lane] : (T)0;
#pragma unroll
            for (int k = 0; k < TP; k++)
#pragma unroll
                for (int i = k + 1; i < TP; i++)
                    if (i < kb) v[i] = v[i] - tri[(i * (i - 1) / 2 + k) * 32 + lane] * v[k];
#pragma unroll
            for (int i = 0; i < TP; i++)
                if (i < kb) yt[(j0 + i) * 32 + lane] = v[i];
        }
        __syncthreads();
        for (int32_t ii = j0 + kb + w; ii < NT; ii += nwarp) {
            T lv[TP];
#pragma unroll
            for (int k = 0; k < TP; k++) lv[k] = k < kb ? lub[(lb[j0 + k] + ii) * S] : (T)0;
            T acc = yt[ii * 32 + lane];
#pragma unroll
            for (int k = 0; k < TP; k++)
                if (k < kb) acc = acc - lv[k] * yt[(j0 + k) * 32 + lane];
            yt[ii * 32 + lane] = acc;
        }
        if (j0 + TP < NT) {
            const int32_t jn = j0 + TP;
            stage_tri_b<T>(tri, lub, lb, jn, (NT - jn) < TP ? (NT - jn) : TP, S, false, w, nwarp, lane);
        }
        __syncthreads();
    }
    // backward, panels descending
    const int32_t last = ((NT - 1) / TP) * TP;
    if (NT > 0) stage_tri_b<T>(tri, lub, lb, last, NT - last, S, true, w, nwarp, lane);
    __syncthreads();
    for (int32_t j0 = last; j0 >= 0; j0 -= TP) {
        const int32_t kb = (NT - j0) < TP ? (NT - j0) : TP;
        if (w == 0) {
            T v[TP];
#pragma unroll
            for (int i = 0; i < TP; i++) v[i] = i < kb ? yt[(j0 + i) * 32 + lane] : (T)0;
#pragma unroll
            for (int j = TP - 1; j >= 0; j--)
                if (j < kb) {
                    v[j] = v[j] * ((T)1 / tri[(j * (j + 1) / 2 + j) * 32 + lane]);
#pragma unroll
                    for (int i = 0; i < j; i++) v[i] = v[i] - tri[(j * (j + 1) / 2 + i) * 32 + lane] * v[j];
                }
#pragma unroll
            for (int i = 0; i < TP; i++)
                if (i < kb) yt[(j0 + i) * 32 + lane] = v[i];
        }
        __syncthreads();
        for (int32_t ii = w; ii < j0; ii += nwarp) {
            T uv[TP];
#pragma unroll
            for (int k = 0; k < TP; k++) uv[k] = k < kb ? lub[(lb[j0 + k] + ii) * S] : (T)0;
            T acc = yt[ii * 32 + lane];
#pragma unroll
            for (int k = TP - 1; k >= 0; k--)
                if (k < kb) acc = acc - uv[k] * yt[(j0 + k) * 32 + lane];
            yt[ii * 32 + lane] = acc;
        }
        if (j0 > 0) stage_tri_b<T>(tri, lub, lb, j0 - TP, TP, S, true, w, nwarp, lane);
        __syncthreads();
    }
    T *zr = z + (int64_t)r * n * S;
    for (int32_t ii = w; ii < NT; ii += nwarp) zr[(int64_t)(t0 + ii) * S + b] = yt[ii * 32 + lane];
    // every right-hand side's block stores the same flags; the backward
    // items read them after this launch has completed
    for (int32_t ii = threadIdx.x; ii < NT; ii += blockDim.x) ta.bready[(int64_t)(t0 + ii) * G + g] = ta.epoch;
}

// ------------------------------------------------------------ refinement
__device__ __forceinline__ unsigned long long abs_bits_b(double v) {
    return (unsigned long long)__double_as_longlong(fabs(v));
}

// Blocks of 32 sets (x) by 8 rows (y): each thread keeps the maximum over
// its rows of one set; the block's maximum per set goes into slot[x] by one
// atomicMax (bit patterns of non-negative doubles order like the values).
__device__ __forceinline__ void block_max_b(unsigned long long *slot, unsigned long long m) {
    __shared__ unsigned long long sm[8][32];
    sm[threadIdx.y][threadIdx.x] = m;
    __syncthreads();
    if (threadIdx.y == 0) {
        for (int w = 1; w < (int)blockDim.y; w++) {
            const unsigned long long u = sm[w][threadIdx.x];
            m = u > m ? u : m;
        }
        if (m) atomicMax(slot + threadIdx.x, m);
    }
    __syncthreads();
}

__global__ void k_csr_values_b(double *__restrict__ out, const double *__restrict__ aT,
                               const int64_t *__restrict__ src, int64_t nnz, int32_t S) {
    const int64_t total = nnz * S;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / S;
        out[t] = aT[src[q] * S + (t - q * S)];
    }
}

// ||A_b||_inf per set b (lane group blockIdx.y)
__global__ void k_anorm_b(const int64_t *__restrict__ rp, const double *__restrict__ av, int32_t n, int32_t S,
                          unsigned long long *anorm) {
    const int32_t b = blockIdx.y * 32 + threadIdx.x;
    unsigned long long m = 0;
    for (int32_t i = blockIdx.x * blockDim.y + threadIdx.y; i < n; i += gridDim.x * blockDim.y) {
        double s = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; p++) s += fabs(av[p * S + b]);
        const unsigned long long u = abs_bits_b(s);
        m = u > m ? u : m;
    }
    block_max_b(anorm + blockIdx.y * 32, m);
}

// r = b - A x per (row, side k = blockIdx.z, set); max |r|, |x| per (side, set)
__global__ void k_residual_b(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const double *__restrict__ av, const double *__restrict__ bb,
                             const double *__restrict__ x, double *__restrict__ r, int32_t n, int32_t S,
                             unsigned long long *rmax, unsigned long long *xmax) {
    const int32_t k = blockIdx.z;
    const int32_t b = blockIdx.y * 32 + threadIdx.x;
    const double *xk = x + (int64_t)k * n * S + b;
    unsigned long long mr = 0, mx = 0;
    for (int32_t i = blockIdx.x * blockDim.y + threadIdx.y; i < n; i += gridDim.x * blockDim.y) {
        double s = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; p++) s = fma(av[p * S + b], xk[(int64_t)ci[p] * S], s);
        const int64_t t = ((int64_t)k * n + i) * S + b;
        const double v = bb[t] - s;
        r[t] = v;
        const unsigned long long ur = abs_bits_b(v), ux = abs_bits_b(x[t]);
        mr = ur > mr ? ur : mr;
        mx = ux > mx ? ux : mx;
    }
    block_max_b(rmax + (int64_t)k * S + blockIdx.y * 32, mr);
    block_max_b(xmax + (int64_t)k * S + blockIdx.y * 32, mx);
}

__global__ void k_absmax_b(const double *__restrict__ v, int32_t n, int32_t S, unsigned long long *out) {
    const int32_t k = blockIdx.z;
    const int32_t b = blockIdx.y * 32 + threadIdx.x;
    unsigned long long m = 0;
    for (int32_t i = blockIdx.x * blockDim.y + threadIdx.y; i < n; i += gridDim.x * blockDim.y) {
        const unsigned long long u = abs_bits_b(v[((int64_t)k * n + i) * S + b]);
        m = u > m ? u : m;
    }
    block_max_b(out + (int64_t)k * S + blockIdx.y * 32, m);
}

__global__ void k_check_b(const unsigned long long *rmax, const unsigned long long *xmax,
                          const unsigned long long *bmax, const unsigned long long *anorm, int32_t nrhs, int32_t B,
                          int32_t S, double tol, int32_t *done, double *berr, int32_t *ndone) {
    const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nrhs * S) return;
    const int32_t b = t % S;
    if (b >= B) {
        done[t] = 1;
        berr[t] = 0.0;
        return;
    }
    const double den = __longlong_as_double((long long)anorm[b]) * __longlong_as_double((long long)xmax[t]) +
                       __longlong_as_double((long long)bmax[t]);
    const double e = den > 0.0 ? __longlong_as_double((long long)rmax[t]) / den : 0.0;
    berr[t] = e;
    const int d = e <= tol ? 1 : 0;
    done[t] = d;
    if (d) atomicAdd(ndone, 1);
}

__global__ void k_update_b(double *__restrict__ x, const double *__restrict__ d, const int32_t *__restrict__ done,
                           int32_t n, int32_t nrhs, int32_t S) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * nrhs * S) return;
    const int64_t ri = t / S;
    const int32_t b = (int32_t)(t - ri * S);
    if (!done[(ri / n) * S + b]) x[t] += d[t];
}

// row-parallel reductions over (row blocks, lane groups, sides): about eight
// blocks per SM in all
dim3 row_grid_b(int32_t n, int32_t nrhs, int32_t S) {
    const int64_t groups = (int64_t)(S / 32) * (nrhs > 0 ? nrhs : 1);
    int64_t rb = ((int64_t)n + 7) / 8;
    const int64_t cap = (int64_t)152 * 8 / groups;
    if (rb > cap) rb = cap;
    if (rb < 1) rb = 1;
    return dim3((unsigned)rb, (unsigned)(S / 32), (unsigned)(nrhs > 0 ? nrhs : 1));
}

unsigned grid_b(int64_t work) {
    int64_t g = (work + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_values_in(double *aT, const double *v, int64_t nnz, int32_t B, int64_t ld, int32_t S,
                             cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    dim3 grid((unsigned)((nnz + 31) / 32), (unsigned)(S / 32));
    k_values_in<<<grid, dim3(32, 8), 0, s>>>(aT, v, nnz, B, ld, S);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_b(T *lu, const double *aT, const int32_t *gsrc, int64_t nnz, int32_t S, cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    k_gather_b<T><<<grid_b(nnz * S), 256, 0, s>>>(lu, aT, gsrc, nnz, S);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_level_b(const FactorArgs<T> &a, int lookup, const LevelRange &r, int32_t S, int num_sms,
                           cudaStream_t s) {
    const int64_t items = ((int64_t)(r.t_end - r.t_begin) + (r.n_end - r.n_begin)) * (S / 32);
    if (items <= 0) return cudaSuccess;
    // one item per warp: the items' costs vary widely, and the block
    // scheduler balances them better than a grid-stride split (6 % on the
    // 256-set workload against 16 blocks per SM)
    const int64_t blocks = (items + 3) / 4;
    (void)num_sms;
    if (lookup == 2) k_level_b<T, uint16_t><<<(unsigned)blocks, 128, 0, s>>>(a, r, S);
    else if (lookup == 4) k_level_b<T, uint32_t><<<(unsigned)blocks, 128, 0, s>>>(a, r, S);
    else k_level_b<T, Run><<<(unsigned)blocks, 128, 0, s>>>(a, r, S);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pivot_b(const T *lu, const int64_t *diag_pos, int32_t n, int32_t B, int32_t S,
                           unsigned long long *err, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_pivot_b<T><<<(unsigned)(((int64_t)n * S + 255) / 256), 256, 0, s>>>(lu, diag_pos, n, B, S, err);
    return cudaGetLastError();
}

cudaError_t launch_rhs_in(double *out, const double *in, int32_t n, int32_t nrhs, int32_t B, int32_t S,
                          cudaStream_t s) {
    k_rhs_in<<<grid_b((int64_t)n * nrhs * S), 256, 0, s>>>(out, in, n, nrhs, B, S);
    return cudaGetLastError();
}

cudaError_t launch_rhs_out(double *out, const double *in, int32_t n, int32_t nrhs, int32_t B, int32_t S,
                           cudaStream_t s) {
    k_rhs_out<<<grid_b((int64_t)n * nrhs * S), 256, 0, s>>>(out, in, n, nrhs, B, S);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_b(const SolveArgs<T> &sa, const DFSolveArgs &a, int32_t nfwd,
                           const TailArgs &ta, const double *in, double *out, T *y, T *z, const int32_t *perm,
                           int32_t nrhs, int32_t S, int num_sms, cudaStream_t s) {
    const int32_t n = sa.n;
    k_perm_in_b<T><<<grid_b((int64_t)n * nrhs * S), 256, 0, s>>>(y, in, perm, n, nrhs, S);
    // forward items, the tail, backward items
    for (int part = 0; part < 2; part++) {
        DFSolveArgs d = a;
        if (part == 0) d.nitems = nfwd;
        else {
            d.items = a.items + nfwd;
            d.nitems = a.nitems - nfwd;
        }
        if (d.nitems > 0) {
            cudaError_t e = cudaMemsetAsync(a.ticket, 0, sizeof(unsigned), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(a.abort, 0, sizeof(unsigned), s);
            if (e != cudaSuccess) return e;
            int64_t blocks = ((int64_t)d.nitems * (S / 32) * 32 + 127) / 128;
            if (blocks > (int64_t)num_sms * 8) blocks = (int64_t)num_sms * 8;
            k_solve_df_b<T><<<(unsigned)blocks, 128, 0, s>>>(sa, d, y, z, nrhs, S);
        }
        if (part == 0 && ta.t0 < n) {
            const int32_t nt = n - ta.t0;
            const size_t smem = (size_t)nt * sizeof(int64_t) + ((size_t)nt + TRI_B) * 32 * sizeof(T);
            cudaError_t e = cudaFuncSetAttribute(k_solve_tail_b<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
            if (nrhs > 0)
                k_solve_tail_b<T><<<dim3((unsigned)(S / 32), (unsigned)nrhs), 512, smem, s>>>(
                    sa, ta, static_cast<const T *>(a.fpartial_v), y, z, nrhs, S);
        }
    }
    k_perm_out_b<T><<<grid_b((int64_t)n * nrhs * S), 256, 0, s>>>(out, z, perm, n, nrhs, S);
    return cudaGetLastError();
}

cudaError_t launch_ir_b(int op, const int64_t *rp, const int32_t *ci, const double *av, const double *aT,
                        const int64_t *src, int64_t nnz, const double *bb, double *x, double *r, const double *d,
                        int32_t n, int32_t nrhs, int32_t B, int32_t S, unsigned long long *anorm,
                        unsigned long long *rmax, unsigned long long *xmax, unsigned long long *bmax, double tol,
                        int32_t *done, double *berr, int32_t *ndone, cudaStream_t s) {
    const int64_t w = (int64_t)n * nrhs * S;
    switch (op) {
        case 0:   // values in compressed-row order, ||A||, ||b||
            if (nnz > 0) k_csr_values_b<<<grid_b(nnz * S), 256, 0, s>>>(const_cast<double *>(av), aT, src, nnz, S);
            if (n > 0) k_anorm_b<<<row_grid_b(n, 1, S), dim3(32, 8), 0, s>>>(rp, av, n, S, anorm);
            if (w > 0) k_absmax_b<<<row_grid_b(n, nrhs, S), dim3(32, 8), 0, s>>>(bb, n, S, bmax);
            break;
        case 1:   // residual and check
            if (w > 0) k_residual_b<<<row_grid_b(n, nrhs, S), dim3(32, 8), 0, s>>>(rp, ci, av, bb, x, r, n, S, rmax, xmax);
            k_check_b<<<(unsigned)((nrhs * S + 127) / 128), 128, 0, s>>>(rmax, xmax, bmax, anorm, nrhs, B, S, tol, done,
                                                                         berr, ndone);
            break;
        case 2:   // update
            if (w > 0) k_update_b<<<(unsigned)((w + 255) / 256), 256, 0, s>>>(x, d, done, n, nrhs, S);
            break;
    }
    return cudaGetLastError();
}

template cudaError_t launch_gather_b<double>(double *, const double *, const int32_t *, int64_t, int32_t, cudaStream_t);
template cudaError_t launch_gather_b<float>(float *, const double *, const int32_t *, int64_t, int32_t, cudaStream_t);
template cudaError_t launch_level_b<double>(const FactorArgs<double> &, int, const LevelRange &, int32_t, int,
                                            cudaStream_t);
template cudaError_t launch_level_b<float>(const FactorArgs<float> &, int, const LevelRange &, int32_t, int,
                                           cudaStream_t);
template cudaError_t launch_pivot_b<double>(const double *, const int64_t *, int32_t, int32_t, int32_t,
                                            unsigned long long *, cudaStream_t);
template cudaError_t launch_pivot_b<float>(const float *, const int64_t *, int32_t, int32_t, int32_t,
                                           unsigned long long *, cudaStream_t);
template cudaError_t launch_solve_b<double>(const SolveArgs<double> &, const DFSolveArgs &, int32_t,
                                            const TailArgs &, const double *, double *, double *, double *,
                                            const int32_t *, int32_t, int32_t, int, cudaStream_t);
template cudaError_t launch_solve_b<float>(const SolveArgs<float> &, const DFSolveArgs &, int32_t,
                                           const TailArgs &, const double *, double *, float *, float *,
                                           const int32_t *, int32_t, int32_t, int, cudaStream_t);

}  // namespace glu
