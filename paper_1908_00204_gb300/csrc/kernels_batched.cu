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
            for (int32_t t = ni.t0; t < ni.t1; t++) {
                T *p = lu + (dj + 1 + t) * S + b;
                *p = *p * rd;
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

// sum over entries p0..p1-1 of M[pos[p]] * v[col[p]] for this lane's set;
// entries in sequence, BU independent loads in flight
template <typename T>
__device__ __forceinline__ T dot_b(const T *__restrict__ lu, const int64_t *__restrict__ pos,
                                   const int32_t *__restrict__ col, const T *v, int64_t p0, int64_t p1, int32_t S) {
    T acc = (T)0;
    for (int64_t pb = p0; pb < p1; pb += BU) {
        T lv[BU], yv[BU];
#pragma unroll
        for (int u = 0; u < BU; u++)
            if (pb + u < p1) {
                lv[u] = lu[pos[pb + u] * S];
                yv[u] = __ldcg(v + (int64_t)col[pb + u] * S);
            }
#pragma unroll
        for (int u = 0; u < BU; u++)
            if (pb + u < p1) acc += lv[u] * yv[u];
    }
    return acc;
}

// Dataflow solve for all sets: work item (DF item, lane group).  Flags are per
// (row, group) and per (chunk, group).  Forward writes y, backward z.  The
// lanes of a warp acquire the flags of an item's entries together, then each
// lane runs the entries in sequence for its own set.
template <typename T>
__global__ void __launch_bounds__(128) k_solve_df_b(const SolveArgs<T> s, const DFSolveArgs a, T *y, T *z,
                                                    int32_t nrhs, int32_t S) {
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
        const int64_t *pos = bwd ? s.urow_pos : s.lrow_pos;
        const int32_t *col = bwd ? s.urow_col : s.lrow_col;
        int32_t *ready = bwd ? a.bready : a.fready;
        const T *src = bwd ? z : y;
        const T *lub = s.lu + b;
        if (it.flags & DF_BLOCK) {
            // a dense diagonal block [c0, c1) of at most SN_MAX_B rows for this
            // group: lane = set, the block's values of the set in registers,
            // swept a column at a time (forward: rows below subtract L(i, jj)
            // y(jj); backward: z(jj) = y(jj) / U(jj, jj), rows above subtract)
            const int32_t c0 = it.row, ns = it.cb - it.row;
            const int32_t *snx = (bwd ? a.bsnx : a.fsnx) + it.ce;
            const int32_t *crd = bwd ? a.bchunk_ready : a.fchunk_ready;
            for (int32_t c = snx[0] + lane; c < snx[ns]; c += 32) wait_b(crd + (int64_t)c * G + g, a);
            __syncwarp();
            const T *partial = static_cast<const T *>(bwd ? a.bpartial_v : a.fpartial_v);
            for (int32_t r = 0; r < nrhs; r++) {
                T v[SN_MAX_B];
#pragma unroll
                for (int kk = 0; kk < SN_MAX_B; kk++) {
                    T x = (T)0;
                    if (kk < ns) {
                        x = __ldcg(y + ((int64_t)r * n + c0 + kk) * S + b);
                        for (int32_t c = snx[kk]; c < snx[kk + 1]; c++)
                            x -= __ldcg(partial + (((int64_t)c * nrhs) + r) * S + b);
                    }
                    v[kk] = x;
                }
                if (!bwd) {
#pragma unroll
                    for (int jj = 0; jj < SN_MAX_B; jj++) {
                        if (jj + 1 < ns) {
                            const int64_t base = s.diag_pos[c0 + jj] - jj;
#pragma unroll
                            for (int ii = jj + 1; ii < SN_MAX_B; ii++)
                                if (ii < ns) v[ii] = v[ii] - lub[(base + ii) * S] * v[jj];
                        }
                    }
                } else {
#pragma unroll
                    for (int jj = SN_MAX_B - 1; jj >= 0; jj--) {
                        if (jj < ns) {
                            const int64_t dp = s.diag_pos[c0 + jj];
                            v[jj] = v[jj] / lub[dp * S];
                            const int64_t base = dp - jj;
#pragma unroll
                            for (int ii = 0; ii < jj; ii++) v[ii] = v[ii] - lub[(base + ii) * S] * v[jj];
                        }
                    }
                }
                T *out = (bwd ? z : y) + ((int64_t)r * n + c0) * S + b;
#pragma unroll
                for (int kk = 0; kk < SN_MAX_B; kk++)
                    if (kk < ns) out[(int64_t)kk * S] = v[kk];
            }
            __syncwarp();
            for (int32_t kk = lane; kk < ns; kk += 32) st_release_b(ready + (int64_t)(c0 + kk) * G + g, a.epoch);
            continue;
        }
        if (it.flags & DF_CHUNK) {
            const SolveChunk ch = (bwd ? a.bchunks : a.fchunks)[it.chunk];
            T *partial = static_cast<T *>(bwd ? a.bpartial_v : a.fpartial_v);
            for (int64_t p = ch.p0 + lane; p < ch.p1; p += 32) wait_b(ready + (int64_t)col[p] * G + g, a);
            __syncwarp();
            for (int32_t r = 0; r < nrhs; r++)
                partial[(((int64_t)it.chunk * nrhs) + r) * S + b] =
                    dot_b<T>(lub, pos, col, src + (int64_t)r * n * S + b, ch.p0, ch.p1, S);
            __syncwarp();
            if (lane == 0) st_release_b((bwd ? a.bchunk_ready : a.fchunk_ready) + (int64_t)it.chunk * G + g, a.epoch);
            continue;
        }
        const int32_t i = it.row;
        const int64_t p0 = rptr[i], p1 = rptr[i + 1];
        const int32_t *crd = bwd ? a.bchunk_ready : a.fchunk_ready;
        if (lane == 0 && bwd) wait_b(a.fready + (int64_t)i * G + g, a);
        if (it.ce > it.cb) {
            for (int32_t c = it.cb + lane; c < it.ce; c += 32) wait_b(crd + (int64_t)c * G + g, a);
        } else {
            for (int64_t p = p0 + lane; p < p1; p += 32) wait_b(ready + (int64_t)col[p] * G + g, a);
        }
        __syncwarp();
        const T d = bwd ? s.lu[s.diag_pos[i] * S + b] : (T)1;
        const T *partial = static_cast<const T *>(bwd ? a.bpartial_v : a.fpartial_v);
        for (int32_t r = 0; r < nrhs; r++) {
            T acc = (T)0;
            if (it.ce > it.cb) {
                for (int32_t c = it.cb; c < it.ce; c++) acc += __ldcg(partial + (((int64_t)c * nrhs) + r) * S + b);
            } else {
                acc = dot_b<T>(lub, pos, col, src + (int64_t)r * n * S + b, p0, p1, S);
            }
            const T v = __ldcg(y + ((int64_t)r * n + i) * S + b);
            (bwd ? z : y)[((int64_t)r * n + i) * S + b] = bwd ? (v - acc) / d : v - acc;
        }
        __syncwarp();
        if (lane == 0) st_release_b(ready + (int64_t)i * G + g, a.epoch);
    }
}

// The dense tail [t0, n) for one group of 32 sets per block: warp w takes
// rows w, w+32, ...; lane = set.  The tail's values of the group stay in
// shared memory; one barrier per column forward, two backward.
template <typename T>
__global__ void __launch_bounds__(1024) k_solve_tail_b(const SolveArgs<T> s, const int64_t *__restrict__ lu_colptr,
                                                       const TailArgs ta, const T *__restrict__ fpartial, const T *y,
                                                       T *z, int32_t nrhs, int32_t S) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int32_t n = s.n, t0 = ta.t0, NT = n - t0, G = S / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int32_t g = blockIdx.x;
    const int32_t b = g * 32 + lane;
    T *yt = reinterpret_cast<T *>(smem_raw);      // [NT][32]
    T *zc = yt + (int64_t)NT * 32;                 // [32]: z of the current column
    for (int32_t r = 0; r < nrhs; r++) {
        for (int32_t ii = w; ii < NT; ii += nwarp) {
            T v = __ldcg(y + ((int64_t)r * n + t0 + ii) * S + b);
            for (int32_t c = ta.cb[ii]; c < ta.ce[ii]; c++) v -= __ldcg(fpartial + (((int64_t)c * nrhs) + r) * S + b);
            yt[ii * 32 + lane] = v;
        }
        __syncthreads();
        for (int32_t jj = 0; jj < NT; jj++) {
            const int64_t lb = s.diag_pos[t0 + jj] - jj;
            const T vj = yt[jj * 32 + lane];
            for (int32_t ii = jj + 1 + w; ii < NT; ii += nwarp)
                yt[ii * 32 + lane] = yt[ii * 32 + lane] - s.lu[(lb + ii) * S + b] * vj;
            __syncthreads();
        }
        T *zr = z + (int64_t)r * n * S;
        for (int32_t jj = NT - 1; jj >= 0; jj--) {
            const int32_t j = t0 + jj;
            if (w == 0) {
                const T zj = yt[jj * 32 + lane] / s.lu[s.diag_pos[j] * S + b];
                zc[lane] = zj;
                zr[(int64_t)j * S + b] = zj;
            }
            __syncthreads();
            const int64_t ub = lu_colptr[j + 1] - NT;
            const T zj = zc[lane];
            for (int32_t ii = w; ii < jj; ii += nwarp)
                yt[ii * 32 + lane] = yt[ii * 32 + lane] - s.lu[(ub + ii) * S + b] * zj;
            __syncthreads();
        }
    }
    for (int32_t ii = threadIdx.x; ii < NT; ii += blockDim.x) ta.bready[(int64_t)(t0 + ii) * G + g] = ta.epoch;
}

// ------------------------------------------------------------ refinement
__device__ __forceinline__ void max_abs_b(unsigned long long *slot, double v) {
    atomicMax(slot, (unsigned long long)__double_as_longlong(fabs(v)));
}

__global__ void k_csr_values_b(double *__restrict__ out, const double *__restrict__ aT,
                               const int64_t *__restrict__ src, int64_t nnz, int32_t S) {
    const int64_t total = nnz * S;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t / S;
        out[t] = aT[src[q] * S + (t - q * S)];
    }
}

__global__ void k_anorm_b(const int64_t *__restrict__ rp, const double *__restrict__ av, int32_t n, int32_t S,
                          unsigned long long *anorm) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * S) return;
    const int32_t i = (int32_t)(t / S);
    const int32_t b = (int32_t)(t - (int64_t)i * S);
    double s = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) s += fabs(av[p * S + b]);
    max_abs_b(anorm + b, s);
}

// r = b - A x per (row, side, set); max |r|, |x| per (side, set)
__global__ void k_residual_b(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const double *__restrict__ av, const double *__restrict__ bb,
                             const double *__restrict__ x, double *__restrict__ r, int32_t n, int32_t nrhs, int32_t S,
                             unsigned long long *rmax, unsigned long long *xmax) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * nrhs * S) return;
    const int64_t ri = t / S;
    const int32_t b = (int32_t)(t - ri * S);
    const int32_t k = (int32_t)(ri / n);
    const int32_t i = (int32_t)(ri - (int64_t)k * n);
    const double *xk = x + (int64_t)k * n * S + b;
    double s = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) s = fma(av[p * S + b], xk[(int64_t)ci[p] * S], s);
    const double v = bb[t] - s;
    r[t] = v;
    max_abs_b(rmax + (int64_t)k * S + b, v);
    max_abs_b(xmax + (int64_t)k * S + b, x[t]);
}

__global__ void k_absmax_b(const double *__restrict__ v, int32_t n, int32_t nrhs, int32_t S,
                           unsigned long long *out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * nrhs * S) return;
    const int64_t ri = t / S;
    const int32_t b = (int32_t)(t - ri * S);
    max_abs_b(out + (ri / n) * S + b, v[t]);
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
    int64_t blocks = (items + 3) / 4;
    if (blocks > (int64_t)num_sms * 16) blocks = (int64_t)num_sms * 16;
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
cudaError_t launch_solve_b(const SolveArgs<T> &sa, const DFSolveArgs &a, int32_t nfwd, const int64_t *lu_colptr,
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
            const size_t smem = ((size_t)(n - ta.t0) * 32 + 32) * sizeof(T);
            cudaError_t e = cudaFuncSetAttribute(k_solve_tail_b<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
            k_solve_tail_b<T><<<(unsigned)(S / 32), 1024, smem, s>>>(sa, lu_colptr, ta,
                                                                     static_cast<const T *>(a.fpartial_v), y, z,
                                                                     nrhs, S);
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
            if (n > 0) k_anorm_b<<<(unsigned)(((int64_t)n * S + 255) / 256), 256, 0, s>>>(rp, av, n, S, anorm);
            if (w > 0) k_absmax_b<<<(unsigned)((w + 255) / 256), 256, 0, s>>>(bb, n, nrhs, S, bmax);
            break;
        case 1:   // residual and check
            if (w > 0) k_residual_b<<<(unsigned)((w + 255) / 256), 256, 0, s>>>(rp, ci, av, bb, x, r, n, nrhs, S, rmax, xmax);
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
template cudaError_t launch_solve_b<double>(const SolveArgs<double> &, const DFSolveArgs &, int32_t, const int64_t *,
                                            const TailArgs &, const double *, double *, double *, double *,
                                            const int32_t *, int32_t, int32_t, int, cudaStream_t);
template cudaError_t launch_solve_b<float>(const SolveArgs<float> &, const DFSolveArgs &, int32_t, const int64_t *,
                                           const TailArgs &, const double *, double *, float *, float *,
                                           const int32_t *, int32_t, int32_t, int, cudaStream_t);

}  // namespace glu
