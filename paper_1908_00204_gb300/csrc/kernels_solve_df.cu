// kernels_solve_df.cu -- dataflow ("sync-free") triangular solves (sm_103a).
//
// The two triangular systems of Section I: forward (unit L) items in one
// launch, the dense tail, then backward (U) items in a second launch, so a
// backward row finds its own forward value final.  Work items -- a row, or a
// chunk of a long row's dot
// product -- are listed in a topological order (each item after everything it
// reads) and handed out by an atomic ticket, so a warp waits only on items
// that running warps already hold: no level barriers, no co-residency
// assumption.  A finished row publishes a flag with release semantics; a
// reader acquires it before loading the value.  Flags hold the call's epoch,
// so they need no reset between calls.  Every wait is bounded: past the limit
// the kernel records GLU_ERR_TIMEOUT, raises an abort flag that ends all other
// waits, publishes its own result and carries on, so the launch always ends.
// The backward sweep writes its own vector z (y keeps the forward values).
// A backward step multiplies by the reciprocal of U's diagonal, taken before
// the step's waits, so no division sits on the dependency chain.
#include <cuda_runtime.h>

#include <cstdint>

#include "glu_device.cuh"

namespace glu {
namespace {

__device__ __forceinline__ int ld_acquire(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int32_t *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ T ld_cg(const T *p) { return __ldcg(p); }

template <typename T>
__device__ __forceinline__ T warp_sum_df(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Wait until *flag == epoch; false once the wait gave up (timeout or abort).
__device__ __forceinline__ bool wait_flag(const int32_t *flag, int epoch, const DFSolveArgs &a) {
    if (ld_acquire(flag) == epoch) return true;
    const long long t0 = clock64();
    int spins = 0;
    while (true) {
        __nanosleep(32);
        if (ld_acquire(flag) == epoch) return true;
        if ((++spins & 63) == 0) {
            if (*(volatile const unsigned *)a.abort) return false;
            if (clock64() - t0 > a.spin_limit_cycles) {
                atomicOr(a.abort, 1u);
                atomicMin(a.err, ((unsigned long long)0xffffffu << 8) | DEVERR_TIMEOUT);
                return false;
            }
        }
    }
}

__device__ __forceinline__ int ld_relaxed(const int32_t *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Poll *flag (relaxed reads) until it holds epoch; false once the wait gave
// up.  The caller fences afterwards.
__device__ __forceinline__ bool spin_flag(const int32_t *flag, int epoch, const DFSolveArgs &a) {
    const long long t0 = clock64();
    int spins = 0;
    while (true) {
        __nanosleep(32);
        if (ld_relaxed(flag) == epoch) return true;
        if ((++spins & 63) == 0) {
            if (*(volatile const unsigned *)a.abort) return false;
            if (clock64() - t0 > a.spin_limit_cycles) {
                atomicOr(a.abort, 1u);
                atomicMin(a.err, ((unsigned long long)0xffffffu << 8) | DEVERR_TIMEOUT);
                return false;
            }
        }
    }
}

// Rows without chunks and chunks hold at most SOLVE_CHUNK = 4 x 32 entries.
constexpr int DF_PER_LANE = 4;

// The entries p0..p1-1 of a row of L or U, up to DF_PER_LANE per lane: their
// columns and values do not depend on other rows, so they are loaded before
// any wait.  j = -1 marks an empty slot.
template <typename T>
__device__ __forceinline__ void load_entries(const SolveArgs<T> &s, const int32_t *col, const int64_t *pos,
                                             int64_t p0, int64_t p1, int lane, int32_t (&j)[DF_PER_LANE],
                                             T (&l)[DF_PER_LANE]) {
#pragma unroll
    for (int k = 0; k < DF_PER_LANE; k++) {
        const int64_t p = p0 + lane + 32 * k;
        j[k] = p < p1 ? col[p] : -1;
    }
#pragma unroll
    for (int k = 0; k < DF_PER_LANE; k++) {
        const int64_t p = p0 + lane + 32 * k;
        l[k] = p < p1 ? s.lu[pos[p]] : (T)0;
    }
}

// Wait for the ready flags of a lane's columns: all first reads go out at
// once, then any flag not yet set is polled; one fence after the relaxed
// reads completes the acquire, so the writers' values are visible.
__device__ __forceinline__ void wait_cols(const int32_t *ready, const int32_t (&j)[DF_PER_LANE], int epoch,
                                          const DFSolveArgs &a) {
    int v[DF_PER_LANE];
#pragma unroll
    for (int k = 0; k < DF_PER_LANE; k++) v[k] = j[k] >= 0 ? ld_relaxed(ready + j[k]) : epoch;
#pragma unroll
    for (int k = 0; k < DF_PER_LANE; k++)
        if (v[k] != epoch) spin_flag(ready + j[k], epoch, a);
    fence_acq_rel();
}

template <typename T>
__device__ __forceinline__ T dot_entries(const int32_t (&j)[DF_PER_LANE], const T (&l)[DF_PER_LANE], const T *yr) {
    T acc = (T)0;
#pragma unroll
    for (int k = 0; k < DF_PER_LANE; k++)
        if (j[k] >= 0) acc += l[k] * ld_cg(yr + j[k]);
    return warp_sum_df(acc);
}

// A dense diagonal block [c0, c1) of at most SN_MAX rows, one warp: lane l
// keeps rows l, l + 32, ... in registers.  After the partial sums of the
// rows' entries outside the block (chunk items) are ready, the block's own
// triangle is swept a column at a time: the owner of row jj holds its final
// value, a shuffle broadcasts it, every other row of the block subtracts
// L(i, jj) times it (forward), or, backward, z(jj) = y(jj) times the
// reciprocal of U(jj, jj) and the rows above subtract U(i, jj) z(jj).  The block being dense, column c0+jj's
// entries in rows c0..c1-1 are contiguous in the CSC values, at
// diag_pos[c0+jj] - jj + i; the coefficients of BLK_PF columns are loaded
// together, ahead of their steps.
constexpr int BLK_K = SN_MAX / 32;   // rows per lane
#ifndef GLU_BLK_PF
#define GLU_BLK_PF 4
#endif
constexpr int BLK_PF = GLU_BLK_PF;   // columns whose coefficients load together

template <typename T>
__device__ __forceinline__ void block_item(const SolveArgs<T> &s, const DFSolveArgs &a, const DFItem &it, T *y, T *z,
                                           int32_t nrhs, int lane) {
    const bool bwd = it.flags & DF_BACKWARD;
    const int32_t c0 = it.row, ns = it.cb - it.row;
    const int32_t *snx = (bwd ? a.bsnx : a.fsnx) + it.ce;
    const int32_t *chunk_ready = bwd ? a.bchunk_ready : a.fchunk_ready;
    const T *partial = static_cast<const T *>(bwd ? a.bpartial_v : a.fpartial_v);
    int32_t *ready = bwd ? a.bready : a.fready;
    const int n = s.n;
    for (int32_t c = snx[0] + lane; c < snx[ns]; c += 32)
        if (ld_relaxed(chunk_ready + c) != a.epoch) spin_flag(chunk_ready + c, a.epoch, a);
    fence_acq_rel();
    __syncwarp();
    int32_t cb[BLK_K], ce[BLK_K];
    int64_t bj[BLK_K];   // lane l, slot k: diag_pos of column c0 + 32k + l, minus its offset
    T d[BLK_K];
#pragma unroll
    for (int k = 0; k < BLK_K; k++) {
        const int32_t ii = k * 32 + lane;
        cb[k] = ce[k] = 0;
        bj[k] = 0;
        d[k] = (T)1;
        if (ii < ns) {
            cb[k] = snx[ii];
            ce[k] = snx[ii + 1];
            const int64_t dp = s.diag_pos[c0 + ii];
            bj[k] = dp - ii;
            if (bwd) d[k] = (T)1 / s.lu[dp];   // the reciprocal of U(ii, ii)
        }
    }
    for (int32_t r = 0; r < nrhs; r++) {
        T v[BLK_K];
#pragma unroll
        for (int k = 0; k < BLK_K; k++) {
            const int32_t ii = k * 32 + lane;
            T x = (T)0;
            if (ii < ns) {
                x = ld_cg(y + (int64_t)r * n + c0 + ii);
                // the row's chunk partial sums in chunk order, eight loads in flight
                for (int32_t c = cb[k]; c < ce[k]; c += 8) {
                    T pv[8];
#pragma unroll
                    for (int u = 0; u < 8; u++)
                        pv[u] = c + u < ce[k] ? ld_cg(partial + (int64_t)(c + u) * nrhs + r) : (T)0;
#pragma unroll
                    for (int u = 0; u < 8; u++)
                        if (c + u < ce[k]) x -= pv[u];
                }
            }
            v[k] = x;
        }
        if (!bwd) {
#pragma unroll
            for (int kj = 0; kj < BLK_K; kj++) {
                for (int32_t tg = 0; tg < 32; tg += BLK_PF) {
                    const int32_t jj0 = kj * 32 + tg;
                    if (jj0 >= ns) break;
                    T cf[BLK_PF][BLK_K];
#pragma unroll
                    for (int u = 0; u < BLK_PF; u++) {
                        const int32_t jj = jj0 + u;
                        const int64_t base = __shfl_sync(0xffffffffu, bj[kj], tg + u);
#pragma unroll
                        for (int kk = 0; kk < BLK_K; kk++) {
                            const int32_t ii = kk * 32 + lane;
                            cf[u][kk] = (kk >= kj && ii > jj && ii < ns) ? s.lu[base + ii] : (T)0;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < BLK_PF; u++) {
                        const int32_t jj = jj0 + u;
                        const T vj = __shfl_sync(0xffffffffu, v[kj], tg + u);
                        if (jj < ns) {
#pragma unroll
                            for (int kk = 0; kk < BLK_K; kk++)
                                if (kk >= kj && kk * 32 + lane > jj) v[kk] = v[kk] - cf[u][kk] * vj;
                        }
                    }
                }
            }
        } else {
#pragma unroll
            for (int kj = BLK_K - 1; kj >= 0; kj--) {
                for (int32_t tg = 32 - BLK_PF; tg >= 0; tg -= BLK_PF) {
                    if (kj * 32 + tg >= ns) continue;
                    T cf[BLK_PF][BLK_K];
#pragma unroll
                    for (int u = 0; u < BLK_PF; u++) {
                        const int32_t t = tg + BLK_PF - 1 - u;   // columns descending
                        const int32_t jj = kj * 32 + t;
                        const int64_t base = __shfl_sync(0xffffffffu, bj[kj], t);
#pragma unroll
                        for (int kk = 0; kk < BLK_K; kk++) {
                            const int32_t ii = kk * 32 + lane;
                            cf[u][kk] = (kk <= kj && jj < ns && ii < jj) ? s.lu[base + ii] : (T)0;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < BLK_PF; u++) {
                        const int32_t t = tg + BLK_PF - 1 - u;
                        const int32_t jj = kj * 32 + t;
                        const T zo = v[kj] * d[kj];
                        const T zj = __shfl_sync(0xffffffffu, zo, t);
                        if (jj < ns) {
                            if (lane == t) v[kj] = zj;
#pragma unroll
                            for (int kk = 0; kk < BLK_K; kk++)
                                if (kk <= kj && kk * 32 + lane < jj) v[kk] = v[kk] - cf[u][kk] * zj;
                        }
                    }
                }
            }
        }
        T *out = (bwd ? z : y) + (int64_t)r * n + c0;
#pragma unroll
        for (int k = 0; k < BLK_K; k++)
            if (k * 32 + lane < ns) out[k * 32 + lane] = v[k];
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < BLK_K; k++) {
        const int32_t i = c0 + k * 32 + lane;
        if (k * 32 + lane < ns && i != a.fault_row) st_release(ready + i, a.epoch);
    }
}

template <typename T>
__global__ void __launch_bounds__(128) k_solve_df(const SolveArgs<T> s, const DFSolveArgs a, T *y, T *z, int32_t nrhs) {
    const int lane = threadIdx.x & 31;
    const int n = s.n;
    while (true) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(a.ticket, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= a.nitems) break;
        const DFItem it = a.items[t];
        const bool bwd = it.flags & DF_BACKWARD;
        const int64_t *rptr = bwd ? s.urow_ptr : s.lrow_ptr;
        const int64_t *pos = bwd ? s.urow_pos : s.lrow_pos;
        const int32_t *col = bwd ? s.urow_col : s.lrow_col;
        int32_t *ready = bwd ? a.bready : a.fready;
        const T *src = bwd ? z : y;   // values the dot products read
        if (it.flags & DF_BLOCK) {
            block_item<T>(s, a, it, y, z, nrhs, lane);
            continue;
        }
        int32_t j[DF_PER_LANE];
        T l[DF_PER_LANE];
        if (it.flags & DF_CHUNK) {
            // partial dot product of entries p0..p1-1 of a long row
            const SolveChunk ch = (bwd ? a.bchunks : a.fchunks)[it.chunk];
            T *partial = static_cast<T *>(bwd ? a.bpartial_v : a.fpartial_v);
            load_entries<T>(s, col, pos, ch.p0, ch.p1, lane, j, l);
            wait_cols(ready, j, a.epoch, a);
            for (int32_t r = 0; r < nrhs; r++) {
                const T acc = dot_entries<T>(j, l, src + (int64_t)r * n);
                if (lane == 0) partial[(int64_t)it.chunk * nrhs + r] = acc;
            }
            __syncwarp();
            if (lane == 0) st_release((bwd ? a.bchunk_ready : a.fchunk_ready) + it.chunk, a.epoch);
            continue;
        }
        const int32_t i = it.row;
        // a backward launch follows the forward one and the tail, so its own
        // row's forward value is final; d: the reciprocal of U(i, i)
        T d = (T)1, v0 = (T)0;
        if (lane == 0) {
            if (bwd) d = (T)1 / s.lu[s.diag_pos[i]];
            v0 = ld_cg(y + i);    // c(i) forward, y(i) backward, first side
        }
        if (it.ce > it.cb) {
            // a long row: the sum of its chunks' partials, in chunk order
            const T *partial = static_cast<const T *>(bwd ? a.bpartial_v : a.fpartial_v);
            const int32_t *chunk_ready = bwd ? a.bchunk_ready : a.fchunk_ready;
            for (int32_t c = it.cb + lane; c < it.ce; c += 32)
                if (ld_relaxed(chunk_ready + c) != a.epoch) spin_flag(chunk_ready + c, a.epoch, a);
            fence_acq_rel();
            __syncwarp();
            if (lane == 0) {
                for (int32_t r = 0; r < nrhs; r++) {
                    T acc = (T)0;
                    for (int32_t c = it.cb; c < it.ce; c++) acc += ld_cg(partial + (int64_t)c * nrhs + r);
                    const T v = r == 0 ? v0 : ld_cg(y + (int64_t)r * n + i);
                    (bwd ? z : y)[(int64_t)r * n + i] = bwd ? (v - acc) * d : v - acc;
                }
            }
        } else {
            const int64_t b = rptr[i], e = rptr[i + 1];
            load_entries<T>(s, col, pos, b, e, lane, j, l);
            wait_cols(ready, j, a.epoch, a);
            for (int32_t r = 0; r < nrhs; r++) {
                const T acc = dot_entries<T>(j, l, src + (int64_t)r * n);
                if (lane == 0) {
                    const T v = r == 0 ? v0 : ld_cg(y + (int64_t)r * n + i);
                    (bwd ? z : y)[(int64_t)r * n + i] = bwd ? (v - acc) * d : v - acc;
                }
            }
        }
        __syncwarp();
        if (lane == 0 && i != a.fault_row) st_release(ready + i, a.epoch);
    }
}

// The dense tail, one block, one tail row per thread (at most 1024 rows),
// its running value in a register, columns taken TAIL_TB at a time.  For a
// panel of columns j0..j0+TB-1 the warp owning the panel's rows solves the
// panel's triangle with shuffles (row j0+u is final after the panel's
// columns before u), publishes the values in shared memory, and after one
// barrier every row below subtracts the panel's columns in order.  The
// backward sweep mirrors it (z(jj) = y(jj) times the reciprocal of U(jj, jj),
// taken once per row before the sweeps; rows above, columns descending).
// Each row applies the columns in the same order as a column-at-a-time
// sweep.  The tail column jj's entries are contiguous in the CSC values: the
// block is prefetched into L2 first, and every thread copies its own row's
// coefficients of the next panel into shared memory (cp.async) while the
// current panel runs.
constexpr int TAIL_TB = 8;

__device__ __forceinline__ void cp_async_tail(void *dst, const void *src, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// barrier 1 over the first `threads` threads of the block (whole warps)
__device__ __forceinline__ void tail_bar(int threads) { asm volatile("bar.sync 1, %0;" ::"r"(threads) : "memory"); }

// Row ii's coefficients in the panel at j0 (forward: L(ii, j0+u) for ii > j0+u;
// backward: U(ii, j0+u) for ii < j0+u) into buf[u * NT + ii], one commit group.
template <typename T>
__device__ __forceinline__ void tail_panel_issue(T *buf, const T *lu, const int64_t *colbase, int32_t j0, int32_t NT,
                                                 int32_t ii, bool bwd) {
    if (ii < NT) {
        const int32_t jn = min(TAIL_TB, NT - j0);
#pragma unroll
        for (int u = 0; u < TAIL_TB; u++)
            if (u < jn && (bwd ? ii < j0 + u : ii > j0 + u))
                cp_async_tail(buf + u * NT + ii, lu + colbase[j0 + u] + ii, (int)sizeof(T));
    }
    cp_async_commit();
}

template <typename T>
__global__ void __launch_bounds__(1024) k_solve_tail(const SolveArgs<T> s, const int64_t *__restrict__ lu_colptr,
                                                     const TailArgs ta, const T *__restrict__ fpartial, T *y, T *z,
                                                     int32_t nrhs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int32_t n = s.n, t0 = ta.t0, NT = n - t0;
    int64_t *lcol = reinterpret_cast<int64_t *>(smem_raw);   // L(t0+ii, t0+jj) at lcol[jj] + ii
    int64_t *ucol = lcol + NT;                                // U(t0+ii, t0+jj) at ucol[jj] + ii
    T *bc = reinterpret_cast<T *>(ucol + NT);                 // published values
    T *cf = bc + NT;                                          // [2][TAIL_TB][NT]: panel coefficients
    const int32_t ii = threadIdx.x, nwarp = blockDim.x >> 5;
    const bool own = ii < NT;
    for (int32_t q = ii; q < NT; q += blockDim.x) {
        lcol[q] = s.diag_pos[t0 + q] - q;
        ucol[q] = lu_colptr[t0 + q + 1] - NT;
    }
    __syncthreads();
    // the tail block's values (NT contiguous entries per column) into L2
    // ahead of the panels, kept there over the streaming sweeps
    {
        const int32_t lines = (int32_t)(((int64_t)NT * sizeof(T) + 127) / 128) + 1;
        for (int64_t q = ii; q < (int64_t)NT * lines; q += blockDim.x) {
            const int32_t j = (int32_t)(q / lines), k = (int32_t)(q - (int64_t)j * lines);
            const char *p0 = reinterpret_cast<const char *>(s.lu + lcol[j]);
            const char *pl = p0 + (int64_t)k * 128;
            if (pl < reinterpret_cast<const char *>(s.lu + lcol[j] + NT))
                asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(pl));
        }
    }
    // the reciprocal of the row's diagonal, taken once off the panels' chains
    const T rd = own ? (T)1 / s.lu[lcol[ii] + ii] : (T)1;
    const int32_t npanel = (NT + TAIL_TB - 1) / TAIL_TB;
    for (int32_t r = 0; r < nrhs; r++) {
        T v = (T)0;
        if (own) {
            v = __ldcg(y + (int64_t)r * n + t0 + ii);
            // the row's chunk partial sums, in chunk order, eight loads in flight
            for (int32_t c = ta.cb[ii]; c < ta.ce[ii]; c += 8) {
                T pv[8];
#pragma unroll
                for (int u = 0; u < 8; u++)
                    pv[u] = c + u < ta.ce[ii] ? __ldcg(fpartial + (int64_t)(c + u) * nrhs + r) : (T)0;
#pragma unroll
                for (int u = 0; u < 8; u++)
                    if (c + u < ta.ce[ii]) v -= pv[u];
            }
        }
        // forward, panels j0 = 0, TB, 2TB, ... (a panel's rows lie in one
        // warp); a warp whose rows all lie above the panel is done with the
        // sweep and leaves it, the others meet at a barrier sized to them
        const int32_t w = ii >> 5;
        tail_panel_issue<T>(cf, s.lu, lcol, 0, NT, ii, false);
        for (int32_t p = 0; p < npanel; p++) {
            const int32_t j0 = p * TAIL_TB, jn = min(TAIL_TB, NT - j0);
            if (w < (j0 >> 5)) {
                cp_async_wait_all();
                break;
            }
            T *cur = cf + (p & 1) * TAIL_TB * NT;
            if (p + 1 < npanel) {
                tail_panel_issue<T>(cf + ((p + 1) & 1) * TAIL_TB * NT, s.lu, lcol, j0 + TAIL_TB, NT, ii, false);
                cp_async_wait_prev();
            } else {
                cp_async_wait_all();
            }
            T lv[TAIL_TB];
#pragma unroll
            for (int u = 0; u < TAIL_TB; u++) lv[u] = (own && u < jn && ii > j0 + u) ? cur[u * NT + ii] : (T)0;
            if (w == (j0 >> 5)) {
                const int base = j0 & 31;
                const bool inside = own && ii >= j0 && ii < j0 + jn;
#pragma unroll
                for (int u = 0; u < TAIL_TB; u++) {
                    if (u < jn) {
                        const T vu = __shfl_sync(0xffffffffu, v, base + u);
                        if (inside && ii > j0 + u) v = v - lv[u] * vu;
                    }
                }
                if (inside) bc[ii] = v;
            }
            tail_bar((nwarp - (j0 >> 5)) * 32);
            if (own && ii >= j0 + jn) {
#pragma unroll
                for (int u = 0; u < TAIL_TB; u++)
                    if (u < jn) v = v - lv[u] * bc[j0 + u];
            }
        }
        __syncthreads();
        // backward, panels from the last (aligned) one down; a warp whose rows
        // all lie below the panel is done
        T *zr = z + (int64_t)r * n;
        tail_panel_issue<T>(cf, s.lu, ucol, (npanel - 1) * TAIL_TB, NT, ii, true);
        for (int32_t p = npanel - 1, k = 0; p >= 0; p--, k++) {
            const int32_t j0 = p * TAIL_TB, jn = min(TAIL_TB, NT - j0);
            const int32_t wlast = (j0 + jn - 1) >> 5;
            if (w > wlast) {
                cp_async_wait_all();
                break;
            }
            T *cur = cf + (k & 1) * TAIL_TB * NT;
            if (p > 0) {
                tail_panel_issue<T>(cf + ((k + 1) & 1) * TAIL_TB * NT, s.lu, ucol, j0 - TAIL_TB, NT, ii, true);
                cp_async_wait_prev();
            } else {
                cp_async_wait_all();
            }
            T lv[TAIL_TB];
#pragma unroll
            for (int u = 0; u < TAIL_TB; u++) lv[u] = (own && u < jn && ii < j0 + u) ? cur[u * NT + ii] : (T)0;
            if (w == (j0 >> 5)) {
                const int base = j0 & 31;
                const bool inside = own && ii >= j0 && ii < j0 + jn;
#pragma unroll
                for (int u = TAIL_TB - 1; u >= 0; u--) {
                    if (u < jn) {
                        if (inside && ii == j0 + u) v = v * rd;
                        const T zu = __shfl_sync(0xffffffffu, v, base + u);
                        if (inside && ii < j0 + u) v = v - lv[u] * zu;
                    }
                }
                if (inside) {
                    bc[ii] = v;
                    zr[t0 + ii] = v;
                }
            }
            tail_bar((wlast + 1) * 32);
            if (own && ii < j0) {
#pragma unroll
                for (int u = TAIL_TB - 1; u >= 0; u--)
                    if (u < jn) v = v - lv[u] * bc[j0 + u];
            }
        }
        __syncthreads();
    }
    if (own) ta.bready[t0 + ii] = ta.epoch;
}

}  // namespace

template <typename T>
cudaError_t launch_solve_tail(const SolveArgs<T> &s, const int64_t *lu_colptr, const TailArgs &t, const T *fpartial,
                              T *y, T *z, int32_t nrhs, cudaStream_t st) {
    const int32_t NT = s.n - t.t0;
    if (NT <= 0) return cudaSuccess;
    if (NT > 1024) return cudaErrorInvalidValue;
    const size_t smem = 2 * (size_t)NT * sizeof(int64_t) + (size_t)NT * (1 + 2 * TAIL_TB) * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k_solve_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // one thread per tail row, whole warps
    k_solve_tail<T><<<1, (unsigned)((NT + 31) / 32 * 32), smem, st>>>(s, lu_colptr, t, fpartial, y, z, nrhs);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_df(const SolveArgs<T> &s, const DFSolveArgs &a, T *y, T *z, int32_t nrhs, int num_sms,
                            cudaStream_t st) {
    if (a.nitems == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(a.ticket, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(a.abort, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    int64_t blocks = ((int64_t)a.nitems * 32 + 127) / 128;
    const int64_t cap = (int64_t)num_sms * 8;
    if (blocks > cap) blocks = cap;
    k_solve_df<T><<<(unsigned)blocks, 128, 0, st>>>(s, a, y, z, nrhs);
    return cudaGetLastError();
}

template cudaError_t launch_solve_tail<double>(const SolveArgs<double> &, const int64_t *, const TailArgs &,
                                               const double *, double *, double *, int32_t, cudaStream_t);
template cudaError_t launch_solve_tail<float>(const SolveArgs<float> &, const int64_t *, const TailArgs &,
                                              const float *, float *, float *, int32_t, cudaStream_t);
template cudaError_t launch_solve_df<double>(const SolveArgs<double> &, const DFSolveArgs &, double *, double *,
                                             int32_t, int, cudaStream_t);
template cudaError_t launch_solve_df<float>(const SolveArgs<float> &, const DFSolveArgs &, float *, float *, int32_t,
                                            int, cudaStream_t);

}  // namespace glu
