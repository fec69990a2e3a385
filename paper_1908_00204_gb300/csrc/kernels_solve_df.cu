// kernels_solve_df.cu -- dataflow ("sync-free") triangular solves (sm_103a).
//
// The two triangular systems of Section I, forward (unit L) then backward
// (U), in one launch.  Work items -- a row, or a chunk of a long row's dot
// product -- are listed in a topological order (each item after everything it
// reads) and handed out by an atomic ticket, so a warp waits only on items
// that running warps already hold: no level barriers, no co-residency
// assumption.  A finished row publishes a flag with release semantics; a
// reader acquires it before loading the value.  Flags hold the call's epoch,
// so they need no reset between calls.  Every wait is bounded: past the limit
// the kernel records GLU_ERR_TIMEOUT, raises an abort flag that ends all other
// waits, publishes its own result and carries on, so the launch always ends.
// The backward sweep writes its own vector z: with an unsymmetric pattern a
// backward row can be ready while a forward row still reads the forward value
// of that row, so the two sweeps must not share storage.
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
        if (it.flags & DF_CHUNK) {
            // partial dot product of entries p0..p1-1 of a long row
            const SolveChunk ch = (bwd ? a.bchunks : a.fchunks)[it.chunk];
            T *partial = static_cast<T *>(bwd ? a.bpartial_v : a.fpartial_v);
            for (int32_t r = 0; r < nrhs; r++) {
                const T *yr = (bwd ? z : y) + (int64_t)r * n;
                T acc = (T)0;
                for (int64_t p = ch.p0 + lane; p < ch.p1; p += 32) {
                    const int32_t j = col[p];
                    if (r == 0) wait_flag(ready + j, a.epoch, a);
                    acc += s.lu[pos[p]] * ld_cg(yr + j);
                }
                acc = warp_sum_df(acc);
                if (lane == 0) partial[(int64_t)it.chunk * nrhs + r] = acc;
            }
            __syncwarp();
            if (lane == 0) st_release((bwd ? a.bchunk_ready : a.fchunk_ready) + it.chunk, a.epoch);
            continue;
        }
        const int32_t i = it.row;
        // the backward row needs the forward result of its own row
        if (bwd && lane == 0) wait_flag(a.fready + i, a.epoch, a);
        __syncwarp();
        const T d = bwd ? s.lu[s.diag_pos[i]] : (T)1;
        const T *partial = static_cast<const T *>(bwd ? a.bpartial_v : a.fpartial_v);
        const int32_t *chunk_ready = bwd ? a.bchunk_ready : a.fchunk_ready;
        if (it.ce > it.cb && lane == 0)
            for (int32_t c = it.cb; c < it.ce; c++) wait_flag(chunk_ready + c, a.epoch, a);
        const int64_t b = rptr[i], e = rptr[i + 1];
        for (int32_t r = 0; r < nrhs; r++) {
            const T *yr = (bwd ? z : y) + (int64_t)r * n;   // values the row reads
            T *out = (bwd ? z : y) + (int64_t)r * n;
            T acc = (T)0;
            if (it.ce > it.cb) {
                if (lane == 0)
                    for (int32_t c = it.cb; c < it.ce; c++) acc += ld_cg(partial + (int64_t)c * nrhs + r);
            } else {
                for (int64_t p = b + lane; p < e; p += 32) {
                    const int32_t j = col[p];
                    if (r == 0) wait_flag(ready + j, a.epoch, a);
                    acc += s.lu[pos[p]] * ld_cg(yr + j);
                }
                acc = warp_sum_df(acc);
            }
            if (lane == 0) {
                const T v = ld_cg(y + (int64_t)r * n + i);   // c(i) forward, y(i) backward
                out[i] = bwd ? (v - acc) / d : v - acc;
            }
        }
        __syncwarp();
        if (lane == 0 && i != a.fault_row) st_release(ready + i, a.epoch);
    }
}

// The dense tail, one block.  Tail column j's rows below (and, in U, above
// from t0) are contiguous in the CSC values, so a column sweep reads them
// coalesced; the tail's values stay in shared memory; one barrier per column
// forward, two backward (the pivot division is done once).
template <typename T>
__global__ void __launch_bounds__(1024) k_solve_tail(const SolveArgs<T> s, const int64_t *__restrict__ lu_colptr,
                                                     const TailArgs ta, const T *__restrict__ fpartial, T *y, T *z,
                                                     int32_t nrhs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int32_t n = s.n, t0 = ta.t0, NT = n - t0;
    T *yt = reinterpret_cast<T *>(smem_raw);
    T *zt = yt + NT;
    for (int32_t r = 0; r < nrhs; r++) {
        const T *yr = y + (int64_t)r * n;
        T *zr = z + (int64_t)r * n;
        for (int32_t ii = threadIdx.x; ii < NT; ii += blockDim.x) {
            T v = __ldcg(yr + t0 + ii);
            for (int32_t c = ta.cb[ii]; c < ta.ce[ii]; c++) v -= __ldcg(fpartial + (int64_t)c * nrhs + r);
            yt[ii] = v;
        }
        __syncthreads();
        // forward: y(i) -= L(i,j) y(j) for the rows i > j of the tail
        for (int32_t jj = 0; jj < NT; jj++) {
            const int64_t lb = s.diag_pos[t0 + jj] + 1 - (jj + 1);   // L(t0+ii, t0+jj) at lb + ii
            const T vj = yt[jj];
            for (int32_t ii = jj + 1 + threadIdx.x; ii < NT; ii += blockDim.x)
                yt[ii] = yt[ii] - s.lu[lb + ii] * vj;
            __syncthreads();
        }
        // backward: z(j) = y(j) / U(j,j); y(i) -= U(i,j) z(j) for the rows t0 <= i < j
        for (int32_t jj = NT - 1; jj >= 0; jj--) {
            const int32_t j = t0 + jj;
            if (threadIdx.x == 0) zt[jj] = yt[jj] / s.lu[s.diag_pos[j]];
            __syncthreads();
            const int64_t ub = lu_colptr[j + 1] - NT;                 // U(t0+ii, j) at ub + ii
            const T zj = zt[jj];
            for (int32_t ii = threadIdx.x; ii < jj; ii += blockDim.x) yt[ii] = yt[ii] - s.lu[ub + ii] * zj;
            __syncthreads();
        }
        for (int32_t ii = threadIdx.x; ii < NT; ii += blockDim.x) zr[t0 + ii] = zt[ii];
        __syncthreads();
    }
    for (int32_t ii = threadIdx.x; ii < NT; ii += blockDim.x) ta.bready[t0 + ii] = ta.epoch;
}

}  // namespace

template <typename T>
cudaError_t launch_solve_tail(const SolveArgs<T> &s, const int64_t *lu_colptr, const TailArgs &t, const T *fpartial,
                              T *y, T *z, int32_t nrhs, cudaStream_t st) {
    const int32_t NT = s.n - t.t0;
    if (NT <= 0) return cudaSuccess;
    const size_t smem = 2 * (size_t)NT * sizeof(T);
    k_solve_tail<T><<<1, 1024, smem, st>>>(s, lu_colptr, t, fpartial, y, z, nrhs);
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
