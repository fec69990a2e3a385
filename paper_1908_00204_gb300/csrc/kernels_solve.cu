// kernels_solve.cu -- level-scheduled triangular solves (sm_103a).
//
// x follows from the two triangular systems (Section I): c = P b; L y = c
// with unit L (forward); U z = y (backward); x = P^T z.  Both sweeps pull
// along rows: row i of a level reads only rows of earlier levels, so the
// rows of one level run in parallel, one warp per row and right-hand side
// loop inside; the sum over a row is a fixed-order warp reduction, so the
// result is the same run to run.
#include <cuda_runtime.h>

#include <cstdint>

#include "glu_device.cuh"

namespace glu {
namespace {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__global__ void k_permute_in(T *__restrict__ y, const double *__restrict__ b, const int32_t *__restrict__ perm,
                             int32_t n, int32_t nrhs) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)n * nrhs;
    for (; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = i / n, row = i - r * n;
        y[i] = (T)b[r * n + perm[row]];
    }
}

template <typename T>
__global__ void k_permute_out(double *__restrict__ x, const T *__restrict__ y, const int32_t *__restrict__ perm,
                              int32_t n, int32_t nrhs) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)n * nrhs;
    for (; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = i / n, row = i - r * n;
        x[r * n + perm[row]] = (double)y[i];
    }
}

constexpr int SOLVE_UNROLL = 4;

// sum over entries p0..p1-1 of val[pos[p]] * y[col[p]], lanes strided,
// SOLVE_UNROLL independent loads in flight per lane; fixed-order warp sum.
template <typename T>
__device__ __forceinline__ T row_dot(const T *__restrict__ lu, const int64_t *__restrict__ pos,
                                     const int32_t *__restrict__ col, const T *__restrict__ y, int64_t p0, int64_t p1,
                                     int lane) {
    T s = (T)0;
    for (int64_t pb = p0 + lane; pb < p1; pb += 32 * SOLVE_UNROLL) {
        int64_t ps[SOLVE_UNROLL];
        int32_t cs[SOLVE_UNROLL];
#pragma unroll
        for (int u = 0; u < SOLVE_UNROLL; u++) {
            const int64_t p = pb + 32 * u;
            if (p < p1) {
                ps[u] = pos[p];
                cs[u] = col[p];
            }
        }
#pragma unroll
        for (int u = 0; u < SOLVE_UNROLL; u++)
            if (pb + 32 * u < p1) s += lu[ps[u]] * y[cs[u]];
    }
    return warp_sum(s);
}

// Partial dot products of the long rows of one level.
template <typename T>
__global__ void k_solve_chunks(const T *__restrict__ lu, const int64_t *__restrict__ pos,
                               const int32_t *__restrict__ col, const SolveChunk *__restrict__ chunks, int32_t c0,
                               int32_t c1, const T *y, int32_t n, int32_t nrhs, T *__restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t c = c0 + w;
    if (c >= c1) return;
    const SolveChunk ch = chunks[c];
    for (int32_t r = 0; r < nrhs; r++) {
        const T s = row_dot<T>(lu, pos, col, y + (int64_t)r * n, ch.p0, ch.p1, lane);
        if (lane == 0) partial[c * nrhs + r] = s;
    }
}

// One level: y[i] = (y[i] - sum_j M(i,j) y[j]) * scale, one warp per row;
// long rows add up their partials in chunk order.  Forward: unit diagonal;
// backward: divide by the pivot.
template <typename T, bool BACKWARD>
__global__ void k_solve_level(const SolveArgs<T> a, T *y, int32_t nrhs, const SolveRow *__restrict__ items,
                              int32_t nitems, const T *__restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nitems) return;
    const SolveRow it = items[w];
    const int32_t i = it.row;
    const int64_t *rptr = BACKWARD ? a.urow_ptr : a.lrow_ptr;
    const int64_t *pos = BACKWARD ? a.urow_pos : a.lrow_pos;
    const int32_t *col = BACKWARD ? a.urow_col : a.lrow_col;
    const T d = BACKWARD ? (T)1 / a.lu[a.diag_pos[i]] : (T)1;   // the reciprocal of U(i, i)
    for (int32_t r = 0; r < nrhs; r++) {
        T *yr = y + (int64_t)r * a.n;
        T s;
        if (it.ce > it.cb) {
            s = (T)0;
            if (lane == 0)
                for (int32_t c = it.cb; c < it.ce; c++) s += partial[(int64_t)c * nrhs + r];
        } else {
            s = row_dot<T>(a.lu, pos, col, yr, rptr[i], rptr[i + 1], lane);
        }
        if (lane == 0) yr[i] = BACKWARD ? (yr[i] - s) * d : yr[i] - s;
    }
}

unsigned grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

template <typename T>
cudaError_t launch_permute_in(T *y, const double *b, const int32_t *perm, int32_t n, int32_t nrhs, cudaStream_t s) {
    if ((int64_t)n * nrhs == 0) return cudaSuccess;
    k_permute_in<T><<<grid_for((int64_t)n * nrhs, 256), 256, 0, s>>>(y, b, perm, n, nrhs);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_permute_out(double *x, const T *y, const int32_t *perm, int32_t n, int32_t nrhs,
                               cudaStream_t s) {
    if ((int64_t)n * nrhs == 0) return cudaSuccess;
    k_permute_out<T><<<grid_for((int64_t)n * nrhs, 256), 256, 0, s>>>(x, y, perm, n, nrhs);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_level(const SolveArgs<T> &a, bool backward, T *y, int32_t nrhs, const SolveRow *items,
                               int32_t nitems, const SolveChunk *chunks, int32_t c0, int32_t c1, T *partial,
                               cudaStream_t s, int *launched) {
    *launched = 0;
    if (c1 > c0) {
        const int64_t threads = (int64_t)(c1 - c0) * 32;
        k_solve_chunks<T><<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(
            a.lu, backward ? a.urow_pos : a.lrow_pos, backward ? a.urow_col : a.lrow_col, chunks, c0, c1, y, a.n,
            nrhs, partial);
        (*launched)++;
    }
    if (nitems > 0) {
        const unsigned blocks = (unsigned)(((int64_t)nitems * 32 + 127) / 128);
        if (backward) k_solve_level<T, true><<<blocks, 128, 0, s>>>(a, y, nrhs, items, nitems, partial);
        else k_solve_level<T, false><<<blocks, 128, 0, s>>>(a, y, nrhs, items, nitems, partial);
        (*launched)++;
    }
    return cudaGetLastError();
}

template cudaError_t launch_permute_in<double>(double *, const double *, const int32_t *, int32_t, int32_t,
                                               cudaStream_t);
template cudaError_t launch_permute_in<float>(float *, const double *, const int32_t *, int32_t, int32_t,
                                              cudaStream_t);
template cudaError_t launch_permute_out<double>(double *, const double *, const int32_t *, int32_t, int32_t,
                                                cudaStream_t);
template cudaError_t launch_permute_out<float>(double *, const float *, const int32_t *, int32_t, int32_t,
                                               cudaStream_t);
template cudaError_t launch_solve_level<double>(const SolveArgs<double> &, bool, double *, int32_t,
                                                const SolveRow *, int32_t, const SolveChunk *, int32_t, int32_t,
                                                double *, cudaStream_t, int *);
template cudaError_t launch_solve_level<float>(const SolveArgs<float> &, bool, float *, int32_t, const SolveRow *,
                                               int32_t, const SolveChunk *, int32_t, int32_t, float *, cudaStream_t,
                                               int *);

}  // namespace glu
