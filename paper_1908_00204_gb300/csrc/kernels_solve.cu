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

template <typename T>
__global__ void k_lsolve_level(const SolveArgs<T> a, T *y, int32_t nrhs, const int32_t *__restrict__ rows,
                               int32_t nrows) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nrows) return;
    const int32_t i = rows[w];
    const int64_t b = a.lrow_ptr[i], e = a.lrow_ptr[i + 1];
    for (int32_t r = 0; r < nrhs; r++) {
        T *yr = y + (int64_t)r * a.n;
        T s = (T)0;
        for (int64_t p = b + lane; p < e; p += 32) s += a.lu[a.lrow_pos[p]] * yr[a.lrow_col[p]];
        s = warp_sum(s);
        if (lane == 0) yr[i] = yr[i] - s;
    }
}

template <typename T>
__global__ void k_usolve_level(const SolveArgs<T> a, T *y, int32_t nrhs, const int32_t *__restrict__ rows,
                               int32_t nrows) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nrows) return;
    const int32_t i = rows[w];
    const int64_t b = a.urow_ptr[i], e = a.urow_ptr[i + 1];
    const T d = a.lu[a.diag_pos[i]];
    for (int32_t r = 0; r < nrhs; r++) {
        T *yr = y + (int64_t)r * a.n;
        T s = (T)0;
        for (int64_t p = b + lane; p < e; p += 32) s += a.lu[a.urow_pos[p]] * yr[a.urow_col[p]];
        s = warp_sum(s);
        if (lane == 0) yr[i] = (yr[i] - s) / d;
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
cudaError_t launch_lsolve_level(const SolveArgs<T> &a, T *y, int32_t nrhs, const int32_t *rows, int32_t nrows,
                                cudaStream_t s) {
    if (nrows == 0) return cudaSuccess;
    k_lsolve_level<T><<<(unsigned)(((int64_t)nrows * 32 + 127) / 128), 128, 0, s>>>(a, y, nrhs, rows, nrows);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_usolve_level(const SolveArgs<T> &a, T *y, int32_t nrhs, const int32_t *rows, int32_t nrows,
                                cudaStream_t s) {
    if (nrows == 0) return cudaSuccess;
    k_usolve_level<T><<<(unsigned)(((int64_t)nrows * 32 + 127) / 128), 128, 0, s>>>(a, y, nrhs, rows, nrows);
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
template cudaError_t launch_lsolve_level<double>(const SolveArgs<double> &, double *, int32_t, const int32_t *,
                                                 int32_t, cudaStream_t);
template cudaError_t launch_lsolve_level<float>(const SolveArgs<float> &, float *, int32_t, const int32_t *,
                                                int32_t, cudaStream_t);
template cudaError_t launch_usolve_level<double>(const SolveArgs<double> &, double *, int32_t, const int32_t *,
                                                 int32_t, cudaStream_t);
template cudaError_t launch_usolve_level<float>(const SolveArgs<float> &, float *, int32_t, const int32_t *,
                                                int32_t, cudaStream_t);

}  // namespace glu
