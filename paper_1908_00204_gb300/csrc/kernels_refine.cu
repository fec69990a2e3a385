// kernels_refine.cu -- FP64 pieces of mixed-precision iterative refinement.
//
// The factors are FP32; the residual r = b - A x, its norms and the update
// x += d stay in FP64 on the GPU.  Norm maxima use the bit pattern of
// non-negative doubles, which orders like the values, so an integer maximum
// (within a block by shuffles, across blocks by one atomicMax each) is exact
// and independent of order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "glu_device.cuh"

namespace glu {
namespace {

__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(fabs(v));
}

__device__ __forceinline__ double as_double(unsigned long long u) { return __longlong_as_double((long long)u); }

// The block's maximum of m (bit patterns of non-negative doubles) into *slot:
// shuffles within each warp, then shared memory, one atomic per block.
__device__ __forceinline__ void block_max(unsigned long long *slot, unsigned long long m) {
    __shared__ unsigned long long wmax[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, m, o);
        m = u > m ? u : m;
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) wmax[w] = m;
    __syncthreads();
    if (w == 0) {
        m = lane < (int)(blockDim.x >> 5) ? wmax[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long u = __shfl_xor_sync(0xffffffffu, m, o);
            m = u > m ? u : m;
        }
        if (lane == 0 && m) atomicMax(slot, m);
    }
    __syncthreads();   // wmax is reused by the next call
}

// A's values in compressed-row order (gathered once per factorization).
__global__ void k_csr_values(double *__restrict__ out, const double *__restrict__ aval,
                             const int64_t *__restrict__ src, int64_t nnz) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = aval[src[q]];
}

// ||A||_inf = max over rows of sum |a_ij|.
__global__ void k_anorm(const int64_t *__restrict__ rp, const double *__restrict__ av, int32_t n,
                        unsigned long long *anorm) {
    unsigned long long m = 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; p++) s += fabs(av[p]);
        const unsigned long long u = abs_bits(s);
        m = u > m ? u : m;
    }
    block_max(anorm, m);
}

// r = b - A x for right-hand side k = blockIdx.y; also max |r| and max |x|.
__global__ void k_residual(const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ av, const double *__restrict__ b, const double *__restrict__ x,
                           double *__restrict__ r, int32_t n, unsigned long long *rmax, unsigned long long *xmax) {
    const int32_t k = blockIdx.y;
    const double *xk = x + (int64_t)k * n;
    unsigned long long mr = 0, mx = 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; p++) s = fma(av[p], xk[ci[p]], s);
        const int64_t t = (int64_t)k * n + i;
        const double v = b[t] - s;
        r[t] = v;
        const unsigned long long ur = abs_bits(v), ux = abs_bits(xk[i]);
        mr = ur > mr ? ur : mr;
        mx = ux > mx ? ux : mx;
    }
    block_max(rmax + k, mr);
    block_max(xmax + k, mx);
}

__global__ void k_absmax(const double *__restrict__ v, int32_t n, unsigned long long *out) {
    const int32_t k = blockIdx.y;
    unsigned long long m = 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned long long u = abs_bits(v[(int64_t)k * n + i]);
        m = u > m ? u : m;
    }
    block_max(out + k, m);
}

// Normwise backward error per side, ||r|| / (||A|| ||x|| + ||b||); a side is
// done once it is at or below tol.  ndone counts the sides done.
__global__ void k_check(const unsigned long long *rmax, const unsigned long long *xmax,
                        const unsigned long long *bmax, const unsigned long long *anorm, int32_t nrhs, double tol,
                        int32_t *done, double *berr, int32_t *ndone) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrhs) return;
    const double den = as_double(*anorm) * as_double(xmax[k]) + as_double(bmax[k]);
    const double e = den > 0.0 ? as_double(rmax[k]) / den : 0.0;
    berr[k] = e;
    const int d = (e <= tol) ? 1 : 0;
    done[k] = d;
    if (d) atomicAdd(ndone, 1);
}

// x += d on the sides not done yet.
__global__ void k_update(double *__restrict__ x, const double *__restrict__ d, const int32_t *__restrict__ done,
                         int32_t n, int32_t nrhs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * nrhs) return;
    if (!done[t / n]) x[t] += d[t];
}

unsigned blocks_for(int64_t work) {
    int64_t b = (work + 255) / 256;
    return (unsigned)(b < 1 ? 1 : b);
}

// row-parallel reductions: at most eight blocks per SM in all
unsigned row_blocks(int32_t n, int32_t nrhs) {
    int64_t b = ((int64_t)n + 255) / 256;
    const int64_t cap = std::max<int64_t>(1, (int64_t)152 * 8 / std::max<int32_t>(nrhs, 1));
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_csr_values(double *out, const double *aval, const int64_t *src, int64_t nnz, cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    int64_t b = (nnz + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    k_csr_values<<<(unsigned)b, 256, 0, s>>>(out, aval, src, nnz);
    return cudaGetLastError();
}

cudaError_t launch_anorm(const int64_t *rp, const double *av, int32_t n, unsigned long long *anorm, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_anorm<<<row_blocks(n, 1), 256, 0, s>>>(rp, av, n, anorm);
    return cudaGetLastError();
}

cudaError_t launch_residual(const int64_t *rp, const int32_t *ci, const double *av, const double *b, const double *x,
                            double *r, int32_t n, int32_t nrhs, unsigned long long *rmax, unsigned long long *xmax,
                            cudaStream_t s) {
    if ((int64_t)n * nrhs == 0) return cudaSuccess;
    k_residual<<<dim3(row_blocks(n, nrhs), (unsigned)nrhs), 256, 0, s>>>(rp, ci, av, b, x, r, n, rmax, xmax);
    return cudaGetLastError();
}

cudaError_t launch_absmax(const double *v, int32_t n, int32_t nrhs, unsigned long long *out, cudaStream_t s) {
    if ((int64_t)n * nrhs == 0) return cudaSuccess;
    k_absmax<<<dim3(row_blocks(n, nrhs), (unsigned)nrhs), 256, 0, s>>>(v, n, out);
    return cudaGetLastError();
}

cudaError_t launch_check(const unsigned long long *rmax, const unsigned long long *xmax,
                         const unsigned long long *bmax, const unsigned long long *anorm, int32_t nrhs, double tol,
                         int32_t *done, double *berr, int32_t *ndone, cudaStream_t s) {
    k_check<<<(nrhs + 127) / 128, 128, 0, s>>>(rmax, xmax, bmax, anorm, nrhs, tol, done, berr, ndone);
    return cudaGetLastError();
}

cudaError_t launch_update(double *x, const double *d, const int32_t *done, int32_t n, int32_t nrhs, cudaStream_t s) {
    const int64_t w = (int64_t)n * nrhs;
    if (w == 0) return cudaSuccess;
    k_update<<<blocks_for(w), 256, 0, s>>>(x, d, done, n, nrhs);
    return cudaGetLastError();
}

}  // namespace glu
