// kernels_dense.cu -- the dense trailing block of the factorization.
//
// Under a nested-dissection order the last separator (and the supply nets)
// fill in completely: the trailing columns [t0, n) form a dense block in
// which each column depends on the one before it, so the level sweep would
// spend one level -- one launch -- per column there.  The analysis accepts
// the block only when no column before t0 sits in a level at or after
// level(t0); once the levels before level(t0) and the normalizations of
// level(t0) have run, every update from outside the block has been applied
// and what remains is the dense LU, without pivoting, of the block itself
// (Algorithm 2 restricted to it).  It runs here as one cooperative launch,
// a right-looking blocked LU with panels of nb columns and three phases per
// panel, separated by grid barriers:
//   A  block 0 factors the panel (rows c0..nt-1, columns c0..c1-1) in
//      shared memory, one thread per row;
//   B  every block computes U12 = L11^-1 A12, one warp per column;
//   C  every block updates A22 -= L21 U12 in 32 x 64 tiles.
// The values stay in place in the CSC factor storage.  Data written by one
// block is read by others after a grid barrier, so every read of the factor
// values bypasses L1 (ld.global.cg).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "glu_device.cuh"

namespace glu {
namespace {

constexpr int DT_THREADS = 512;
constexpr int DT_TM = 32, DT_TN = 64, DT_TNP = DT_TN + 1;
constexpr size_t DT_PANEL_BYTES = 200 * 1024;   // shared memory for the panel

template <typename T>
__device__ __forceinline__ T *dcol(T *lu, const DenseTailArgs &d, int32_t k) {
    return lu + (__ldg(d.colptr + d.t0 + k + 1) - d.nt);
}

template <typename T>
__global__ void __launch_bounds__(DT_THREADS) k_dense_tail(T *lu, const DenseTailArgs d, int32_t nb,
                                                           GridBarrier bar) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    __shared__ int s_stop;
    const int32_t nt = d.nt;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    constexpr int NWB = DT_THREADS / 32;
    unsigned arrivals = 0;
    for (int32_t c0 = 0; c0 < nt; c0 += nb) {
        const int32_t w = min(nb, nt - c0), c1 = c0 + w, rows = nt - c0;
        // ---- A: the panel, in shared memory as [column][row - c0]
        if (blockIdx.x == 0) {
            for (int32_t idx = tid; idx < rows * w; idx += DT_THREADS) {
                const int32_t c = idx / rows, r = idx - c * rows;
                sm[idx] = __ldcg(dcol(lu, d, c0 + c) + c0 + r);
            }
            __syncthreads();
            for (int32_t c = 0; c < w; c++) {
                const T *pc = sm + (int64_t)c * rows;
                const T piv = pc[c];
                // row r > c: L(r, c) = A(r, c) / A(c, c), then the rest of
                // the panel's row r loses L(r, c) U(c, cc); row c is final
                for (int32_t r = c + 1 + tid; r < rows; r += DT_THREADS) {
                    const T l = sm[(int64_t)c * rows + r] / piv;
                    sm[(int64_t)c * rows + r] = l;
                    for (int32_t cc = c + 1; cc < w; cc++) {
                        T *p = sm + (int64_t)cc * rows;
                        p[r] = p[r] - l * p[c];
                    }
                }
                __syncthreads();
            }
            for (int32_t idx = tid; idx < rows * w; idx += DT_THREADS) {
                const int32_t c = idx / rows, r = idx - c * rows;
                dcol(lu, d, c0 + c)[c0 + r] = sm[idx];
            }
        }
        arrivals += gridDim.x;
        if (!grid_sync(bar, arrivals, &s_stop)) return;
        if (c1 >= nt) break;
        // ---- B: U12 = L11^-1 A12 (unit lower L11), one warp per column
        for (int32_t idx = tid; idx < w * w; idx += DT_THREADS) {
            const int32_t c = idx / w, r = idx - c * w;
            sm[c * 32 + r] = __ldcg(dcol(lu, d, c0 + c) + c0 + r);
        }
        __syncthreads();
        for (int32_t k = c1 + (int32_t)blockIdx.x * NWB + wib; k < nt; k += (int32_t)gridDim.x * NWB) {
            T *col = dcol(lu, d, k) + c0;
            T x = lane < w ? __ldcg(col + lane) : T(0);
            for (int32_t c = 0; c + 1 < w; c++) {
                const T xc = __shfl_sync(0xffffffffu, x, c);
                if (lane > c && lane < w) x = x - sm[c * 32 + lane] * xc;
            }
            if (lane < w) col[lane] = x;
        }
        arrivals += gridDim.x;
        if (!grid_sync(bar, arrivals, &s_stop)) return;
        // ---- C: A22 -= L21 U12, tiles of DT_TM rows x DT_TN columns
        {
            const int32_t m = nt - c1;
            const int32_t ntr = (m + DT_TM - 1) / DT_TM, ntc = (m + DT_TN - 1) / DT_TN;
            T *Ls = sm;                    // [w][DT_TM]
            T *Us = sm + 32 * DT_TM;       // [w][DT_TNP]
            const int32_t r = tid % DT_TM, cg = tid / DT_TM;   // cg: 0..15, one per warp
            for (int32_t t = blockIdx.x; t < ntr * ntc; t += gridDim.x) {
                const int32_t r0 = c1 + (t % ntr) * DT_TM, k0 = c1 + (t / ntr) * DT_TN;
                __syncthreads();
                for (int32_t idx = tid; idx < w * DT_TM; idx += DT_THREADS) {
                    const int32_t c = idx / DT_TM, rr = idx - c * DT_TM;
                    Ls[c * DT_TM + rr] = (r0 + rr < nt) ? __ldcg(dcol(lu, d, c0 + c) + r0 + rr) : T(0);
                }
                for (int32_t idx = tid; idx < w * DT_TN; idx += DT_THREADS) {
                    const int32_t kk = idx / w, c = idx - kk * w;
                    Us[c * DT_TNP + kk] = (k0 + kk < nt) ? __ldcg(dcol(lu, d, k0 + kk) + c0 + c) : T(0);
                }
                __syncthreads();
                T acc[DT_TN / 16];
#pragma unroll
                for (int j = 0; j < DT_TN / 16; j++) acc[j] = T(0);
                for (int32_t c = 0; c < w; c++) {
                    const T a = Ls[c * DT_TM + r];
#pragma unroll
                    for (int j = 0; j < DT_TN / 16; j++) acc[j] = fma(a, Us[c * DT_TNP + cg + 16 * j], acc[j]);
                }
                if (r0 + r < nt) {
#pragma unroll
                    for (int j = 0; j < DT_TN / 16; j++) {
                        const int32_t k = k0 + cg + 16 * j;
                        if (k < nt) {
                            T *p = dcol(lu, d, k) + r0 + r;
                            *p = __ldcg(p) - acc[j];
                        }
                    }
                }
            }
        }
        arrivals += gridDim.x;
        if (!grid_sync(bar, arrivals, &s_stop)) return;
    }
}

}  // namespace

// Panel width: the widest of 32, 16, 8 whose panel (nt rows) fits the
// shared-memory budget.
template <typename T>
int32_t dense_tail_panel(int32_t nt) {
    for (int32_t nb = 32; nb >= 8; nb /= 2)
        if ((size_t)nt * nb * sizeof(T) <= DT_PANEL_BYTES) return nb;
    return 0;
}

template <typename T>
cudaError_t launch_dense_tail(T *lu, const DenseTailArgs &d, const GridBarrier &bar, int num_sms, cudaStream_t s) {
    if (d.nt <= 0) return cudaSuccess;
    const int32_t nb = dense_tail_panel<T>(d.nt);
    if (nb == 0) return cudaErrorInvalidValue;
    const size_t smem = std::max<size_t>((size_t)d.nt * nb, 32 * DT_TM + 32 * DT_TNP) * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k_dense_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_tail<T>, DT_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    e = cudaMemsetAsync(bar.count, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bar.abort, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)num_sms);
    cfg.blockDim = dim3(DT_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_dense_tail<T>, lu, d, nb, bar);
}

template int32_t dense_tail_panel<double>(int32_t);
template int32_t dense_tail_panel<float>(int32_t);
template cudaError_t launch_dense_tail<double>(double *, const DenseTailArgs &, const GridBarrier &, int,
                                               cudaStream_t);
template cudaError_t launch_dense_tail<float>(float *, const DenseTailArgs &, const GridBarrier &, int,
                                              cudaStream_t);

}  // namespace glu
