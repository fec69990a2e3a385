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
// (Algorithm 2 restricted to it).  It runs here as one cooperative launch, a
// right-looking blocked LU with panels of 32 columns and grid barriers:
//   A  the panel's 32 x 32 diagonal block is factored by four warps of
//      block 0 in shared memory (row r of column c: L(r, c) = A(r, c) times
//      the reciprocal of U(c, c), then the columns to its right lose
//      L(r, c) U(c, cc));
//   B  every block: L21 = A21 U11^-1 (one warp per row, lane = column) and
//      U12 = L11^-1 A12 (one warp per column, lane = row), each row and
//      column taking the panel's columns in the order of step A;
//   C  every block updates A22 -= L21 U12 in tiles of 32 rows by 64, 32 or
//      16 columns, the width that spreads the panel's work best.
// Step A of the next panel needs only the tile of step C that holds the next
// diagonal block: block 0 takes that tile first and factors the block right
// after it while the other blocks are still in step C (look-ahead), so a
// panel costs two grid barriers.  The values stay in place in the CSC factor
// storage.  Data written by one block is read by others after a grid
// barrier, so every read of the factor values bypasses L1 (ld.global.cg).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "glu_device.cuh"

namespace glu {
namespace {

constexpr int DT_THREADS = 512;
constexpr int DT_NB = 32;                       // panel width
constexpr int DT_TM = 32, DT_TN = 64, DT_TNP = DT_TN + 1;

template <typename T>
__device__ __forceinline__ T *dcol(T *lu, const DenseTailArgs &d, int32_t k) {
    return lu + (__ldg(d.colptr + d.t0 + k + 1) - d.nt);
}

// barrier 1 over the block's first `threads` threads (whole warps)
__device__ __forceinline__ void dt_bar(int threads) { asm volatile("bar.sync 1, %0;" ::"r"(threads) : "memory"); }

// Step A: the diagonal block [c0, c0 + w)^2, by threads 0..127 of the block
// (warps 0..3; column cc's updates belong to warp cc mod 4), through
// sm[c * 32 + r] (column-major).  Column c stays unscaled while step c reads
// it; L(r, c) = A(r, c) times the reciprocal of U(c, c) is formed by every
// warp for its own updates and stored at the end.  The owner of column c + 1
// updates that column first and takes the next pivot's reciprocal before
// its other columns, so one barrier per step suffices.
template <typename T>
__device__ __forceinline__ void dt_factor_diag(T *lu, const DenseTailArgs &d, int32_t c0, int32_t w, T *sm) {
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    T *rps = sm + DT_NB * DT_NB;   // reciprocals of the pivots
    for (int idx = tid; idx < DT_NB * DT_NB; idx += 128) {
        const int c = idx >> 5, r = idx & 31;
        sm[idx] = (c < w && r < w) ? __ldcg(dcol(lu, d, c0 + c) + c0 + r) : T(0);
    }
    dt_bar(128);
    if (tid == 0) rps[0] = T(1) / sm[0];
    dt_bar(128);
    for (int c = 0; c + 1 < w; c++) {
        const T l = lane > c ? sm[c * 32 + lane] * rps[c] : T(0);
        int cc = c + 1 + ((wib - c - 1) & 3);
        if (cc == c + 1) {
            if (lane > c) sm[cc * 32 + lane] = sm[cc * 32 + lane] - l * sm[cc * 32 + c];
            __syncwarp();
            if (lane == 0) rps[cc] = T(1) / sm[cc * 32 + cc];
            cc += 4;
        }
        for (; cc < w; cc += 4)
            if (lane > c) sm[cc * 32 + lane] = sm[cc * 32 + lane] - l * sm[cc * 32 + c];
        dt_bar(128);
    }
    for (int idx = tid; idx < DT_NB * DT_NB; idx += 128) {
        const int c = idx >> 5, r = idx & 31;
        if (c < w && r < w) dcol(lu, d, c0 + c)[c0 + r] = r > c ? sm[idx] * rps[c] : sm[idx];
    }
}

// Step C's tile width (columns) for an m x m trailing update on g blocks: of
// 64, 32 and 16, the one with the fewest rounds of equal tiles times the
// work of a tile, the widest among equals.
__device__ __forceinline__ int32_t dt_tile_width(int32_t m, int32_t g) {
    const int32_t ntr = (m + DT_TM - 1) / DT_TM;
    int32_t best = DT_TN;
    int64_t best_cost = -1;
    for (int32_t tn = DT_TN; tn >= 16; tn >>= 1) {
        const int64_t tiles = (int64_t)ntr * ((m + tn - 1) / tn);
        const int64_t cost = ((tiles + g - 1) / g) * tn;
        if (best_cost < 0 || cost < best_cost) {
            best = tn;
            best_cost = cost;
        }
    }
    return best;
}

// One tile of step C: rows r0..r0+31, columns k0..k0+tn-1 of A22 lose
// L21(rows, panel) U12(panel, columns).  Thread: row tid % 32, columns
// tid / 32 + 16 j.
template <typename T>
__device__ __forceinline__ void dt_tile(T *lu, const DenseTailArgs &d, int32_t c0, int32_t w, int32_t r0, int32_t k0,
                                        int32_t tn, T *Ls, T *Us) {
    const int32_t nt = d.nt;
    const int tid = threadIdx.x;
    const int32_t tnp = tn + 1;
    __syncthreads();
    for (int32_t idx = tid; idx < w * DT_TM; idx += DT_THREADS) {
        const int32_t c = idx / DT_TM, rr = idx - c * DT_TM;
        Ls[c * DT_TM + rr] = (r0 + rr < nt) ? __ldcg(dcol(lu, d, c0 + c) + r0 + rr) : T(0);
    }
    for (int32_t idx = tid; idx < w * tn; idx += DT_THREADS) {
        const int32_t kk = idx / w, c = idx - kk * w;
        Us[c * tnp + kk] = (k0 + kk < nt) ? __ldcg(dcol(lu, d, k0 + kk) + c0 + c) : T(0);
    }
    __syncthreads();
    const int32_t r = tid % DT_TM, cg = tid / DT_TM;   // cg: 0..15, one per warp
    T acc[DT_TN / 16];
#pragma unroll
    for (int j = 0; j < DT_TN / 16; j++) acc[j] = T(0);
    for (int32_t c = 0; c < w; c++) {
        const T a = Ls[c * DT_TM + r];
#pragma unroll
        for (int j = 0; j < DT_TN / 16; j++)
            if (16 * j < tn) acc[j] = fma(a, Us[c * tnp + cg + 16 * j], acc[j]);
    }
    if (r0 + r < nt) {
#pragma unroll
        for (int j = 0; j < DT_TN / 16; j++) {
            const int32_t k = k0 + cg + 16 * j;
            if (16 * j < tn && k < nt) {
                T *p = dcol(lu, d, k) + r0 + r;
                *p = __ldcg(p) - acc[j];
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(DT_THREADS, 1) k_dense_tail(T *lu, const DenseTailArgs d, GridBarrier bar) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);   // diagonal block [32][32], then 32 reciprocals
    T *rps = sm + DT_NB * DT_NB;
    __shared__ int s_stop;
    const int32_t nt = d.nt;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    constexpr int NWB = DT_THREADS / 32;
    unsigned arrivals = 0;
    if (blockIdx.x == 0 && tid < 128) dt_factor_diag<T>(lu, d, 0, min(DT_NB, nt), sm);
    arrivals += gridDim.x;
    if (!grid_sync(bar, arrivals, &s_stop)) return;
    for (int32_t c0 = 0; c0 < nt; c0 += DT_NB) {
        const int32_t w = min(DT_NB, nt - c0), c1 = c0 + w, m = nt - c1;
        if (m <= 0) break;
        // ---- B: the factored diagonal block and its pivots' reciprocals
        __syncthreads();
        for (int idx = tid; idx < DT_NB * DT_NB; idx += DT_THREADS) {
            const int c = idx >> 5, r = idx & 31;
            sm[idx] = (c < w && r < w) ? __ldcg(dcol(lu, d, c0 + c) + c0 + r) : T(0);
        }
        __syncthreads();
        if (tid < w) rps[tid] = T(1) / sm[tid * 32 + tid];
        __syncthreads();
        // warp tasks: rows c1.. of L21, then columns c1.. of U12
        for (int32_t t = (int32_t)blockIdx.x * NWB + wib; t < 2 * m; t += (int32_t)gridDim.x * NWB) {
            if (t < m) {
                const int32_t rr = c1 + t;   // L21 row: lane = column
                T *pc = lane < w ? dcol(lu, d, c0 + lane) + rr : nullptr;
                T x = lane < w ? __ldcg(pc) : T(0);
                for (int c = 0; c < w; c++) {
                    const T l = __shfl_sync(0xffffffffu, x, c) * rps[c];
                    if (lane == c) x = l;
                    if (lane > c && lane < w) x = x - l * sm[lane * 32 + c];
                }
                if (lane < w) *pc = x;
            } else {
                T *col = dcol(lu, d, c1 + (t - m)) + c0;   // U12 column: lane = row
                T x = lane < w ? __ldcg(col + lane) : T(0);
                for (int c = 0; c + 1 < w; c++) {
                    const T xc = __shfl_sync(0xffffffffu, x, c);
                    if (lane > c && lane < w) x = x - sm[c * 32 + lane] * xc;
                }
                if (lane < w) col[lane] = x;
            }
        }
        arrivals += gridDim.x;
        if (!grid_sync(bar, arrivals, &s_stop)) return;
        // ---- C: A22 -= L21 U12.  Block 0 updates the next diagonal block
        // (rows and columns c1..c1+31) and factors it right away; the other
        // blocks take the rest in tiles of 32 rows by the width of least
        // makespan (row tile 0 starts 32 columns further right)
        {
            const int32_t G = (int32_t)gridDim.x, gr = G > 1 ? G - 1 : 1;
            const int32_t tn = dt_tile_width(m, gr);
            const int32_t ntr = (m + DT_TM - 1) / DT_TM;
            const int32_t n0 = m > DT_NB ? (m - DT_NB + tn - 1) / tn : 0, nrow = (m + tn - 1) / tn;
            const int32_t nreg = n0 + (ntr - 1) * nrow;
            T *Ls = sm;                    // [w][DT_TM]
            T *Us = sm + 32 * DT_TM;       // [w][tn + 1]
            if (blockIdx.x == 0) {
                dt_tile<T>(lu, d, c0, w, c1, c1, DT_NB, Ls, Us);
                __threadfence();
                __syncthreads();
                if (tid < 128) dt_factor_diag<T>(lu, d, c1, min(DT_NB, m), sm + 32 * DT_TM + 32 * DT_TNP);
            }
            if (blockIdx.x > 0 || G == 1)
                for (int32_t u = G > 1 ? (int32_t)blockIdx.x - 1 : 0; u < nreg; u += gr) {
                    int32_t r0, k0;
                    if (u < n0) {
                        r0 = c1;
                        k0 = c1 + DT_NB + u * tn;
                    } else {
                        const int32_t q = u - n0;
                        r0 = c1 + (1 + q / nrow) * DT_TM;
                        k0 = c1 + (q % nrow) * tn;
                    }
                    dt_tile<T>(lu, d, c0, w, r0, k0, tn, Ls, Us);
                }
        }
        arrivals += gridDim.x;
        if (!grid_sync(bar, arrivals, &s_stop)) return;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_dense_tail(T *lu, const DenseTailArgs &d, const GridBarrier &bar, int num_sms, cudaStream_t s) {
    if (d.nt <= 0) return cudaSuccess;
    // step C's tiles, then the look-ahead diagonal block behind them
    const size_t smem = (size_t)(32 * DT_TM + 32 * DT_TNP + DT_NB * DT_NB + DT_NB) * sizeof(T);
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
    return cudaLaunchKernelEx(&cfg, k_dense_tail<T>, lu, d, bar);
}

template cudaError_t launch_dense_tail<double>(double *, const DenseTailArgs &, const GridBarrier &, int,
                                               cudaStream_t);
template cudaError_t launch_dense_tail<float>(float *, const DenseTailArgs &, const GridBarrier &, int,
                                              cudaStream_t);

}  // namespace glu
