// kernels_blocks.cu -- the supernodal ("block") factorization.
//
// Under a nested-dissection order every separator is a run of columns whose
// diagonal block is dense and whose columns share the rows below the run.
// Column by column (Algorithm 2 scheduled by the levels of Algorithm 4) such
// a run is a chain of levels, and every entry of its targets is read and
// written once per column of the run.  Here a run of up to BSN_MAX columns is
// one node of the contracted dependency graph and is processed as a dense
// panel -- the same right-looking arithmetic in another order:
//   k_bdiag    the diagonal block, LU without pivoting (a warp per run, one
//              row per lane, in registers);
//   k_bpanel   the rows below it, L21 = A21 U11^-1 (a warp per 32 rows, one
//              row per lane), and for every target column k the rows of the
//              run, U12(:, k) = L11^-1 A12(:, k) (a warp per target);
//   k_bupdate  A(R_B, k) -= L21 U12(:, k), one read-modify-write of each
//              target entry per run; a warp task owns BCHUNK positions of a
//              column and applies the level's runs in order (no atomics).
// The dense block being contiguous in every column of the run, the diagonal
// block's column c0+m starts at diag_pos[c0+m] - m, and L21's column at
// colptr[c0+m+1] - |R_B|.
#include <cuda_runtime.h>

#include <cstdint>

#include "glu_device.cuh"

namespace glu {
namespace {

constexpr int BW = 4;   // warps per block

__device__ __forceinline__ void raise_err_bk(unsigned long long *err, int32_t col, unsigned code) {
    atomicMin(err, ((unsigned long long)(uint32_t)col << 8) | code);
}

template <typename T>
__global__ void __launch_bounds__(BW * 32) k_bdiag(const BlockArgs<T> a, int32_t b0, int32_t b1) {
    const int lane = threadIdx.x & 31;
    const int32_t warp = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int32_t nw = (int32_t)((gridDim.x * blockDim.x) >> 5);
    for (int32_t it = b0 + warp; it < b1; it += nw) {
        const int32_t q = a.bdiag[it];
        const int32_t c0 = a.sn_c0[q], s = a.sn_c0[q + 1] - c0;
        const bool own = lane < s;
        T x[BSN_MAX];   // lane r: row c0 + r of the diagonal block
#pragma unroll
        for (int m = 0; m < BSN_MAX; m++) x[m] = (own && m < s) ? a.lu[a.diag_pos[c0 + m] - m + lane] : (T)0;
#pragma unroll
        for (int jj = 0; jj + 1 < BSN_MAX; jj++) {
            if (jj + 1 < s) {
                const T piv = __shfl_sync(0xffffffffu, x[jj], jj);
                const bool below = own && lane > jj;
                T l = (T)0;
                if (below) {
                    l = x[jj] / piv;
                    x[jj] = l;
                }
#pragma unroll
                for (int m = jj + 1; m < BSN_MAX; m++) {
                    const T u = __shfl_sync(0xffffffffu, x[m], jj);
                    if (below && m < s) x[m] = x[m] - l * u;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < BSN_MAX; m++)
            if (own && m < s) a.lu[a.diag_pos[c0 + m] - m + lane] = x[m];
    }
}

constexpr int U11_LD = BSN_MAX + 1;   // padded row length of the shared U11 copy

template <typename T>
__global__ void __launch_bounds__(BW * 32) k_bpanel(const BlockArgs<T> a, int32_t i0, int32_t i1) {
    __shared__ T u11s[BW][BSN_MAX * U11_LD];
    const int lane = threadIdx.x & 31;
    const int32_t warp = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int32_t nw = (int32_t)((gridDim.x * blockDim.x) >> 5);
    T *u11 = u11s[threadIdx.x >> 5];
    for (int32_t it = i0 + warp; it < i1; it += nw) {
        const BItem bi = a.bitems[it];
        const int32_t q = bi.sn;
        const int32_t c0 = a.sn_c0[q], s = a.sn_c0[q + 1] - c0, r = a.sn_r[q];
        if (bi.kind == 0) {
            // U11 (rows <= columns) into this warp's shared copy: column m's
            // block rows start at diag_pos[c0 + m] - m
            for (int32_t m = 0; m < s; m++) {
                const int64_t base = a.diag_pos[c0 + m] - m;
                if (lane <= m) u11[lane * U11_LD + m] = a.lu[base + lane];
            }
            __syncwarp();
            // the diagonal kept as reciprocals: one division per column, not per row
            if (lane < s) u11[lane * U11_LD + lane] = (T)1 / u11[lane * U11_LD + lane];
            __syncwarp();
            // rows bi.a .. bi.b-1 of R_B: x U11 = a, solved left to right
            const int32_t t = bi.a + lane;
            const bool own = t < bi.b;
            T x[BSN_MAX];
#pragma unroll
            for (int m = 0; m < BSN_MAX; m++) x[m] = (own && m < s) ? a.lu[a.colptr[c0 + m + 1] - r + t] : (T)0;
#pragma unroll
            for (int jj = 0; jj < BSN_MAX; jj++) {
                if (jj < s) {
                    x[jj] = x[jj] * u11[jj * U11_LD + jj];
#pragma unroll
                    for (int m = jj + 1; m < BSN_MAX; m++)
                        if (m < s) x[m] = x[m] - x[jj] * u11[jj * U11_LD + m];
                }
            }
            __syncwarp();
#pragma unroll
            for (int m = 0; m < BSN_MAX; m++)
                if (own && m < s) a.lu[a.colptr[c0 + m + 1] - r + t] = x[m];
        } else {
            // the rows f..s-1 of the run in target column k: L11 x = a
            const BPair bp = a.bpairs[bi.a];
            const int32_t m = lane;
            const bool own = m >= bp.f && m < s;
            T x = own ? a.lu[bp.upos + (m - bp.f)] : (T)0;
            // lane m's row of L11, loaded before the sweep
            T l11[BSN_MAX];
#pragma unroll
            for (int jj = 0; jj < BSN_MAX; jj++)
                l11[jj] = (own && jj >= bp.f && jj < m) ? a.lu[a.diag_pos[c0 + jj] + (m - jj)] : (T)0;
#pragma unroll
            for (int jj = 0; jj + 1 < BSN_MAX; jj++) {
                if (jj >= bp.f && jj + 1 < s) {
                    const T xj = __shfl_sync(0xffffffffu, x, jj);
                    if (own && m > jj) x = x - l11[jj] * xj;
                }
            }
            if (own) a.lu[bp.upos + (m - bp.f)] = x;
        }
    }
}

constexpr int BU_ROWS = BCHUNK / 32;   // target rows per lane in one segment

template <typename T, typename M>
__global__ void __launch_bounds__(BW * 32) k_bupdate(const BlockArgs<T> a, int32_t k0, int32_t k1) {
    const int lane = threadIdx.x & 31;
    const int32_t warp = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int32_t nw = (int32_t)((gridDim.x * blockDim.x) >> 5);
    const M *__restrict__ map = static_cast<const M *>(a.map);
    for (int32_t it = k0 + warp; it < k1; it += nw) {
        const BTask tk = a.btasks[it];
        for (int32_t sg = tk.seg_begin; sg < tk.seg_end; sg++) {
            const BSeg seg = a.bsegs[sg];
            const BPair bp = a.bpairs[seg.pair];
            const int32_t q = bp.sn;
            const int32_t c0 = a.sn_c0[q], s = a.sn_c0[q + 1] - c0, r = a.sn_r[q];
            // lane m (f <= m < s): U12(m, k) and where L21's column m starts
            T um = (T)0;
            int64_t lc = 0;
            if (lane >= bp.f && lane < s) {
                um = a.lu[bp.upos + (lane - bp.f)];
                lc = a.colptr[c0 + lane + 1] - r;
            }
            // the targets' offsets and values first: they do not depend on
            // the products, so their loads overlap the L21 loop below
            T *tgt = a.lu + a.colptr[bp.k];
            const M *mp = map + bp.mb;
            uint32_t off[BU_ROWS];
            T tv[BU_ROWS];
#pragma unroll
            for (int u = 0; u < BU_ROWS; u++) {
                const int32_t t = seg.t0 + lane + 32 * u;
                if (t < seg.t1) off[u] = mp[t];
            }
#pragma unroll
            for (int u = 0; u < BU_ROWS; u++)
                if (seg.t0 + lane + 32 * u < seg.t1) tv[u] = tgt[off[u]];
            T acc[BU_ROWS];
#pragma unroll
            for (int u = 0; u < BU_ROWS; u++) acc[u] = (T)0;
            for (int32_t m = bp.f; m < s; m++) {
                const T um_b = __shfl_sync(0xffffffffu, um, m);
                const int64_t lcm = __shfl_sync(0xffffffffu, lc, m);
#pragma unroll
                for (int u = 0; u < BU_ROWS; u++) {
                    const int32_t t = seg.t0 + lane + 32 * u;
                    if (t < seg.t1) acc[u] = fma(a.lu[lcm + t], um_b, acc[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < BU_ROWS; u++)
                if (seg.t0 + lane + 32 * u < seg.t1) tgt[off[u]] = tv[u] - acc[u];
            __syncwarp();
        }
    }
}

// Offsets in column k of the rows R_B, a warp per pair (binary search).
template <typename M>
__global__ void k_bmap_build(const BlockArgs<double> a, int64_t npairs) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    M *map = static_cast<M *>(const_cast<void *>(a.map));
    for (int64_t p = w; p < npairs; p += nw) {
        const BPair bp = a.bpairs[p];
        const int32_t q = bp.sn;
        const int32_t r = a.sn_r[q];
        const int32_t *R = a.rowidx + a.colptr[a.sn_c0[q + 1]] - r;
        const int64_t cb = a.colptr[bp.k];
        const int32_t *rows = a.rowidx + cb;
        const int64_t len = a.colptr[bp.k + 1] - cb;
        for (int32_t t = lane; t < r; t += 32) {
            const int32_t row = R[t];
            int64_t lo = 0, hi = len;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (rows[mid] < row) lo = mid + 1;
                else hi = mid;
            }
            if (lo >= len || rows[lo] != row) {
                raise_err_bk(a.err, bp.k, DEVERR_INTERNAL);
                lo = 0;
            }
            map[bp.mb + t] = (M)lo;
        }
    }
}

// One work item per warp: the items' costs vary widely, and the block
// scheduler balances them better than a grid-stride split (200k workload
// 65.7 -> 58.5 ms FP64 against 8 blocks per SM)
unsigned warps_grid(int64_t warps, int num_sms) {
    (void)num_sms;
    const int64_t blocks = (warps + BW - 1) / BW;
    return (unsigned)(blocks < 1 ? 1 : blocks);
}

}  // namespace

template <typename T>
cudaError_t launch_block_level(const BlockArgs<T> &a, int map_bytes, int32_t d0, int32_t d1, int32_t i0,
                               int32_t i1, int32_t k0, int32_t k1, int num_sms, cudaStream_t s, int *launched) {
    *launched = 0;
    if (d1 > d0) {
        k_bdiag<T><<<warps_grid(d1 - d0, num_sms), BW * 32, 0, s>>>(a, d0, d1);
        ++*launched;
    }
    if (i1 > i0) {
        k_bpanel<T><<<warps_grid(i1 - i0, num_sms), BW * 32, 0, s>>>(a, i0, i1);
        ++*launched;
    }
    if (k1 > k0) {
        if (map_bytes == 2) k_bupdate<T, uint16_t><<<warps_grid(k1 - k0, num_sms), BW * 32, 0, s>>>(a, k0, k1);
        else k_bupdate<T, uint32_t><<<warps_grid(k1 - k0, num_sms), BW * 32, 0, s>>>(a, k0, k1);
        ++*launched;
    }
    return cudaGetLastError();
}

cudaError_t launch_bmap_build(const BlockArgs<double> &a, int map_bytes, int64_t npairs, int num_sms, cudaStream_t s) {
    if (npairs <= 0) return cudaSuccess;
    int64_t blocks = (npairs * 32 + 255) / 256;
    if (blocks > (int64_t)num_sms * 16) blocks = (int64_t)num_sms * 16;
    if (map_bytes == 2) k_bmap_build<uint16_t><<<(unsigned)blocks, 256, 0, s>>>(a, npairs);
    else k_bmap_build<uint32_t><<<(unsigned)blocks, 256, 0, s>>>(a, npairs);
    return cudaGetLastError();
}

template cudaError_t launch_block_level<double>(const BlockArgs<double> &, int, int32_t, int32_t, int32_t, int32_t,
                                                int32_t, int32_t, int, cudaStream_t, int *);
template cudaError_t launch_block_level<float>(const BlockArgs<float> &, int, int32_t, int32_t, int32_t, int32_t,
                                               int32_t, int32_t, int, cudaStream_t, int *);

}  // namespace glu
