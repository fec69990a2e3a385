// analyze_gpu.cu -- Algorithm 4 (relaxed dependency detection) and the
// longest-path levels on the GPU (option gpu_analysis).
//
// Column k depends on column i < k when U(i,k) != 0 and column i of L is not
// empty (looking up), or when L(k,i) != 0 (looking left) -- Section III-A,
// Algorithm 4.  Both candidate lists are sorted: the rows above the diagonal
// of column k, and row k of L.  A warp per column forms their union without
// repeats by ranks: an up-looking candidate a that is kept and not in row k
// lands at (kept candidates before it) + (row-k entries below a); a row-k
// entry b lands at its index + (kept candidates below b).  A count pass, a
// prefix sum on the host, then the fill pass.  The levels: level(k) = 0
// without dependencies, else 1 + the largest level of its dependencies; a
// ticket hands out the columns in increasing order (every dependency of k
// has a smaller ticket, so a warp only waits on columns already handed out),
// each column waits for its dependencies' levels (bounded) and publishes its
// own with release semantics.  The results equal the host's bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "glu_device.cuh"

namespace glu {
namespace {

struct DepArgs {
    const int64_t *colptr;    // n + 1
    const int32_t *rowidx;
    const int64_t *diag;      // n
    const int64_t *lrow_ptr;  // n + 1: row k of L
    const int32_t *lrow_col;
    int32_t *scratch;         // per entry of the fill: kept-and-new up-looking candidates before it
    const int64_t *dep_ptr;   // fill pass
    int32_t *dep_cnt;         // count pass
    int32_t *dep_idx;
    int32_t n;
};

__device__ __forceinline__ bool has_l(const DepArgs &a, int32_t i) { return a.colptr[i + 1] - 1 > a.diag[i]; }

// first index in v[0, len) with v[idx] >= x
__device__ __forceinline__ int64_t lower(const int32_t *v, int64_t len, int32_t x) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (v[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_deps(const DepArgs a, int fill) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = w; k < a.n; k += nw) {
        const int32_t *A = a.rowidx + a.colptr[k];
        const int64_t na = a.diag[k] - a.colptr[k];
        const int32_t *B = a.lrow_col + a.lrow_ptr[k];
        const int64_t nb = a.lrow_ptr[k + 1] - a.lrow_ptr[k];
        int32_t *S = a.scratch + a.colptr[k];
        int64_t carry = 0;     // kept up-looking candidates not in row k, so far
        const int64_t base = fill ? a.dep_ptr[k] : 0;
        for (int64_t t0 = 0; t0 < na; t0 += 32) {
            const int64_t t = t0 + lane;
            bool add = false;
            int32_t v = 0;
            int64_t p = 0;
            if (t < na) {
                v = A[t];
                p = lower(B, nb, v);
                add = has_l(a, v) && !(p < nb && B[p] == v);
            }
            const unsigned m = __ballot_sync(0xffffffffu, add);
            const int64_t before = carry + __popc(m & ((1u << lane) - 1));
            if (fill && t < na) {
                S[t] = (int32_t)before;
                if (add) a.dep_idx[base + before + p] = v;
            }
            carry += __popc(m);
        }
        if (!fill) {
            if (lane == 0) a.dep_cnt[k] = (int32_t)(carry + nb);
            continue;
        }
        __syncwarp();
        for (int64_t j = lane; j < nb; j += 32) {
            const int32_t v = B[j];
            const int64_t p = lower(A, na, v);
            const int64_t kept_below = p < na ? (int64_t)S[p] : carry;
            a.dep_idx[base + j + kept_below] = v;
        }
    }
}

struct LevelArgs {
    const int64_t *dep_ptr;
    const int32_t *dep_idx;
    int32_t *level;           // n, -1 until published
    int32_t n;
    unsigned *ticket;
    unsigned *abort;
    int32_t *timed_out;
    long long spin_limit_cycles;
};

__device__ __forceinline__ int ld_acq(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__global__ void k_levels(const LevelArgs a) {
    const int lane = threadIdx.x & 31;
    while (true) {
        int32_t k = 0;
        if (lane == 0) k = (int32_t)atomicAdd(a.ticket, 1u);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= a.n) break;
        int32_t lv = -1;    // the largest dependency level seen by this lane
        bool ok = true;
        for (int64_t p = a.dep_ptr[k] + lane; p < a.dep_ptr[k + 1]; p += 32) {
            const int32_t *q = a.level + a.dep_idx[p];
            int v = ld_acq(q);
            if (v < 0) {
                const long long t0 = clock64();
                int spins = 0;
                while ((v = ld_acq(q)) < 0) {
                    __nanosleep(64);
                    if ((++spins & 63) == 0) {
                        if (*(volatile const unsigned *)a.abort) break;
                        if (clock64() - t0 > a.spin_limit_cycles) {
                            atomicOr(a.abort, 1u);
                            atomicExch(a.timed_out, 1);
                            break;
                        }
                    }
                }
            }
            if (v < 0) ok = false;
            lv = max(lv, v);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lv = max(lv, __shfl_xor_sync(0xffffffffu, lv, o));
        (void)ok;
        if (lane == 0) asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(a.level + k), "r"(lv + 1) : "memory");
    }
}

template <typename T, typename A>
cudaError_t up(T **d, const std::vector<T, A> &v) {
    cudaError_t e = cudaMalloc(d, std::max<size_t>(v.size(), 1) * sizeof(T));
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

}  // namespace

// Algorithm 4 and the levels of P (fill and row views already computed) on
// the current GPU: fills P.dep_ptr, P.dep_idx and P.level_of.  GLU_OK,
// GLU_ERR_CUDA / GLU_ERR_OOM (why says which call), GLU_ERR_TIMEOUT.
int gpu_dependencies_levels(HostPlan &P, int32_t spin_limit_us, std::string &why) {
    const int32_t n = P.n;
    long long spin_limit_cycles = 0;
    {
        int dev = 0, khz = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
        const long long us = spin_limit_us > 0 ? spin_limit_us : 2000000;
        spin_limit_cycles = us * (long long)(khz > 0 ? khz : 2000000) / 1000;
    }
    P.dep_ptr.assign((size_t)n + 1, 0);
    P.dep_idx.clear();
    P.level_of.assign((size_t)n, 0);
    if (n == 0) return GLU_OK;
    int64_t *d_cp = nullptr, *d_diag = nullptr, *d_lrp = nullptr, *d_dp = nullptr;
    int32_t *d_ri = nullptr, *d_lrc = nullptr, *d_s = nullptr, *d_cnt = nullptr, *d_idx = nullptr, *d_lv = nullptr;
    unsigned *d_w = nullptr;
    int rc = GLU_OK;
    auto fail = [&](cudaError_t e, const char *what) {
        why = std::string("gpu analysis: ") + what + ": " + cudaGetErrorString(e);
        rc = e == cudaErrorMemoryAllocation ? GLU_ERR_OOM : GLU_ERR_CUDA;
    };
    cudaError_t e;
    do {
        if ((e = up(&d_cp, P.lu_colptr)) != cudaSuccess) { fail(e, "upload"); break; }
        if ((e = up(&d_ri, P.lu_rowidx)) != cudaSuccess) { fail(e, "upload"); break; }
        if ((e = up(&d_diag, P.diag_pos)) != cudaSuccess) { fail(e, "upload"); break; }
        if ((e = up(&d_lrp, P.lrow_ptr)) != cudaSuccess) { fail(e, "upload"); break; }
        if ((e = up(&d_lrc, P.lrow_col)) != cudaSuccess) { fail(e, "upload"); break; }
        if ((e = cudaMalloc(&d_s, std::max<size_t>(P.lu_rowidx.size(), 1) * sizeof(int32_t))) != cudaSuccess) {
            fail(e, "scratch");
            break;
        }
        if ((e = cudaMalloc(&d_cnt, (size_t)n * sizeof(int32_t))) != cudaSuccess) { fail(e, "counts"); break; }
        DepArgs a{d_cp, d_ri, d_diag, d_lrp, d_lrc, d_s, nullptr, d_cnt, nullptr, n};
        const unsigned blocks = (unsigned)std::min<int64_t>(((int64_t)n * 32 + 255) / 256, 152 * 32);
        k_deps<<<blocks, 256>>>(a, 0);
        std::vector<int32_t> cnt((size_t)n);
        if ((e = cudaMemcpy(cnt.data(), d_cnt, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess) {
            fail(e, "dependency counts");
            break;
        }
        for (int32_t k = 0; k < n; k++) P.dep_ptr[(size_t)k + 1] = P.dep_ptr[(size_t)k] + cnt[(size_t)k];
        const int64_t nd = P.dep_ptr[(size_t)n];
        if ((e = up(&d_dp, P.dep_ptr)) != cudaSuccess) { fail(e, "upload"); break; }
        if ((e = cudaMalloc(&d_idx, std::max<int64_t>(nd, 1) * sizeof(int32_t))) != cudaSuccess) {
            fail(e, "dependency lists");
            break;
        }
        a.dep_ptr = d_dp;
        a.dep_idx = d_idx;
        k_deps<<<blocks, 256>>>(a, 1);
        if ((e = cudaMalloc(&d_lv, (size_t)n * sizeof(int32_t))) != cudaSuccess) { fail(e, "levels"); break; }
        if ((e = cudaMalloc(&d_w, 4 * sizeof(unsigned))) != cudaSuccess) { fail(e, "levels"); break; }
        cudaMemset(d_lv, 0xff, (size_t)n * sizeof(int32_t));
        cudaMemset(d_w, 0, 4 * sizeof(unsigned));
        LevelArgs la{d_dp, d_idx, d_lv, n, d_w, d_w + 1, reinterpret_cast<int32_t *>(d_w + 2), spin_limit_cycles};
        k_levels<<<152 * 8, 128>>>(la);
        P.dep_idx.resize((size_t)nd);
        if ((e = cudaMemcpy(P.dep_idx.data(), d_idx, nd * sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess) {
            fail(e, "dependency lists");
            break;
        }
        if ((e = cudaMemcpy(P.level_of.data(), d_lv, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost)) !=
            cudaSuccess) {
            fail(e, "levels");
            break;
        }
        unsigned w[4];
        if ((e = cudaMemcpy(w, d_w, sizeof(w), cudaMemcpyDeviceToHost)) != cudaSuccess) { fail(e, "levels"); break; }
        if (w[2] != 0) {
            why = "gpu analysis: a bounded wait of the level kernel timed out";
            rc = GLU_ERR_TIMEOUT;
        }
    } while (false);
    cudaFree(d_cp);
    cudaFree(d_ri);
    cudaFree(d_diag);
    cudaFree(d_lrp);
    cudaFree(d_lrc);
    cudaFree(d_s);
    cudaFree(d_cnt);
    cudaFree(d_dp);
    cudaFree(d_idx);
    cudaFree(d_lv);
    cudaFree(d_w);
    return rc;
}

}  // namespace glu
