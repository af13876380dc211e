// General permutation of a CSR matrix, Y = P X Q^T: Y[row_perm[i],
// col_perm[j]] = X[i, j].  The random relabelling of rows and columns turns
// a structured matrix (diagonal bands) into an unstructured one whose 2D
// tiles carry even shares of the nonzeros (Sec. 5, the permuted HV15R
// experiment).
//
// Steps: both maps are checked to be permutations (every target hit exactly
// once, on the device, before any entry of Y is written); Y's row lengths
// are X's moved to their new rows, scanned into Y.row_ptr; every row is
// copied with its columns mapped and re-sorted.  Rows of up to 1024 entries
// are sorted by one warp (bitonic network over (column, source position)
// pairs in shared memory); longer rows by one block that ranks every entry
// against the whole row (columns are distinct, so ranks are a permutation).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace tsg {

constexpr int kPermWarpMax = 1024;  // longest row one warp sorts on chip (8 KB of keys)
constexpr int kPermWarps = 4;       // warps per block of the row kernel (32 KB of keys)
constexpr int kPermLongThreads = 512;
constexpr int kPermLongMax = 65536;  // longest row ranked (quadratic: ~10 ms per row at this length)

__global__ void k_perm_hits(const int* __restrict__ perm, int n, int* hits, unsigned* status) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p = __ldg(perm + i);
        if (p < 0 || p >= n) {
            atomicOr(status, kStatusBadMap);
            continue;
        }
        atomicAdd(hits + p, 1);
    }
}

__global__ void k_perm_verify(const int* __restrict__ hits, int n, unsigned* status) {
    bool bad = false;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) bad |= hits[t] != 1;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusBadMap);
}

// ylen[row_perm[i]] = |X_i|; rows longer than one warp's capacity are listed.
__global__ void k_perm_len(const int* __restrict__ rp, const int* __restrict__ row_perm, int n, int* ylen,
                           int* long_count, int* long_list, const unsigned* status) {
    if (*status & kStatusBadMap) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int len = __ldg(rp + i + 1) - __ldg(rp + i);
        ylen[row_perm ? __ldg(row_perm + i) : i] = len;
        if (len > kPermWarpMax) long_list[atomicAdd(long_count, 1)] = i;
    }
}

template <typename T>
__global__ void __launch_bounds__(32 * kPermWarps) k_perm_rows(const int* __restrict__ rp,
                                                                const int* __restrict__ col,
                                                                const T* __restrict__ val, int n,
                                                                const int* __restrict__ row_perm,
                                                                const int* __restrict__ col_perm,
                                                                const int* __restrict__ yrp, int* ycol, T* yval,
                                                                const unsigned* status) {
    __shared__ unsigned long long keys[kPermWarps][kPermWarpMax];
    if (*status & kStatusBadMap) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long* s = keys[w];
    for (int i = blockIdx.x * kPermWarps + w; i < n; i += gridDim.x * kPermWarps) {
        const int x0 = __ldg(rp + i), len = __ldg(rp + i + 1) - x0;
        if (len == 0 || len > kPermWarpMax) continue;
        const int dst = __ldg(yrp + (row_perm ? __ldg(row_perm + i) : i));
        if (!col_perm) {
            // columns keep their order: a straight copy
            for (int e = lane; e < len; e += 32) {
                ycol[dst + e] = __ldg(col + x0 + e);
                if (val) yval[dst + e] = __ldg(val + x0 + e);
            }
            continue;
        }
        int N = 32;
        while (N < len) N <<= 1;
        for (int e = lane; e < N; e += 32)
            s[e] = e < len ? ((unsigned long long)(unsigned)__ldg(col_perm + __ldg(col + x0 + e)) << 32) | (unsigned)e
                           : ~0ull;
        __syncwarp();
        for (int k = 2; k <= N; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int t = lane; t < N; t += 32) {
                    const int u = t ^ j;
                    if (u > t) {
                        const unsigned long long a = s[t], b = s[u];
                        if ((a > b) == ((t & k) == 0)) {
                            s[t] = b;
                            s[u] = a;
                        }
                    }
                }
                __syncwarp();
            }
        }
        for (int e = lane; e < len; e += 32) {
            const unsigned long long kv = s[e];
            ycol[dst + e] = (int)(kv >> 32);
            if (val) yval[dst + e] = __ldg(val + x0 + (int)(kv & 0xffffffffu));
        }
        __syncwarp();
    }
}

// One block per listed long row: rank of every entry among the row's mapped
// columns (distinct), then each entry written at its rank.
template <typename T>
__global__ void __launch_bounds__(kPermLongThreads) k_perm_long(const int* __restrict__ rp,
                                                                const int* __restrict__ col,
                                                                const T* __restrict__ val,
                                                                const int* __restrict__ row_perm,
                                                                const int* __restrict__ col_perm,
                                                                const int* __restrict__ yrp, int* ycol, T* yval,
                                                                const int* long_count,
                                                                const int* __restrict__ long_list, int* rank,
                                                                unsigned* status) {
    if (*status & kStatusBadMap) return;
    const int nl = *long_count;
    for (int l = blockIdx.x; l < nl; l += gridDim.x) {
        const int i = long_list[l];
        const int x0 = __ldg(rp + i), len = __ldg(rp + i + 1) - x0;
        const int dst = __ldg(yrp + (row_perm ? __ldg(row_perm + i) : i));
        if (col_perm && len > kPermLongMax) {
            if (threadIdx.x == 0) atomicOr(status, kStatusCapacity);
            continue;
        }
        if (!col_perm) {
            for (int e = threadIdx.x; e < len; e += blockDim.x) {
                ycol[dst + e] = __ldg(col + x0 + e);
                if (val) yval[dst + e] = __ldg(val + x0 + e);
            }
            continue;
        }
        // mapped columns, unsorted, staged in Y's own row
        for (int e = threadIdx.x; e < len; e += blockDim.x)
            ycol[dst + e] = col_perm ? __ldg(col_perm + __ldg(col + x0 + e)) : __ldg(col + x0 + e);
        __syncthreads();
        for (int e = threadIdx.x; e < len; e += blockDim.x) {
            const int key = ycol[dst + e];
            int r = 0;
            for (int q = 0; q < len; ++q) r += ycol[dst + q] < key;
            rank[x0 + e] = r;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < len; e += blockDim.x) {
            const int r = rank[x0 + e];
            ycol[dst + r] = col_perm ? __ldg(col_perm + __ldg(col + x0 + e)) : __ldg(col + x0 + e);
            if (val) yval[dst + r] = __ldg(val + x0 + e);
        }
        __syncthreads();
    }
}

cudaError_t launch_permute(const PermuteArgs& p, cudaStream_t s) {
    const int threads = 256;
    auto grid = [&](long long n) { return (int)std::min<long long>((n + threads - 1) / threads, (long long)p.sms * 8); };
    if (p.row_perm && p.nrows > 0) k_perm_hits<<<grid(p.nrows), threads, 0, s>>>(p.row_perm, p.nrows, p.hits_r, p.status);
    if (p.col_perm && p.ncols > 0) k_perm_hits<<<grid(p.ncols), threads, 0, s>>>(p.col_perm, p.ncols, p.hits_c, p.status);
    if (p.row_perm && p.nrows > 0) k_perm_verify<<<grid(p.nrows), threads, 0, s>>>(p.hits_r, p.nrows, p.status);
    if (p.col_perm && p.ncols > 0) k_perm_verify<<<grid(p.ncols), threads, 0, s>>>(p.hits_c, p.ncols, p.status);
    if (p.nrows > 0)
        k_perm_len<<<grid(p.nrows), threads, 0, s>>>(p.rp, p.row_perm, p.nrows, p.ylen, p.long_count, p.long_list,
                                                      p.status);
    cudaError_t e = launch_scan(p.ylen, p.nrows, p.bsum, p.ex, s);
    if (e != cudaSuccess) return e;
    e = launch_ll_to_int(p.ex, (long long)p.nrows + 1, p.yrp, s);
    if (e != cudaSuccess) return e;
    if (p.nrows > 0 && p.nnz > 0) {
        const int blocks = (int)std::min<long long>(((long long)p.nrows + kPermWarps - 1) / kPermWarps,
                                                    (long long)p.sms * 8);
        if (p.dtype == 1) {
            k_perm_rows<double><<<blocks, 32 * kPermWarps, 0, s>>>(
                p.rp, p.col, static_cast<const double*>(p.val), p.nrows, p.row_perm, p.col_perm, p.yrp, p.ycol,
                static_cast<double*>(p.yval), p.status);
            k_perm_long<double><<<p.sms, kPermLongThreads, 0, s>>>(
                p.rp, p.col, static_cast<const double*>(p.val), p.row_perm, p.col_perm, p.yrp, p.ycol,
                static_cast<double*>(p.yval), p.long_count, p.long_list, p.rank, p.status);
        } else {
            k_perm_rows<float><<<blocks, 32 * kPermWarps, 0, s>>>(
                p.rp, p.col, static_cast<const float*>(p.val), p.nrows, p.row_perm, p.col_perm, p.yrp, p.ycol,
                static_cast<float*>(p.yval), p.status);
            k_perm_long<float><<<p.sms, kPermLongThreads, 0, s>>>(
                p.rp, p.col, static_cast<const float*>(p.val), p.row_perm, p.col_perm, p.yrp, p.ycol,
                static_cast<float*>(p.yval), p.long_count, p.long_list, p.rank, p.status);
        }
    }
    return cudaGetLastError();
}

}  // namespace tsg
