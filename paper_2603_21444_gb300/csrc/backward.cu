// Backward pass of C = A B on fixed patterns, and the CSR transpose.
//
// For a scalar loss L with upstream gradient G_ij = dL/dC_ij on pat(C), the
// chain rule on C_ij = sum_k a_ik b_kj (paper Sec. 2) gives
//   dA_ik = sum_{j in B_k} G_ij b_kj        on pat(A)   ((G B^T) sampled)
//   dB_kj = sum_{i : k in A_i} a_ik G_ij    on pat(B)   ((A^T G) sampled)
//
// k_bwd_rows: one warp per row i.  Row i of C (sorted columns and G) is
// staged in shared memory; each lane owns one entry (i, k) of A and walks
// B row k in stored order, finding G_ij by binary search in the staged row.
// dA_ik is the running sum in that order (product rounded, then added,
// starting from zero).  With scatter_db, a_ik G_ij is added to dB_kj with a
// device atomic (order not fixed).
// k_bwd_db: deterministic dB from A^T (rows sorted by i): one lane per B
// entry (k, j) sums a_ik G_ij over i ascending, G_ij found by binary search
// in row i of C in global memory.
#include <algorithm>

#include "internal.h"

namespace tsg {

constexpr int kBwdWarps = 4;
constexpr int kBwdStage = 768;  // C-row entries staged per warp (36 KB per block for double)

__device__ __forceinline__ int lower_bound_i(const int* __restrict__ a, int lo, int hi, int x) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

template <typename T>
__global__ void __launch_bounds__(32 * kBwdWarps) k_bwd_rows(BwdArgs a) {
    __shared__ int s_col[kBwdWarps][kBwdStage];
    __shared__ T s_g[kBwdWarps][kBwdStage];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T* aval = reinterpret_cast<const T*>(a.aval);
    const T* bval = reinterpret_cast<const T*>(a.bval);
    const T* g = reinterpret_cast<const T*>(a.g);
    T* da = reinterpret_cast<T*>(a.da);
    T* db = reinterpret_cast<T*>(a.db);
    for (int i = blockIdx.x * kBwdWarps + w; i < a.m; i += gridDim.x * kBwdWarps) {
        const int c0 = __ldg(a.crp + i), c1 = __ldg(a.crp + i + 1);
        const int cl = c1 - c0;
        const bool staged = cl <= kBwdStage;
        if (staged) {
            for (int q = lane; q < cl; q += 32) {
                s_col[w][q] = __ldg(a.ccol + c0 + q);
                s_g[w][q] = __ldg(g + c0 + q);
            }
        }
        __syncwarp();
        const int a0 = __ldg(a.arp + i), a1 = __ldg(a.arp + i + 1);
        for (int e = a0 + lane; e < a1; e += 32) {
            const int k = __ldg(a.acol + e);
            const T av = __ldg(aval + e);
            const int f0 = __ldg(a.brp + k), f1 = __ldg(a.brp + k + 1);
            T s = T(0);
            for (int f = f0; f < f1; ++f) {
                const int j = __ldg(a.bcol + f);
                T gij;
                if (staged) {
                    const int pos = lower_bound_i(s_col[w], 0, cl, j);
                    if (pos >= cl || s_col[w][pos] != j) {
                        atomicOr(a.status, kStatusInternal);
                        continue;
                    }
                    gij = s_g[w][pos];
                } else {
                    const int pos = lower_bound_i(a.ccol, c0, c1, j);
                    if (pos >= c1 || __ldg(a.ccol + pos) != j) {
                        atomicOr(a.status, kStatusInternal);
                        continue;
                    }
                    gij = __ldg(g + pos);
                }
                if (da) s = add_rn(s, mul_rn(gij, __ldg(bval + f)));
                if (db && a.scatter_db) atomicAdd(db + f, mul_rn(av, gij));
            }
            if (da) da[e] = s;
        }
        __syncwarp();
    }
}

template <typename T>
__global__ void k_bwd_db(BwdArgs a) {
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    const T* bval = reinterpret_cast<const T*>(a.bval);
    (void)bval;
    const T* g = reinterpret_cast<const T*>(a.g);
    const T* tval = reinterpret_cast<const T*>(a.tval);
    T* db = reinterpret_cast<T*>(a.db);
    for (int k = blockIdx.x * warps + (threadIdx.x >> 5); k < a.kdim; k += gridDim.x * warps) {
        const int f0 = __ldg(a.brp + k), f1 = __ldg(a.brp + k + 1);
        const int t0 = __ldg(a.trp + k), t1 = __ldg(a.trp + k + 1);
        for (int f = f0 + lane; f < f1; f += 32) {
            const int j = __ldg(a.bcol + f);
            T s = T(0);
            for (int t = t0; t < t1; ++t) {
                const int i = __ldg(a.tcol + t);
                const int c0 = __ldg(a.crp + i), c1 = __ldg(a.crp + i + 1);
                const int pos = lower_bound_i(a.ccol, c0, c1, j);
                if (pos >= c1 || __ldg(a.ccol + pos) != j) {
                    atomicOr(a.status, kStatusInternal);
                    continue;
                }
                s = add_rn(s, mul_rn(__ldg(tval + t), __ldg(g + pos)));
            }
            db[f] = s;
        }
    }
}

template <typename T>
__global__ void k_zero(T* p, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = T(0);
}

cudaError_t launch_backward(int dtype, const BwdArgs& a, int sms, cudaStream_t s) {
    const int threads = 32 * kBwdWarps;
    const long long need = ((long long)a.m + kBwdWarps - 1) / kBwdWarps;
    const int blocks = (int)std::min<long long>(std::max<long long>(need, 1), (long long)sms * 8);
    if (a.db && a.scatter_db) {
        const int zb = (int)std::min<long long>((a.nnzb + 255) / 256 + 1, (long long)sms * 16);
        if (dtype == 1) k_zero<double><<<zb, 256, 0, s>>>(static_cast<double*>(a.db), a.nnzb);
        else k_zero<float><<<zb, 256, 0, s>>>(static_cast<float*>(a.db), a.nnzb);
    }
    if (a.m > 0 && (a.da || (a.db && a.scatter_db))) {
        if (dtype == 1) k_bwd_rows<double><<<blocks, threads, 0, s>>>(a);
        else k_bwd_rows<float><<<blocks, threads, 0, s>>>(a);
    }
    if (a.db && !a.scatter_db && a.kdim > 0) {
        const long long needk = ((long long)a.kdim + 7) / 8;
        const int kb = (int)std::min<long long>(needk, (long long)sms * 8);
        if (dtype == 1) k_bwd_db<double><<<kb, 256, 0, s>>>(a);
        else k_bwd_db<float><<<kb, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------- transpose
//
// X^T in CSR: count per column, scan, scatter (arrival order), then sort
// each row of X^T by its column (the row index of X): element rank = number
// of entries of the row with a smaller key, one warp per row.

__global__ void k_tr_count(const int* __restrict__ col, long long nnz, int* cnt) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz; e += (long long)gridDim.x * blockDim.x)
        atomicAdd(cnt + __ldg(col + e), 1);
}

template <typename T>
__global__ void k_tr_scatter(const int* __restrict__ rp, const int* __restrict__ col, const T* __restrict__ val,
                             int nrows, const int* __restrict__ trp, int* cursor, int* tcol, T* tval) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    for (int e = __ldg(rp + r); e < __ldg(rp + r + 1); ++e) {
        const int k = __ldg(col + e);
        const int pos = __ldg(trp + k) + atomicAdd(cursor + k, 1);
        tcol[pos] = r;
        if (val) tval[pos] = __ldg(val + e);
    }
}

// Rows of X^T up to kTrShort entries: one warp per row, each entry ranked by
// a scan of its row (len^2 / 32 compares per lane).  Longer rows (a dense or
// power-law column of X) go to k_tr_sort_long.
constexpr int kTrShort = 1024;
constexpr int kTrLongThreads = 1024;
constexpr int kTrWindow = 1 << 19;          // keys per bitmap pass
constexpr int kTrWords = kTrWindow / 32;    // 16384 words: 64 KB bitmap + 64 KB prefixes
constexpr int kTrLongSmem = 2 * kTrWords * 4;

// rows are sorted into tmp then copied back; keys within a row are distinct
template <typename T>
__global__ void k_tr_sort(const int* __restrict__ trp, int nrows_t, int* tcol, T* tval, int* tmpc, T* tmpv,
                          bool has_val) {
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    for (int k = blockIdx.x * warps + (threadIdx.x >> 5); k < nrows_t; k += gridDim.x * warps) {
        const int lo = __ldg(trp + k), hi = __ldg(trp + k + 1);
        if (hi - lo > kTrShort) continue;
        for (int e = lo + lane; e < hi; e += 32) {
            const int key = tcol[e];
            int rank = 0;
            for (int q = lo; q < hi; ++q) rank += tcol[q] < key;
            tmpc[lo + rank] = key;
            if (has_val) tmpv[lo + rank] = tval[e];
        }
        __syncwarp();
        for (int e = lo + lane; e < hi; e += 32) {
            tcol[e] = tmpc[e];
            if (has_val) tval[e] = tmpv[e];
        }
        __syncwarp();
    }
}

// Long rows of X^T, one block each: the row's keys (distinct row indices of
// X, in [0, nkeys)) are marked in a shared-memory bitmap over a window of
// kTrWindow keys, the words' popcounts are scanned, and each entry's rank is
// the keys below it -- earlier windows, earlier words, lower bits of its
// word.  O(len + nkeys / 32) per window and row, for any row length.  Blocks
// find the long rows by checking kTrLongThreads rows at a time.
template <typename T>
__global__ void __launch_bounds__(kTrLongThreads, 1)
    k_tr_sort_long(const int* __restrict__ trp, int nrows_t, int nkeys, int* tcol, T* tval, int* tmpc, T* tmpv,
                   bool has_val) {
    extern __shared__ __align__(16) unsigned trsm[];
    unsigned* bm = trsm;
    unsigned* pre = trsm + kTrWords;
    __shared__ int scratch[34];
    __shared__ int longs[kTrLongThreads];
    __shared__ int nlong;
    const int tid = threadIdx.x;
    for (long long k0 = (long long)blockIdx.x * kTrLongThreads; k0 < nrows_t;
         k0 += (long long)gridDim.x * kTrLongThreads) {
        if (tid == 0) nlong = 0;
        __syncthreads();
        const long long kk = k0 + tid;
        if (kk < nrows_t && __ldg(trp + kk + 1) - __ldg(trp + kk) > kTrShort) longs[atomicAdd(&nlong, 1)] = (int)kk;
        __syncthreads();
        const int nl = nlong;
        for (int x = 0; x < nl; ++x) {
            const int k = longs[x];
            const int lo = __ldg(trp + k), hi = __ldg(trp + k + 1);
            int base = 0;  // keys in earlier windows
            for (int w0 = 0; w0 < nkeys; w0 += kTrWindow) {
                const int words = min(kTrWords, (nkeys - w0 + 31) / 32);
                for (int i = tid; i < words; i += kTrLongThreads) bm[i] = 0u;
                __syncthreads();
                for (int e = lo + tid; e < hi; e += kTrLongThreads) {
                    const unsigned r = (unsigned)(tcol[e] - w0);
                    if (r < (unsigned)kTrWindow) atomicOr(bm + (r >> 5), 1u << (r & 31));
                }
                __syncthreads();
                constexpr int per = kTrWords / kTrLongThreads;
                const int beg = tid * per;
                int loc = 0;
                for (int i = beg; i < beg + per && i < words; ++i) loc += __popc(bm[i]);
                int tot;
                int run = Team<kTrLongThreads>::scan_excl(loc, &tot, scratch);
                for (int i = beg; i < beg + per && i < words; ++i) {
                    pre[i] = (unsigned)run;
                    run += __popc(bm[i]);
                }
                __syncthreads();
                for (int e = lo + tid; e < hi; e += kTrLongThreads) {
                    const int key = tcol[e];
                    const unsigned r = (unsigned)(key - w0);
                    if (r < (unsigned)kTrWindow) {
                        const int rank = base + (int)pre[r >> 5] + __popc(bm[r >> 5] & ((1u << (r & 31)) - 1u));
                        tmpc[lo + rank] = key;
                        if (has_val) tmpv[lo + rank] = tval[e];
                    }
                }
                base += tot;
                __syncthreads();
            }
            for (int e = lo + tid; e < hi; e += kTrLongThreads) {
                tcol[e] = tmpc[e];
                if (has_val) tval[e] = tmpv[e];
            }
            __syncthreads();
        }
    }
}

cudaError_t launch_transpose(int dtype, const int* rp, const int* col, const void* val, int nrows, int ncols,
                             long long nnz, int* trp, int* tcol, void* tval, int* work, void* workv, long long* bsum,
                             long long* ex, int sms, cudaStream_t s) {
    // work: ncols ints (counts, then cursors); ex: ncols + 1 long longs
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(int) * (size_t)std::max(ncols, 1), s);
    if (e != cudaSuccess) return e;
    if (nnz > 0) k_tr_count<<<(int)std::min<long long>((nnz + 255) / 256, (long long)sms * 16), 256, 0, s>>>(col, nnz, work);
    e = launch_scan(work, ncols, bsum, ex, s);
    if (e != cudaSuccess) return e;
    // row_ptr of X^T from the 64-bit exclusive sums (nnz fits int32)
    e = launch_ll_to_int(ex, ncols + 1, trp, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(work, 0, sizeof(int) * (size_t)std::max(ncols, 1), s);
    if (e != cudaSuccess) return e;
    if (nrows > 0) {
        if (dtype == 1)
            k_tr_scatter<double><<<(nrows + 127) / 128, 128, 0, s>>>(rp, col, static_cast<const double*>(val), nrows, trp,
                                                                     work, tcol, static_cast<double*>(tval));
        else
            k_tr_scatter<float><<<(nrows + 127) / 128, 128, 0, s>>>(rp, col, static_cast<const float*>(val), nrows, trp,
                                                                    work, tcol, static_cast<float*>(tval));
    }
    if (ncols > 0 && nnz > 0) {
        const int blocks = (int)std::min<long long>(((long long)ncols + 7) / 8, (long long)sms * 8);
        int* tmpc = reinterpret_cast<int*>(workv);
        void* tmpv = static_cast<char*>(workv) + ((sizeof(int) * (size_t)nnz + 15) & ~size_t(15));
        if (dtype == 1)
            k_tr_sort<double><<<blocks, 256, 0, s>>>(trp, ncols, tcol, static_cast<double*>(tval), tmpc,
                                                     static_cast<double*>(tmpv), val != nullptr);
        else
            k_tr_sort<float><<<blocks, 256, 0, s>>>(trp, ncols, tcol, static_cast<float*>(tval), tmpc,
                                                    static_cast<float*>(tmpv), val != nullptr);
        // rows longer than kTrShort exist only if nnz exceeds it
        if (nnz > kTrShort) {
            const int lb = (int)std::min<long long>(((long long)ncols + kTrLongThreads - 1) / kTrLongThreads, sms);
            if (dtype == 1) {
                cudaFuncSetAttribute(k_tr_sort_long<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrLongSmem);
                k_tr_sort_long<double><<<lb, kTrLongThreads, kTrLongSmem, s>>>(
                    trp, ncols, nrows, tcol, static_cast<double*>(tval), tmpc, static_cast<double*>(tmpv),
                    val != nullptr);
            } else {
                cudaFuncSetAttribute(k_tr_sort_long<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrLongSmem);
                k_tr_sort_long<float><<<lb, kTrLongThreads, kTrLongSmem, s>>>(
                    trp, ncols, nrows, tcol, static_cast<float*>(tval), tmpc, static_cast<float*>(tmpv),
                    val != nullptr);
            }
        }
    }
    return cudaGetLastError();
}

}  // namespace tsg
