// One Markov-clustering iteration (paper Sec. 5.6) fused into the expansion.
//
// The Markov matrix M is stored transposed (row r = column r of M), so the
// expansion (M M)^T = Mt Mt and every column operation are row-local.  Per
// row r (one block):
//   expand    e_j = sum_k Mt[r,k] Mt[k,j]: float products, double sums, in a
//             dense double accumulator private to the block (atomic adds in
//             L2), with a bitmap and a list of the touched columns
//   inflate   w_j = e_j^r (r = 2: e_j * e_j), v_j = w_j / sum w
//   prune     keep v_j >= prune; none kept -> keep the largest
//   top-k     more than k kept -> keep the k largest (radix selection on the
//             double's bits), equal values: smaller column first
//   renorm    out_j = float(v_j / sum of kept v)
//   write     the kept entries sorted by column (bitonic sort in shared
//             memory) at the row's upper-bound slot min(u_r, k)
// A second kernel compacts the kept rows into the caller's CSR.
// All keep/drop decisions are taken in double.
#include <algorithm>

#include "internal.h"

namespace tsg {

constexpr int kMclThreads = 256;
constexpr int kMclMaxK = 1024;

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < kMclThreads / 32 ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) sh[0] = t;
    }
    __syncthreads();
    t = sh[0];
    __syncthreads();
    return t;
}

__device__ __forceinline__ int block_sum_i(int v, int* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    int t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < kMclThreads / 32 ? sh[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) sh[0] = t;
    }
    __syncthreads();
    t = sh[0];
    __syncthreads();
    return t;
}

struct MclArgs {
    int n;
    const int* rp;
    const int* col;
    const float* val;
    const long long* ub_off;  // n + 1: slot of each row's kept entries
    int* tmp_col;
    float* tmp_val;
    int* kept;                // kept entries per row
    double* dense;            // per block: n doubles
    unsigned* bitmap;         // per block: ceil(n / 32) words
    int* touched;             // per block: n ints
    long long stride;         // n rounded up
    long long bm_words;
    int* row_counter;
    double inflation;
    double prune;
    int topk;
    unsigned* status;
};

struct MclShared {
    int row, cnt;
    unsigned long long prefix;
    int kk;
    int bestj;
    double red[32];
    int ired[32];
    unsigned hist[256];
    int kcol[kMclMaxK];
    float kval[kMclMaxK];
};

__global__ void __launch_bounds__(kMclThreads) k_mcl_rows(MclArgs a) {
    __shared__ MclShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* D = a.dense + (long long)blockIdx.x * a.stride;
    unsigned* BM = a.bitmap + (long long)blockIdx.x * a.bm_words;
    int* L = a.touched + (long long)blockIdx.x * a.stride;
    const bool square = a.inflation == 2.0;
    for (;;) {
        if (tid == 0) {
            sh.row = atomicAdd(a.row_counter, 1);
            sh.cnt = 0;
        }
        __syncthreads();
        const int r = sh.row;
        if (r >= a.n) break;

        // ---- expansion into the dense accumulator
        const int e0 = __ldg(a.rp + r), e1 = __ldg(a.rp + r + 1);
        for (int e = e0 + warp; e < e1; e += kMclThreads / 32) {
            const int k = __ldg(a.col + e);
            const float av = __ldg(a.val + e);
            const int f0 = __ldg(a.rp + k), f1 = __ldg(a.rp + k + 1);
            for (int f = f0 + lane; f < f1; f += 32) {
                const int j = __ldg(a.col + f);
                const double p = (double)__fmul_rn(av, __ldg(a.val + f));
                atomicAdd(D + j, p);
                const unsigned bit = 1u << (j & 31);
                if (!(atomicOr(BM + (j >> 5), bit) & bit)) L[atomicAdd(&sh.cnt, 1)] = j;
            }
        }
        __threadfence();
        __syncthreads();
        const int c = sh.cnt;

        // ---- inflation: v_j = w_j / sum w
        double loc = 0.0;
        for (int i = tid; i < c; i += kMclThreads) {
            const double x = __ldcg(D + L[i]);
            loc += square ? x * x : pow(x, a.inflation);
        }
        const double s = block_sum_d(loc, sh.red);
        auto vof = [&](int j) {
            const double x = __ldcg(D + j);
            return (square ? x * x : pow(x, a.inflation)) / s;
        };

        // ---- prune count and the largest entry (ties: smaller column)
        int nk = 0;
        double vmax = -1.0;
        int jmax = 0x7fffffff;
        for (int i = tid; i < c; i += kMclThreads) {
            const int j = L[i];
            const double v = vof(j);
            nk += v >= a.prune;
            if (v > vmax || (v == vmax && j < jmax)) {
                vmax = v;
                jmax = j;
            }
        }
        const int nkeep = block_sum_i(nk, sh.ired);
        // arg-max over the block: the largest double, then the smallest column
        {
            double bv = vmax;
            int bj = jmax;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
                if (ov > bv || (ov == bv && oj < bj)) {
                    bv = ov;
                    bj = oj;
                }
            }
            if (lane == 0) {
                sh.red[warp] = bv;
                sh.ired[warp] = bj;
            }
            __syncthreads();
            if (tid == 0) {
                double gv = sh.red[0];
                int gj = sh.ired[0];
                for (int w = 1; w < kMclThreads / 32; ++w)
                    if (sh.red[w] > gv || (sh.red[w] == gv && sh.ired[w] < gj)) {
                        gv = sh.red[w];
                        gj = sh.ired[w];
                    }
                sh.bestj = gj;
            }
            __syncthreads();
        }

        // ---- the keep rule: mode 0 prune only, 1 largest only, 2 top-k
        int mode = nkeep == 0 ? 1 : (nkeep > a.topk ? 2 : 0);
        unsigned long long tkey = 0;  // top-k: the k-th largest value's bits
        int tie_j = 0x7fffffff;       // and the last column kept among ties
        if (mode == 2) {
            // radix selection of the k-th largest key among kept candidates
            if (tid == 0) {
                sh.prefix = 0ull;
                sh.kk = a.topk;
            }
            unsigned long long mask = 0ull;
            for (int shift = 56; shift >= 0; shift -= 8) {
                for (int b = tid; b < 256; b += kMclThreads) sh.hist[b] = 0u;
                __syncthreads();
                const unsigned long long pre = sh.prefix;
                for (int i = tid; i < c; i += kMclThreads) {
                    const double v = vof(L[i]);
                    if (v < a.prune) continue;
                    const unsigned long long key = (unsigned long long)__double_as_longlong(v);
                    if ((key & mask) == pre) atomicAdd(&sh.hist[(key >> shift) & 255u], 1u);
                }
                __syncthreads();
                if (tid == 0) {
                    int kk = sh.kk;
                    int d = 255;
                    for (; d > 0; --d) {
                        if ((int)sh.hist[d] >= kk) break;
                        kk -= sh.hist[d];
                    }
                    sh.kk = kk;
                    sh.prefix = pre | ((unsigned long long)d << shift);
                }
                mask |= 0xffull << shift;
                __syncthreads();
            }
            tkey = sh.prefix;
            const int need = sh.kk;  // entries equal to the cut that are kept
            __syncthreads();         // everyone has the cut before it is reused
            // among entries equal to the cut, keep the `need` smallest columns
            if (tid == 0) {
                sh.prefix = 0ull;
                sh.kk = need;
            }
            unsigned jmask = 0u;
            __syncthreads();
            for (int shift = 24; shift >= 0; shift -= 8) {
                for (int b = tid; b < 256; b += kMclThreads) sh.hist[b] = 0u;
                __syncthreads();
                const unsigned pre = (unsigned)sh.prefix;
                for (int i = tid; i < c; i += kMclThreads) {
                    const int j = L[i];
                    const double v = vof(j);
                    if ((unsigned long long)__double_as_longlong(v) != tkey) continue;
                    if (((unsigned)j & jmask) == pre) atomicAdd(&sh.hist[((unsigned)j >> shift) & 255u], 1u);
                }
                __syncthreads();
                if (tid == 0) {
                    int kk = sh.kk;
                    int d = 0;
                    for (; d < 255; ++d) {
                        if ((int)sh.hist[d] >= kk) break;
                        kk -= sh.hist[d];
                    }
                    sh.kk = kk;
                    sh.prefix = pre | ((unsigned)d << shift);
                }
                jmask |= 0xffu << shift;
                __syncthreads();
            }
            tie_j = (int)sh.prefix;
        }
        const int bestj = sh.bestj;
        auto keep = [&](int j, double v) {
            if (mode == 1) return j == bestj;
            if (v < a.prune) return false;
            if (mode == 0) return true;
            const unsigned long long key = (unsigned long long)__double_as_longlong(v);
            return key > tkey || (key == tkey && j <= tie_j);
        };

        // ---- renormalise over the kept entries and gather them
        double kl = 0.0;
        for (int i = tid; i < c; i += kMclThreads) {
            const int j = L[i];
            const double v = vof(j);
            if (keep(j, v)) kl += v;
        }
        const double t = block_sum_d(kl, sh.red);
        if (tid == 0) sh.cnt = 0;
        __syncthreads();
        for (int i = tid; i < c; i += kMclThreads) {
            const int j = L[i];
            const double v = vof(j);
            if (keep(j, v)) {
                const int q = atomicAdd(&sh.cnt, 1);
                if (q < kMclMaxK) {
                    sh.kcol[q] = j;
                    sh.kval[q] = (float)(v / t);
                }
            }
        }
        __syncthreads();
        const int nout = sh.cnt;
        const long long slot = __ldg(a.ub_off + r);
        const int cap = (int)(__ldg(a.ub_off + r + 1) - slot);
        if (nout > kMclMaxK || nout > cap) {
            if (tid == 0) atomicOr(a.status, kStatusInternal);
        } else {
            // bitonic sort of the kept entries by column (padding sorts last)
            int P = 1;
            while (P < nout) P <<= 1;
            for (int i = nout + tid; i < P; i += kMclThreads) sh.kcol[i] = 0x7fffffff;
            __syncthreads();
            for (int size = 2; size <= P; size <<= 1) {
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    for (int i = tid; i < P; i += kMclThreads) {
                        const int pj = i ^ stride;
                        if (pj > i) {
                            const bool up = (i & size) == 0;
                            const int ci = sh.kcol[i], cj = sh.kcol[pj];
                            if ((ci > cj) == up) {
                                sh.kcol[i] = cj;
                                sh.kcol[pj] = ci;
                                const float t2 = sh.kval[i];
                                sh.kval[i] = sh.kval[pj];
                                sh.kval[pj] = t2;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            for (int q = tid; q < nout; q += kMclThreads) {
                a.tmp_col[slot + q] = sh.kcol[q];
                a.tmp_val[slot + q] = sh.kval[q];
            }
            if (tid == 0) a.kept[r] = nout;
        }
        // ---- clear the accumulator for the next row
        __syncthreads();
        for (int i = tid; i < c; i += kMclThreads) {
            const int j = L[i];
            __stcg(D + j, 0.0);
            BM[j >> 5] = 0u;
        }
        __threadfence();
        __syncthreads();
    }
}

__global__ void k_mcl_bounds(const int* __restrict__ rp, const int* __restrict__ col, int n, int topk, int* ub) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    long long u = 0;
    for (int e = __ldg(rp + r); e < __ldg(rp + r + 1) && u < topk; ++e) {
        const int k = __ldg(col + e);
        u += __ldg(rp + k + 1) - __ldg(rp + k);
    }
    ub[r] = (int)(u < topk ? u : topk);
}

__global__ void k_mcl_collect(int n, const long long* __restrict__ ub_off, const int* __restrict__ tmp_col,
                              const float* __restrict__ tmp_val, const int* __restrict__ orp, int* ocol,
                              float* oval) {
    const int lane = threadIdx.x & 31;
    for (int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += gridDim.x * (blockDim.x >> 5)) {
        const long long s = __ldg(ub_off + r);
        const int o = __ldg(orp + r), len = __ldg(orp + r + 1) - o;
        for (int q = lane; q < len; q += 32) {
            ocol[o + q] = __ldg(tmp_col + s + q);
            oval[o + q] = __ldg(tmp_val + s + q);
        }
    }
}

cudaError_t launch_mcl_bounds(const int* rp, const int* col, int n, int topk, int* ub, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_mcl_bounds<<<(n + 255) / 256, 256, 0, s>>>(rp, col, n, topk, ub);
    return cudaGetLastError();
}

cudaError_t launch_mcl_rows(const MclLaunch& l, int blocks, cudaStream_t s) {
    MclArgs a;
    a.n = l.n;
    a.rp = l.rp;
    a.col = l.col;
    a.val = l.val;
    a.ub_off = l.ub_off;
    a.tmp_col = l.tmp_col;
    a.tmp_val = l.tmp_val;
    a.kept = l.kept;
    a.dense = l.dense;
    a.bitmap = l.bitmap;
    a.touched = l.touched;
    a.stride = l.stride;
    a.bm_words = l.bm_words;
    a.row_counter = l.row_counter;
    a.inflation = l.inflation;
    a.prune = l.prune;
    a.topk = l.topk;
    a.status = l.status;
    k_mcl_rows<<<blocks, kMclThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mcl_collect(int n, const long long* ub_off, const int* tmp_col, const float* tmp_val,
                               const int* orp, int* ocol, float* oval, int sms, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (int)std::min<long long>(((long long)n + 7) / 8, (long long)sms * 16);
    k_mcl_collect<<<blocks, 256, 0, s>>>(n, ub_off, tmp_col, tmp_val, orp, ocol, oval);
    return cudaGetLastError();
}

}  // namespace tsg
