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
// All keep/drop decisions are taken in double.  The double pipe is narrow on
// this part, so each touched entry costs one square, one add and two
// compares per pass: the quotient v = w / s is formed only for the
// entries that can reach the prune or the maximum, and the prune survivors
// (at most about 1 / prune of them, as the v sum to 1) go to a compact
// candidate list that the top-k passes and the gather read.
#include <algorithm>

#include "internal.h"

namespace tsg {

constexpr int kMclThreads = 256;
constexpr int kMclMaxK = 1024;
constexpr int kMclUnroll = 4;

// fire-and-forget double add in L2 (no value returned to the thread)
__device__ __forceinline__ void red_add_f64(double* p, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

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

__device__ __forceinline__ double block_max_d(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = sh[0];
    for (int i = 1; i < kMclThreads / 32; ++i) t = fmax(t, sh[i]);
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
    unsigned long long* ckey; // per block: ccap candidate values (double bits) ...
    int* ccol;                // ... and their columns
    int ccap;
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
    double bestv;
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
            // four products per lane in flight: the bitmap's fetch-or must
            // return before its column can be listed, so its round trips
            // are overlapped four at a time; the sums need no return
            for (int f = f0 + lane; f < f1; f += 32 * kMclUnroll) {
                int jj[kMclUnroll];
                unsigned old[kMclUnroll];
#pragma unroll
                for (int u = 0; u < kMclUnroll; ++u) {
                    const int g = f + 32 * u;
                    jj[u] = g < f1 ? __ldg(a.col + g) : -1;
                    if (jj[u] >= 0) {
                        const double p = (double)__fmul_rn(av, __ldg(a.val + g));
                        red_add_f64(D + jj[u], p);
                        old[u] = atomicOr(BM + (jj[u] >> 5), 1u << (jj[u] & 31));
                    }
                }
#pragma unroll
                for (int u = 0; u < kMclUnroll; ++u)
                    if (jj[u] >= 0 && !(old[u] & (1u << (jj[u] & 31)))) L[atomicAdd(&sh.cnt, 1)] = jj[u];
            }
        }
        __threadfence();
        __syncthreads();
        const int c = sh.cnt;

        // ---- inflation: w_j = e_j^r; s = sum w (w is formed again from e
        // in the next pass rather than stored and reloaded)
        double loc = 0.0, wtop = 0.0;
        for (int i = tid; i < c; i += kMclThreads) {
            const double x = __ldcg(D + L[i]);
            const double w = square ? x * x : pow(x, a.inflation);
            loc += w;
            wtop = fmax(wtop, w);
        }
        const double s = block_sum_d(loc, sh.red);
        const double wmax = block_max_d(wtop, sh.red);

        // ---- v_j = w_j / s; candidates v_j >= prune; the largest v (ties:
        // smaller column).  With s > 0 the division is monotone, so only the
        // entries whose w is within 2^-45 (relative) of prune * s or of the
        // largest w can reach the prune or the maximum: the others are
        // skipped without dividing (their rounded quotient stays below).
        // (normal-range products only: there the two roundings stay far
        // inside the 2^-45 margin)
        const bool filt = a.prune >= 0.0 && s > 0.0 && s <= 1.7e308 && wmax >= 0x1p-1000 && wmax <= 1.7e308 &&
                          (a.prune == 0.0 || a.prune * s >= 0x1p-1000);
        const double wlo = filt ? a.prune * s * (1.0 - 0x1p-45) : 0.0;
        const double whi = filt ? wmax * (1.0 - 0x1p-45) : 0.0;
        unsigned long long* CK = a.ckey + (long long)blockIdx.x * a.ccap;
        int* CC = a.ccol + (long long)blockIdx.x * a.ccap;
        if (tid == 0) sh.cnt = 0;
        __syncthreads();
        double vmax = -1.0;
        int jmax = 0x7fffffff;
        for (int i = tid; i < c; i += kMclThreads) {
            const int j = L[i];
            const double x = __ldcg(D + j);
            const double w = square ? x * x : pow(x, a.inflation);
            if (filt && !(w >= wlo) && !(w >= whi)) continue;
            const double v = w / s;
            if (v >= a.prune) {
                const int q = atomicAdd(&sh.cnt, 1);
                if (q < a.ccap) {
                    CK[q] = (unsigned long long)__double_as_longlong(v);
                    CC[q] = j;
                }
            }
            if (v > vmax || (v == vmax && j < jmax)) {
                vmax = v;
                jmax = j;
            }
        }
        __syncthreads();
        const int nkeep = sh.cnt;
        const int ncand = nkeep < a.ccap ? nkeep : a.ccap;
        if (tid == 0 && nkeep > a.ccap) atomicOr(a.status, kStatusInternal);

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
                sh.bestv = gv;
            }
            __syncthreads();
        }

        // ---- the keep rule: mode 0 prune only, 1 largest only, 2 top-k
        const int mode = nkeep == 0 ? 1 : (nkeep > a.topk ? 2 : 0);
        unsigned long long tkey = 0;  // top-k: the k-th largest value's bits
        int tie_j = 0x7fffffff;       // and the last column kept among ties
        if (mode == 2) {
            // radix selection of the k-th largest key among the candidates
            // (non-negative doubles: the bit patterns order as the values)
            if (tid == 0) {
                sh.prefix = 0ull;
                sh.kk = a.topk;
            }
            unsigned long long mask = 0ull;
            for (int shift = 56; shift >= 0; shift -= 8) {
                for (int b = tid; b < 256; b += kMclThreads) sh.hist[b] = 0u;
                __syncthreads();
                const unsigned long long pre = sh.prefix;
                for (int q = tid; q < ncand; q += kMclThreads) {
                    const unsigned long long key = CK[q];
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
                for (int q = tid; q < ncand; q += kMclThreads) {
                    if (CK[q] != tkey) continue;
                    const unsigned j = (unsigned)CC[q];
                    if ((j & jmask) == pre) atomicAdd(&sh.hist[(j >> shift) & 255u], 1u);
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
        auto kept_q = [&](int q) {
            if (mode == 0) return true;
            const unsigned long long key = CK[q];
            return key > tkey || (key == tkey && CC[q] <= tie_j);
        };

        // ---- renormalise over the kept entries and gather them
        double kl = 0.0;
        if (mode == 1) {
            if (tid == 0 && bestj != 0x7fffffff) kl = sh.bestv;
        } else {
            for (int q = tid; q < ncand; q += kMclThreads)
                if (kept_q(q)) kl += __longlong_as_double((long long)CK[q]);
        }
        const double t = block_sum_d(kl, sh.red);
        if (tid == 0) sh.cnt = 0;
        __syncthreads();
        if (mode == 1) {
            if (tid == 0 && bestj != 0x7fffffff) {
                sh.kcol[0] = bestj;
                sh.kval[0] = (float)(sh.bestv / t);
                sh.cnt = 1;
            }
        } else {
            for (int q = tid; q < ncand; q += kMclThreads) {
                if (!kept_q(q)) continue;
                const int o = atomicAdd(&sh.cnt, 1);
                if (o < kMclMaxK) {
                    sh.kcol[o] = CC[q];
                    sh.kval[o] = (float)(__longlong_as_double((long long)CK[q]) / t);
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
        // ---- clear the accumulator and the bitmap for the next row (a pass
        // of its own: a store right behind the load of the same word in the
        // candidate pass held every iteration for the load's round trip)
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
    a.ckey = l.ckey;
    a.ccol = l.ccol;
    a.ccap = l.ccap;
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
