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

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    unsigned long long t = sh[0];
    for (int i = 1; i < kMclThreads / 32; ++i) t = sh[i] > t ? sh[i] : t;
    __syncthreads();
    return t;
}

// The double pipe is narrow on this part: zero tests and threshold tests
// run on the bit patterns.  |x| as bits orders as |x| (NaN above +inf).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
// Bits of a bound on |x| below which the rounded square x * x stays below
// w (w >= 0, normal or zero): sqrt(w) less a 2^-40 margin, far beyond the
// roundings of the root, the product and the square.
__device__ __forceinline__ unsigned long long sq_bound_bits(double w) {
    return w > 0.0 ? abs_bits(sqrt(w) * (1.0 - 0x1p-40)) : 0ull;
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
    const unsigned char* heavy;  // row flags: 1 batched path, 2 window-summed path
    int skip;                    // flags (bits) whose rows this kernel leaves
    int positive;                // every value is positive and no product underflows to 0
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
};

// Keep rule, renormalisation and output of row r from its candidates (the
// entries with v >= prune: CK their values' bits, CC their columns; nkeep of
// them found, the first ncand stored) and, when none reached the prune, the
// largest entry sh.bestj / sh.bestv.  Called by every thread of the block.
__device__ void mcl_finish_row(const MclArgs& a, MclShared& sh, int* kcol, float* kval, int r,
                               const unsigned long long* CK, const int* CC, int nkeep, int ncand) {
    const int tid = threadIdx.x;
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
            kcol[0] = bestj;
            kval[0] = (float)(sh.bestv / t);
            sh.cnt = 1;
        }
    } else {
        for (int q = tid; q < ncand; q += kMclThreads) {
            if (!kept_q(q)) continue;
            const int o = atomicAdd(&sh.cnt, 1);
            if (o < kMclMaxK) {
                kcol[o] = CC[q];
                kval[o] = (float)(__longlong_as_double((long long)CK[q]) / t);
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
        for (int i = nout + tid; i < P; i += kMclThreads) kcol[i] = 0x7fffffff;
        __syncthreads();
        for (int size = 2; size <= P; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = tid; i < P; i += kMclThreads) {
                    const int pj = i ^ stride;
                    if (pj > i) {
                        const bool up = (i & size) == 0;
                        const int ci = kcol[i], cj = kcol[pj];
                        if ((ci > cj) == up) {
                            kcol[i] = cj;
                            kcol[pj] = ci;
                            const float t2 = kval[i];
                            kval[i] = kval[pj];
                            kval[pj] = t2;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int q = tid; q < nout; q += kMclThreads) {
            a.tmp_col[slot + q] = kcol[q];
            a.tmp_val[slot + q] = kval[q];
        }
        if (tid == 0) a.kept[r] = nout;
    }
}

__global__ void __launch_bounds__(kMclThreads) k_mcl_rows(MclArgs a) {
    __shared__ MclShared sh;
    __shared__ int kcol[kMclMaxK];
    __shared__ float kval[kMclMaxK];
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
        if (a.heavy && (a.heavy[r] & a.skip)) {
            __syncthreads();  // every thread has read the row before the next is drawn
            continue;
        }

        // ---- expansion into the dense accumulator
        const int e0 = __ldg(a.rp + r), e1 = __ldg(a.rp + r + 1);
        for (int e = e0 + warp; e < e1; e += kMclThreads / 32) {
            const int k = __ldg(a.col + e);
            const float av = __ldg(a.val + e);
            const int f0 = __ldg(a.rp + k), f1 = __ldg(a.rp + k + 1);
            // four products per lane in flight: the first-touch test must
            // return before its column can be listed, so the round trips are
            // overlapped four at a time
            if (a.positive) {
                // every value is positive, so a sum is positive once touched:
                // the add's old value 0 marks the first touch (one atomic per
                // product, no bitmap)
                for (int f = f0 + lane; f < f1; f += 32 * kMclUnroll) {
                    int jj[kMclUnroll];
                    double old[kMclUnroll];
#pragma unroll
                    for (int u = 0; u < kMclUnroll; ++u) {
                        const int g = f + 32 * u;
                        jj[u] = g < f1 ? __ldg(a.col + g) : -1;
                        if (jj[u] >= 0) old[u] = atomicAdd(D + jj[u], (double)__fmul_rn(av, __ldg(a.val + g)));
                    }
#pragma unroll
                    for (int u = 0; u < kMclUnroll; ++u)
                        if (jj[u] >= 0 && old[u] == 0.0) L[atomicAdd(&sh.cnt, 1)] = jj[u];
                }
                continue;
            }
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
        // (square: one fused multiply-add per entry; the largest w is the
        // square of the largest |x|, found on the bits)
        double loc = 0.0, wtop = 0.0;
        unsigned long long amax = 0;
        for (int i = tid; i < c; i += kMclThreads) {
            const double x = __ldcg(D + L[i]);
            if (square) {
                loc = fma(x, x, loc);
                const unsigned long long ax = abs_bits(x);
                amax = ax > amax ? ax : amax;
            } else {
                const double w = pow(x, a.inflation);
                loc += w;
                wtop = fmax(wtop, w);
            }
        }
        const double s = block_sum_d(loc, sh.red);
        double wmax;
        if (square) {
            const double xm = __longlong_as_double(
                (long long)block_max_u64(amax, reinterpret_cast<unsigned long long*>(sh.red)));
            wmax = xm * xm;
        } else {
            wmax = block_max_d(wtop, sh.red);
        }

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
        const unsigned long long xlo = filt && square ? sq_bound_bits(wlo) : 0ull;
        const unsigned long long xhi = filt && square ? sq_bound_bits(whi) : 0ull;
        const unsigned long long xskip = xlo < xhi ? xlo : xhi;
        unsigned long long* CK = a.ckey + (long long)blockIdx.x * a.ccap;
        int* CC = a.ccol + (long long)blockIdx.x * a.ccap;
        if (tid == 0) sh.cnt = 0;
        __syncthreads();
        double vmax = -1.0;
        int jmax = 0x7fffffff;
        for (int i = tid; i < c; i += kMclThreads) {
            const int j = L[i];
            const double x = __ldcg(D + j);
            if (abs_bits(x) < xskip) continue;
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

        mcl_finish_row(a, sh, kcol, kval, r, CK, CC, nkeep, ncand);
        // ---- clear the accumulator and the bitmap for the next row (a pass
        // of its own: a store right behind the load of the same word in the
        // candidate pass held every iteration for the load's round trip)
        __syncthreads();
        for (int i = tid; i < c; i += kMclThreads) {
            const int j = L[i];
            __stcg(D + j, 0.0);
            if (!a.positive) BM[j >> 5] = 0u;
        }
        __threadfence();
        __syncthreads();
    }
}

// ------------------------------------------------------ bucketed mid rows
//
// Rows between the small and the heavy thresholds, positive values only.
// The row's products are counted per column window of W = 2^lw columns,
// scattered into a staging buffer in window order (column, float product:
// 8 bytes), and each window is then summed in shared memory, where the add
// that finds 0 lists the column; the window's entries are emitted as a
// compact (column, e) list in column-window order, which the prune and
// top-k passes read contiguously.  Every global access but the B-row reads
// is a stream, where the per-block kernel's random adds into an 8 MB
// accumulator miss L2.

__host__ __device__ inline size_t mcl_window_bytes(int lw) {
    const size_t b = 8 * ((size_t)1 << lw);
    return b > 8 * (size_t)kMclMaxK ? b : 8 * (size_t)kMclMaxK;
}

struct MclBucketArgs {
    const int* list;     // the rows of this path
    int count;           // how many
    int* counter;        // next row to take
    int2* stage;         // per block: cap entries (column, float product bits)
    int* ej;             // per block: cap emitted columns (values overwrite stage)
    long long cap;
    int lw;              // log2 of the window width
    int nbk;             // windows: ceil(n / W)
};

__global__ void __launch_bounds__(kMclThreads) k_mcl_rows_bucket(MclArgs a, MclBucketArgs bk) {
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ MclShared sh;
    __shared__ int s_row, s_lc[2];
    const int W = 1 << bk.lw, NB = bk.nbk;
    // window sums (at least 8 KB: the row's kept entries are gathered there
    // at the end) | window-local touched columns | window offsets, cursors
    const size_t wb = mcl_window_bytes(bk.lw);
    double* win = reinterpret_cast<double*>(dyn);
    unsigned short* tl = reinterpret_cast<unsigned short*>(dyn + wb);
    int* off = reinterpret_cast<int*>(dyn + wb + 2 * (size_t)W);  // NB + 1
    int* cur = off + NB + 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int2* stage = bk.stage + (long long)blockIdx.x * bk.cap;
    double* ex = reinterpret_cast<double*>(stage);
    int* ej = bk.ej + (long long)blockIdx.x * bk.cap;
    unsigned long long* CK = a.ckey + (long long)blockIdx.x * a.ccap;
    int* CC = a.ccol + (long long)blockIdx.x * a.ccap;
    const bool square = a.inflation == 2.0;
    for (int i = tid; i < W; i += kMclThreads) win[i] = 0.0;
    if (tid == 0) {
        s_lc[0] = 0;
        s_lc[1] = 0;
    }
    for (;;) {
        if (tid == 0) s_row = atomicAdd(bk.counter, 1);
        for (int i = tid; i < NB; i += kMclThreads) cur[i] = 0;
        __syncthreads();
        const int q = s_row;
        if (q >= bk.count) break;
        const int r = bk.list[q];
        const int e0 = __ldg(a.rp + r), e1 = __ldg(a.rp + r + 1);
        // ---- products per window
        for (int e = e0 + warp; e < e1; e += kMclThreads / 32) {
            const int k = __ldg(a.col + e);
            const int f0 = __ldg(a.rp + k), f1 = __ldg(a.rp + k + 1);
            for (int f = f0 + lane; f < f1; f += 32) atomicAdd(cur + (__ldg(a.col + f) >> bk.lw), 1);
        }
        __syncthreads();
        // ---- window offsets (one warp, 32 windows per step)
        if (warp == 0) {
            int run = 0;
            for (int b0 = 0; b0 < NB; b0 += 32) {
                const int b = b0 + lane;
                const int v = b < NB ? cur[b] : 0;
                int x = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                if (b < NB) off[b] = run + x - v;
                run += __shfl_sync(0xffffffffu, x, 31);
            }
            if (lane == 0) off[NB] = run;
        }
        __syncthreads();
        for (int i = tid; i < NB; i += kMclThreads) cur[i] = off[i];
        __syncthreads();
        // ---- scatter the products in window order
        for (int e = e0 + warp; e < e1; e += kMclThreads / 32) {
            const int k = __ldg(a.col + e);
            const float av = __ldg(a.val + e);
            const int f0 = __ldg(a.rp + k), f1 = __ldg(a.rp + k + 1);
            for (int f = f0 + lane; f < f1; f += 32) {
                const int j = __ldg(a.col + f);
                const float p = __fmul_rn(av, __ldg(a.val + f));
                const int pos = atomicAdd(cur + (j >> bk.lw), 1);
                stage[pos] = make_int2(j, __float_as_int(p));
            }
        }
        __syncthreads();
        // ---- each window: sums in shared memory, then the touched columns out
        double loc = 0.0;
        unsigned long long amax = 0;
        int c = 0, par = 0;
        for (int b = 0; b < NB; ++b) {
            const int o0 = off[b], o1 = off[b + 1];
            if (o0 == o1) continue;
            for (int i = o0 + tid; i < o1; i += kMclThreads) {
                const int2 ent = stage[i];
                const int jl = ent.x & (W - 1);
                if (atomicAdd(win + jl, (double)__int_as_float(ent.y)) == 0.0)
                    tl[atomicAdd(s_lc + par, 1)] = (unsigned short)jl;
            }
            __syncthreads();
            const int lc = s_lc[par];
            if (tid == 0) s_lc[par ^ 1] = 0;
            for (int t = tid; t < lc; t += kMclThreads) {
                const int jl = tl[t];
                const double x = win[jl];
                win[jl] = 0.0;
                ex[c + t] = x;  // slots of windows already summed
                ej[c + t] = (b << bk.lw) | jl;
                if (square) {
                    loc = fma(x, x, loc);
                    const unsigned long long ax = abs_bits(x);
                    amax = ax > amax ? ax : amax;
                }
            }
            c += lc;
            par ^= 1;
            __syncthreads();
        }
        if (tid == 0) {
            s_lc[0] = 0;
            s_lc[1] = 0;
        }
        // non-square inflation: the sum and the largest w from the list
        double wtop = 0.0;
        if (!square) {
            for (int i = tid; i < c; i += kMclThreads) {
                const double w = pow(ex[i], a.inflation);
                loc += w;
                wtop = fmax(wtop, w);
            }
        }
        const double s = block_sum_d(loc, sh.red);
        double wmax;
        if (square) {
            const double xm = __longlong_as_double(
                (long long)block_max_u64(amax, reinterpret_cast<unsigned long long*>(sh.red)));
            wmax = xm * xm;
        } else {
            wmax = block_max_d(wtop, sh.red);
        }

        // ---- candidates and the largest entry, as in k_mcl_rows
        const bool filt = a.prune >= 0.0 && s > 0.0 && s <= 1.7e308 && wmax >= 0x1p-1000 && wmax <= 1.7e308 &&
                          (a.prune == 0.0 || a.prune * s >= 0x1p-1000);
        const double wlo = filt ? a.prune * s * (1.0 - 0x1p-45) : 0.0;
        const double whi = filt ? wmax * (1.0 - 0x1p-45) : 0.0;
        const unsigned long long xlo = filt && square ? sq_bound_bits(wlo) : 0ull;
        const unsigned long long xhi = filt && square ? sq_bound_bits(whi) : 0ull;
        const unsigned long long xskip = xlo < xhi ? xlo : xhi;
        if (tid == 0) sh.cnt = 0;
        __syncthreads();
        double vmax = -1.0;
        int jmax = 0x7fffffff;
        for (int i = tid; i < c; i += kMclThreads) {
            const double x = ex[i];
            if (abs_bits(x) < xskip) continue;
            const double w = square ? x * x : pow(x, a.inflation);
            if (filt && !(w >= wlo) && !(w >= whi)) continue;
            const int j = ej[i];
            const double v = w / s;
            if (v >= a.prune) {
                const int qq = atomicAdd(&sh.cnt, 1);
                if (qq < a.ccap) {
                    CK[qq] = (unsigned long long)__double_as_longlong(v);
                    CC[qq] = j;
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
        // the kept entries are gathered in the window buffer (the windows
        // are done), which is zero again before the next row
        mcl_finish_row(a, sh, reinterpret_cast<int*>(win), reinterpret_cast<float*>(win) + kMclMaxK, r, CK, CC,
                       nkeep, ncand);
        __syncthreads();
        for (int i = tid; i < kMclMaxK; i += kMclThreads) win[i] = 0.0;
        __syncthreads();
    }
}

// Pilot of the window-summed path: block b expands row rows[b * step] into
// its private accumulator (positive values: the add that finds 0 counts a
// distinct column), adds the row's products and distinct columns to tot[0]
// and tot[1], and clears what it touched.  Rows whose products pile onto
// few columns (a clustered iterate) are summed faster by k_mcl_rows, whose
// accumulator footprint is then small and stays in L2.
__global__ void __launch_bounds__(kMclThreads) k_mcl_pilot(MclArgs a, const int* rows, int step,
                                                           unsigned long long* tot) {
    __shared__ int cnt;
    __shared__ unsigned long long prods;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* D = a.dense + (long long)blockIdx.x * a.stride;
    int* L = a.touched + (long long)blockIdx.x * a.stride;
    const int r = rows[(long long)blockIdx.x * step];
    if (tid == 0) {
        cnt = 0;
        prods = 0;
    }
    __syncthreads();
    const int e0 = __ldg(a.rp + r), e1 = __ldg(a.rp + r + 1);
    unsigned long long u = 0;
    for (int e = e0 + warp; e < e1; e += kMclThreads / 32) {
        const int k = __ldg(a.col + e);
        const float av = __ldg(a.val + e);
        const int f0 = __ldg(a.rp + k), f1 = __ldg(a.rp + k + 1);
        if (lane == 0) u += f1 - f0;
        for (int f = f0 + lane; f < f1; f += 32) {
            const int j = __ldg(a.col + f);
            if (atomicAdd(D + j, (double)__fmul_rn(av, __ldg(a.val + f))) == 0.0) L[atomicAdd(&cnt, 1)] = j;
        }
    }
    if (lane == 0) atomicAdd(&prods, u);
    __threadfence();
    __syncthreads();
    const int c = cnt;
    for (int i = tid; i < c; i += kMclThreads) __stcg(D + L[i], 0.0);
    if (tid == 0) {
        atomicAdd(tot, prods);
        atomicAdd(tot + 1, (unsigned long long)c);
    }
}


// ---------------------------------------------------------------- heavy rows
//
// Rows with many products (their distinct columns a large part of n) run in
// batches of a few rows whose dense accumulators stay resident in L2: the
// whole GPU expands the batch with return-free double adds (no bitmap, no
// touched list), then the accumulators are scanned densely for the sum and
// the largest w, then for the candidates (v >= prune) and the entries near
// the largest w, and one block per row takes the keep rule on those.  A row
// here decides exactly as in k_mcl_rows: untouched columns read 0 and are
// skipped, which with prune > 0 drops nothing the touched list would keep.

struct MclHeavyArgs {
    MclArgs a;
    const int* rows;          // the batch's rows
    int nb;                   // rows in the batch
    double* D;                // nb x stride dense accumulators, zero on entry
    double* s;                // per row: sum of w
    unsigned long long* wmax; // per row: bits of the largest w
    unsigned* flags;          // per row: 1 a negative or NaN w, 2 near-max list overflow
    int* ncand;               // per row: candidates found
    int* nmax;                // per row: near-max entries found
    unsigned long long* ck;   // per row: ccap candidate value bits
    int* cc;                  // per row: ccap candidate columns
    int* mlist;               // per row: kMclMaxList near-max columns
};

constexpr int kMclLongB = 512;  // B rows longer than this are split over the block

// Products of the batch: 8 A entries per block step, one per warp; a B row of
// at most kMclLongB entries is added by its warp, a longer one by the whole
// block (after the short ones), four products per lane per step.
__global__ void __launch_bounds__(kMclThreads) k_mcl_heavy_expand(MclHeavyArgs h) {
    __shared__ long long pre[kMclBatch + 1];
    __shared__ int lk[kMclThreads / 32], lb[kMclThreads / 32];
    __shared__ float lav[kMclThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const MclArgs& a = h.a;
    if (tid == 0) {
        long long t = 0;
        for (int b = 0; b < h.nb; ++b) {
            pre[b] = t;
            const int r = h.rows[b];
            t += __ldg(a.rp + r + 1) - __ldg(a.rp + r);
        }
        pre[h.nb] = t;
    }
    __syncthreads();
    const long long E = pre[h.nb];
    for (long long g = (long long)blockIdx.x * (kMclThreads / 32); g < E; g += (long long)gridDim.x * (kMclThreads / 32)) {
        const long long t = g + warp;
        lk[warp] = -1;
        if (t < E) {
            int b = 0;
            while (pre[b + 1] <= t) ++b;
            const int e = __ldg(a.rp + h.rows[b]) + (int)(t - pre[b]);
            const int k = __ldg(a.col + e);
            const float av = __ldg(a.val + e);
            const int f0 = __ldg(a.rp + k), f1 = __ldg(a.rp + k + 1);
            double* Db = h.D + (long long)b * a.stride;
            if (f1 - f0 <= kMclLongB) {
                for (int f = f0 + lane; f < f1; f += 32)
                    red_add_f64(Db + __ldg(a.col + f), (double)__fmul_rn(av, __ldg(a.val + f)));
            } else if (lane == 0) {
                lk[warp] = k;
                lb[warp] = b;
                lav[warp] = av;
            }
        }
        __syncthreads();
        for (int w = 0; w < kMclThreads / 32; ++w) {
            const int k = lk[w];
            if (k < 0) continue;
            const float av = lav[w];
            double* Db = h.D + (long long)lb[w] * a.stride;
            const int f0 = __ldg(a.rp + k), f1 = __ldg(a.rp + k + 1);
            for (int f = f0 + tid; f < f1; f += kMclThreads * kMclUnroll) {
#pragma unroll
                for (int u = 0; u < kMclUnroll; ++u) {
                    const int q = f + kMclThreads * u;
                    if (q < f1) red_add_f64(Db + __ldg(a.col + q), (double)__fmul_rn(av, __ldg(a.val + q)));
                }
            }
        }
        __syncthreads();
    }
}

// Dense passes: each thread takes chunks of 8 doubles (four 16-byte loads
// in flight); the rows are zero past n up to the stride, a multiple of 32.

// Dense pass 1 over row blockIdx.y of the batch: sum of w and the largest w
// over the touched (nonzero) columns.
__global__ void __launch_bounds__(kMclThreads) k_mcl_heavy_sums(MclHeavyArgs h) {
    __shared__ double red[32];
    const int b = blockIdx.y;
    const double2* D2 = reinterpret_cast<const double2*>(h.D + (long long)b * h.a.stride);
    const bool square = h.a.inflation == 2.0;
    const long long nch = h.a.stride / 8;
    double loc = 0.0, top = 0.0;
    unsigned long long amax = 0;
    bool bad = false;
    for (long long c = (long long)blockIdx.x * kMclThreads + threadIdx.x; c < nch; c += (long long)gridDim.x * kMclThreads) {
        double2 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = __ldcg(D2 + 4 * c + u);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const double x = (u & 1) ? q[u >> 1].y : q[u >> 1].x;
            const unsigned long long ax = abs_bits(x);
            if (ax == 0) continue;  // untouched (or a zero sum)
            if (square) {
                loc = fma(x, x, loc);
                amax = ax > amax ? ax : amax;
            } else {
                const double w = pow(x, h.a.inflation);
                loc += w;
                top = fmax(top, w);
                bad |= !(w >= 0.0);
            }
        }
    }
    const double ssum = block_sum_d(loc, red);
    double smax;
    if (square) {
        const double xm = __longlong_as_double((long long)block_max_u64(amax, reinterpret_cast<unsigned long long*>(red)));
        smax = xm * xm;
    } else {
        smax = block_max_d(top, red);
    }
    const int nbad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        atomicAdd(h.s + b, ssum);
        atomicMax(h.wmax + b, (unsigned long long)__double_as_longlong(smax));
        if (nbad) atomicOr(h.flags + b, 1u);
    }
}

// Dense pass 2: candidates v >= prune and the columns whose w is near the
// largest (the only ones that can hold the largest v), each appended with
// one atomic per warp and element position.
__global__ void __launch_bounds__(kMclThreads) k_mcl_heavy_cand(MclHeavyArgs h) {
    const int b = blockIdx.y, lane = threadIdx.x & 31;
    const MclArgs& a = h.a;
    const double2* D2 = reinterpret_cast<const double2*>(h.D + (long long)b * a.stride);
    const bool square = a.inflation == 2.0;
    const double s = __ldcg(h.s + b);
    const double wmax = __longlong_as_double((long long)__ldcg(h.wmax + b));
    const bool filt = !(__ldcg(h.flags + b) & 1u) && a.prune >= 0.0 && s > 0.0 && s <= 1.7e308 &&
                      wmax >= 0x1p-1000 && wmax <= 1.7e308 && (a.prune == 0.0 || a.prune * s >= 0x1p-1000);
    const double wlo = filt ? a.prune * s * (1.0 - 0x1p-45) : 0.0;
    const double whi = filt ? wmax * (1.0 - 0x1p-45) : 0.0;
    const unsigned long long xlo = filt && square ? sq_bound_bits(wlo) : 0ull;
    const unsigned long long xhi = filt && square ? sq_bound_bits(whi) : 0ull;
    const unsigned long long xskip = xlo < xhi ? xlo : xhi;
    unsigned long long* ck = h.ck + (long long)b * a.ccap;
    int* cc = h.cc + (long long)b * a.ccap;
    int* ml = h.mlist + (long long)b * kMclMaxList;
    const long long nch = a.stride / 8, nch32 = (nch + 31) & ~31ll;
    // whole warps walk the row (the appends are warp-wide)
    for (long long c0 = (long long)blockIdx.x * kMclThreads + (threadIdx.x & ~31); c0 < nch32;
         c0 += (long long)gridDim.x * kMclThreads) {
        const long long c = c0 + lane;
        double2 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = c < nch ? __ldcg(D2 + 4 * c + u) : make_double2(0.0, 0.0);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const double x = (u & 1) ? q[u >> 1].y : q[u >> 1].x;
            const int j = (int)(8 * c + u);
            bool cand = false, near = false;
            double v = 0.0;
            const unsigned long long ax = abs_bits(x);
            if (ax != 0 && ax >= xskip) {
                const double w = square ? x * x : pow(x, a.inflation);
                near = !filt || w >= whi;
                if (!filt || w >= wlo || near) {
                    v = w / s;
                    cand = v >= a.prune;
                }
            }
            const unsigned mc = __ballot_sync(0xffffffffu, cand);
            if (mc) {
                int base = 0;
                if (lane == 0) base = atomicAdd(h.ncand + b, __popc(mc));
                base = __shfl_sync(0xffffffffu, base, 0);
                const int qq = base + __popc(mc & ((1u << lane) - 1u));
                if (cand && qq < a.ccap) {
                    ck[qq] = (unsigned long long)__double_as_longlong(v);
                    cc[qq] = j;
                }
            }
            const unsigned mn = __ballot_sync(0xffffffffu, near);
            if (mn) {
                int base = 0;
                if (lane == 0) base = atomicAdd(h.nmax + b, __popc(mn));
                base = __shfl_sync(0xffffffffu, base, 0);
                const int qq = base + __popc(mn & ((1u << lane) - 1u));
                if (near) {
                    if (qq < kMclMaxList) ml[qq] = j;
                    else atomicOr(h.flags + b, 2u);
                }
            }
        }
    }
}

// One block per row of the batch: the largest entry when nothing reached
// the prune (from the near-max list, or the whole row after an overflow),
// then the keep rule and the output as in k_mcl_rows.
__global__ void __launch_bounds__(kMclThreads) k_mcl_heavy_select(MclHeavyArgs h) {
    __shared__ MclShared sh;
    __shared__ int kcol[kMclMaxK];
    __shared__ float kval[kMclMaxK];
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const MclArgs& a = h.a;
    const int r = h.rows[b];
    const int nkeep = __ldcg(h.ncand + b);
    const int ncand = nkeep < a.ccap ? nkeep : a.ccap;
    if (tid == 0 && nkeep > a.ccap) atomicOr(a.status, kStatusInternal);
    if (nkeep == 0) {
        const double* Db = h.D + (long long)b * a.stride;
        const bool square = a.inflation == 2.0;
        const double s = __ldcg(h.s + b);
        const bool all = (__ldcg(h.flags + b) & 2u) != 0;
        const int nm = all ? 0 : __ldcg(h.nmax + b);
        const long long cnt = all ? a.n : (long long)(nm < kMclMaxList ? nm : kMclMaxList);
        double bv = -1.0;
        int bj = 0x7fffffff;
        for (long long i = tid; i < cnt; i += kMclThreads) {
            const int j = all ? (int)i : h.mlist[(long long)b * kMclMaxList + i];
            const double x = __ldcg(Db + j);
            if (x == 0.0) continue;
            const double v = (square ? x * x : pow(x, a.inflation)) / s;
            if (v > bv || (v == bv && j < bj)) {
                bv = v;
                bj = j;
            }
        }
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
    mcl_finish_row(a, sh, kcol, kval, r, h.ck + (long long)b * a.ccap, h.cc + (long long)b * a.ccap, nkeep, ncand);
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

namespace {
MclArgs mcl_args(const MclLaunch& l) {
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
    a.heavy = l.heavy;
    a.skip = l.skip;
    a.positive = l.positive;
    return a;
}

MclHeavyArgs heavy_args(const MclLaunch& l, const MclHeavyLaunch& hb) {
    MclHeavyArgs h;
    h.a = mcl_args(l);
    h.rows = hb.rows;
    h.nb = hb.nb;
    h.D = hb.D;
    h.s = hb.s;
    h.wmax = hb.wmax;
    h.flags = hb.flags;
    h.ncand = hb.ncand;
    h.nmax = hb.nmax;
    h.ck = hb.ck;
    h.cc = hb.cc;
    h.mlist = hb.mlist;
    return h;
}
}  // namespace

cudaError_t launch_mcl_pilot(const MclLaunch& l, const int* rows, int nrows, int step, unsigned long long* tot,
                             cudaStream_t s) {
    if (nrows <= 0 || step <= 0) return cudaErrorInvalidValue;
    k_mcl_pilot<<<nrows, kMclThreads, 0, s>>>(mcl_args(l), rows, step, tot);
    return cudaGetLastError();
}

cudaError_t launch_mcl_rows(const MclLaunch& l, int blocks, cudaStream_t s) {
    k_mcl_rows<<<blocks, kMclThreads, 0, s>>>(mcl_args(l));
    return cudaGetLastError();
}

// flag := 1 if a value is not in [2^-63, FLT_MAX] (zero, negative, tiny,
// infinite or NaN): then a product may be 0 or a sum may return to 0
__global__ void k_mcl_check_positive(const float* __restrict__ val, long long nnz, int* flag) {
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (long long)gridDim.x * blockDim.x) {
        const float v = __ldg(val + i);
        bad |= !(v >= 0x1p-63f && v <= 3.4028234e38f);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

cudaError_t launch_mcl_check_positive(const float* val, long long nnz, int* flag, int sms, cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    const int blocks = (int)std::min<long long>((nnz + 255) / 256, (long long)sms * 8);
    k_mcl_check_positive<<<blocks, 256, 0, s>>>(val, nnz, flag);
    return cudaGetLastError();
}

// per row, by its product count u: u >= heavy -> 1 (batched path, listed in
// hlist); bucket_lo <= u < bucket_hi and every value positive (*notpos == 0)
// -> 2 (bucketed path, listed in blist); else 0 (per-block kernel)
__global__ void k_mcl_mark(const int* __restrict__ rp, const int* __restrict__ col, int n, long long heavy,
                           long long bucket_lo, long long bucket_hi, const int* notpos, unsigned char* flags,
                           int* hlist, int* hcount, int* blist, int* bcount) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const long long stop = heavy > bucket_hi ? heavy : bucket_hi;
    long long u = 0;
    for (int e = __ldg(rp + r); e < __ldg(rp + r + 1) && u < stop; ++e) {
        const int k = __ldg(col + e);
        u += __ldg(rp + k + 1) - __ldg(rp + k);
    }
    unsigned char f = 0;
    if (u >= heavy) {
        f = 1;
        hlist[atomicAdd(hcount, 1)] = r;
    } else if (u >= bucket_lo && u < bucket_hi && *notpos == 0) {
        f = 2;
        blist[atomicAdd(bcount, 1)] = r;
    }
    flags[r] = f;
}

cudaError_t launch_mcl_mark(const int* rp, const int* col, int n, long long heavy, long long bucket_lo,
                            long long bucket_hi, const int* notpos, unsigned char* flags, int* hlist, int* hcount,
                            int* blist, int* bcount, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_mcl_mark<<<(n + 255) / 256, 256, 0, s>>>(rp, col, n, heavy, bucket_lo, bucket_hi, notpos, flags, hlist, hcount,
                                               blist, bcount);
    return cudaGetLastError();
}

size_t mcl_bucket_smem(int lw, int nbk) {
    return mcl_window_bytes(lw) + 2 * ((size_t)1 << lw) + 4 * (2 * (size_t)nbk + 1);
}

int mcl_bucket_blocks_per_sm(int lw, int nbk) {
    const size_t dyn = mcl_bucket_smem(lw, nbk);
    if (cudaFuncSetAttribute(k_mcl_rows_bucket, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_mcl_rows_bucket, kMclThreads, dyn) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t launch_mcl_bucket(const MclLaunch& l, const MclBucketLaunch& b, int blocks, cudaStream_t s) {
    if (blocks <= 0 || b.lw < 5 || b.lw > 13) return cudaErrorInvalidValue;
    MclBucketArgs bk;
    bk.list = b.list;
    bk.count = b.count;
    bk.counter = b.counter;
    bk.stage = b.stage;
    bk.ej = b.ej;
    bk.cap = b.cap;
    bk.lw = b.lw;
    bk.nbk = b.nbk;
    k_mcl_rows_bucket<<<blocks, kMclThreads, mcl_bucket_smem(b.lw, b.nbk), s>>>(mcl_args(l), bk);
    return cudaGetLastError();
}

cudaError_t launch_mcl_heavy_batch(const MclLaunch& l, const MclHeavyLaunch& hb, int sms, cudaStream_t s) {
    if (hb.nb <= 0 || hb.nb > kMclBatch) return cudaErrorInvalidValue;
    // six blocks per SM (30 registers, 8 fit): room is left for the previous
    // batch's scans and selection on the other stream
    k_mcl_heavy_expand<<<sms * 6, kMclThreads, 0, s>>>(heavy_args(l, hb));
    return cudaGetLastError();
}

cudaError_t launch_mcl_heavy_scans(const MclLaunch& l, const MclHeavyLaunch& hb, int sms, cudaStream_t s) {
    if (hb.nb <= 0 || hb.nb > kMclBatch) return cudaErrorInvalidValue;
    const MclHeavyArgs h = heavy_args(l, hb);
    const long long tiles = (l.stride / 8 + kMclThreads - 1) / kMclThreads;  // chunks of 8 per thread
    const int gx = (int)std::max<long long>(1, std::min<long long>(tiles, (8ll * sms + hb.nb - 1) / hb.nb));
    k_mcl_heavy_sums<<<dim3(gx, hb.nb), kMclThreads, 0, s>>>(h);
    k_mcl_heavy_cand<<<dim3(gx, hb.nb), kMclThreads, 0, s>>>(h);
    return cudaGetLastError();
}

cudaError_t launch_mcl_heavy_select(const MclLaunch& l, const MclHeavyLaunch& hb, cudaStream_t s) {
    if (hb.nb <= 0 || hb.nb > kMclBatch) return cudaErrorInvalidValue;
    k_mcl_heavy_select<<<hb.nb, kMclThreads, 0, s>>>(heavy_args(l, hb));
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
