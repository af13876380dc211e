// Row analysis and binning, the scan of row counts into row pointers, and
// input validation.
#include "internal.h"

namespace tsg {

// ----------------------------------------------------------------- analysis
//
// u_i = sum over the row's A entries k of |B_k| (merge: the sum of the
// partials' row lengths) and the row's A-entry count pick the bin.
__global__ void k_analysis(AnalysisArgs a) {
    const long long unit = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int bin = -1;
    if (unit < a.nunits) {
        const int g = unit_group(a.unit_base, a.ngroups, unit);
        const GroupDev& G = a.groups[g];
        const int rho = (int)(unit - a.unit_base[g]);
        long long u = 0, nA = 0;
        for (int t = 0; t < G.inst_count; ++t) {
            const InstDev& I = a.inst[G.inst_begin + t];
            if (a.merge) {
                u += __ldg(I.brp + rho + 1) - __ldg(I.brp + rho);
                nA += 1;
            } else {
                const int a0 = __ldg(I.arp + rho), a1 = __ldg(I.arp + rho + 1);
                nA += a1 - a0;
                // unrolled so that the loads of several A entries are in flight at once
#pragma unroll 8
                for (int e = a0; e < a1; ++e) {
                    const int k = __ldg(I.acol + e);
                    u += __ldg(I.brp + k + 1) - __ldg(I.brp + k);
                }
            }
        }
        const int nb = a.bt.nbins;
        if (u == 0) {
            bin = nb + 1;
        } else {
            bin = nb;
            for (int b = 0; b < nb; ++b)
                if (u <= a.bt.upper[b] && nA <= a.bt.amax[b]) {
                    bin = b;
                    break;
                }
        }
        a.bin_of[unit] = (unsigned char)bin;
        if (bin == nb + 1 && a.sizing) a.counts[unit] = 0;
        if (a.total_u && u) atomicAdd(a.total_u, (unsigned long long)u);
    }
    const unsigned active = __ballot_sync(0xffffffffu, bin >= 0);
    if (bin >= 0) {
        const unsigned peers = __match_any_sync(active, bin);
        if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(a.hist + bin, __popc(peers));
    }
}

cudaError_t launch_analysis(const AnalysisArgs& a, cudaStream_t s) {
    const int threads = 256;
    const long long blocks = (a.nunits + threads - 1) / threads;
    k_analysis<<<(unsigned)blocks, threads, 0, s>>>(a);
    return cudaGetLastError();
}

__global__ void k_bin_offsets(int* hist, int* off, int* cursor, int nslots) {
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < nslots; ++b) {
            off[b] = acc;
            acc += hist[b];
            cursor[b] = 0;
        }
        off[nslots] = acc;
    }
}

cudaError_t launch_bin_offsets(int* hist, int* off, int* cursor, int nslots, cudaStream_t s) {
    k_bin_offsets<<<1, 32, 0, s>>>(hist, off, cursor, nslots);
    return cudaGetLastError();
}

// Append every unit to its bin's list (warp-aggregated cursors, so the units
// of a warp stay in ascending order within a bin).
__global__ void k_bin_fill(const unsigned char* __restrict__ bin_of, long long nunits, const int* __restrict__ off,
                           int* cursor, int* list) {
    const long long unit = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int bin = unit < nunits ? (int)bin_of[unit] : -1;
    const unsigned active = __ballot_sync(0xffffffffu, bin >= 0);
    if (bin < 0) return;
    const unsigned peers = __match_any_sync(active, bin);
    const int leader = __ffs(peers) - 1;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == leader) base = atomicAdd(cursor + bin, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    list[off[bin] + base + __popc(peers & lanemask_lt())] = (int)unit;
}

cudaError_t launch_bin_fill(const unsigned char* bin_of, long long nunits, const int* off, int* cursor, int* list,
                            cudaStream_t s) {
    const int threads = 256;
    const long long blocks = (nunits + threads - 1) / threads;
    k_bin_fill<<<(unsigned)blocks, threads, 0, s>>>(bin_of, nunits, off, cursor, list);
    return cudaGetLastError();
}

// --------------------------------------------------------------------- scan

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanSpan = kScanThreads * kScanPer;

long long scan_blocks(long long n) { return (n + kScanSpan - 1) / kScanSpan; }

__device__ __forceinline__ long long block_scan_excl_ll(long long v, long long* total, long long* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = kScanThreads / 32;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const long long w = lane < NW ? sh[lane] : 0;
        long long z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < NW) sh[lane] = z - w;
        if (lane == 31) sh[32] = z;
    }
    __syncthreads();
    const long long r = sh[warp] + x - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int* __restrict__ counts, long long n,
                                                               long long* bsum) {
    __shared__ long long sh[33];
    const long long base = blockIdx.x * (long long)kScanSpan + threadIdx.x * (long long)kScanPer;
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i)
        if (base + i < n) s += counts[base + i];
    long long tot;
    block_scan_excl_ll(s, &tot, sh);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(long long* bsum, long long nb) {
    __shared__ long long sh[33];
    long long carry = 0;
    for (long long b0 = 0; b0 < nb; b0 += kScanThreads) {
        const long long b = b0 + threadIdx.x;
        const long long v = b < nb ? bsum[b] : 0;
        long long tot;
        const long long ex = block_scan_excl_ll(v, &tot, sh);
        if (b < nb) bsum[b] = carry + ex;
        carry += tot;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int* __restrict__ counts, long long n,
                                                              const long long* __restrict__ boff, long long* ex) {
    __shared__ long long sh[33];
    const long long base = blockIdx.x * (long long)kScanSpan + threadIdx.x * (long long)kScanPer;
    int c[kScanPer];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        c[i] = base + i < n ? counts[base + i] : 0;
        s += c[i];
    }
    long long tot;
    long long run = boff[blockIdx.x] + block_scan_excl_ll(s, &tot, sh);
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (base + i < n) ex[base + i] = run;
        run += c[i];
        if (base + i == n - 1) ex[n] = run;
    }
}

cudaError_t launch_scan(const int* counts, long long n, long long* bsum, long long* ex, cudaStream_t s) {
    if (n <= 0) return cudaMemsetAsync(ex, 0, sizeof(long long), s);  // ex[0] = 0
    const long long nb = scan_blocks(n);
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(counts, n, bsum);
    k_scan_top<<<1, kScanThreads, 0, s>>>(bsum, nb);
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(counts, n, bsum, ex);
    return cudaGetLastError();
}

__global__ void k_rowptr(const GroupDev* __restrict__ groups, const long long* __restrict__ unit_base, int ngroups,
                         long long n, const long long* __restrict__ ex, long long* nnz_out) {
    const long long unit = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (unit >= n) return;
    const int g = unit_group(unit_base, ngroups, unit);
    const GroupDev& G = groups[g];
    const long long u0 = unit_base[g];
    const int rho = (int)(unit - u0);
    const long long b0 = ex[u0];
    G.crp[rho] = (int)(ex[unit] - b0);
    if (rho == G.nrows - 1) {
        const long long t = ex[unit + 1] - b0;
        G.crp[G.nrows] = (int)t;
        nnz_out[g] = t;
    }
}

cudaError_t launch_rowptr(const GroupDev* groups, const long long* unit_base, int ngroups, long long n,
                          const long long* ex, long long* nnz_out, cudaStream_t s) {
    const int threads = 256;
    k_rowptr<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(groups, unit_base, ngroups, n, ex, nnz_out);
    return cudaGetLastError();
}

__global__ void k_ll_to_int(const long long* __restrict__ src, long long n, int* dst) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (int)src[i];
}

cudaError_t launch_ll_to_int(const long long* src, long long n, int* dst, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_ll_to_int<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, n, dst);
    return cudaGetLastError();
}

// ------------------------------------------------------------- validation

__global__ void k_validate(const int* __restrict__ rp, const int* __restrict__ col, int nrows, int ncols, int nnz,
                           unsigned* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > nrows) return;
    bool bad = false;
    const int a = rp[i];
    if (i == 0 && a != 0) bad = true;
    if (i == nrows && a != nnz) bad = true;
    if (i < nrows) {
        const int b = rp[i + 1];
        if (b < a || a < 0 || b > nnz) {
            bad = true;
        } else {
            for (int e = a; e < b; ++e) {
                const int c = col[e];
                if (c < 0 || c >= ncols) {
                    bad = true;
                    break;
                }
            }
        }
    }
    if (bad) atomicOr(status, kStatusNotCanonical);
}

cudaError_t launch_validate(const int* rp, const int* col, int nrows, int ncols, int nnz, unsigned* status,
                            cudaStream_t s) {
    const int threads = 256;
    k_validate<<<(nrows + 1 + threads - 1) / threads, threads, 0, s>>>(rp, col, nrows, ncols, nnz, status);
    return cudaGetLastError();
}

// Small device-to-host reads (counts, histograms, status words) stored by a
// kernel into mapped page-locked memory: a copy-engine read would queue
// behind whatever large device-to-host copy another stream has in flight.
__global__ void k_readback(const unsigned* __restrict__ src, unsigned* dst, int nwords) {
    for (int i = threadIdx.x; i < nwords; i += blockDim.x) dst[i] = src[i];
}

cudaError_t launch_readback(void* dst_mapped, const void* src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    if (bytes % 4 || bytes > (size_t(1) << 20)) return cudaErrorInvalidValue;
    k_readback<<<1, 256, 0, s>>>(static_cast<const unsigned*>(src), static_cast<unsigned*>(dst_mapped),
                                 (int)(bytes / 4));
    return cudaGetLastError();
}

}  // namespace tsg
