// Trident partitioning (paper Sec. 3.2) on the device: a CSR matrix is cut
// into a grid of tiles along given row and column boundaries, each tile a CSR
// matrix with block-local column indices.  The A operand is cut into q*lambda
// row slices x q column tiles (A_{i r k}); the B operand into q x q tiles
// (B_{r j}: on one device the allgathered tile of Alg. 2 is extracted whole).
//
// Sizing: per row, the number of entries in each column part; the units of
// the scan are (column part, row) so that tile (rp, cp) owns a contiguous
// range of units and the shared scan kernels produce every tile's row_ptr.
// Fill: per row, entries go to their tile in stored order.
#include "internal.h"

namespace tsg {

constexpr int kMaxParts = 64;

__device__ __forceinline__ int part_of(const int* __restrict__ bounds, int nparts, int x) {
    int lo = 0, hi = nparts;  // bounds[lo] <= x < bounds[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(bounds + mid) <= x) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_split_count(const int* __restrict__ rp, const int* __restrict__ col, int nrows,
                              const int* __restrict__ cb, int ncp, int* counts) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    int c[kMaxParts];
    for (int p = 0; p < ncp; ++p) c[p] = 0;
    const int e1 = rp[r + 1];
    for (int e = rp[r]; e < e1; ++e) ++c[part_of(cb, ncp, __ldg(col + e))];
    for (int p = 0; p < ncp; ++p) counts[(long long)p * nrows + r] = c[p];
}

template <typename T>
__global__ void k_split_fill(const int* __restrict__ rp, const int* __restrict__ col, const T* __restrict__ val,
                             int nrows, const int* __restrict__ rb, int nrp, const int* __restrict__ cb, int ncp,
                             const GroupDev* __restrict__ tiles) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const int p_r = part_of(rb, nrp, r);
    const int local = r - __ldg(rb + p_r);
    const GroupDev* row_tiles = tiles + (long long)p_r * ncp;
    int off[kMaxParts];
    for (int p = 0; p < ncp; ++p) off[p] = __ldg(row_tiles[p].crp + local);
    const int e1 = rp[r + 1];
    for (int e = rp[r]; e < e1; ++e) {
        const int c = __ldg(col + e);
        const int p = part_of(cb, ncp, c);
        const GroupDev& Tt = row_tiles[p];
        Tt.ccol[off[p]] = c - __ldg(cb + p);
        if (val) reinterpret_cast<T*>(Tt.cval)[off[p]] = __ldg(val + e);
        ++off[p];
    }
}

cudaError_t launch_split_count(const int* rp, const int* col, int nrows, const int* cb, int ncp, int* counts,
                               cudaStream_t s) {
    const int threads = 128;
    k_split_count<<<(nrows + threads - 1) / threads, threads, 0, s>>>(rp, col, nrows, cb, ncp, counts);
    return cudaGetLastError();
}

cudaError_t launch_split_fill(int dtype, const int* rp, const int* col, const void* val, int nrows, const int* rb,
                              int nrp, const int* cb, int ncp, const GroupDev* tiles, cudaStream_t s) {
    const int threads = 128;
    const int blocks = (nrows + threads - 1) / threads;
    if (dtype == 1)
        k_split_fill<double><<<blocks, threads, 0, s>>>(rp, col, static_cast<const double*>(val), nrows, rb, nrp, cb,
                                                        ncp, tiles);
    else
        k_split_fill<float><<<blocks, threads, 0, s>>>(rp, col, static_cast<const float*>(val), nrows, rb, nrp, cb,
                                                       ncp, tiles);
    return cudaGetLastError();
}

}  // namespace tsg
