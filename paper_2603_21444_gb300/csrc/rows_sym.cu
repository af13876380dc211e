// Symbolic row kernels: per-row distinct-column counts (hash set per team),
// plus the heavy-row bitmap counter.
#include "rows_launch.cuh"

namespace tsg {

int warp_variant_max_wpb(int variant, int per_warp_bytes, bool symbolic) {
    if (variant_team(variant) != 32) return 1;
    const int per = variant_per(variant);
    // the kernels' launch bounds: symbolic 256 threads up to 12 per lane
    // (registers for 5 resp. 3 blocks per SM), numeric 1024 up to 8
    const int by_threads = symbolic ? (per <= 12 ? 8 : 16) : (per <= 8 ? 32 : (per == 12 ? 8 : 16));
    const int by_smem = (227 * 1024) / per_warp_bytes;
    return by_smem < by_threads ? by_smem : by_threads;
}

int sym_smem_bytes(int variant, int wpb) {
    int bytes = 0;
    dispatch_variant(variant, [&](auto S) {
        using SS = decltype(S);
        if constexpr (SS::TEAM == 1)
            bytes = 0;  // static shared memory
        else
            bytes = SS::TEAM == 32 ? WSymLayout<SS::CAP>::bytes * wpb : SymLayout<SS::CAP>::bytes;
        return cudaSuccess;
    });
    return bytes;
}

int sym_blocks_per_sm(int variant, int wpb) {
    int nb = 0;
    dispatch_variant(variant, [&](auto S) {
        using SS = decltype(S);
        if constexpr (SS::TEAM == 1) {
            nb = blocks_per_sm(k_sym_thread, kThreadRows, 0);
        } else {
            const int threads = SS::TEAM == 32 ? 32 * wpb : SS::TEAM;
            nb = blocks_per_sm(k_sym_rows<SS::TEAM, SS::PER>, threads, sym_smem_bytes(variant, wpb));
        }
        return cudaSuccess;
    });
    return nb;
}

cudaError_t launch_sym_rows(int variant, const RowLaunchArgs& l, int blocks, int wpb, cudaStream_t s) {
    const RowArgs a = to_row_args(l);
    return dispatch_variant(variant, [&](auto S) {
        using SS = decltype(S);
        if constexpr (SS::TEAM == 1) {
            k_sym_thread<<<blocks, kThreadRows, 0, s>>>(a);
        } else {
            const int threads = SS::TEAM == 32 ? 32 * wpb : SS::TEAM;
            const int smem = sym_smem_bytes(variant, wpb);
            cudaFuncSetAttribute(k_sym_rows<SS::TEAM, SS::PER>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            k_sym_rows<SS::TEAM, SS::PER><<<blocks, threads, smem, s>>>(a);
        }
        return cudaGetLastError();
    });
}

// Thread-per-row rows: sorted columns in the thread's column of a shared
// array, distinct ones counted.
__global__ void __launch_bounds__(kThreadRows) k_sym_thread(RowArgs a) {
    __shared__ int cols[kThreadCap * kThreadRows];
    int* sc = cols + threadIdx.x;
    const int begin = a.bin_off[a.bin], end = a.bin_off[a.bin + 1];
    for (int i = begin + blockIdx.x * kThreadRows + threadIdx.x; i < end; i += gridDim.x * kThreadRows) {
        const int unit = __ldg(a.list + i);
        const int g = unit_group(a.unit_base, a.ngroups, unit);
        const GroupDev& G = a.groups[g];
        const int rho = (int)(unit - a.unit_base[g]);
        const int n = thread_gather<false, float>(a, G, rho, sc, nullptr, nullptr);
        if (n < 0) {
            atomicOr(a.status, kStatusInternal);
            a.counts[unit] = 0;
            continue;
        }
        for (int x = 1; x < n; ++x) {
            const int c = sc[x * kThreadRows];
            int y = x - 1;
            while (y >= 0 && sc[y * kThreadRows] > c) {
                sc[(y + 1) * kThreadRows] = sc[y * kThreadRows];
                --y;
            }
            sc[(y + 1) * kThreadRows] = c;
        }
        int distinct = 0;
        for (int x = 0; x < n; ++x) distinct += x == 0 || sc[x * kThreadRows] != sc[(x - 1) * kThreadRows];
        a.counts[unit] = distinct;
    }
}

// Heavy rows: one block per row, a bitmap of `chunk` columns per pass.
__global__ void __launch_bounds__(kHeavyThreads, 1) k_sym_heavy(RowArgs a, int chunk) {
    extern __shared__ __align__(16) unsigned bm[];
    __shared__ int scratch[34];
    const int words = chunk >> 5;
    const int begin = a.bin_off[a.bin], end = a.bin_off[a.bin + 1];
    for (int i = begin + blockIdx.x; i < end; i += gridDim.x) {
        const int unit = __ldg(a.list + i);
        const int g = unit_group(a.unit_base, a.ngroups, unit);
        const GroupDev& G = a.groups[g];
        const int rho = (int)(unit - a.unit_base[g]);
        long long total = 0;
        for (long long c0 = 0; c0 < G.ncols; c0 += chunk) {
            for (int w = threadIdx.x; w < words; w += blockDim.x) bm[w] = 0u;
            __syncthreads();
            int fresh = 0;
            heavy_products<false, float>(a, G, rho, [&](int col, float) {
                const unsigned rel = (unsigned)((long long)col - c0);
                if (rel < (unsigned)chunk) {
                    const unsigned bit = 1u << (rel & 31);
                    if (!(atomicOr(bm + (rel >> 5), bit) & bit)) ++fresh;
                }
            });
            total += Team<kHeavyThreads>::sum(fresh, scratch);
            __syncthreads();
        }
        if (threadIdx.x == 0) a.counts[unit] = (int)total;
    }
}

int heavy_chunk_for(int ncols) {
    int c = 32;
    while (c < ncols && c < kHeavyChunk) c <<= 1;
    return c;
}

cudaError_t launch_sym_heavy(const RowLaunchArgs& l, int blocks, int chunk, cudaStream_t s) {
    const RowArgs a = to_row_args(l);
    const int smem = (chunk / 32) * 4;
    cudaFuncSetAttribute(k_sym_heavy, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_sym_heavy<<<blocks, kHeavyThreads, smem, s>>>(a, chunk);
    return cudaGetLastError();
}

}  // namespace tsg
