// Launch helpers for the row kernels (included by the per-dtype .cu files).
#pragma once

#include "internal.h"
#include "rows.cuh"
#include "rows_team.cuh"

namespace tsg {

inline RowArgs to_row_args(const RowLaunchArgs& l) {
    RowArgs a;
    a.inst = l.inst;
    a.groups = l.groups;
    a.unit_base = l.unit_base;
    a.ngroups = l.ngroups;
    a.list = l.list;
    a.bin_off = l.bin_off;
    a.bin = l.bin;
    a.merge = l.merge;
    a.status = l.status;
    a.counts = l.counts;
    a.tick = l.tick;
    a.glist = l.glist;
    a.gcount = l.gcount;
    return a;
}

template <int V>
struct VariantShape {
    static constexpr int TEAM = variant_team(V);
    static constexpr int PER = variant_per(V);
    static constexpr int CAP = TEAM * PER;
    static constexpr bool TEAMK = variant_is_team(V);  // block team running the warp counting sort
    static constexpr bool STAGED = variant_is_staged(V);  // ... with its B rows staged by TMA
};

// Calls f(std::integral_constant-like tag) for the runtime variant v.
template <typename F>
inline cudaError_t dispatch_variant(int v, F&& f) {
    switch (v) {
        case 0: return f(VariantShape<0>());
        case 1: return f(VariantShape<1>());
        case 2: return f(VariantShape<2>());
        case 3: return f(VariantShape<3>());
        case 4: return f(VariantShape<4>());
        case 5: return f(VariantShape<5>());
        case 6: return f(VariantShape<6>());
        case 7: return f(VariantShape<7>());
        case 8: return f(VariantShape<8>());
        case 9: return f(VariantShape<9>());
        case 10: return f(VariantShape<10>());
        case 11: return f(VariantShape<11>());
        case 12: return f(VariantShape<12>());
        case 13: return f(VariantShape<13>());
        case 14: return f(VariantShape<14>());
        case 15: return f(VariantShape<15>());
        case 16: return f(VariantShape<16>());
        case 17: return f(VariantShape<17>());
        case 18: return f(VariantShape<18>());
        case 19: return f(VariantShape<19>());
        default: return cudaErrorInvalidValue;
    }
}

template <typename K>
inline int blocks_per_sm(K kernel, int threads, int smem) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

}  // namespace tsg
