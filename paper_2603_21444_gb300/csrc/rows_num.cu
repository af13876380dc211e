// Numeric row kernels (deterministic sort accumulator) and the heavy-row
// dense accumulator, for float and double values.
#include "rows_launch.cuh"

namespace tsg {

template <typename T>
static int num_smem_bytes_t(int variant, int wpb) {
    int bytes = 0;
    dispatch_variant(variant, [&](auto S) {
        using SS = decltype(S);
        if constexpr (SS::TEAM == 1)
            bytes = ThreadNumLayout<T>::bytes;
        else if constexpr (SS::TEAMK)
            bytes = SS::STAGED ? TNumLayout<SS::CAP, T>::bytes_staged : TNumLayout<SS::CAP, T>::bytes;
        else
            bytes = SS::TEAM == 32 ? WNumLayout<SS::CAP, T>::bytes * wpb : NumLayout<SS::CAP, T>::bytes;
        return cudaSuccess;
    });
    return bytes;
}

int num_smem_bytes(int variant, int dtype, int wpb) {
    return dtype == 1 ? num_smem_bytes_t<double>(variant, wpb) : num_smem_bytes_t<float>(variant, wpb);
}

template <typename T>
static int num_blocks_per_sm_t(int variant, int wpb) {
    int nb = 0;
    dispatch_variant(variant, [&](auto S) {
        using SS = decltype(S);
        if constexpr (SS::TEAM == 1) {
            nb = blocks_per_sm(k_num_thread<T>, kThreadRows, ThreadNumLayout<T>::bytes);
        } else if constexpr (SS::TEAMK) {
            nb = blocks_per_sm(k_num_team<SS::TEAM / 32, T, SS::STAGED>, SS::TEAM, num_smem_bytes_t<T>(variant, wpb));
        } else {
            const int threads = SS::TEAM == 32 ? 32 * wpb : SS::TEAM;
            nb = blocks_per_sm(k_num_rows<SS::TEAM, SS::PER, T>, threads, num_smem_bytes_t<T>(variant, wpb));
        }
        return cudaSuccess;
    });
    return nb;
}

int num_blocks_per_sm(int variant, int dtype, int wpb) {
    return dtype == 1 ? num_blocks_per_sm_t<double>(variant, wpb) : num_blocks_per_sm_t<float>(variant, wpb);
}

template <typename T>
static cudaError_t launch_num_rows_t(int variant, const RowLaunchArgs& l, int blocks, int wpb, cudaStream_t s) {
    const RowArgs a = to_row_args(l);
    return dispatch_variant(variant, [&](auto S) {
        using SS = decltype(S);
        if constexpr (SS::TEAM == 1) {
            const int smem = ThreadNumLayout<T>::bytes;
            cudaFuncSetAttribute(k_num_thread<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            k_num_thread<T><<<blocks, kThreadRows, smem, s>>>(a);
        } else if constexpr (SS::TEAMK) {
            const int smem = num_smem_bytes_t<T>(variant, wpb);
            cudaFuncSetAttribute(k_num_team<SS::TEAM / 32, T, SS::STAGED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
            k_num_team<SS::TEAM / 32, T, SS::STAGED><<<blocks, SS::TEAM, smem, s>>>(a);
        } else {
            const int threads = SS::TEAM == 32 ? 32 * wpb : SS::TEAM;
            const int smem = num_smem_bytes_t<T>(variant, wpb);
            cudaFuncSetAttribute(k_num_rows<SS::TEAM, SS::PER, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            k_num_rows<SS::TEAM, SS::PER, T><<<blocks, threads, smem, s>>>(a);
        }
        return cudaGetLastError();
    });
}

cudaError_t launch_num_rows(int variant, int dtype, const RowLaunchArgs& l, int blocks, int wpb, cudaStream_t s) {
    return dtype == 1 ? launch_num_rows_t<double>(variant, l, blocks, wpb, s)
                      : launch_num_rows_t<float>(variant, l, blocks, wpb, s);
}

template <typename T>
static cudaError_t launch_num_fused_t(int variant, const RowLaunchArgs& l, const FusedCtl& fc, int blocks, int wpb,
                                      cudaStream_t s) {
    const RowArgs a = to_row_args(l);
    return dispatch_variant(variant, [&](auto S) {
        using SS = decltype(S);
        if constexpr (SS::TEAM != 32) {
            return cudaErrorInvalidValue;
        } else {
            const int smem = WNumLayout<SS::CAP, T>::bytes * wpb;
            cudaFuncSetAttribute(k_num_fused<SS::PER, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            k_num_fused<SS::PER, T><<<blocks, 32 * wpb, smem, s>>>(a, fc);
            return cudaGetLastError();
        }
    });
}

cudaError_t launch_num_fused(int variant, int dtype, const RowLaunchArgs& l, const FusedCtl& fc, int blocks, int wpb,
                             cudaStream_t s) {
    return dtype == 1 ? launch_num_fused_t<double>(variant, l, fc, blocks, wpb, s)
                      : launch_num_fused_t<float>(variant, l, fc, blocks, wpb, s);
}

template <typename T>
static int num_fused_blocks_per_sm_t(int variant, int wpb) {
    int nb = 0;
    dispatch_variant(variant, [&](auto S) {
        using SS = decltype(S);
        if constexpr (SS::TEAM == 32)
            nb = blocks_per_sm(k_num_fused<SS::PER, T>, 32 * wpb, WNumLayout<SS::CAP, T>::bytes * wpb);
        return cudaSuccess;
    });
    return nb;
}

int num_fused_blocks_per_sm(int variant, int dtype, int wpb) {
    return dtype == 1 ? num_fused_blocks_per_sm_t<double>(variant, wpb) : num_fused_blocks_per_sm_t<float>(variant, wpb);
}

cudaError_t launch_num_grouped(int dtype, const RowLaunchArgs& l, int sms, cudaStream_t s) {
    const RowArgs a = to_row_args(l);
    auto go = [&](auto tag) {
        using T = decltype(tag);
        const int smem = GroupedLayout<T>::bytes * kGroupedWarps;
        cudaFuncSetAttribute(k_num_grouped<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int nb = blocks_per_sm(k_num_grouped<T>, 32 * kGroupedWarps, smem);
        if (nb < 1) nb = 1;
        k_num_grouped<T><<<sms * nb, 32 * kGroupedWarps, smem, s>>>(a);
        return cudaGetLastError();
    };
    return dtype == 1 ? go(double()) : go(float());
}

cudaError_t launch_num_heavy(int dtype, const RowLaunchArgs& l, void* dense, int blocks, int chunk, cudaStream_t s) {
    const RowArgs a = to_row_args(l);
    const int smem = (chunk / 32) * 4;
    if (dtype == 1) {
        cudaFuncSetAttribute(k_num_heavy<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_num_heavy<double><<<blocks, kHeavyThreads, smem, s>>>(a, reinterpret_cast<double*>(dense), chunk);
    } else {
        cudaFuncSetAttribute(k_num_heavy<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_num_heavy<float><<<blocks, kHeavyThreads, smem, s>>>(a, reinterpret_cast<float*>(dense), chunk);
    }
    return cudaGetLastError();
}

}  // namespace tsg
