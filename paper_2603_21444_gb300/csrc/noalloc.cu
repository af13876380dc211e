// An allocation-free variant of the CSR transpose for callers that may not
// allocate device memory.
//
// Who needs it: code whose device memory is owned by an outside pool or
// budget that forbids allocations behind its back, and latency-critical
// paths where an allocation's implicit device synchronisation is not
// acceptable.  Such a caller passes inputs and outputs it allocated itself;
// all working memory comes from one fixed array compiled into this library.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (kNoAllocScratchBytes) until the process exits.  In host
// code the variable's name is only a host-side stand-in, never a device
// address, so its address is obtained with cudaGetSymbolAddress, once per
// device, with that device current, by the first call on that device.  That
// first call must therefore come before any stream capture begins.  The
// address is cached for the life of the process; a device reset
// (cudaDeviceReset) invalidates it, and the entry point must not be called
// again afterwards.
//
// Every call uses the same array and leaves its contents behind; the parts
// that must start at zero (column counts and cursors) are cleared on the
// stream by every call.  Calls whose work overlaps on the GPU (different
// streams, or different host threads without ordering) race on the array.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "trident_spgemm.h"

namespace tsg {

constexpr size_t kNoAllocScratchBytes = SPGEMM_NOALLOC_SCRATCH_BYTES;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};
int g_noalloc_sms[kNoAllocMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch array and the SM count for the current device.
cudaError_t noalloc_setup(void** ptr, int* sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
        g_noalloc_sms[dev] = n;
    }
    *ptr = g_noalloc_ptr[dev];
    *sms = g_noalloc_sms[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace tsg

extern "C" spgemm_status spgemm_csr_transpose_noalloc(spgemm_dtype dtype, const spgemm_csr_in* X,
                                                      spgemm_csr_out* XT, spgemm_stream_t stream) {
    using namespace tsg;
    if (!X || X->nrows < 0 || X->ncols < 0 || X->nnz < 0 || !X->row_ptr || (X->nnz > 0 && !X->col_idx))
        return SPGEMM_ERR_INVALID_ARG;
    if (!XT || !XT->row_ptr || (X->nnz > 0 && !XT->col_idx)) return SPGEMM_ERR_INVALID_ARG;
    if (dtype != SPGEMM_F32 && dtype != SPGEMM_F64) return SPGEMM_ERR_DTYPE;
    if (XT->nrows != X->ncols || XT->ncols != X->nrows) return SPGEMM_ERR_SHAPE;
    if (X->val && X->nnz > 0 && !XT->val) return SPGEMM_ERR_INVALID_ARG;
    // scratch layout: column counts/cursors | 64-bit sums | scan partials | sort buffers
    const long long nc = X->ncols, nnz = X->nnz;
    const size_t esz = dtype == SPGEMM_F64 ? 8 : 4;
    const size_t o_work = 0;
    const size_t o_ex = o_work + align256(4 * (size_t)std::max<long long>(nc, 1));
    const size_t o_bsum = o_ex + align256(8 * (size_t)(nc + 1));
    const size_t o_tmp = o_bsum + align256(8 * (size_t)scan_blocks(std::max<long long>(nc, 1)));
    const size_t need = o_tmp + align256(4 * (size_t)std::max<long long>(nnz, 1)) +
                        align256(esz * (size_t)std::max<long long>(nnz, 1));
    if (need > kNoAllocScratchBytes) return SPGEMM_ERR_UNSUPPORTED;
    if (nc == 0) {
        // X^T has no rows: its row pointer is the single entry 0
        return cudaMemsetAsync(XT->row_ptr, 0, sizeof(int), reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
                   ? SPGEMM_OK
                   : SPGEMM_ERR_CUDA;
    }
    void* base = nullptr;
    int sms = 0;
    if (noalloc_setup(&base, &sms) != cudaSuccess) {
        cudaGetLastError();
        return SPGEMM_ERR_CUDA;
    }
    char* b = static_cast<char*>(base);
    const cudaError_t e = launch_transpose(dtype, X->row_ptr, X->col_idx, X->val, X->nrows, X->ncols, nnz,
                                           XT->row_ptr, XT->col_idx, X->val ? XT->val : nullptr,
                                           reinterpret_cast<int*>(b + o_work), b + o_tmp,
                                           reinterpret_cast<long long*>(b + o_bsum),
                                           reinterpret_cast<long long*>(b + o_ex), sms,
                                           reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}
