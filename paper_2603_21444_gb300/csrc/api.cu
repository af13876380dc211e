// C ABI of the trident SpGEMM library: handles, argument checking, workspace,
// and the host-side flow of symbolic / numeric / merge / batched calls.
//
// Flow of one call (all on the caller's stream):
//   descriptors -> device (one small copy)
//   [validate]      k_validate per input matrix
//   analysis        k_analysis (u_i, A-row length -> bin), k_bin_offsets,
//                   k_bin_fill (per-bin unit lists)
//   sizing call     k_sym_rows per bin + k_sym_heavy, k_scan_* (counts ->
//                   exclusive sums), k_rowptr (per-group row_ptr, nnz),
//                   one device->host copy and one stream synchronisation
//   fill call       k_num_rows per non-empty bin + k_num_heavy
// A fill call that follows the sizing call of the same problem on the same
// handle reuses its bin lists (no second analysis, no host round trip).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "trident_spgemm.h"

using namespace tsg;

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
};

struct PhaseEvent {
    int phase;
    cudaEvent_t a, b;
};

constexpr int kNumPhases = SPGEMM_NUM_PHASES;

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// The handle's per-unit workspace for `cap` units: bin id (1 B) | list
// entry (4 B) | count (4 B) | 64-bit exclusive sum (8 B, cap + 1) |
// deferred-row list (4 B).  Every user sizes it with this one function, so
// the offsets derived from units_cap stay inside the allocation.
size_t units_bytes(long long cap) {
    return align16(cap) + align16(4 * cap) + align16(4 * cap) + align16(8 * (cap + 1)) + align16(4 * cap);
}

}  // namespace

struct spgemm_handle {
    int device = 0;
    int sms = 0;
    spgemm_tune tune{};
    DevBuf units;   // bin_of | list | counts | ex
    long long units_cap = -1;
    DevBuf small;
    DevBuf dense;
    DevBuf status;  // the device status word latched by kernels
    DevBuf tr;      // transpose work and the A^T of the deterministic backward
    DevBuf mcl;     // Markov clustering: bounds, offsets, kept entries
    DevBuf mcl_acc; // Markov clustering: per-block dense accumulators
    DevBuf mcl_heavy;  // ... row flags, heavy and bucket lists, two buffers of batch accumulators
    DevBuf mcl_bucket; // ... bucketed rows: staging and emitted columns per block
    long long mcl_heavy_key = -1;  // layout whose batch accumulators are known to be zero
    double mcl_pilot_ratio = 0.0;  // products per distinct column of the last pilot (0: none ran)
    long long mcl_paths[3] = {};   // rows of the last expand per path: per-block, window-summed, batched
    cudaStream_t mcl_side = nullptr;  // heavy-row selection, overlapping the next batch
    cudaEvent_t mcl_ev[5] = {};       // batch ready (2), buffer cleared (2), join
    DevBuf perm;    // permutation: target hits, row lengths, scan, long-row list, ranks
    DevBuf hx;      // product from host memory: device copies of A, B and C's row_ptr
    DevBuf hc;      // ... and of C's columns and values
    const void* hx_key[4] = {};  // host A.row_ptr, A.col, B.row_ptr, B.col of the last sizing call
    bool hx_sized = false;
    const void* hv_key[2] = {};  // host A.val, B.val whose copies the last sizing call started
    int hv_dtype = -1;
    bool hv_ready = false;
    cudaEvent_t hv_ev = nullptr;  // ... recorded on `copy` after them
    cudaStream_t copy = nullptr;  // value uploads during the sizing; copies of finished row panels out
    std::vector<cudaEvent_t> panel_ev;
    int mcl_n = -1;
    long long mcl_acc_key = -1;  // accumulator layout (stride, slots) whose arrays are known to be zero
    long long mcl_total = 0;
    void* pinned = nullptr;      // mapped page-locked words the kernels' small results are stored into
    void* pinned_dev = nullptr;  // ... the device address of the same memory
    size_t pinned_n = 0;
    // plan cache (bin lists of the last sizing call)
    uint64_t plan_sig = 0;
    bool plan_valid = false;
    std::vector<int> plan_hist;
    int64_t launches = 0;
    bool timing = false;
    long long ws_limit = -1;              // cap on the device bytes held by the buffers above (-1: none)
    int wait_limit = kLookbackSpinLimit;  // polls of a look-back wait of the single-pass product
    int hold_tile = -1;                   // fault injection: a look-back entry never published
    int only_bin = -1;                    // autotuner: a fill call launches this bin's kernel alone
    std::vector<PhaseEvent> pending;
    std::vector<cudaEvent_t> spare;
    cudaStream_t last_stream = nullptr;
    int occ_wpb = -1;
    int occ_sym[kNumVariants];
    int occ_num[2][kNumVariants];
    std::vector<cudaStream_t> streams_used;
    // branches for the per-bin launches of one call: bins hold disjoint rows,
    // so their kernels run concurrently (forked from the call's stream,
    // joined back before anything that needs every bin)
    bool concurrent_bins = true;
    cudaStream_t side[kMaxBins + 1] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kMaxBins + 1] = {};
    // the last descriptor block copied to the device (identical blocks are
    // not copied again, so a repeated fill call launches kernels only)
    std::vector<char> last_stage;
    const void* last_stage_dst = nullptr;
};

namespace {

spgemm_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SPGEMM_OK;
    if (e == cudaErrorMemoryAllocation) return SPGEMM_ERR_OOM;
    return SPGEMM_ERR_CUDA;
}

#define TSG_CHECK(expr)                                   \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess) return cuda_status(e_);    \
    } while (0)

#define TSG_TRY(expr)                                     \
    do {                                                  \
        spgemm_status s_ = (expr);                        \
        if (s_ != SPGEMM_OK) return s_;                   \
    } while (0)

// Device bytes the handle's workspace buffers hold.
size_t held_bytes(const spgemm_handle* h) {
    return h->units.n + h->small.n + h->dense.n + h->status.n + h->tr.n + h->mcl.n + h->mcl_acc.n + h->perm.n +
           h->hx.n + h->hc.n;
}

// Grows b (one of h's buffers, or a buffer that will replace one) to at
// least `bytes`.  A growth that would take the bytes held over the handle's
// workspace limit returns SPGEMM_ERR_OOM and leaves b as it was; a failed
// cudaMalloc returns SPGEMM_ERR_OOM with b empty.
spgemm_status grow(spgemm_handle* h, DevBuf& b, size_t bytes, cudaStream_t zero_on = nullptr, bool zero = false) {
    if (b.n >= bytes) return SPGEMM_OK;
    const size_t want = std::max(bytes, size_t(1) << 16);
    if (h->ws_limit >= 0 && held_bytes(h) - b.n + want > (size_t)h->ws_limit) return SPGEMM_ERR_OOM;
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        b.p = nullptr;
        b.n = 0;
        if (e != cudaSuccess) return cuda_status(e);
    }
    const size_t n = want;
    if (cudaMalloc(&b.p, n) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return SPGEMM_ERR_OOM;
    }
    b.n = n;
    if (zero) TSG_CHECK(cudaMemsetAsync(b.p, 0, n, zero_on));
    return SPGEMM_OK;
}

spgemm_status grow_pinned(spgemm_handle* h, size_t bytes) {
    if (h->pinned_n >= bytes) return SPGEMM_OK;
    if (h->pinned) cudaFreeHost(h->pinned);
    h->pinned = nullptr;
    h->pinned_dev = nullptr;
    h->pinned_n = 0;
    size_t n = std::max(bytes, size_t(4096));
    if (cudaHostAlloc(&h->pinned, n, cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        h->pinned = nullptr;
        return SPGEMM_ERR_OOM;
    }
    if (cudaHostGetDevicePointer(&h->pinned_dev, h->pinned, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(h->pinned);
        h->pinned = nullptr;
        return SPGEMM_ERR_CUDA;
    }
    h->pinned_n = n;
    return SPGEMM_OK;
}

// Reads `bytes` of device memory into h->pinned at host address p (inside
// h->pinned) with a kernel on st, so that the read never waits behind a
// large copy-engine transfer of another stream; the caller synchronises st.
cudaError_t readback(spgemm_handle* h, void* p, const void* d, size_t bytes, cudaStream_t st) {
    const size_t off = static_cast<size_t>(static_cast<char*>(p) - static_cast<char*>(h->pinned));
    if (!h->pinned || static_cast<char*>(p) < static_cast<char*>(h->pinned) || off + bytes > h->pinned_n)
        return cudaErrorInvalidValue;
    ++h->launches;
    return launch_readback(static_cast<char*>(h->pinned_dev) + off, d, bytes, st);
}

void default_tune(spgemm_tune* t) {
    std::memset(t, 0, sizeof(*t));
    const int upper[12] = {16, 32, 64, 128, 256, 320, 384, 512, 1024, 2048, 4096, 8192};
    const int kernel[12] = {10, 0, 1, 2, 3, 15, 9, 4, 11, 12, 13, 14};
    t->num_bins = 12;
    for (int b = 0; b < 12; ++b) {
        t->bin_upper[b] = upper[b];
        t->bin_kernel[b] = kernel[b];
    }
    t->accumulator = SPGEMM_ACC_SORT;
    t->warps_per_block = 16;
    t->validate = 0;
    t->sym_warps_per_block = 8;
}

spgemm_status check_tune(const spgemm_tune* t) {
    if (t->num_bins < 1 || t->num_bins > SPGEMM_MAX_BINS) return SPGEMM_ERR_INVALID_ARG;
    if (t->accumulator != SPGEMM_ACC_SORT) return SPGEMM_ERR_INVALID_ARG;
    if (t->warps_per_block < 1 || t->warps_per_block > 32) return SPGEMM_ERR_INVALID_ARG;
    if (t->sym_warps_per_block < 0 || t->sym_warps_per_block > 32) return SPGEMM_ERR_INVALID_ARG;
    for (int b = 0; b < t->num_bins; ++b) {
        const int v = t->bin_kernel[b];
        if (v < 0 || v >= kNumVariants) return SPGEMM_ERR_INVALID_ARG;
        if (t->bin_upper[b] < 1 || t->bin_upper[b] > variant_cap(v)) return SPGEMM_ERR_INVALID_ARG;
        if (b > 0 && t->bin_upper[b] <= t->bin_upper[b - 1]) return SPGEMM_ERR_INVALID_ARG;
    }
    return SPGEMM_OK;
}

BinTable bins_of(const spgemm_tune& t) {
    BinTable bt{};
    bt.nbins = t.num_bins;
    for (int b = 0; b < t.num_bins; ++b) {
        bt.upper[b] = t.bin_upper[b];
        // warp and block teams keep one meta entry per A entry (capacity / 2);
        // a thread walks its A row directly
        bt.amax[b] = variant_team(t.bin_kernel[b]) == 1 ? (1 << 30) : variant_cap(t.bin_kernel[b]) / 2;
    }
    return bt;
}

uint64_t fnv(uint64_t h, const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= c[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct PhaseScope {
    spgemm_handle* h;
    int phase;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    PhaseScope(spgemm_handle* h_, int phase_, cudaStream_t s_) : h(h_), phase(phase_), s(s_) {
        if (!h->timing) return;
        a = take();
        b = take();
        if (a) cudaEventRecord(a, s);
    }
    cudaEvent_t take() {
        if (!h->spare.empty()) {
            cudaEvent_t e = h->spare.back();
            h->spare.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return e;
    }
    ~PhaseScope() {
        if (!h->timing) return;
        if (a && b) {
            cudaEventRecord(b, s);
            h->pending.push_back({phase, a, b});
        } else {
            if (a) h->spare.push_back(a);
            if (b) h->spare.push_back(b);
        }
    }
};

// warps per block of variant v for the requested setting (clamped to what
// the variant's launch bound and shared memory allow)
int sym_wpb(int v, int wpb) { return std::min(wpb, warp_variant_max_wpb(v, sym_smem_bytes(v, 1), true)); }
int num_wpb(int v, int dtype, int wpb) {
    return std::min(wpb, warp_variant_max_wpb(v, num_smem_bytes(v, dtype, 1), false));
}

void occupancy(spgemm_handle* h, int wpb, int swpb) {
    if (h->occ_wpb == wpb * 64 + swpb) return;
    for (int v = 0; v < kNumVariants; ++v) {
        h->occ_sym[v] = std::max(1, sym_blocks_per_sm(v, sym_wpb(v, swpb)));
        h->occ_num[0][v] = std::max(1, num_blocks_per_sm(v, 0, num_wpb(v, 0, wpb)));
        h->occ_num[1][v] = std::max(1, num_blocks_per_sm(v, 1, num_wpb(v, 1, wpb)));
    }
    h->occ_wpb = wpb * 64 + swpb;
}

int teams_per_block(int v, int wpb) {
    return variant_team(v) == 32 ? wpb : (variant_team(v) == 1 ? kThreadRows : 1);
}

void note_stream(spgemm_handle* h, cudaStream_t s) {
    h->last_stream = s;
    if (std::find(h->streams_used.begin(), h->streams_used.end(), s) == h->streams_used.end())
        h->streams_used.push_back(s);
}

// Fork / join of the per-bin launches.  next() hands out a branch stream
// that first waits for everything issued on st so far; join() makes st wait
// for every branch handed out.  With concurrency off every branch is st.
// Under stream capture the branches become parallel graph nodes.
struct BinFork {
    spgemm_handle* h;
    cudaStream_t st;
    bool on;
    int used = 0;
    cudaError_t err = cudaSuccess;
    BinFork(spgemm_handle* h_, cudaStream_t st_) : h(h_), st(st_), on(h_->concurrent_bins) {
        if (!on) return;
        if (!h->fork_ev) err = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming);
        if (err == cudaSuccess) err = cudaEventRecord(h->fork_ev, st);
        if (err != cudaSuccess) on = false;
    }
    cudaStream_t next() {
        if (!on || used > kMaxBins) return st;
        const int i = used;
        if (!h->side[i]) {
            cudaError_t e = cudaStreamCreateWithFlags(&h->side[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join_ev[i], cudaEventDisableTiming);
            if (e != cudaSuccess) {
                err = e;
                return st;
            }
        }
        if (cudaStreamWaitEvent(h->side[i], h->fork_ev, 0) != cudaSuccess) return st;
        ++used;
        return h->side[i];
    }
    cudaError_t join() {
        for (int i = 0; i < used; ++i) {
            cudaError_t e = cudaEventRecord(h->join_ev[i], h->side[i]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->join_ev[i], 0);
            if (e != cudaSuccess) return e;
        }
        used = 0;
        return err;
    }
};

struct Validate {
    const int* rp;
    const int* col;
    int nrows, ncols, nnz;
};

// One call of the engine: product (merge == false) or ordered sum of partials.
// fused_cap >= 0: single-pass product (one group) into that many entries;
// SPGEMM_ERR_UNSUPPORTED when the rows do not fit the warp-team variants.
// products_only: analysis only, *c_nnz = sum of the rows' product counts.
spgemm_status run(spgemm_handle* h, int dtype, bool merge, const std::vector<InstDev>& inst,
                  std::vector<GroupDev> groups, bool sizing, int64_t* c_nnz, const spgemm_tune& tune,
                  const std::vector<Validate>& checks, cudaStream_t st, long long fused_cap = -1,
                  bool products_only = false) {
    for (GroupDev& G : groups) G.ncols_inv = (1ull << 63) / (unsigned long long)std::max(G.ncols, 1);
    int dev = -1;
    TSG_CHECK(cudaGetDevice(&dev));
    if (dev != h->device) return SPGEMM_ERR_INVALID_ARG;
    note_stream(h, st);
    const int ngroups = (int)groups.size();
    const int ninst = (int)inst.size();
    std::vector<long long> unit_base(ngroups + 1);
    long long U = 0;
    int max_ncols = 1;
    for (int g = 0; g < ngroups; ++g) {
        unit_base[g] = U;
        U += groups[g].nrows;
        max_ncols = std::max(max_ncols, groups[g].ncols);
    }
    unit_base[ngroups] = U;
    if (U >= (1ll << 31) - 1) return SPGEMM_ERR_UNSUPPORTED;
    const int nb = tune.num_bins;
    const int nslots = nb + 2;  // regular bins, heavy, empty

    if (sizing) {
        // row_ptr of groups without rows is the single entry 0
        for (int g = 0; g < ngroups; ++g)
            if (groups[g].nrows == 0) TSG_CHECK(cudaMemsetAsync(groups[g].crp, 0, sizeof(int), st));
    }
    if (U == 0) {
        if ((sizing || products_only) && c_nnz)
            for (int g = 0; g < ngroups; ++g) c_nnz[g] = 0;
        if (fused_cap >= 0) {
            for (int g = 0; g < ngroups; ++g) TSG_CHECK(cudaMemsetAsync(groups[g].crp, 0, sizeof(int), st));
            if (c_nnz) c_nnz[0] = 0;
        }
        return SPGEMM_OK;
    }

    // ---- workspace
    if (U > h->units_cap) {
        // a failed growth may leave the buffer empty: units_cap follows it
        h->units_cap = h->units.n >= units_bytes(U) ? h->units_cap : -1;
        h->plan_valid = false;
        TSG_TRY(grow(h, h->units, units_bytes(U)));
        h->units_cap = U;
    }
    char* ub = static_cast<char*>(h->units.p);
    unsigned char* d_bin_of = reinterpret_cast<unsigned char*>(ub);
    int* d_list = reinterpret_cast<int*>(ub + align16(h->units_cap));
    int* d_counts = reinterpret_cast<int*>(ub + align16(h->units_cap) + align16(4 * h->units_cap));
    long long* d_ex =
        reinterpret_cast<long long*>(ub + align16(h->units_cap) + 2 * align16(4 * h->units_cap));
    int* d_glist = reinterpret_cast<int*>(ub + align16(h->units_cap) + 2 * align16(4 * h->units_cap) +
                                          align16(8 * (h->units_cap + 1)));

    const long long nblk = scan_blocks(U);
    size_t o_hist = 0;
    size_t o_off = o_hist + align16(4 * (kMaxBins + 2));
    size_t o_cur = o_off + align16(4 * (kMaxBins + 3));
    size_t o_status = o_cur + align16(4 * (kMaxBins + 2));
    size_t o_tick = o_status + 16;
    size_t o_bsum = o_tick + align16(4 * (kMaxBins + 3));  // per-bin tickets, then the deferred-row count
    size_t o_nnz = o_bsum + align16(8 * nblk);
    size_t o_ubase = o_nnz + align16(8 * ngroups);
    size_t o_inst = o_ubase + align16(8 * (ngroups + 1));
    size_t o_groups = o_inst + align16(sizeof(InstDev) * ninst);
    size_t small_bytes = o_groups + align16(sizeof(GroupDev) * ngroups);
    if (h->small.n < small_bytes) {
        h->plan_valid = false;
        h->last_stage_dst = nullptr;
    }
    TSG_TRY(grow(h, h->small, small_bytes));
    char* sb = static_cast<char*>(h->small.p);
    int* d_hist = reinterpret_cast<int*>(sb + o_hist);
    int* d_off = reinterpret_cast<int*>(sb + o_off);
    int* d_cur = reinterpret_cast<int*>(sb + o_cur);
    int* d_tick = reinterpret_cast<int*>(sb + o_tick);
    TSG_TRY(grow(h, h->status, 16, st, true));
    unsigned* d_status = static_cast<unsigned*>(h->status.p);
    long long* d_bsum = reinterpret_cast<long long*>(sb + o_bsum);
    long long* d_nnz = reinterpret_cast<long long*>(sb + o_nnz);
    long long* d_ubase = reinterpret_cast<long long*>(sb + o_ubase);
    InstDev* d_inst = reinterpret_cast<InstDev*>(sb + o_inst);
    GroupDev* d_groups = reinterpret_cast<GroupDev*>(sb + o_groups);

    const size_t pinned_bytes = align16(8 * ngroups) + align16(4 * (kMaxBins + 2)) + 16;
    TSG_TRY(grow_pinned(h, pinned_bytes));
    long long* p_nnz = static_cast<long long*>(h->pinned);
    int* p_hist = reinterpret_cast<int*>(static_cast<char*>(h->pinned) + align16(8 * ngroups));
    unsigned* p_status =
        reinterpret_cast<unsigned*>(static_cast<char*>(h->pinned) + align16(8 * ngroups) + align16(4 * (kMaxBins + 2)));

    // ---- descriptors (pageable source: the copy is staged before the call returns)
    {
        std::vector<char> stage(small_bytes - o_ubase);
        std::memcpy(stage.data(), unit_base.data(), 8 * (ngroups + 1));
        if (ninst) std::memcpy(stage.data() + (o_inst - o_ubase), inst.data(), sizeof(InstDev) * ninst);
        std::memcpy(stage.data() + (o_groups - o_ubase), groups.data(), sizeof(GroupDev) * ngroups);
        if (h->last_stage_dst != sb + o_ubase || h->last_stage != stage) {
            TSG_CHECK(cudaMemcpyAsync(sb + o_ubase, stage.data(), stage.size(), cudaMemcpyHostToDevice, st));
            h->last_stage.swap(stage);
            h->last_stage_dst = sb + o_ubase;
        }
    }
    // ---- plan signature (input patterns, output row_ptr, bins)
    uint64_t sig = 1469598103934665603ull;
    sig = fnv(sig, &merge, sizeof(merge));
    for (const InstDev& I : inst) {
        const void* ptrs[4] = {I.arp, I.acol, I.brp, I.bcol};
        sig = fnv(sig, ptrs, sizeof(ptrs));
    }
    for (const GroupDev& G : groups) {
        const int shape[4] = {G.inst_begin, G.inst_count, G.nrows, G.ncols};
        sig = fnv(sig, shape, sizeof(shape));
        sig = fnv(sig, &G.crp, sizeof(G.crp));
    }
    sig = fnv(sig, tune.bin_upper, sizeof(int) * nb);
    sig = fnv(sig, tune.bin_kernel, sizeof(int) * nb);

    if (tune.validate) {
        // nothing else may read a bad input: check, wait, then proceed
        for (const Validate& v : checks) {
            TSG_CHECK(launch_validate(v.rp, v.col, v.nrows, v.ncols, v.nnz, d_status, st));
            ++h->launches;
        }
        TSG_CHECK(readback(h, p_status, d_status, 4, st));
        TSG_CHECK(cudaStreamSynchronize(st));
        if (*p_status & kStatusNotCanonical) {
            h->plan_valid = false;
            TSG_CHECK(cudaMemsetAsync(d_status, 0, 4, st));
            return SPGEMM_ERR_NOT_CANONICAL;
        }
    }

    const bool reuse = !sizing && fused_cap < 0 && !products_only && h->plan_valid && h->plan_sig == sig;
    if (!reuse) {
        h->plan_valid = false;
        PhaseScope ps(h, 0, st);
        TSG_CHECK(cudaMemsetAsync(d_hist, 0, 4 * nslots, st));
        AnalysisArgs aa;
        aa.inst = d_inst;
        aa.groups = d_groups;
        aa.unit_base = d_ubase;
        aa.ngroups = ngroups;
        aa.nunits = U;
        aa.merge = merge ? 1 : 0;
        aa.bt = bins_of(tune);
        aa.bin_of = d_bin_of;
        aa.hist = d_hist;
        aa.counts = d_counts;
        aa.sizing = sizing ? 1 : 0;
        aa.total_u = nullptr;
        if (products_only) {
            aa.total_u = reinterpret_cast<unsigned long long*>(d_nnz);
            TSG_CHECK(cudaMemsetAsync(d_nnz, 0, 8, st));
        }
        TSG_CHECK(launch_analysis(aa, st));
        TSG_CHECK(launch_bin_offsets(d_hist, d_off, d_cur, nslots, st));
        TSG_CHECK(launch_bin_fill(d_bin_of, U, d_off, d_cur, d_list, st));
        h->launches += 3;
    }

    const int wpb = tune.warps_per_block;
    const int swpb = tune.sym_warps_per_block > 0 ? tune.sym_warps_per_block : wpb;
    occupancy(h, wpb, swpb);
    RowLaunchArgs la;
    la.inst = d_inst;
    la.groups = d_groups;
    la.unit_base = d_ubase;
    la.ngroups = ngroups;
    la.list = d_list;
    la.bin_off = d_off;
    la.merge = merge ? 1 : 0;
    la.status = d_status;
    la.counts = d_counts;
    la.tick = d_tick;
    la.glist = nullptr;  // deferral only in the numeric pass of the two-pass product
    la.gcount = d_tick + nslots;
    const int chunk = heavy_chunk_for(max_ncols);

    if (products_only) {
        TSG_CHECK(readback(h, p_nnz, d_nnz, 8, st));
        TSG_CHECK(cudaStreamSynchronize(st));
        *c_nnz = p_nnz[0];
        return SPGEMM_OK;
    }
    if (fused_cap >= 0) {
        // single pass: all rows must sit in warp-team bins of increasing capacity
        h->plan_valid = false;
        TSG_CHECK(readback(h, p_hist, d_hist, 4 * nslots, st));
        TSG_CHECK(cudaStreamSynchronize(st));
        if (ngroups != 1 || p_hist[nb] > 0) return SPGEMM_ERR_UNSUPPORTED;
        int bmax = -1;
        for (int b = 0; b < nb; ++b)
            if (p_hist[b] > 0) bmax = b;
        if (bmax < 0) bmax = 0;
        const int v = tune.bin_kernel[bmax];
        if (variant_team(v) != 32) return SPGEMM_ERR_UNSUPPORTED;
        for (int b = 0; b < bmax; ++b)
            if (p_hist[b] > 0 && variant_cap(tune.bin_kernel[b]) > variant_cap(v)) return SPGEMM_ERR_UNSUPPORTED;
        const int wv = num_wpb(v, dtype, wpb);
        int* d_ticket = reinterpret_cast<int*>(sb + o_status);
        TSG_CHECK(cudaMemsetAsync(d_ticket, 0, 16, st));
        const long long ntiles = (U + wv - 1) / wv;  // look-back entries: one per tile of wv rows
        TSG_CHECK(cudaMemsetAsync(d_ex, 0, 8 * ntiles, st));
        FusedCtl fc;
        fc.ticket = d_ticket;
        fc.lb = reinterpret_cast<unsigned long long*>(d_ex);
        fc.cap = fused_cap;
        fc.nunits = (int)U;
        fc.crp = groups[0].crp;
        fc.spin_limit = h->wait_limit;
        fc.hold_tile = h->hold_tile;
        const int occ = std::max(1, num_fused_blocks_per_sm(v, dtype, wv));
        const int blocks = (int)std::min<long long>(ntiles, (long long)h->sms * occ);
        {
            PhaseScope ps(h, 3, st);
            TSG_CHECK(launch_num_fused(v, dtype, la, fc, blocks, wv, st));
            ++h->launches;
        }
        int* p_total = reinterpret_cast<int*>(p_nnz);
        TSG_CHECK(readback(h, p_total, groups[0].crp + U, 4, st));
        TSG_CHECK(readback(h, p_status, d_status, 4, st));
        TSG_CHECK(cudaStreamSynchronize(st));
        const unsigned status = *p_status;
        if (status) TSG_CHECK(cudaMemsetAsync(d_status, 0, 4, st));
        if (status & kStatusTimeout) return SPGEMM_ERR_DEVICE_TIMEOUT;
        if (status & kStatusCapacity) return SPGEMM_ERR_CAPACITY;
        if (status & kStatusInternal) return SPGEMM_ERR_INTERNAL;
        if (c_nnz) c_nnz[0] = *p_total;
        return SPGEMM_OK;
    }

    if (sizing) {
        {
            PhaseScope ps(h, 1, st);
            BinFork fork(h, st);
            for (int b = 0; b < nb; ++b) {
                const int v = tune.bin_kernel[b];
                la.bin = b;
                TSG_CHECK(launch_sym_rows(v, la, h->sms * h->occ_sym[v], sym_wpb(v, swpb), fork.next()));
                ++h->launches;
            }
            la.bin = nb;
            TSG_CHECK(launch_sym_heavy(la, h->sms, chunk, fork.next()));
            ++h->launches;
            TSG_CHECK(fork.join());
        }
        {
            PhaseScope ps(h, 2, st);
            TSG_CHECK(cudaMemsetAsync(d_nnz, 0, 8 * ngroups, st));
            TSG_CHECK(launch_scan(d_counts, U, d_bsum, d_ex, st));
            TSG_CHECK(launch_rowptr(d_groups, d_ubase, ngroups, U, d_ex, d_nnz, st));
            h->launches += 4;
        }
        TSG_CHECK(readback(h, p_nnz, d_nnz, 8 * ngroups, st));
        TSG_CHECK(readback(h, p_hist, d_hist, 4 * nslots, st));
        TSG_CHECK(readback(h, p_status, d_status, 4, st));
        TSG_CHECK(cudaStreamSynchronize(st));
        const unsigned status = *p_status;
        // a latched error (this call's or an earlier asynchronous call's) is
        // reported once, then cleared
        if (status) TSG_CHECK(cudaMemsetAsync(d_status, 0, 4, st));
        if (status & kStatusNotCanonical) return SPGEMM_ERR_NOT_CANONICAL;
        if (status & kStatusHashOverflow) return SPGEMM_ERR_HASH_OVERFLOW;
        if (status & kStatusInternal) return SPGEMM_ERR_INTERNAL;
        bool overflow = false;
        for (int g = 0; g < ngroups; ++g) {
            if (c_nnz) c_nnz[g] = p_nnz[g];
            if (p_nnz[g] > 2147483647ll) overflow = true;
        }
        if (overflow) return SPGEMM_ERR_INDEX_OVERFLOW;
        h->plan_hist.assign(p_hist, p_hist + nslots);
        h->plan_sig = sig;
        h->plan_valid = true;
        return SPGEMM_OK;
    }

    // ---- fill call
    std::vector<int> hist;
    if (reuse) {
        hist = h->plan_hist;
    } else {
        TSG_CHECK(readback(h, p_hist, d_hist, 4 * nslots, st));
        TSG_CHECK(cudaStreamSynchronize(st));
        hist.assign(p_hist, p_hist + nslots);
    }
    const int only = h->only_bin;  // >= 0: the autotuner times one bin's kernel
    if (hist[nb] > 0 && only < 0) {
        PhaseScope ps(h, 4, st);
        const int blocks = std::min(hist[nb], h->sms);
        const size_t esz = dtype == SPGEMM_F64 ? 8 : 4;
        TSG_TRY(grow(h, h->dense, (size_t)blocks * chunk * esz, st, true));
        // blocks beyond the allocation would share slots: size the grid to it
        const int slots = (int)std::min<size_t>(blocks, h->dense.n / ((size_t)chunk * esz));
        la.bin = nb;
        TSG_CHECK(launch_num_heavy(dtype, la, h->dense.p, slots, chunk, st));
        ++h->launches;
    }
    {
        PhaseScope ps(h, 3, st);
        TSG_CHECK(cudaMemsetAsync(d_tick, 0, 4 * (nslots + 1), st));
        la.glist = d_glist;
        BinFork fork(h, st);
        for (int b = 0; b < nb; ++b) {
            if (hist[b] == 0 || (only >= 0 && b != only)) continue;
            const int v = tune.bin_kernel[b];
            const int wv = num_wpb(v, dtype, wpb);
            const int tpb = teams_per_block(v, wv);
            const long long need = (hist[b] + tpb - 1) / tpb;
            const int blocks = (int)std::min<long long>(need, (long long)h->sms * h->occ_num[dtype][v]);
            la.bin = b;
            TSG_CHECK(launch_num_rows(v, dtype, la, blocks, wv, fork.next()));
            ++h->launches;
        }
        TSG_CHECK(fork.join());
        // rows the bins deferred (clustered columns, many repeats)
        if (only < 0) {
            TSG_CHECK(launch_num_grouped(dtype, la, h->sms, st));
            ++h->launches;
        }
        la.glist = nullptr;
    }
    if (tune.validate) {
        TSG_CHECK(readback(h, p_status, d_status, 4, st));
        TSG_CHECK(cudaStreamSynchronize(st));
        const unsigned status = *p_status;
        if (status) TSG_CHECK(cudaMemsetAsync(d_status, 0, 4, st));
        if (status & kStatusNotCanonical) return SPGEMM_ERR_NOT_CANONICAL;
        if (status & kStatusInternal) return SPGEMM_ERR_INTERNAL;
    }
    return SPGEMM_OK;
}

bool csr_in_ok(const spgemm_csr_in* X, bool need_val) {
    if (!X || X->nrows < 0 || X->ncols < 0 || X->nnz < 0 || !X->row_ptr) return false;
    if (X->nnz > 0 && (!X->col_idx || (need_val && !X->val))) return false;
    return true;
}

}  // namespace

namespace {

// Offsets of the device copies in h->hx: A row_ptr | A col | A val | B row_ptr
// | B col | B val | C row_ptr (values sized for 8 bytes).
struct HostLayout {
    size_t arp, acol, aval, brp, bcol, bval, crp, bytes;
    HostLayout(const spgemm_csr_in* A, const spgemm_csr_in* B) {
        arp = 0;
        acol = arp + align16(4 * ((size_t)A->nrows + 1));
        aval = acol + align16(4 * (size_t)A->nnz);
        brp = aval + align16(8 * (size_t)A->nnz);
        bcol = brp + align16(4 * ((size_t)B->nrows + 1));
        bval = bcol + align16(4 * (size_t)B->nnz);
        crp = bval + align16(8 * (size_t)B->nnz);
        bytes = crp + align16(4 * ((size_t)A->nrows + 1));
    }
};

bool host_in_ok(const spgemm_csr_in* X, bool need_val) {
    if (!csr_in_ok(X, false)) return false;
    return !(need_val && X->nnz > 0 && !X->val);
}

spgemm_csr_in dev_view(const spgemm_csr_in* X, char* base, size_t rp, size_t col, size_t val, bool vals) {
    spgemm_csr_in d = *X;
    d.row_ptr = reinterpret_cast<const int32_t*>(base + rp);
    d.col_idx = reinterpret_cast<const int32_t*>(base + col);
    d.val = vals ? static_cast<const void*>(base + val) : nullptr;
    return d;
}

}  // namespace

// ====================================================================== ABI

extern "C" {

const char* spgemm_status_str(spgemm_status s) {
    switch (s) {
        case SPGEMM_OK: return "ok";
        case SPGEMM_ERR_INVALID_ARG: return "invalid argument";
        case SPGEMM_ERR_SHAPE: return "shape mismatch";
        case SPGEMM_ERR_DTYPE: return "unknown dtype";
        case SPGEMM_ERR_INDEX_OVERFLOW: return "output nnz exceeds int32";
        case SPGEMM_ERR_OOM: return "out of device memory";
        case SPGEMM_ERR_CUDA: return "CUDA runtime error";
        case SPGEMM_ERR_DEVICE_TIMEOUT: return "device wait timed out";
        case SPGEMM_ERR_HASH_OVERFLOW: return "accumulator overflow";
        case SPGEMM_ERR_NOT_CANONICAL: return "input is not a valid CSR matrix";
        case SPGEMM_ERR_INTERNAL: return "device consistency check failed";
        case SPGEMM_ERR_UNSUPPORTED: return "unsupported request";
        case SPGEMM_ERR_CAPACITY: return "output capacity too small";
    }
    return "unknown status";
}

const char* spgemm_version(void) { return "trident-spgemm-gb300 0.1 (sm_103a)"; }

spgemm_status spgemm_default_tune(spgemm_tune* t) {
    if (!t) return SPGEMM_ERR_INVALID_ARG;
    default_tune(t);
    return SPGEMM_OK;
}

spgemm_status spgemm_create(spgemm_handle** out) {
    if (!out) return SPGEMM_ERR_INVALID_ARG;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SPGEMM_ERR_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        return SPGEMM_ERR_CUDA;
    }
    spgemm_handle* h = new (std::nothrow) spgemm_handle();
    if (!h) return SPGEMM_ERR_OOM;
    h->device = dev;
    h->sms = sms;
    default_tune(&h->tune);
    *out = h;
    return SPGEMM_OK;
}

spgemm_status spgemm_destroy(spgemm_handle* h) {
    if (!h) return SPGEMM_OK;
    for (cudaStream_t s : h->streams_used) cudaStreamSynchronize(s);
    for (int i = 0; i <= kMaxBins; ++i) {
        if (h->side[i]) {
            cudaStreamSynchronize(h->side[i]);
            cudaStreamDestroy(h->side[i]);
        }
        if (h->join_ev[i]) cudaEventDestroy(h->join_ev[i]);
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    for (const PhaseEvent& p : h->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (cudaEvent_t e : h->spare) cudaEventDestroy(e);
    if (h->units.p) cudaFree(h->units.p);
    if (h->small.p) cudaFree(h->small.p);
    if (h->dense.p) cudaFree(h->dense.p);
    if (h->status.p) cudaFree(h->status.p);
    if (h->tr.p) cudaFree(h->tr.p);
    if (h->mcl.p) cudaFree(h->mcl.p);
    if (h->mcl_acc.p) cudaFree(h->mcl_acc.p);
    if (h->mcl_side) {
        cudaStreamSynchronize(h->mcl_side);
        cudaStreamDestroy(h->mcl_side);
    }
    for (cudaEvent_t e : h->mcl_ev)
        if (e) cudaEventDestroy(e);
    if (h->mcl_heavy.p) cudaFree(h->mcl_heavy.p);
    if (h->mcl_bucket.p) cudaFree(h->mcl_bucket.p);
    if (h->perm.p) cudaFree(h->perm.p);
    if (h->hx.p) cudaFree(h->hx.p);
    if (h->hc.p) cudaFree(h->hc.p);
    if (h->copy) {
        cudaStreamSynchronize(h->copy);
        cudaStreamDestroy(h->copy);
    }
    for (cudaEvent_t e : h->panel_ev) cudaEventDestroy(e);
    if (h->hv_ev) cudaEventDestroy(h->hv_ev);
    if (h->pinned) cudaFreeHost(h->pinned);
    delete h;
    return SPGEMM_OK;
}

spgemm_status spgemm_set_tune(spgemm_handle* h, const spgemm_tune* t) {
    if (!h) return SPGEMM_ERR_INVALID_ARG;
    if (!t) {
        default_tune(&h->tune);
        return SPGEMM_OK;
    }
    TSG_TRY(check_tune(t));
    h->tune = *t;
    return SPGEMM_OK;
}

spgemm_status spgemm_get_tune(const spgemm_handle* h, spgemm_tune* t) {
    if (!h || !t) return SPGEMM_ERR_INVALID_ARG;
    *t = h->tune;
    return SPGEMM_OK;
}

spgemm_status spgemm_symbolic(spgemm_handle* h, const spgemm_csr_in* A, const spgemm_csr_in* B, int32_t* c_row_ptr,
                              int64_t* c_nnz, spgemm_stream_t stream) {
    if (!h || !csr_in_ok(A, false) || !csr_in_ok(B, false) || !c_row_ptr || !c_nnz) return SPGEMM_ERR_INVALID_ARG;
    if (A->ncols != B->nrows) return SPGEMM_ERR_SHAPE;
    std::vector<InstDev> inst{{A->row_ptr, A->col_idx, A->val, B->row_ptr, B->col_idx, B->val, B->nnz}};
    std::vector<GroupDev> groups{{0, 1, A->nrows, B->ncols, c_row_ptr, nullptr, nullptr, 0}};
    std::vector<Validate> checks{{A->row_ptr, A->col_idx, A->nrows, A->ncols, A->nnz},
                                 {B->row_ptr, B->col_idx, B->nrows, B->ncols, B->nnz}};
    return run(h, 0, false, inst, groups, true, c_nnz, h->tune, checks, reinterpret_cast<cudaStream_t>(stream));
}

spgemm_status spgemm_numeric(spgemm_handle* h, spgemm_dtype dtype, const spgemm_csr_in* A, const spgemm_csr_in* B,
                             spgemm_csr_out* C, spgemm_stream_t stream) {
    if (!h || !csr_in_ok(A, true) || !csr_in_ok(B, true) || !C || !C->row_ptr) return SPGEMM_ERR_INVALID_ARG;
    if (dtype != SPGEMM_F32 && dtype != SPGEMM_F64) return SPGEMM_ERR_DTYPE;
    if (A->ncols != B->nrows || C->nrows != A->nrows || C->ncols != B->ncols) return SPGEMM_ERR_SHAPE;
    std::vector<InstDev> inst{{A->row_ptr, A->col_idx, A->val, B->row_ptr, B->col_idx, B->val, B->nnz}};
    std::vector<GroupDev> groups{{0, 1, A->nrows, B->ncols, C->row_ptr, C->col_idx, C->val, 0}};
    std::vector<Validate> checks{{A->row_ptr, A->col_idx, A->nrows, A->ncols, A->nnz},
                                 {B->row_ptr, B->col_idx, B->nrows, B->ncols, B->nnz}};
    return run(h, dtype, false, inst, groups, false, nullptr, h->tune, checks,
               reinterpret_cast<cudaStream_t>(stream));
}

spgemm_status spgemm_host_symbolic(spgemm_handle* h, int32_t value_dtype, const spgemm_csr_in* A,
                                   const spgemm_csr_in* B, int32_t* c_row_ptr, int64_t* c_nnz,
                                   spgemm_stream_t stream) {
    if (!h || !host_in_ok(A, false) || !host_in_ok(B, false) || !c_row_ptr || !c_nnz) return SPGEMM_ERR_INVALID_ARG;
    if (value_dtype != -1 && value_dtype != SPGEMM_F32 && value_dtype != SPGEMM_F64) return SPGEMM_ERR_DTYPE;
    if (A->ncols != B->nrows) return SPGEMM_ERR_SHAPE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    h->hx_sized = false;
    h->hv_ready = false;
    // an earlier call's uploads into the buffers must be over before they move
    if (h->copy) TSG_CHECK(cudaStreamSynchronize(h->copy));
    const HostLayout L(A, B);
    TSG_TRY(grow(h, h->hx, L.bytes));
    char* x = static_cast<char*>(h->hx.p);
    const bool vals = value_dtype != -1 && (A->nnz == 0 || A->val) && (B->nnz == 0 || B->val);
    if (vals) {
        // the values are not needed for the sizing: their upload runs on the
        // second stream meanwhile, and the numeric call waits for it
        const size_t esz = value_dtype == SPGEMM_F64 ? 8 : 4;
        if (!h->copy) TSG_CHECK(cudaStreamCreateWithFlags(&h->copy, cudaStreamNonBlocking));
        if (!h->hv_ev) TSG_CHECK(cudaEventCreateWithFlags(&h->hv_ev, cudaEventDisableTiming));
        if (B->nnz) TSG_CHECK(cudaMemcpyAsync(x + L.bval, B->val, esz * (size_t)B->nnz, cudaMemcpyHostToDevice, h->copy));
        if (A->nnz) TSG_CHECK(cudaMemcpyAsync(x + L.aval, A->val, esz * (size_t)A->nnz, cudaMemcpyHostToDevice, h->copy));
        TSG_CHECK(cudaEventRecord(h->hv_ev, h->copy));
    }
    TSG_CHECK(cudaMemcpyAsync(x + L.arp, A->row_ptr, 4 * ((size_t)A->nrows + 1), cudaMemcpyHostToDevice, st));
    if (A->nnz) TSG_CHECK(cudaMemcpyAsync(x + L.acol, A->col_idx, 4 * (size_t)A->nnz, cudaMemcpyHostToDevice, st));
    TSG_CHECK(cudaMemcpyAsync(x + L.brp, B->row_ptr, 4 * ((size_t)B->nrows + 1), cudaMemcpyHostToDevice, st));
    if (B->nnz) TSG_CHECK(cudaMemcpyAsync(x + L.bcol, B->col_idx, 4 * (size_t)B->nnz, cudaMemcpyHostToDevice, st));
    const spgemm_csr_in dA = dev_view(A, x, L.arp, L.acol, L.aval, false);
    const spgemm_csr_in dB = dev_view(B, x, L.brp, L.bcol, L.bval, false);
    TSG_TRY(spgemm_symbolic(h, &dA, &dB, reinterpret_cast<int32_t*>(x + L.crp), c_nnz, stream));
    TSG_CHECK(cudaMemcpyAsync(c_row_ptr, x + L.crp, 4 * ((size_t)A->nrows + 1), cudaMemcpyDeviceToHost, st));
    TSG_CHECK(cudaStreamSynchronize(st));
    h->hx_key[0] = A->row_ptr;
    h->hx_key[1] = A->col_idx;
    h->hx_key[2] = B->row_ptr;
    h->hx_key[3] = B->col_idx;
    h->hx_sized = true;
    if (vals) {
        h->hv_key[0] = A->val;
        h->hv_key[1] = B->val;
        h->hv_dtype = value_dtype;
        h->hv_ready = true;
    }
    return SPGEMM_OK;
}

spgemm_status spgemm_host_numeric(spgemm_handle* h, spgemm_dtype dtype, const spgemm_csr_in* A,
                                  const spgemm_csr_in* B, spgemm_csr_out* C, int32_t panels,
                                  spgemm_stream_t stream) {
    if (!h || !host_in_ok(A, true) || !host_in_ok(B, true) || !C || !C->row_ptr) return SPGEMM_ERR_INVALID_ARG;
    if (dtype != SPGEMM_F32 && dtype != SPGEMM_F64) return SPGEMM_ERR_DTYPE;
    if (A->ncols != B->nrows || C->nrows != A->nrows || C->ncols != B->ncols) return SPGEMM_ERR_SHAPE;
    if (panels < 0 || panels > 1024) return SPGEMM_ERR_INVALID_ARG;
    if (panels == 0) panels = 8;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int m = A->nrows;
    const long long nnz = C->row_ptr[m];
    if (nnz < 0 || nnz > 2147483647ll) return SPGEMM_ERR_INVALID_ARG;
    if (nnz > 0 && (!C->col_idx || !C->val)) return SPGEMM_ERR_INVALID_ARG;
    const size_t esz = dtype == SPGEMM_F64 ? 8 : 4;
    const HostLayout L(A, B);
    const bool same = h->hx_sized && h->hx.n >= L.bytes && h->hx_key[0] == A->row_ptr &&
                      h->hx_key[1] == A->col_idx && h->hx_key[2] == B->row_ptr && h->hx_key[3] == B->col_idx;
    const bool have_vals = same && h->hv_ready && h->hv_dtype == (int)dtype && h->hv_key[0] == A->val &&
                           h->hv_key[1] == B->val;
    h->hx_sized = false;
    h->hv_ready = false;
    if (!same) {
        if (h->copy) TSG_CHECK(cudaStreamSynchronize(h->copy));
        TSG_TRY(grow(h, h->hx, L.bytes));
    }
    TSG_TRY(grow(h, h->hc, align16(4 * (size_t)nnz) + esz * (size_t)nnz));
    char* x = static_cast<char*>(h->hx.p);
    int32_t* ccol = static_cast<int32_t*>(h->hc.p);
    char* cval = static_cast<char*>(h->hc.p) + align16(4 * (size_t)nnz);
    if (!same) {
        // not the sizing call's inputs: indices and C's row_ptr again
        TSG_CHECK(cudaMemcpyAsync(x + L.arp, A->row_ptr, 4 * ((size_t)m + 1), cudaMemcpyHostToDevice, st));
        if (A->nnz) TSG_CHECK(cudaMemcpyAsync(x + L.acol, A->col_idx, 4 * (size_t)A->nnz, cudaMemcpyHostToDevice, st));
        TSG_CHECK(cudaMemcpyAsync(x + L.brp, B->row_ptr, 4 * ((size_t)B->nrows + 1), cudaMemcpyHostToDevice, st));
        if (B->nnz) TSG_CHECK(cudaMemcpyAsync(x + L.bcol, B->col_idx, 4 * (size_t)B->nnz, cudaMemcpyHostToDevice, st));
        TSG_CHECK(cudaMemcpyAsync(x + L.crp, C->row_ptr, 4 * ((size_t)m + 1), cudaMemcpyHostToDevice, st));
    }
    if (have_vals) {
        TSG_CHECK(cudaStreamWaitEvent(st, h->hv_ev, 0));  // uploaded during the sizing call
    } else {
        if (A->nnz) TSG_CHECK(cudaMemcpyAsync(x + L.aval, A->val, esz * (size_t)A->nnz, cudaMemcpyHostToDevice, st));
        if (B->nnz) TSG_CHECK(cudaMemcpyAsync(x + L.bval, B->val, esz * (size_t)B->nnz, cudaMemcpyHostToDevice, st));
    }
    if (!h->copy) TSG_CHECK(cudaStreamCreateWithFlags(&h->copy, cudaStreamNonBlocking));
    while ((int)h->panel_ev.size() < panels) {
        cudaEvent_t e;
        TSG_CHECK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        h->panel_ev.push_back(e);
    }
    const spgemm_csr_in dB = dev_view(B, x, L.brp, L.bcol, L.bval, true);
    // A panel's row_ptr view starts at an absolute offset, which the input
    // check would reject: the whole matrices are checked once (here, or by
    // the sizing call on the same arrays) and the panels run unchecked.
    spgemm_tune tp = h->tune;
    if (tp.validate && !same) {
        const spgemm_csr_in fA = dev_view(A, x, L.arp, L.acol, L.aval, false);
        TSG_TRY(grow(h, h->status, 16, st, true));
        TSG_TRY(grow_pinned(h, 16));
        unsigned* d_status = static_cast<unsigned*>(h->status.p);
        for (const spgemm_csr_in* X : {&fA, &dB}) {
            TSG_CHECK(launch_validate(X->row_ptr, X->col_idx, X->nrows, X->ncols, (int)X->nnz, d_status, st));
            ++h->launches;
        }
        TSG_CHECK(readback(h, h->pinned, d_status, 4, st));
        TSG_CHECK(cudaStreamSynchronize(st));
        if (*static_cast<const unsigned*>(h->pinned) & kStatusNotCanonical) {
            TSG_CHECK(cudaMemsetAsync(d_status, 0, 4, st));
            return SPGEMM_ERR_NOT_CANONICAL;
        }
    }
    tp.validate = 0;
    spgemm_status rc = SPGEMM_OK;
    for (int p = 0; p < panels && rc == SPGEMM_OK; ++p) {
        // the first panel is half the others: the copies out start sooner
        const long long den = 2ll * panels - 1;
        const int r0 = p == 0 ? 0 : (int)((2ll * p - 1) * m / den);
        const int r1 = (int)((2ll * p + 1) * m / den);
        if (r1 <= r0) continue;
        // rows [r0, r1): row pointers are absolute offsets into the full arrays
        spgemm_csr_in dA = dev_view(A, x, L.arp, L.acol, L.aval, true);
        dA.nrows = r1 - r0;
        dA.row_ptr += r0;
        int32_t* crp = reinterpret_cast<int32_t*>(x + L.crp) + r0;
        std::vector<InstDev> inst{{dA.row_ptr, dA.col_idx, dA.val, dB.row_ptr, dB.col_idx, dB.val, dB.nnz}};
        std::vector<GroupDev> groups{{0, 1, dA.nrows, dB.ncols, crp, ccol, cval, 0}};
        rc = run(h, dtype, false, inst, groups, false, nullptr, tp, {}, st);
        if (rc != SPGEMM_OK) break;
        const long long e0 = C->row_ptr[r0], e1 = C->row_ptr[r1];
        if (e1 <= e0) continue;
        TSG_CHECK(cudaEventRecord(h->panel_ev[p], st));
        TSG_CHECK(cudaStreamWaitEvent(h->copy, h->panel_ev[p], 0));
        TSG_CHECK(cudaMemcpyAsync(C->col_idx + e0, ccol + e0, 4 * (size_t)(e1 - e0), cudaMemcpyDeviceToHost, h->copy));
        TSG_CHECK(cudaMemcpyAsync(static_cast<char*>(C->val) + esz * e0, cval + esz * e0, esz * (size_t)(e1 - e0),
                                  cudaMemcpyDeviceToHost, h->copy));
    }
    const cudaError_t e1 = cudaStreamSynchronize(h->copy);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    if (rc != SPGEMM_OK) return rc;
    TSG_CHECK(e1);
    TSG_CHECK(e2);
    return spgemm_device_status(h);
}

spgemm_status spgemm_products(spgemm_handle* h, const spgemm_csr_in* A, const spgemm_csr_in* B, int64_t* total,
                              spgemm_stream_t stream) {
    if (!h || !csr_in_ok(A, false) || !csr_in_ok(B, false) || !total) return SPGEMM_ERR_INVALID_ARG;
    if (A->ncols != B->nrows) return SPGEMM_ERR_SHAPE;
    std::vector<InstDev> inst{{A->row_ptr, A->col_idx, A->val, B->row_ptr, B->col_idx, B->val, B->nnz}};
    std::vector<GroupDev> groups{{0, 1, A->nrows, B->ncols, nullptr, nullptr, nullptr, 0}};
    return run(h, 0, false, inst, groups, false, total, h->tune, {}, reinterpret_cast<cudaStream_t>(stream), -1, true);
}

spgemm_status spgemm_fused(spgemm_handle* h, spgemm_dtype dtype, const spgemm_csr_in* A, const spgemm_csr_in* B,
                           spgemm_csr_out* C, int64_t capacity, int64_t* c_nnz, spgemm_stream_t stream) {
    if (!h || !csr_in_ok(A, true) || !csr_in_ok(B, true) || !C || !C->row_ptr || !c_nnz || capacity < 0)
        return SPGEMM_ERR_INVALID_ARG;
    if (capacity > 0 && (!C->col_idx || !C->val)) return SPGEMM_ERR_INVALID_ARG;
    if (dtype != SPGEMM_F32 && dtype != SPGEMM_F64) return SPGEMM_ERR_DTYPE;
    if (A->ncols != B->nrows || C->nrows != A->nrows || C->ncols != B->ncols) return SPGEMM_ERR_SHAPE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::vector<InstDev> inst{{A->row_ptr, A->col_idx, A->val, B->row_ptr, B->col_idx, B->val, B->nnz}};
    std::vector<GroupDev> groups{{0, 1, A->nrows, B->ncols, C->row_ptr, C->col_idx, C->val, 0}};
    std::vector<Validate> checks{{A->row_ptr, A->col_idx, A->nrows, A->ncols, A->nnz},
                                 {B->row_ptr, B->col_idx, B->nrows, B->ncols, B->nnz}};
    spgemm_status rc = run(h, dtype, false, inst, groups, false, c_nnz, h->tune, checks, st, capacity);
    if (rc != SPGEMM_ERR_UNSUPPORTED) return rc;
    // two-pass route
    TSG_TRY(spgemm_symbolic(h, A, B, C->row_ptr, c_nnz, stream));
    if (*c_nnz > capacity) return SPGEMM_ERR_CAPACITY;
    return spgemm_numeric(h, dtype, A, B, C, stream);
}

spgemm_status spgemm_merge(spgemm_handle* h, spgemm_dtype dtype, int32_t nparts, const spgemm_csr_in* parts,
                           spgemm_csr_out* C, int64_t* c_nnz, spgemm_stream_t stream) {
    if (!h || !parts || !C || !C->row_ptr || nparts < 1 || nparts > kMaxGroupInst) return SPGEMM_ERR_INVALID_ARG;
    if (dtype != SPGEMM_F32 && dtype != SPGEMM_F64) return SPGEMM_ERR_DTYPE;
    const bool sizing = C->col_idx == nullptr;
    if (sizing && !c_nnz) return SPGEMM_ERR_INVALID_ARG;
    std::vector<InstDev> inst;
    std::vector<Validate> checks;
    for (int t = 0; t < nparts; ++t) {
        const spgemm_csr_in* P = parts + t;
        if (!csr_in_ok(P, !sizing)) return SPGEMM_ERR_INVALID_ARG;
        if (P->nrows != C->nrows || P->ncols != C->ncols) return SPGEMM_ERR_SHAPE;
        inst.push_back({nullptr, nullptr, nullptr, P->row_ptr, P->col_idx, P->val, P->nnz});
        checks.push_back({P->row_ptr, P->col_idx, P->nrows, P->ncols, P->nnz});
    }
    if (!sizing && !C->val) return SPGEMM_ERR_INVALID_ARG;
    std::vector<GroupDev> groups{{0, nparts, C->nrows, C->ncols, C->row_ptr, C->col_idx, C->val, 0}};
    return run(h, dtype, true, inst, groups, sizing, c_nnz, h->tune, checks, reinterpret_cast<cudaStream_t>(stream));
}

spgemm_status spgemm_batched(spgemm_handle* h, spgemm_dtype dtype, int32_t ninst, const spgemm_csr_in* A,
                             const spgemm_csr_in* B, int32_t ngroups, const int32_t* group_ptr, spgemm_csr_out* C,
                             int64_t* c_nnz, const spgemm_tune* tune, spgemm_stream_t stream) {
    if (!h || ninst < 1 || ninst > (1 << 20) || !A || !B || !C) return SPGEMM_ERR_INVALID_ARG;
    if (dtype != SPGEMM_F32 && dtype != SPGEMM_F64) return SPGEMM_ERR_DTYPE;
    if (group_ptr == nullptr) {
        if (ngroups != ninst) return SPGEMM_ERR_INVALID_ARG;
    } else {
        if (ngroups < 1 || group_ptr[0] != 0 || group_ptr[ngroups] != ninst) return SPGEMM_ERR_INVALID_ARG;
    }
    spgemm_tune tn = h->tune;
    if (tune) {
        TSG_TRY(check_tune(tune));
        tn = *tune;
    }
    const bool sizing = c_nnz != nullptr;
    std::vector<InstDev> inst;
    std::vector<GroupDev> groups;
    std::vector<Validate> checks;
    inst.reserve(ninst);
    groups.reserve(ngroups);
    for (int g = 0; g < ngroups; ++g) {
        const int t0 = group_ptr ? group_ptr[g] : g;
        const int t1 = group_ptr ? group_ptr[g + 1] : g + 1;
        if (t1 <= t0 || t1 - t0 > kMaxGroupInst) return SPGEMM_ERR_INVALID_ARG;
        const spgemm_csr_out& Cg = C[g];
        if (!Cg.row_ptr) return SPGEMM_ERR_INVALID_ARG;
        for (int t = t0; t < t1; ++t) {
            if (!csr_in_ok(A + t, !sizing) || !csr_in_ok(B + t, !sizing)) return SPGEMM_ERR_INVALID_ARG;
            if (A[t].ncols != B[t].nrows || A[t].nrows != Cg.nrows || B[t].ncols != Cg.ncols) return SPGEMM_ERR_SHAPE;
        }
        groups.push_back({t0, t1 - t0, Cg.nrows, Cg.ncols, Cg.row_ptr, sizing ? nullptr : Cg.col_idx,
                          sizing ? nullptr : Cg.val, 0});
    }
    for (int t = 0; t < ninst; ++t) {
        inst.push_back({A[t].row_ptr, A[t].col_idx, A[t].val, B[t].row_ptr, B[t].col_idx, B[t].val, B[t].nnz});
        if (tn.validate) {
            checks.push_back({A[t].row_ptr, A[t].col_idx, A[t].nrows, A[t].ncols, A[t].nnz});
            checks.push_back({B[t].row_ptr, B[t].col_idx, B[t].nrows, B[t].ncols, B[t].nnz});
        }
    }
    return run(h, dtype, false, inst, groups, sizing, c_nnz, tn, checks, reinterpret_cast<cudaStream_t>(stream));
}

spgemm_status spgemm_tile_split(spgemm_handle* h, spgemm_dtype dtype, const spgemm_csr_in* X, int32_t nrp,
                                const int32_t* row_bounds, int32_t ncp, const int32_t* col_bounds,
                                spgemm_csr_out* tiles, int64_t* tile_nnz, spgemm_stream_t stream) {
    if (!h || !X || !csr_in_ok(X, false) || !row_bounds || !col_bounds || !tiles) return SPGEMM_ERR_INVALID_ARG;
    if (nrp < 1 || ncp < 1 || ncp > 64) return SPGEMM_ERR_INVALID_ARG;
    if (dtype != SPGEMM_F32 && dtype != SPGEMM_F64) return SPGEMM_ERR_DTYPE;
    if (row_bounds[0] != 0 || row_bounds[nrp] != X->nrows || col_bounds[0] != 0 || col_bounds[ncp] != X->ncols)
        return SPGEMM_ERR_SHAPE;
    for (int i = 0; i < nrp; ++i)
        if (row_bounds[i + 1] < row_bounds[i]) return SPGEMM_ERR_INVALID_ARG;
    for (int i = 0; i < ncp; ++i)
        if (col_bounds[i + 1] < col_bounds[i]) return SPGEMM_ERR_INVALID_ARG;
    const bool sizing = tile_nnz != nullptr;
    const int nt = nrp * ncp;
    std::vector<GroupDev> groups(nt);  // indexed by tile (rp, cp)
    for (int rp = 0; rp < nrp; ++rp)
        for (int cp = 0; cp < ncp; ++cp) {
            const spgemm_csr_out& T = tiles[rp * ncp + cp];
            if (!T.row_ptr) return SPGEMM_ERR_INVALID_ARG;
            if (T.nrows != row_bounds[rp + 1] - row_bounds[rp] || T.ncols != col_bounds[cp + 1] - col_bounds[cp])
                return SPGEMM_ERR_SHAPE;
            groups[rp * ncp + cp] = {0, 1, T.nrows, T.ncols, T.row_ptr, T.col_idx, T.val, 0};
        }
    int dev = -1;
    TSG_CHECK(cudaGetDevice(&dev));
    if (dev != h->device) return SPGEMM_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    note_stream(h, st);
    h->plan_valid = false;
    const long long m = X->nrows;
    const long long U = m * ncp;
    if (U >= (1ll << 31) - 1) return SPGEMM_ERR_UNSUPPORTED;
    // scan order: units (cp, row); group order (cp, rp)
    std::vector<GroupDev> sgroups(nt);
    std::vector<long long> ubase(nt + 1);
    for (int cp = 0; cp < ncp; ++cp)
        for (int rp = 0; rp < nrp; ++rp) {
            sgroups[cp * nrp + rp] = groups[rp * ncp + cp];
            ubase[cp * nrp + rp] = cp * m + row_bounds[rp];
        }
    ubase[nt] = U;
    if (m == 0) {
        if (sizing) {
            for (int t = 0; t < nt; ++t) {
                TSG_CHECK(cudaMemsetAsync(groups[t].crp, 0, sizeof(int), st));
                tile_nnz[t] = 0;
            }
        }
        return SPGEMM_OK;
    }
    if (U > h->units_cap) {
        h->units_cap = h->units.n >= units_bytes(U) ? h->units_cap : -1;
        TSG_TRY(grow(h, h->units, units_bytes(U)));
        h->units_cap = U;
    }
    char* ub = static_cast<char*>(h->units.p);
    int* d_counts = reinterpret_cast<int*>(ub + align16(h->units_cap) + align16(4 * h->units_cap));
    long long* d_ex = reinterpret_cast<long long*>(ub + align16(h->units_cap) + 2 * align16(4 * h->units_cap));
    const long long nblk = scan_blocks(U);
    size_t o_bsum = 0;
    size_t o_nnz = o_bsum + align16(8 * nblk);
    size_t o_ubase = o_nnz + align16(8 * nt);
    size_t o_sg = o_ubase + align16(8 * (nt + 1));
    size_t o_tg = o_sg + align16(sizeof(GroupDev) * nt);
    size_t o_rb = o_tg + align16(sizeof(GroupDev) * nt);
    size_t o_cb = o_rb + align16(4 * (nrp + 1));
    size_t bytes = o_cb + align16(4 * (ncp + 1));
    TSG_TRY(grow(h, h->small, bytes));
    h->last_stage_dst = nullptr;
    char* sb = static_cast<char*>(h->small.p);
    std::vector<char> stage(bytes - o_ubase);
    std::memcpy(stage.data(), ubase.data(), 8 * (nt + 1));
    std::memcpy(stage.data() + (o_sg - o_ubase), sgroups.data(), sizeof(GroupDev) * nt);
    std::memcpy(stage.data() + (o_tg - o_ubase), groups.data(), sizeof(GroupDev) * nt);
    std::memcpy(stage.data() + (o_rb - o_ubase), row_bounds, 4 * (nrp + 1));
    std::memcpy(stage.data() + (o_cb - o_ubase), col_bounds, 4 * (ncp + 1));
    TSG_CHECK(cudaMemcpyAsync(sb + o_ubase, stage.data(), stage.size(), cudaMemcpyHostToDevice, st));
    const int* d_rb = reinterpret_cast<const int*>(sb + o_rb);
    const int* d_cb = reinterpret_cast<const int*>(sb + o_cb);
    PhaseScope ps(h, 5, st);
    if (sizing) {
        for (int t = 0; t < nt; ++t)
            if (groups[t].nrows == 0) TSG_CHECK(cudaMemsetAsync(groups[t].crp, 0, sizeof(int), st));
        long long* d_nnz = reinterpret_cast<long long*>(sb + o_nnz);
        TSG_CHECK(cudaMemsetAsync(d_nnz, 0, 8 * nt, st));
        TSG_CHECK(launch_split_count(X->row_ptr, X->col_idx, X->nrows, d_cb, ncp, d_counts, st));
        TSG_CHECK(launch_scan(d_counts, U, reinterpret_cast<long long*>(sb + o_bsum), d_ex, st));
        TSG_CHECK(launch_rowptr(reinterpret_cast<const GroupDev*>(sb + o_sg), reinterpret_cast<const long long*>(sb + o_ubase),
                                nt, U, d_ex, d_nnz, st));
        h->launches += 5;
        TSG_TRY(grow_pinned(h, 8 * nt));
        long long* p_nnz = static_cast<long long*>(h->pinned);
        TSG_CHECK(readback(h, p_nnz, d_nnz, 8 * nt, st));
        TSG_CHECK(cudaStreamSynchronize(st));
        for (int cp = 0; cp < ncp; ++cp)
            for (int rp = 0; rp < nrp; ++rp) tile_nnz[rp * ncp + cp] = p_nnz[cp * nrp + rp];
        return SPGEMM_OK;
    }
    TSG_CHECK(launch_split_fill(dtype, X->row_ptr, X->col_idx, X->val, X->nrows, d_rb, nrp, d_cb, ncp,
                                reinterpret_cast<const GroupDev*>(sb + o_tg), st));
    ++h->launches;
    return SPGEMM_OK;
}

spgemm_status spgemm_trident_bounds(int32_t n, int32_t q, int32_t lambda, int32_t* coarse, int32_t* fine) {
    if (n < 0 || q < 1 || lambda < 1) return SPGEMM_ERR_INVALID_ARG;
    if ((long long)q * lambda > (1 << 20)) return SPGEMM_ERR_INVALID_ARG;
    auto tile = [&](long long t) { return (int32_t)(t * (long long)n / q); };
    if (coarse)
        for (int t = 0; t <= q; ++t) coarse[t] = tile(t);
    if (fine) {
        for (int t = 0; t < q; ++t) {
            const long long lo = tile(t), hi = tile(t + 1);
            for (int sl = 0; sl < lambda; ++sl) fine[t * lambda + sl] = (int32_t)(lo + (long long)sl * (hi - lo) / lambda);
        }
        fine[q * lambda] = n;
    }
    return SPGEMM_OK;
}

spgemm_status spgemm_trident_schedule(int32_t q, int32_t lambda, int32_t* a_tile, int32_t* b_tile,
                                      int32_t* group_ptr) {
    if (q < 1 || lambda < 1 || !a_tile || !b_tile || !group_ptr) return SPGEMM_ERR_INVALID_ARG;
    if ((long long)q * q * lambda * q > (1 << 20)) return SPGEMM_ERR_INVALID_ARG;
    int t = 0, g = 0;
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j)
            for (int k = 0; k < lambda; ++k) {
                group_ptr[g++] = t;
                for (int r = 0; r < q; ++r) {
                    const int rr = (r + i + j) % q;
                    a_tile[t] = (i * lambda + k) * q + rr;
                    b_tile[t] = rr * q + j;
                    ++t;
                }
            }
    group_ptr[g] = t;
    return SPGEMM_OK;
}

namespace {

// Bytes of transpose work for nc columns and nnz entries: column counts,
// exclusive sums, scan partials, sort buffers.  The one formula both users
// of h->tr size it with.
size_t transpose_work_bytes(long long nc, long long nnz, size_t esz) {
    const long long nblk = scan_blocks(std::max<long long>(nc, 1));
    return align16(4 * std::max<long long>(nc, 1)) + align16(8 * (nc + 1)) + align16(8 * nblk) +
           align16(4 * std::max<long long>(nnz, 1)) + align16(esz * std::max<long long>(nnz, 1));
}

// X^T into the given arrays, work from h->tr starting at byte offset `off`
spgemm_status transpose_into(spgemm_handle* h, int dtype, const spgemm_csr_in* X, int* trp, int* tcol, void* tval,
                             size_t off, cudaStream_t st) {
    const long long nnz = X->nnz, nc = X->ncols;
    const size_t esz = dtype == SPGEMM_F64 ? 8 : 4;
    const long long nblk = scan_blocks(std::max<long long>(nc, 1));
    const size_t o_work = off;
    const size_t o_ex = o_work + align16(4 * std::max<long long>(nc, 1));
    const size_t o_bsum = o_ex + align16(8 * (nc + 1));
    const size_t o_tmp = o_bsum + align16(8 * nblk);
    const size_t bytes = off + transpose_work_bytes(nc, nnz, esz);
    TSG_TRY(grow(h, h->tr, bytes));
    char* b = static_cast<char*>(h->tr.p);
    PhaseScope ps(h, 6, st);
    TSG_CHECK(launch_transpose(dtype, X->row_ptr, X->col_idx, X->val, X->nrows, X->ncols, nnz, trp, tcol, tval,
                               reinterpret_cast<int*>(b + o_work), b + o_tmp, reinterpret_cast<long long*>(b + o_bsum),
                               reinterpret_cast<long long*>(b + o_ex), h->sms, st));
    h->launches += 7;
    return SPGEMM_OK;
}

}  // namespace

spgemm_status spgemm_csr_transpose(spgemm_handle* h, spgemm_dtype dtype, const spgemm_csr_in* X,
                                   spgemm_csr_out* XT, spgemm_stream_t stream) {
    if (!h || !csr_in_ok(X, false) || !XT || !XT->row_ptr || (X->nnz > 0 && !XT->col_idx))
        return SPGEMM_ERR_INVALID_ARG;
    if (dtype != SPGEMM_F32 && dtype != SPGEMM_F64) return SPGEMM_ERR_DTYPE;
    if (XT->nrows != X->ncols || XT->ncols != X->nrows) return SPGEMM_ERR_SHAPE;
    if (X->val && X->nnz > 0 && !XT->val) return SPGEMM_ERR_INVALID_ARG;
    int dev = -1;
    TSG_CHECK(cudaGetDevice(&dev));
    if (dev != h->device) return SPGEMM_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    note_stream(h, st);
    return transpose_into(h, dtype, X, XT->row_ptr, XT->col_idx, X->val ? XT->val : nullptr, 0, st);
}

spgemm_status spgemm_csr_permute(spgemm_handle* h, spgemm_dtype dtype, const spgemm_csr_in* X,
                                 const int32_t* row_perm, const int32_t* col_perm, spgemm_csr_out* Y,
                                 spgemm_stream_t stream) {
    if (!h || !csr_in_ok(X, false) || !Y || !Y->row_ptr || (X->nnz > 0 && !Y->col_idx))
        return SPGEMM_ERR_INVALID_ARG;
    if (dtype != SPGEMM_F32 && dtype != SPGEMM_F64) return SPGEMM_ERR_DTYPE;
    if (Y->nrows != X->nrows || Y->ncols != X->ncols) return SPGEMM_ERR_SHAPE;
    if (X->val && X->nnz > 0 && !Y->val) return SPGEMM_ERR_INVALID_ARG;
    int dev = -1;
    TSG_CHECK(cudaGetDevice(&dev));
    if (dev != h->device) return SPGEMM_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    note_stream(h, st);
    const long long nr = X->nrows, nc = X->ncols, nnz = X->nnz;
    // zeroed part first: hits of both maps and the long-row count
    const size_t o_hr = 0;
    const size_t o_hc = o_hr + align16(4 * std::max<long long>(nr, 1));
    const size_t o_cnt = o_hc + align16(4 * std::max<long long>(nc, 1));
    const size_t zero_bytes = o_cnt + 16;
    const size_t o_len = zero_bytes;
    const size_t o_bsum = o_len + align16(4 * std::max<long long>(nr, 1));
    const size_t o_ex = o_bsum + align16(8 * scan_blocks(std::max<long long>(nr, 1)));
    const size_t o_list = o_ex + align16(8 * (nr + 1));
    const size_t o_rank = o_list + align16(4 * std::max<long long>(nr, 1));
    const size_t bytes = o_rank + align16(4 * std::max<long long>(nnz, 1));
    TSG_TRY(grow(h, h->perm, bytes));
    TSG_TRY(grow(h, h->status, 16, st, true));
    char* b = static_cast<char*>(h->perm.p);
    unsigned* d_status = static_cast<unsigned*>(h->status.p);
    PhaseScope ps(h, 6, st);
    TSG_CHECK(cudaMemsetAsync(b, 0, zero_bytes, st));
    PermuteArgs p{};
    p.dtype = dtype == SPGEMM_F64 ? 1 : 0;
    p.nrows = (int)nr;
    p.ncols = (int)nc;
    p.nnz = nnz;
    p.rp = X->row_ptr;
    p.col = X->col_idx;
    p.val = X->val;
    p.row_perm = row_perm;
    p.col_perm = col_perm;
    p.yrp = Y->row_ptr;
    p.ycol = Y->col_idx;
    p.yval = X->val ? Y->val : nullptr;
    p.hits_r = reinterpret_cast<int*>(b + o_hr);
    p.hits_c = reinterpret_cast<int*>(b + o_hc);
    p.long_count = reinterpret_cast<int*>(b + o_cnt);
    p.ylen = reinterpret_cast<int*>(b + o_len);
    p.bsum = reinterpret_cast<long long*>(b + o_bsum);
    p.ex = reinterpret_cast<long long*>(b + o_ex);
    p.long_list = reinterpret_cast<int*>(b + o_list);
    p.rank = reinterpret_cast<int*>(b + o_rank);
    p.status = d_status;
    p.sms = h->sms;
    TSG_CHECK(launch_permute(p, st));
    h->launches += (row_perm ? 2 : 0) + (col_perm ? 2 : 0) + 1 + 4 + 2;
    TSG_TRY(grow_pinned(h, 16));
    TSG_CHECK(readback(h, h->pinned, d_status, 4, st));
    TSG_CHECK(cudaStreamSynchronize(st));
    const unsigned status = *static_cast<const unsigned*>(h->pinned);
    if (status & kStatusBadMap) {
        TSG_CHECK(cudaMemsetAsync(d_status, 0, 4, st));
        return SPGEMM_ERR_INVALID_ARG;
    }
    if (status & kStatusCapacity) {  // a row too long to re-sort
        TSG_CHECK(cudaMemsetAsync(d_status, 0, 4, st));
        return SPGEMM_ERR_UNSUPPORTED;
    }
    return SPGEMM_OK;
}

spgemm_status spgemm_backward(spgemm_handle* h, spgemm_dtype dtype, const spgemm_csr_in* A,
                              const spgemm_csr_in* B, const spgemm_csr_in* C, void* dA, void* dB,
                              int32_t deterministic, spgemm_stream_t stream) {
    if (!h || !csr_in_ok(A, true) || !csr_in_ok(B, true) || !csr_in_ok(C, true)) return SPGEMM_ERR_INVALID_ARG;
    if (dtype != SPGEMM_F32 && dtype != SPGEMM_F64) return SPGEMM_ERR_DTYPE;
    if (A->ncols != B->nrows || C->nrows != A->nrows || C->ncols != B->ncols) return SPGEMM_ERR_SHAPE;
    int dev = -1;
    TSG_CHECK(cudaGetDevice(&dev));
    if (dev != h->device) return SPGEMM_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    note_stream(h, st);
    TSG_TRY(grow(h, h->status, 16, st, true));
    BwdArgs a{};
    a.m = A->nrows;
    a.kdim = B->nrows;
    a.nnzb = B->nnz;
    a.arp = A->row_ptr;
    a.acol = A->col_idx;
    a.aval = A->val;
    a.brp = B->row_ptr;
    a.bcol = B->col_idx;
    a.bval = B->val;
    a.crp = C->row_ptr;
    a.ccol = C->col_idx;
    a.g = C->val;
    a.da = dA;
    a.db = dB;
    a.scatter_db = deterministic ? 0 : 1;
    a.status = static_cast<unsigned*>(h->status.p);
    if (dB && deterministic) {
        // A^T (kdim rows) at the front of h->tr, transpose work after it
        const size_t esz = dtype == SPGEMM_F64 ? 8 : 4;
        const long long nnz = std::max(A->nnz, 1);
        const size_t o_rp = 0;
        const size_t o_col = o_rp + align16(4 * ((long long)A->ncols + 1));
        const size_t o_val = o_col + align16(4 * nnz);
        const size_t o_work = o_val + align16(esz * nnz);
        TSG_TRY(grow(h, h->tr, o_work + 16));
        // the transpose may grow h->tr: compute pointers after it returns
        int* trp = nullptr;
        {
            // grow first to the full size the transpose needs (so that it does
            // not reallocate under the pointers below), then place A^T
            TSG_TRY(grow(h, h->tr, o_work + transpose_work_bytes(A->ncols, A->nnz, esz)));
            char* b = static_cast<char*>(h->tr.p);
            trp = reinterpret_cast<int*>(b + o_rp);
            a.trp = trp;
            a.tcol = reinterpret_cast<int*>(b + o_col);
            a.tval = b + o_val;
        }
        TSG_TRY(transpose_into(h, dtype, A, const_cast<int*>(a.trp), const_cast<int*>(a.tcol),
                               const_cast<void*>(a.tval), o_work, st));
    }
    PhaseScope ps(h, 6, st);
    TSG_CHECK(launch_backward(dtype, a, h->sms, st));
    h->launches += 2;
    return SPGEMM_OK;
}

namespace {

struct MclLayout {
    size_t ub, ub_off, bsum, kept, ex, ctr, tmp_col, tmp_val, bytes;
};

MclLayout mcl_layout(long long n, long long total) {
    MclLayout L;
    L.ub = 0;
    L.ub_off = L.ub + align16(4 * std::max(n, 1ll));
    L.bsum = L.ub_off + align16(8 * (n + 1));
    L.kept = L.bsum + align16(8 * scan_blocks(std::max(n, 1ll)));
    L.ex = L.kept + align16(4 * std::max(n, 1ll));
    L.ctr = L.ex + align16(8 * (n + 1));
    L.tmp_col = L.ctr + 16;
    L.tmp_val = L.tmp_col + align16(4 * std::max(total, 1ll));
    L.bytes = L.tmp_val + align16(4 * std::max(total, 1ll));
    return L;
}

}  // namespace

spgemm_status spgemm_mcl_expand(spgemm_handle* h, const spgemm_csr_in* Mt, const spgemm_mcl_params* prm,
                                int32_t* out_row_ptr, int64_t* out_nnz, spgemm_stream_t stream) {
    if (!h || !csr_in_ok(Mt, true) || !prm || !out_row_ptr || !out_nnz) return SPGEMM_ERR_INVALID_ARG;
    if (Mt->nrows != Mt->ncols) return SPGEMM_ERR_SHAPE;
    if (prm->topk < 1 || prm->topk > 1024 || !(prm->inflation > 0.0) || !(prm->prune >= 0.0) || prm->window < -1 ||
        prm->window > 1)
        return SPGEMM_ERR_INVALID_ARG;
    int dev = -1;
    TSG_CHECK(cudaGetDevice(&dev));
    if (dev != h->device) return SPGEMM_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    note_stream(h, st);
    h->mcl_n = -1;
    h->mcl_pilot_ratio = 0.0;
    for (long long& x : h->mcl_paths) x = 0;
    const long long n = Mt->nrows;
    if (n == 0) {
        TSG_CHECK(cudaMemsetAsync(out_row_ptr, 0, sizeof(int), st));
        *out_nnz = 0;
        h->mcl_n = 0;
        h->mcl_total = 0;
        return SPGEMM_OK;
    }
    if ((long long)prm->topk * n > (1ll << 31) - 1) return SPGEMM_ERR_INDEX_OVERFLOW;
    TSG_TRY(grow(h, h->status, 16, st, true));
    TSG_TRY(grow_pinned(h, 64));
    long long* p_ll = static_cast<long long*>(h->pinned);
    // 1. per-row bound min(products, topk) and its exclusive sums
    MclLayout L0 = mcl_layout(n, 1);
    TSG_TRY(grow(h, h->mcl, L0.bytes));
    char* b = static_cast<char*>(h->mcl.p);
    PhaseScope ps(h, 7, st);
    TSG_CHECK(launch_mcl_bounds(Mt->row_ptr, Mt->col_idx, (int)n, prm->topk, reinterpret_cast<int*>(b + L0.ub), st));
    TSG_CHECK(launch_scan(reinterpret_cast<int*>(b + L0.ub), n, reinterpret_cast<long long*>(b + L0.bsum),
                          reinterpret_cast<long long*>(b + L0.ub_off), st));
    TSG_CHECK(readback(h, p_ll, b + L0.ub_off + 8 * n, 8, st));
    TSG_CHECK(cudaStreamSynchronize(st));
    const long long total = p_ll[0];
    MclLayout L = mcl_layout(n, total);
    if (h->mcl.n < L.bytes) {
        // keep the bounds already computed while growing
        DevBuf nb;
        TSG_TRY(grow(h, nb, L.bytes));
        TSG_CHECK(cudaMemcpyAsync(nb.p, h->mcl.p, L0.tmp_col, cudaMemcpyDeviceToDevice, st));
        TSG_CHECK(cudaStreamSynchronize(st));
        cudaFree(h->mcl.p);
        h->mcl = nb;
    }
    b = static_cast<char*>(h->mcl.p);
    // 2. per-block accumulators: dense doubles, touched list, bitmap
    const long long stride = (n + 31) & ~31ll;
    const long long bm_words = stride / 32;
    const int slots = (int)std::min<long long>(n, (long long)h->sms * 4);
    // candidate list per block: the entries with v >= prune number at most
    // about 1 / prune (the v of a row sum to 1); twice that, and at least
    // 4096, bounds it with room (a row beyond it is reported, not written)
    long long ccap = stride;
    if (prm->prune > 0.0 && 2.0 / prm->prune < (double)stride)
        ccap = std::max<long long>(4096, (long long)std::ceil(2.0 / prm->prune));
    ccap = std::min(ccap, stride);
    const size_t o_bm = 12 * (size_t)stride * slots;
    // candidate lists for the per-block kernel's blocks and for up to six
    // blocks per SM of the window-summed kernel
    const int cslots = (int)std::max<long long>(slots, std::min<long long>(n, (long long)h->sms * 6));
    const size_t o_ck = align16(o_bm + 4 * (size_t)bm_words * slots);
    const size_t o_cc = o_ck + 8 * (size_t)ccap * cslots;
    const size_t acc_bytes = o_cc + 4 * (size_t)ccap * cslots;
    if (h->mcl_acc.n < acc_bytes) {
        TSG_TRY(grow(h, h->mcl_acc, acc_bytes));
        h->mcl_acc_key = -1;
    }
    // the kernel leaves the dense values and the bitmap zero after every row;
    // a different n moves the regions, so they are cleared then
    const long long key = stride * 4096 + slots;
    if (h->mcl_acc_key != key) {
        TSG_CHECK(cudaMemsetAsync(h->mcl_acc.p, 0, o_ck, st));
        h->mcl_acc_key = key;
    }
    char* acc = static_cast<char*>(h->mcl_acc.p);
    TSG_CHECK(cudaMemsetAsync(b + L.kept, 0, 4 * n, st));
    TSG_CHECK(cudaMemsetAsync(b + L.ctr, 0, 16, st));
    MclLaunch ml;
    ml.n = (int)n;
    ml.rp = Mt->row_ptr;
    ml.col = Mt->col_idx;
    ml.val = static_cast<const float*>(Mt->val);
    ml.ub_off = reinterpret_cast<const long long*>(b + L.ub_off);
    ml.tmp_col = reinterpret_cast<int*>(b + L.tmp_col);
    ml.tmp_val = reinterpret_cast<float*>(b + L.tmp_val);
    ml.kept = reinterpret_cast<int*>(b + L.kept);
    ml.dense = reinterpret_cast<double*>(acc);
    ml.touched = reinterpret_cast<int*>(acc + 8 * stride * slots);
    ml.bitmap = reinterpret_cast<unsigned*>(acc + o_bm);
    ml.ckey = reinterpret_cast<unsigned long long*>(acc + o_ck);
    ml.ccol = reinterpret_cast<int*>(acc + o_cc);
    ml.ccap = (int)ccap;
    ml.stride = stride;
    ml.bm_words = bm_words;
    ml.row_counter = reinterpret_cast<int*>(b + L.ctr);
    ml.inflation = prm->inflation;
    ml.prune = prm->prune;
    ml.topk = prm->topk;
    ml.status = static_cast<unsigned*>(h->status.p);
    // 2b. heavy rows (at least `thr` products; prm->heavy > 0 sets it,
    // < 0 turns the path off): batches of R rows whose dense accumulators
    // fit L2 together.  With prune 0 every touched column may be kept, which
    // a dense scan cannot tell from an untouched one: the path is off then.
    const long long thr = prm->heavy > 0 ? (long long)prm->heavy : std::max<long long>(4096, 2 * n);
    const long long acc_row = 8 * stride;
    const bool heavy_on = prm->heavy >= 0 && prm->prune > 0.0 && acc_row <= (64ll << 20);
    int H = 0;
    const int R = (int)std::max<long long>(1, std::min<long long>(kMclBatch, (48ll << 20) / acc_row));
    // flags | heavy list | bucket list | hcount, notpos, bcount, bucket row counter | batch buffers
    const size_t o_hl = align16((size_t)n), o_bl = o_hl + align16(4 * (size_t)n);
    const size_t o_hc = o_bl + align16(4 * (size_t)n);
    const size_t o_sc = (size_t)R * acc_row;  // within a buffer: D | scalars | ck | cc | mlist
    const size_t o_bck = o_sc + align16((size_t)R * (8 + 8 + 4 + 4 + 4));
    const size_t o_bcc = o_bck + 8 * (size_t)R * ccap;
    const size_t buf_bytes = align16(o_bcc + 4 * (size_t)R * ccap + 4 * (size_t)R * kMclMaxList);
    const size_t o_buf = o_hc + 32;  // the 16 bytes after the counters: the pilot's totals
    const size_t heavy_bytes = heavy_on ? o_buf + 2 * buf_bytes : o_buf;
    if (h->mcl_heavy.n < heavy_bytes) {
        TSG_TRY(grow(h, h->mcl_heavy, heavy_bytes));
        h->mcl_heavy_key = -1;
    }
    char* hv = static_cast<char*>(h->mcl_heavy.p);
    int* ctr4 = reinterpret_cast<int*>(hv + o_hc);
    TSG_CHECK(cudaMemsetAsync(ctr4, 0, 16, st));
    // every value in [2^-63, FLT_MAX]: products and sums stay positive, so
    // a column's first add finds 0 (no bitmap), and the bucketed path applies
    TSG_CHECK(launch_mcl_check_positive(static_cast<const float*>(Mt->val), Mt->nnz, ctr4 + 1, h->sms, st));
    ++h->launches;
    // 2c. bucketed mid rows (4096 <= products < the staging capacity 2^21,
    // below the heavy threshold; 12 bytes of staging per product and block):
    // windows of 2^lw columns, at most 64 per row up to n = 2^18 and 4096
    // columns wide beyond
    int lw = 5;
    while (lw < 12 && (n >> lw) > 64) ++lw;
    const int nbk = (int)((n + (1ll << lw) - 1) >> lw);
    const int bps = nbk <= 2048 ? mcl_bucket_blocks_per_sm(lw, nbk) : 0;
    const int bblocks = (int)std::min<long long>(cslots, (long long)h->sms * std::min(bps, 6));
    const long long bcap = heavy_on ? std::min<long long>(1ll << 21, thr) : (1ll << 21);
    const long long blo = bblocks > 0 && prm->window >= 0 ? 4096 : (1ll << 62);
    if (heavy_on) {
        const long long hkey = (long long)stride * 4096 * 32 + (long long)R * 4096 + (ccap & 4095);
        if (h->mcl_heavy_key != hkey) {
            for (int q = 0; q < 2; ++q) TSG_CHECK(cudaMemsetAsync(hv + o_buf + q * buf_bytes, 0, o_bck, st));
            h->mcl_heavy_key = hkey;
        }
    }
    TSG_CHECK(launch_mcl_mark(Mt->row_ptr, Mt->col_idx, (int)n, heavy_on ? thr : (1ll << 62), blo, bcap, ctr4 + 1,
                              reinterpret_cast<unsigned char*>(hv), reinterpret_cast<int*>(hv + o_hl), ctr4,
                              reinterpret_cast<int*>(hv + o_bl), ctr4 + 2, st));
    ++h->launches;
    TSG_CHECK(readback(h, p_ll + 2, ctr4, 12, st));
    TSG_CHECK(cudaStreamSynchronize(st));
    const int* got = reinterpret_cast<const int*>(p_ll + 2);
    H = got[0];
    int NBR = got[2];
    ml.positive = got[1] == 0 ? 1 : 0;
    ml.heavy = H + NBR > 0 ? reinterpret_cast<const unsigned char*>(hv) : nullptr;
    ml.skip = 3;
    if (NBR > 0 && prm->window == 0) {
        // pilot: products per distinct column over up to 32 evenly spaced
        // rows of the window-summed range; above 4 (a clustered iterate,
        // whose many adds to few columns serialise in shared memory while
        // its small accumulator footprint stays in L2 for the per-block
        // kernel) those rows go back to the per-block kernel
        const int ns = std::min(32, NBR);
        unsigned long long* tot = reinterpret_cast<unsigned long long*>(hv + o_hc + 16);
        TSG_CHECK(cudaMemsetAsync(tot, 0, 16, st));
        TSG_CHECK(launch_mcl_pilot(ml, reinterpret_cast<const int*>(hv + o_bl), ns, NBR / ns, tot, st));
        ++h->launches;
        TSG_CHECK(readback(h, p_ll + 4, tot, 16, st));
        TSG_CHECK(cudaStreamSynchronize(st));
        const unsigned long long pp = reinterpret_cast<const unsigned long long*>(p_ll + 4)[0];
        const unsigned long long pd = reinterpret_cast<const unsigned long long*>(p_ll + 4)[1];
        h->mcl_pilot_ratio = pd ? (double)pp / (double)pd : 0.0;
        if (pd == 0 || pp > 4 * pd) {
            ml.skip = 1;
            NBR = 0;
        }
    }
    h->mcl_paths[2] = H;
    h->mcl_paths[1] = NBR;
    h->mcl_paths[0] = n - H - NBR;
    TSG_CHECK(launch_mcl_rows(ml, slots, st));
    if (NBR > 0) {
        const size_t sbytes = (size_t)bblocks * bcap * 8, ebytes = (size_t)bblocks * bcap * 4;
        TSG_TRY(grow(h, h->mcl_bucket, sbytes + ebytes));
        MclBucketLaunch bl;
        bl.list = reinterpret_cast<const int*>(hv + o_bl);
        bl.count = NBR;
        bl.counter = ctr4 + 3;
        bl.stage = reinterpret_cast<int2*>(h->mcl_bucket.p);
        bl.ej = reinterpret_cast<int*>(static_cast<char*>(h->mcl_bucket.p) + sbytes);
        bl.cap = bcap;
        bl.lw = lw;
        bl.nbk = nbk;
        TSG_CHECK(launch_mcl_bucket(ml, bl, bblocks, st));
        ++h->launches;
    }
    if (H > 0) {
        if (!h->mcl_side) TSG_CHECK(cudaStreamCreateWithFlags(&h->mcl_side, cudaStreamNonBlocking));
        for (cudaEvent_t& e : h->mcl_ev)
            if (!e) TSG_CHECK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        const int* hlist = reinterpret_cast<const int*>(hv + o_hl);
        for (int i = 0, bi = 0; i < H; i += R, ++bi) {
            const int q = bi & 1;
            char* bb = hv + o_buf + q * buf_bytes;
            MclHeavyLaunch hb;
            hb.rows = hlist + i;
            hb.nb = std::min(R, H - i);
            hb.D = reinterpret_cast<double*>(bb);
            hb.s = reinterpret_cast<double*>(bb + o_sc);
            hb.wmax = reinterpret_cast<unsigned long long*>(bb + o_sc + 8 * R);
            hb.flags = reinterpret_cast<unsigned*>(bb + o_sc + 16 * R);
            hb.ncand = reinterpret_cast<int*>(bb + o_sc + 20 * R);
            hb.nmax = reinterpret_cast<int*>(bb + o_sc + 24 * R);
            hb.ck = reinterpret_cast<unsigned long long*>(bb + o_bck);
            hb.cc = reinterpret_cast<int*>(bb + o_bcc);
            hb.mlist = reinterpret_cast<int*>(bb + o_bcc + 4 * (size_t)R * ccap);
            // the buffer's previous batch must be selected and cleared
            if (bi >= 2) TSG_CHECK(cudaStreamWaitEvent(st, h->mcl_ev[2 + q], 0));
            // expansion on the caller's stream; the dense scans, the
            // selection and the clear on the second one, overlapping the
            // next batch's expansion into the other buffer
            TSG_CHECK(launch_mcl_heavy_batch(ml, hb, h->sms, st));
            TSG_CHECK(cudaEventRecord(h->mcl_ev[q], st));
            TSG_CHECK(cudaStreamWaitEvent(h->mcl_side, h->mcl_ev[q], 0));
            TSG_CHECK(launch_mcl_heavy_scans(ml, hb, h->sms, h->mcl_side));
            TSG_CHECK(launch_mcl_heavy_select(ml, hb, h->mcl_side));
            TSG_CHECK(cudaMemsetAsync(bb, 0, o_bck, h->mcl_side));
            TSG_CHECK(cudaEventRecord(h->mcl_ev[2 + q], h->mcl_side));
            h->launches += 4;
        }
        TSG_CHECK(cudaEventRecord(h->mcl_ev[4], h->mcl_side));
        TSG_CHECK(cudaStreamWaitEvent(st, h->mcl_ev[4], 0));
    }
    // 3. row pointers of the next iterate
    TSG_CHECK(launch_scan(reinterpret_cast<int*>(b + L.kept), n, reinterpret_cast<long long*>(b + L.bsum),
                          reinterpret_cast<long long*>(b + L.ex), st));
    TSG_CHECK(launch_ll_to_int(reinterpret_cast<long long*>(b + L.ex), n + 1, out_row_ptr, st));
    h->launches += 9;
    unsigned* p_status = reinterpret_cast<unsigned*>(p_ll + 1);
    TSG_CHECK(readback(h, p_ll, b + L.ex + 8 * n, 8, st));
    TSG_CHECK(readback(h, p_status, h->status.p, 4, st));
    TSG_CHECK(cudaStreamSynchronize(st));
    if (*p_status) {
        TSG_CHECK(cudaMemsetAsync(h->status.p, 0, 4, st));
        return SPGEMM_ERR_INTERNAL;
    }
    *out_nnz = p_ll[0];
    h->mcl_n = (int)n;
    h->mcl_total = total;
    return SPGEMM_OK;
}

spgemm_status spgemm_mcl_paths(const spgemm_handle* h, int64_t* rows, double* pilot_ratio) {
    if (!h || !rows || !pilot_ratio) return SPGEMM_ERR_INVALID_ARG;
    for (int i = 0; i < 3; ++i) rows[i] = h->mcl_paths[i];
    *pilot_ratio = h->mcl_pilot_ratio;
    return SPGEMM_OK;
}

spgemm_status spgemm_mcl_collect(spgemm_handle* h, spgemm_csr_out* out, spgemm_stream_t stream) {
    if (!h || !out || !out->row_ptr) return SPGEMM_ERR_INVALID_ARG;
    if (h->mcl_n < 0 || out->nrows != h->mcl_n || out->ncols != h->mcl_n) return SPGEMM_ERR_INVALID_ARG;
    if (h->mcl_n == 0) return SPGEMM_OK;
    if (!out->col_idx || !out->val) return SPGEMM_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    note_stream(h, st);
    const MclLayout L = mcl_layout(h->mcl_n, h->mcl_total);
    char* b = static_cast<char*>(h->mcl.p);
    PhaseScope ps(h, 7, st);
    TSG_CHECK(launch_mcl_collect(h->mcl_n, reinterpret_cast<const long long*>(b + L.ub_off),
                                 reinterpret_cast<const int*>(b + L.tmp_col), reinterpret_cast<const float*>(b + L.tmp_val),
                                 out->row_ptr, out->col_idx, static_cast<float*>(out->val), h->sms, st));
    ++h->launches;
    return SPGEMM_OK;
}

spgemm_status spgemm_launch_count(const spgemm_handle* h, int64_t* count) {
    if (!h || !count) return SPGEMM_ERR_INVALID_ARG;
    *count = h->launches;
    return SPGEMM_OK;
}

spgemm_status spgemm_device_status(spgemm_handle* h) {
    if (!h) return SPGEMM_ERR_INVALID_ARG;
    if (!h->status.p) return SPGEMM_OK;
    TSG_TRY(grow_pinned(h, 16));
    TSG_CHECK(readback(h, h->pinned, h->status.p, 4, h->last_stream));
    TSG_CHECK(cudaStreamSynchronize(h->last_stream));
    const unsigned st = *static_cast<const unsigned*>(h->pinned);
    TSG_CHECK(cudaMemset(h->status.p, 0, 4));
    if (st & kStatusNotCanonical) return SPGEMM_ERR_NOT_CANONICAL;
    if (st & kStatusHashOverflow) return SPGEMM_ERR_HASH_OVERFLOW;
    if (st & kStatusInternal) return SPGEMM_ERR_INTERNAL;
    if (st & kStatusTimeout) return SPGEMM_ERR_DEVICE_TIMEOUT;
    return SPGEMM_OK;
}

spgemm_status spgemm_set_workspace_limit(spgemm_handle* h, int64_t bytes) {
    if (!h) return SPGEMM_ERR_INVALID_ARG;
    h->ws_limit = bytes < 0 ? -1 : bytes;
    return SPGEMM_OK;
}

spgemm_status spgemm_workspace_bytes(const spgemm_handle* h, int64_t* bytes) {
    if (!h || !bytes) return SPGEMM_ERR_INVALID_ARG;
    *bytes = (int64_t)held_bytes(h);
    return SPGEMM_OK;
}

spgemm_status spgemm_set_wait_test(spgemm_handle* h, int32_t spin_limit, int32_t hold_tile) {
    if (!h || hold_tile < -1) return SPGEMM_ERR_INVALID_ARG;
    h->wait_limit = spin_limit > 0 ? spin_limit : kLookbackSpinLimit;
    h->hold_tile = hold_tile;
    return SPGEMM_OK;
}

spgemm_status spgemm_set_timing(spgemm_handle* h, int32_t enable) {
    if (!h) return SPGEMM_ERR_INVALID_ARG;
    h->timing = enable != 0;
    return SPGEMM_OK;
}

spgemm_status spgemm_read_timing(spgemm_handle* h, double* ms, int64_t* count) {
    if (!h || !ms || !count) return SPGEMM_ERR_INVALID_ARG;
    for (int p = 0; p < kNumPhases; ++p) {
        ms[p] = 0.0;
        count[p] = 0;
    }
    spgemm_status rc = SPGEMM_OK;
    for (const PhaseEvent& e : h->pending) {
        if (cudaEventSynchronize(e.b) == cudaSuccess) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, e.a, e.b) == cudaSuccess) {
                ms[e.phase] += t;
                count[e.phase] += 1;
            }
        } else {
            cudaGetLastError();
            rc = SPGEMM_ERR_CUDA;
        }
        h->spare.push_back(e.a);
        h->spare.push_back(e.b);
    }
    h->pending.clear();
    return rc;
}

}  // extern "C"

// ===================================================================== plans

#include <fcntl.h>
#include <unistd.h>

#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <iterator>
#include <map>
#include <mutex>
#include <string>

struct spgemm_plan {
    spgemm_handle* h = nullptr;  // private workspace
    int dtype = 1;
    std::vector<InstDev> inst;
    std::vector<GroupDev> groups;
    spgemm_tune tune{};
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> exec_key;
    int64_t graph_kernels = 0;  // kernels in the captured graph
    cudaStream_t capture = nullptr;  // private stream the graph is captured on
};

namespace {

std::mutex g_tune_mu;
std::map<uint64_t, spgemm_tune> g_tune_cache;

// ---- persistent autotune cache
//
// A text file, one chosen layout per line:
//   tsg-tune-1 <key, 16 hex digits> <num_bins> <warps_per_block>
//              <sym_warps_per_block> <bin_upper[b] bin_kernel[b]> x num_bins
// The key hashes the GPU model (compute capability, SM count), the dtype and
// the shape of the product-count histogram, so an entry applies on any GPU of
// the same model.  Entries are appended (one write per line); on reading,
// lines that do not parse or whose layout fails check_tune are skipped and a
// later line replaces an earlier one with the same key.
constexpr const char* kTuneTag = "tsg-tune-1";
constexpr const char* kTuneEnv = "TRIDENT_SPGEMM_TUNE_CACHE";
std::string g_tune_path;      // file chosen layouts are appended to ("" = none)
bool g_tune_env_done = false;  // the environment variable has been looked at

bool parse_tune_line(const char* line, uint64_t* key, spgemm_tune* t) {
    char tag[16] = {0};
    unsigned long long k = 0;
    int nb = 0, wpb = 0, swpb = 0, used = 0;
    if (std::sscanf(line, "%15s %16llx %d %d %d%n", tag, &k, &nb, &wpb, &swpb, &used) != 5) return false;
    if (std::strcmp(tag, kTuneTag) != 0 || nb < 1 || nb > SPGEMM_MAX_BINS) return false;
    spgemm_tune x;
    default_tune(&x);
    x.num_bins = nb;
    x.warps_per_block = wpb;
    x.sym_warps_per_block = swpb;
    x.validate = 0;
    const char* q = line + used;
    for (int b = 0; b < nb; ++b) {
        int n = 0;
        if (std::sscanf(q, "%d %d%n", &x.bin_upper[b], &x.bin_kernel[b], &n) != 2) return false;
        q += n;
    }
    while (*q == ' ' || *q == '\t' || *q == '\r' || *q == '\n') ++q;
    if (*q != '\0' || check_tune(&x) != SPGEMM_OK) return false;
    *key = (uint64_t)k;
    *t = x;
    return true;
}

std::string format_tune_line(uint64_t key, const spgemm_tune& t) {
    char buf[64];
    std::snprintf(buf, sizeof(buf), "%s %016llx %d %d %d", kTuneTag, (unsigned long long)key, t.num_bins,
                  t.warps_per_block, t.sym_warps_per_block);
    std::string line = buf;
    for (int b = 0; b < t.num_bins; ++b) {
        std::snprintf(buf, sizeof(buf), " %d %d", t.bin_upper[b], t.bin_kernel[b]);
        line += buf;
    }
    return line + "\n";
}

// Adds the file's entries to the cache (caller holds g_tune_mu); returns the
// number taken, or -1 if the file exists but cannot be read.
long long load_tune_file_locked(const std::string& path) {
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return errno == ENOENT ? 0 : -1;
    long long n = 0;
    char line[512];
    while (std::fgets(line, sizeof(line), f)) {
        const size_t len = std::strlen(line);
        if (len + 1 == sizeof(line) && line[len - 1] != '\n') {
            // longer than any valid entry: skip the rest of it
            int c;
            while ((c = std::fgetc(f)) != EOF && c != '\n') {
            }
            continue;
        }
        uint64_t key;
        spgemm_tune t;
        if (parse_tune_line(line, &key, &t)) {
            g_tune_cache[key] = t;
            ++n;
        }
    }
    const bool bad = std::ferror(f) != 0;  // e.g. the path names a directory
    std::fclose(f);
    return bad ? -1 : n;
}

void tune_env_locked() {
    if (g_tune_env_done) return;
    g_tune_env_done = true;
    const char* env = std::getenv(kTuneEnv);
    if (env && *env) {
        g_tune_path = env;
        load_tune_file_locked(g_tune_path);
    }
}

// Records a chosen layout in the cache and appends it to the file, if any
// (caller holds g_tune_mu).  SPGEMM_ERR_INVALID_ARG if the file cannot be
// written.
spgemm_status store_tune_locked(uint64_t key, const spgemm_tune& t) {
    g_tune_cache[key] = t;
    if (g_tune_path.empty()) return SPGEMM_OK;
    const std::string line = format_tune_line(key, t);
    const int fd = ::open(g_tune_path.c_str(), O_WRONLY | O_CREAT | O_APPEND, 0644);
    if (fd < 0) return SPGEMM_ERR_INVALID_ARG;
    const ssize_t w = ::write(fd, line.data(), line.size());
    ::close(fd);
    return w == (ssize_t)line.size() ? SPGEMM_OK : SPGEMM_ERR_INVALID_ARG;
}

spgemm_status plan_bind(spgemm_plan* p, const spgemm_csr_out* C, std::vector<const void*>* key) {
    key->clear();
    for (size_t g = 0; g < p->groups.size(); ++g) {
        const spgemm_csr_out& Cg = C[g];
        if (Cg.row_ptr != p->groups[g].crp || Cg.nrows != p->groups[g].nrows || Cg.ncols != p->groups[g].ncols)
            return SPGEMM_ERR_SHAPE;
        p->groups[g].ccol = Cg.col_idx;
        p->groups[g].cval = Cg.val;
        key->push_back(Cg.col_idx);
        key->push_back(Cg.val);
    }
    return SPGEMM_OK;
}

spgemm_status plan_size(spgemm_plan* p, int64_t* c_nnz, cudaStream_t st) {
    std::vector<GroupDev> g = p->groups;
    for (GroupDev& G : g) {
        G.ccol = nullptr;
        G.cval = nullptr;
    }
    std::vector<int64_t> tmp(g.size());
    return run(p->h, p->dtype, false, p->inst, g, true, c_nnz ? c_nnz : tmp.data(), p->tune, {}, st);
}

void plan_drop_graph(spgemm_plan* p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
    p->exec_key.clear();
}

}  // namespace

extern "C" {

spgemm_status spgemm_plan_create(spgemm_dtype dtype, int32_t ninst, const spgemm_csr_in* A, const spgemm_csr_in* B,
                                 int32_t ngroups, const int32_t* group_ptr, int32_t* const* c_row_ptr,
                                 int64_t* c_nnz, const spgemm_tune* tune, spgemm_stream_t stream,
                                 spgemm_plan** out) {
    if (!out || ninst < 1 || ninst > (1 << 20) || !A || !B || !c_row_ptr || !c_nnz) return SPGEMM_ERR_INVALID_ARG;
    *out = nullptr;
    if (dtype != SPGEMM_F32 && dtype != SPGEMM_F64) return SPGEMM_ERR_DTYPE;
    if (group_ptr == nullptr) {
        if (ngroups != ninst) return SPGEMM_ERR_INVALID_ARG;
    } else if (ngroups < 1 || group_ptr[0] != 0 || group_ptr[ngroups] != ninst) {
        return SPGEMM_ERR_INVALID_ARG;
    }
    spgemm_tune tn;
    default_tune(&tn);
    if (tune) {
        TSG_TRY(check_tune(tune));
        tn = *tune;
    }
    tn.validate = 0;
    spgemm_plan* p = new (std::nothrow) spgemm_plan();
    if (!p) return SPGEMM_ERR_OOM;
    p->dtype = dtype;
    p->tune = tn;
    for (int g = 0; g < ngroups; ++g) {
        const int t0 = group_ptr ? group_ptr[g] : g;
        const int t1 = group_ptr ? group_ptr[g + 1] : g + 1;
        if (t1 <= t0 || t1 - t0 > kMaxGroupInst || !c_row_ptr[g]) {
            delete p;
            return SPGEMM_ERR_INVALID_ARG;
        }
        for (int t = t0; t < t1; ++t) {
            if (!csr_in_ok(A + t, true) || !csr_in_ok(B + t, true)) {
                delete p;
                return SPGEMM_ERR_INVALID_ARG;
            }
            if (A[t].ncols != B[t].nrows || A[t].nrows != A[t0].nrows || B[t].ncols != B[t0].ncols) {
                delete p;
                return SPGEMM_ERR_SHAPE;
            }
        }
        p->groups.push_back({t0, t1 - t0, A[t0].nrows, B[t0].ncols, c_row_ptr[g], nullptr, nullptr, 0});
    }
    for (int t = 0; t < ninst; ++t)
        p->inst.push_back({A[t].row_ptr, A[t].col_idx, A[t].val, B[t].row_ptr, B[t].col_idx, B[t].val, B[t].nnz});
    spgemm_status rc = spgemm_create(&p->h);
    if (rc == SPGEMM_OK) rc = plan_size(p, c_nnz, reinterpret_cast<cudaStream_t>(stream));
    if (rc != SPGEMM_OK) {
        spgemm_destroy(p->h);
        delete p;
        return rc;
    }
    *out = p;
    return SPGEMM_OK;
}

spgemm_status spgemm_plan_execute(spgemm_plan* p, const spgemm_csr_out* C, int32_t use_graph,
                                  spgemm_stream_t stream) {
    if (!p || !C) return SPGEMM_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::vector<const void*> key;
    TSG_TRY(plan_bind(p, C, &key));
    if (use_graph && p->exec && key == p->exec_key) {
        TSG_CHECK(cudaGraphLaunch(p->exec, st));
        p->h->launches += p->graph_kernels;
        return SPGEMM_OK;
    }
    TSG_TRY(run(p->h, p->dtype, false, p->inst, p->groups, false, nullptr, p->tune, {}, st));
    if (!use_graph || !p->h->plan_valid) return SPGEMM_OK;
    // capture the same fill: descriptors and bin lists are already in place,
    // so the captured work is kernel launches only
    plan_drop_graph(p);
    const bool timing = p->h->timing;
    p->h->timing = false;
    // (the caller's stream may be the legacy default stream, which cannot be
    // captured: capture on the plan's own stream, replay on the caller's)
    if (!p->capture) TSG_CHECK(cudaStreamCreateWithFlags(&p->capture, cudaStreamNonBlocking));
    TSG_CHECK(cudaStreamBeginCapture(p->capture, cudaStreamCaptureModeThreadLocal));
    const int64_t before = p->h->launches;
    spgemm_status rc = run(p->h, p->dtype, false, p->inst, p->groups, false, nullptr, p->tune, {}, p->capture);
    p->graph_kernels = p->h->launches - before;
    p->h->launches = before;  // captured, not launched
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->capture, &graph);
    p->h->timing = timing;
    if (rc != SPGEMM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    TSG_CHECK(e);
    e = cudaGraphInstantiate(&p->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        p->exec = nullptr;
        return cuda_status(e);
    }
    p->exec_key = key;
    return SPGEMM_OK;
}

spgemm_status spgemm_plan_autotune(spgemm_plan* p, const spgemm_csr_out* C, spgemm_stream_t stream,
                                   spgemm_tune* chosen) {
    if (!p || !C) return SPGEMM_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::vector<const void*> key;
    TSG_TRY(plan_bind(p, C, &key));
    plan_drop_graph(p);
    // cache key: GPU model, dtype, the problem's product-count histogram
    TSG_TRY(plan_size(p, nullptr, st));
    int dev = 0, cc[3] = {0, 0, p->h->sms};
    TSG_CHECK(cudaGetDevice(&dev));
    TSG_CHECK(cudaDeviceGetAttribute(&cc[0], cudaDevAttrComputeCapabilityMajor, dev));
    TSG_CHECK(cudaDeviceGetAttribute(&cc[1], cudaDevAttrComputeCapabilityMinor, dev));
    uint64_t sig = 1469598103934665603ull;
    sig = fnv(sig, cc, sizeof(cc));
    sig = fnv(sig, &p->dtype, sizeof(p->dtype));
    for (int v : p->h->plan_hist) {
        // histogram shape on a log scale: tunes transfer between similar problems
        int lg = 0;
        while ((1 << lg) < v) ++lg;
        sig = fnv(sig, &lg, sizeof(lg));
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_env_locked();
        auto it = g_tune_cache.find(sig);
        if (it != g_tune_cache.end()) {
            p->tune = it->second;
            if (chosen) *chosen = p->tune;
            return plan_size(p, nullptr, st);
        }
    }
    // Search, per bin of the default layout (a range of row product counts),
    // the kernel variant -- capacity and accumulator kind -- that runs that
    // bin's rows fastest, timing the bin's kernel alone; then the warps per
    // block of the warp variants on whole runs.  Adjacent bins that chose the
    // same variant are merged (their threshold disappears).  Every candidate
    // adds each output entry in the same order: the bits never change.
    spgemm_tune base;
    default_tune(&base);
    base.validate = 0;
    cudaEvent_t e0, e1;
    TSG_CHECK(cudaEventCreate(&e0));
    TSG_CHECK(cudaEventCreate(&e1));
    spgemm_status rc = SPGEMM_OK;
    // time of one fill with tune t: whole (bin < 0) or one bin's kernel
    auto time_fill = [&](const spgemm_tune& t, int bin, float* out_ms) -> spgemm_status {
        p->tune = t;
        TSG_TRY(plan_size(p, nullptr, st));
        TSG_TRY(run(p->h, p->dtype, false, p->inst, p->groups, false, nullptr, p->tune, {}, st));  // warm
        float tb = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            p->h->only_bin = bin;
            cudaEventRecord(e0, st);
            spgemm_status r = run(p->h, p->dtype, false, p->inst, p->groups, false, nullptr, p->tune, {}, st);
            cudaEventRecord(e1, st);
            p->h->only_bin = -1;
            TSG_TRY(r);
            TSG_CHECK(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            tb = std::min(tb, ms);
        }
        *out_ms = tb;
        return SPGEMM_OK;
    };
    // candidate variants of a bin: the default, and every other variant of
    // a capacity between the bin's bound and twice it (other accumulator
    // kinds and the next sizes up)
    auto candidates = [&](int b) {
        std::vector<int> c{base.bin_kernel[b]};
        for (int v = 0; v < kNumVariants; ++v) {
            if (v == base.bin_kernel[b]) continue;
            const int cap = variant_cap(v);
            if (cap >= base.bin_upper[b] && cap <= 2 * base.bin_upper[b] && cap >= 32) c.push_back(v);
        }
        return c;
    };
    spgemm_tune chosen_t = base;
    {
        p->tune = base;
        rc = plan_size(p, nullptr, st);
        const std::vector<int> hist0 = p->h->plan_hist;
        for (int b = 0; b < base.num_bins && rc == SPGEMM_OK; ++b) {
            if (b >= (int)hist0.size() || hist0[b] == 0) continue;
            float best_b = 1e30f;
            for (int v : candidates(b)) {
                spgemm_tune t = chosen_t;
                t.bin_kernel[b] = v;
                float ms = 0.f;
                rc = time_fill(t, b, &ms);
                if (rc != SPGEMM_OK) break;
                if (ms < best_b * 0.98f || (v == base.bin_kernel[b] && ms < best_b)) {
                    best_b = ms;
                    chosen_t.bin_kernel[b] = v;
                }
            }
        }
    }
    // merge neighbours that chose the same variant
    if (rc == SPGEMM_OK) {
        spgemm_tune m = chosen_t;
        int nbm = 0;
        for (int b = 0; b < chosen_t.num_bins; ++b) {
            if (nbm > 0 && m.bin_kernel[nbm - 1] == chosen_t.bin_kernel[b]) {
                m.bin_upper[nbm - 1] = chosen_t.bin_upper[b];
            } else {
                m.bin_upper[nbm] = chosen_t.bin_upper[b];
                m.bin_kernel[nbm] = chosen_t.bin_kernel[b];
                ++nbm;
            }
        }
        m.num_bins = nbm;
        chosen_t = m;
    }
    float best = 1e30f;
    spgemm_tune best_t = chosen_t;
    for (int wpb : {16, 8, 32}) {
        if (rc != SPGEMM_OK) break;
        spgemm_tune t = chosen_t;
        t.warps_per_block = wpb;
        float ms = 0.f;
        rc = time_fill(t, -1, &ms);
        if (rc == SPGEMM_OK && ms < best) {
            best = ms;
            best_t = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SPGEMM_OK) return rc;
    p->tune = best_t;
    spgemm_status stored;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        stored = store_tune_locked(sig, best_t);
    }
    if (chosen) *chosen = best_t;
    TSG_TRY(plan_size(p, nullptr, st));
    return stored;
}

spgemm_status spgemm_tune_cache_open(const char* path, int64_t* loaded) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_env_done = true;
    const char* src = path ? path : std::getenv(kTuneEnv);
    g_tune_path = src ? src : "";
    long long n = g_tune_path.empty() ? 0 : load_tune_file_locked(g_tune_path);
    if (loaded) *loaded = n < 0 ? 0 : n;
    return n < 0 ? SPGEMM_ERR_INVALID_ARG : SPGEMM_OK;
}

spgemm_status spgemm_tune_cache_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache.clear();
    g_tune_path.clear();
    g_tune_env_done = true;
    return SPGEMM_OK;
}

spgemm_status spgemm_tune_cache_store(uint64_t key, const spgemm_tune* t) {
    if (!t) return SPGEMM_ERR_INVALID_ARG;
    TSG_TRY(check_tune(t));
    spgemm_tune x = *t;
    x.validate = 0;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return store_tune_locked(key, x);
}

spgemm_status spgemm_tune_cache_count(int64_t* n) {
    if (!n) return SPGEMM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    *n = (int64_t)g_tune_cache.size();
    return SPGEMM_OK;
}

spgemm_status spgemm_tune_cache_entry(int64_t index, uint64_t* key, spgemm_tune* t) {
    if (!key || !t || index < 0) return SPGEMM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (index >= (int64_t)g_tune_cache.size()) return SPGEMM_ERR_INVALID_ARG;
    auto it = g_tune_cache.begin();
    std::advance(it, index);
    *key = it->first;
    *t = it->second;
    return SPGEMM_OK;
}

spgemm_status spgemm_set_concurrent_bins(spgemm_handle* h, int32_t enable) {
    if (!h) return SPGEMM_ERR_INVALID_ARG;
    h->concurrent_bins = enable != 0;
    return SPGEMM_OK;
}

spgemm_status spgemm_plan_set_concurrent_bins(spgemm_plan* p, int32_t enable) {
    if (!p) return SPGEMM_ERR_INVALID_ARG;
    plan_drop_graph(p);
    p->h->concurrent_bins = enable != 0;
    return SPGEMM_OK;
}

spgemm_status spgemm_plan_launch_count(const spgemm_plan* p, int64_t* count) {
    if (!p || !count) return SPGEMM_ERR_INVALID_ARG;
    *count = p->h->launches;
    return SPGEMM_OK;
}

spgemm_status spgemm_plan_destroy(spgemm_plan* p) {
    if (!p) return SPGEMM_OK;
    plan_drop_graph(p);
    spgemm_destroy(p->h);
    if (p->capture) cudaStreamDestroy(p->capture);
    delete p;
    return SPGEMM_OK;
}

}  // extern "C"
