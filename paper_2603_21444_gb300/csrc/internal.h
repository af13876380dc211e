// Host-side launchers shared between the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace tsg {

struct RowArgs;

struct AnalysisArgs {
    const InstDev* inst;
    const GroupDev* groups;
    const long long* unit_base;
    int ngroups;
    long long nunits;
    int merge;
    BinTable bt;
    unsigned char* bin_of;
    int* hist;      // nbins + 2 counters
    int* counts;    // per-unit row nnz (empty rows written here when sizing)
    int sizing;
    unsigned long long* total_u;  // optional: sum of all rows' product counts
};

// analysis + binning (rows_misc.cu)
cudaError_t launch_analysis(const AnalysisArgs& a, cudaStream_t s);
cudaError_t launch_bin_offsets(int* hist, int* off, int* cursor, int nslots, cudaStream_t s);
cudaError_t launch_bin_fill(const unsigned char* bin_of, long long nunits, const int* off, int* cursor,
                            int* list, cudaStream_t s);

// scan of per-unit counts into per-group row_ptr (rows_misc.cu)
long long scan_blocks(long long nunits);
cudaError_t launch_scan(const int* counts, long long nunits, long long* bsum, long long* ex, cudaStream_t s);
cudaError_t launch_rowptr(const GroupDev* groups, const long long* unit_base, int ngroups, long long nunits,
                          const long long* ex, long long* nnz_out, cudaStream_t s);

// input validation (rows_misc.cu)
cudaError_t launch_validate(const int* rp, const int* col, int nrows, int ncols, int nnz, unsigned* status,
                            cudaStream_t s);

// device-to-host read of `bytes` (a multiple of 4, at most 1 MiB) into mapped
// page-locked memory by a kernel on stream s (rows_misc.cu)
cudaError_t launch_readback(void* dst_mapped, const void* src, size_t bytes, cudaStream_t s);

// row kernels
struct RowLaunchArgs {
    const InstDev* inst;
    const GroupDev* groups;
    const long long* unit_base;
    int ngroups;
    const int* list;
    const int* bin_off;
    int bin;
    int merge;
    unsigned* status;
    int* counts;
    int* tick;  // per-bin row tickets of the numeric warp-team kernels (zeroed before them)
    int* glist;   // rows the numeric kernels defer to the grouped kernel (null: no deferral)
    int* gcount;  // their count (zeroed before the numeric kernels)
};
// warps per block a warp-team variant can take (launch bound and shared memory)
int warp_variant_max_wpb(int variant, int per_warp_bytes, bool symbolic);
int sym_smem_bytes(int variant, int warps_per_block);
int num_smem_bytes(int variant, int dtype, int warps_per_block);
int sym_blocks_per_sm(int variant, int warps_per_block);
int num_blocks_per_sm(int variant, int dtype, int warps_per_block);
cudaError_t launch_sym_rows(int variant, const RowLaunchArgs& a, int blocks, int warps_per_block, cudaStream_t s);
cudaError_t launch_num_rows(int variant, int dtype, const RowLaunchArgs& a, int blocks, int warps_per_block,
                            cudaStream_t s);
// rows the numeric kernels deferred (a.glist, *a.gcount), one warp each
cudaError_t launch_num_grouped(int dtype, const RowLaunchArgs& a, int sms, cudaStream_t s);
cudaError_t launch_num_fused(int variant, int dtype, const RowLaunchArgs& a, const FusedCtl& fc, int blocks,
                             int warps_per_block, cudaStream_t s);
int num_fused_blocks_per_sm(int variant, int dtype, int warps_per_block);
cudaError_t launch_sym_heavy(const RowLaunchArgs& a, int blocks, int chunk, cudaStream_t s);
cudaError_t launch_num_heavy(int dtype, const RowLaunchArgs& a, void* dense, int blocks, int chunk,
                             cudaStream_t s);
int heavy_chunk_for(int ncols);

// int64 exclusive sums -> int32 (rows_misc.cu)
cudaError_t launch_ll_to_int(const long long* src, long long n, int* dst, cudaStream_t s);

// backward (backward.cu)
struct BwdArgs {
    int m;                 // rows of A (= rows of C)
    int kdim;              // rows of B (= columns of A)
    long long nnzb;        // nnz(B)
    const int* arp;
    const int* acol;
    const void* aval;
    const int* brp;
    const int* bcol;
    const void* bval;
    const int* crp;        // pattern of C
    const int* ccol;
    const void* g;         // upstream gradient on pat(C)
    void* da;              // nnz(A) or null
    void* db;              // nnz(B) or null
    int scatter_db;        // 1: atomic scatter; 0: from A^T (deterministic)
    const int* trp;        // A^T (kdim rows), rows sorted
    const int* tcol;
    const void* tval;
    unsigned* status;
};
cudaError_t launch_backward(int dtype, const BwdArgs& a, int sms, cudaStream_t s);
cudaError_t launch_transpose(int dtype, const int* rp, const int* col, const void* val, int nrows, int ncols,
                             long long nnz, int* trp, int* tcol, void* tval, int* work, void* workv, long long* bsum,
                             long long* ex, int sms, cudaStream_t s);

// Markov-clustering iteration (mcl.cu)
struct MclLaunch {
    int n;
    const int* rp;
    const int* col;
    const float* val;
    const long long* ub_off;
    int* tmp_col;
    float* tmp_val;
    int* kept;
    double* dense;
    unsigned* bitmap;
    int* touched;
    unsigned long long* ckey;
    int* ccol;
    int ccap;
    long long stride;
    long long bm_words;
    int* row_counter;
    double inflation;
    double prune;
    int topk;
    unsigned* status;
    const unsigned char* heavy = nullptr;  // row flags: 1 batched, 2 window-summed
    int skip = 0;                          // flag bits whose rows k_mcl_rows leaves
    int positive = 0;                      // every value in [2^-63, FLT_MAX]
};
// batched heavy rows: at most kMclBatch rows per batch, each with a dense
// accumulator; kMclMaxList near-max columns kept per row
constexpr int kMclBatch = 16;
constexpr int kMclMaxList = 1024;
struct MclHeavyLaunch {
    const int* rows;
    int nb;
    double* D;
    double* s;
    unsigned long long* wmax;
    unsigned* flags;
    int* ncand;
    int* nmax;
    unsigned long long* ck;
    int* cc;
    int* mlist;
};
cudaError_t launch_mcl_check_positive(const float* val, long long nnz, int* flag, int sms, cudaStream_t s);
cudaError_t launch_mcl_mark(const int* rp, const int* col, int n, long long heavy, long long bucket_lo,
                            long long bucket_hi, const int* notpos, unsigned char* flags, int* hlist, int* hcount,
                            int* blist, int* bcount, cudaStream_t s);
// bucketed mid rows: staging of cap entries per block, windows of 2^lw columns
struct MclBucketLaunch {
    const int* list;
    int count;
    int* counter;
    int2* stage;
    int* ej;
    long long cap;
    int lw;
    int nbk;
};
cudaError_t launch_mcl_pilot(const MclLaunch& l, const int* rows, int nrows, int step, unsigned long long* tot,
                             cudaStream_t s);
size_t mcl_bucket_smem(int lw, int nbk);
int mcl_bucket_blocks_per_sm(int lw, int nbk);
cudaError_t launch_mcl_bucket(const MclLaunch& l, const MclBucketLaunch& b, int blocks, cudaStream_t s);
cudaError_t launch_mcl_heavy_batch(const MclLaunch& l, const MclHeavyLaunch& hb, int sms, cudaStream_t s);
cudaError_t launch_mcl_heavy_scans(const MclLaunch& l, const MclHeavyLaunch& hb, int sms, cudaStream_t s);
cudaError_t launch_mcl_heavy_select(const MclLaunch& l, const MclHeavyLaunch& hb, cudaStream_t s);
cudaError_t launch_mcl_bounds(const int* rp, const int* col, int n, int topk, int* ub, cudaStream_t s);
cudaError_t launch_mcl_rows(const MclLaunch& l, int blocks, cudaStream_t s);
cudaError_t launch_mcl_collect(int n, const long long* ub_off, const int* tmp_col, const float* tmp_val,
                               const int* orp, int* ocol, float* oval, int sms, cudaStream_t s);

// trident partition (partition.cu)
cudaError_t launch_split_count(const int* rp, const int* col, int nrows, const int* cb, int ncp, int* counts,
                               cudaStream_t s);
cudaError_t launch_split_fill(int dtype, const int* rp, const int* col, const void* val, int nrows, const int* rb,
                              int nrp, const int* cb, int ncp, const GroupDev* tiles, cudaStream_t s);

// ---- permutation Y = P X Q^T (permute.cu)
struct PermuteArgs {
    int dtype;  // 0 float, 1 double
    int nrows, ncols;
    long long nnz;
    const int* rp;
    const int* col;
    const void* val;       // may be null (pattern only)
    const int* row_perm;   // null: identity
    const int* col_perm;   // null: identity
    int* yrp;
    int* ycol;
    void* yval;
    int* hits_r;           // nrows, zeroed
    int* hits_c;           // ncols, zeroed
    int* ylen;             // nrows
    long long* bsum;       // scan_blocks(nrows)
    long long* ex;         // nrows + 1
    int* long_count;       // 1, zeroed
    int* long_list;        // nrows
    int* rank;             // nnz
    unsigned* status;
    int sms;
};
cudaError_t launch_permute(const PermuteArgs& p, cudaStream_t s);

}  // namespace tsg
