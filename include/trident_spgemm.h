/*
 * trident_spgemm.h -- C ABI of the GB300 (sm_103a) trident SpGEMM library.
 *
 * The library computes the local hot path of the trident distributed SpGEMM
 * (Communication-Avoiding SpGEMM via Trident Partitioning, arXiv 2603.21444):
 * the per-block CSR product C_blk = A_blk B_blk (row-wise Gustavson: a
 * symbolic pass that sizes every output row, then a numeric pass) and the
 * ordered sum of the partial products that the sqrt(P/lambda) x
 * sqrt(P/lambda) x lambda trident grid assigns to each output block
 * (Sec. 3.2, Alg. 1, Alg. 2, Sec. 4.4).  On one GPU all blocks run as batched
 * instances; there is no inter-GPU traffic.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Matrices are CSR (Sec. 2): row_ptr (nrows+1 int32), col_idx (nnz int32),
 * val (nnz values, float or double as the call's spgemm_dtype says).
 *
 * Ownership: every array passed in or out is DEVICE memory allocated and
 *   owned by the caller; no call frees or keeps caller memory beyond the
 *   call.  The handle owns only its own workspace (grown on demand with
 *   cudaMalloc, released by spgemm_destroy).  Pointers marked "host" are
 *   ordinary host memory.
 * Streams: all device work is ordered on the stream passed in (a
 *   cudaStream_t; NULL means the legacy default stream).  Calls that return a
 *   size to the host (symbolic, sizing calls) synchronise that stream once.
 * Input canonical form: row_ptr non-decreasing with row_ptr[0] = 0 and
 *   row_ptr[nrows] = nnz, 0 <= col_idx < ncols.  Columns need not be sorted
 *   for the product to be correct, but output rows are always written sorted
 *   ascending and duplicate-free, so outputs are canonical.  With
 *   tune.validate != 0 inputs are checked on the device first and a bad one
 *   gives SPGEMM_ERR_NOT_CANONICAL; with validation off a bad input is
 *   undefined behaviour.
 * Output pattern: structural; an entry exists wherever a product a_ik b_kj
 *   lands, explicit zeros from cancellation are kept.
 * Values: each product is rounded once and the products of an output entry
 *   are added in ascending (instance, k) order, each instance's products
 *   summed first (deterministic accumulator, SPGEMM_ACC_SORT); rows with more
 *   than 8192 products use a dense accumulator with atomic adds whose order is
 *   not fixed (results then agree to rounding, not bit for bit).
 * Sizes: per output matrix nnz must fit int32; otherwise the sizing call
 *   returns SPGEMM_ERR_INDEX_OVERFLOW and no numeric work may follow.
 * Errors: returned, never thrown.  On error the content of the outputs is
 *   unspecified.  A device-side inconsistency is latched in the handle and
 *   reported by spgemm_device_status().
 * Threads: a handle may be used by one host thread at a time.
 */
#ifndef TRIDENT_SPGEMM_H
#define TRIDENT_SPGEMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t without including CUDA headers; NULL = legacy default stream. */
typedef struct CUstream_st* spgemm_stream_t;

typedef enum {
    SPGEMM_OK = 0,
    SPGEMM_ERR_INVALID_ARG = 1,     /* null pointer, negative size, bad enum */
    SPGEMM_ERR_SHAPE = 2,           /* A.ncols != B.nrows, mismatched output shape */
    SPGEMM_ERR_DTYPE = 3,           /* unknown value type */
    SPGEMM_ERR_INDEX_OVERFLOW = 4,  /* an output's nnz exceeds INT32_MAX */
    SPGEMM_ERR_OOM = 5,             /* workspace allocation failed */
    SPGEMM_ERR_CUDA = 6,            /* a CUDA runtime call failed */
    SPGEMM_ERR_DEVICE_TIMEOUT = 7,  /* a bounded device wait ran out */
    SPGEMM_ERR_HASH_OVERFLOW = 8,   /* an accumulator saw more entries than sized for */
    SPGEMM_ERR_NOT_CANONICAL = 9,   /* input failed validation */
    SPGEMM_ERR_INTERNAL = 10,       /* device consistency check failed */
    SPGEMM_ERR_UNSUPPORTED = 11,    /* valid request the library does not handle */
    SPGEMM_ERR_CAPACITY = 12        /* an output buffer is smaller than the result */
} spgemm_status;

typedef enum { SPGEMM_F32 = 0, SPGEMM_F64 = 1 } spgemm_dtype;

/* Input CSR (device pointers).  val may be NULL for the symbolic pass. */
typedef struct {
    int32_t nrows;
    int32_t ncols;
    int32_t nnz;
    const int32_t* row_ptr; /* nrows + 1 */
    const int32_t* col_idx; /* nnz */
    const void* val;        /* nnz values of the call's dtype */
} spgemm_csr_in;

/* Output CSR (device pointers, caller-allocated).  row_ptr is written by the
 * sizing/symbolic call and read by the numeric call. */
typedef struct {
    int32_t nrows;
    int32_t ncols;
    int32_t* row_ptr; /* nrows + 1 */
    int32_t* col_idx; /* nnz (NULL in a sizing call) */
    void* val;        /* nnz */
} spgemm_csr_out;

/* Row bins.  Rows are binned by their intermediate-product count
 * u_i = sum_{k in A_i} |B_k| (and their A-row length).  Bin b serves rows with
 * u <= bin_upper[b] using kernel variant bin_kernel[b] (an index into the
 * variant table below); rows beyond the last bin use the dense heavy-row path.
 * Kernel variants (team = threads cooperating on one row, capacity = most
 * products a team holds on chip):
 *   0: warp,  32   1: warp, 64    2: warp, 128    3: warp, 256    4: warp, 512
 *   5: 128 threads, 1024   6: 256 threads, 2048   7: 512 threads, 4096
 *   8: 512 threads, 8192   9: warp, 384   10: one thread per row, 16
 *   11: 128 threads, 1024  12: 256 threads, 2048  13: 512 threads, 4096
 *   14: 1024 threads, 8192   15: warp, 320
 *   16-19: the block teams 11-14 with the row's B segments staged in shared
 *   memory by TMA bulk copies (rows of at most 128 A entries; others read
 *   from global memory as in 11-14)
 * Two accumulator kinds serve the block teams: variants 5-8 sort 64-bit
 * (column, product) keys by bucket and rank inside each bucket; variants
 * 11-14 keep the products in registers and run the warp teams' counting sort
 * over the whole block (16-bit bucket counters, one bucket per column when
 * the output has fewer columns than buckets, a dense accumulator).  Both
 * add every output entry in the same order, so their results are identical.
 * The default bins are 16, 32, 64, 128, 256, 320, 384, 512, ..., 8192 with
 * variants 10, 0, 1, 2, 3, 15, 9, 4, 11, 12, 13, 14.  A variant whose
 * capacity is below bin_upper is rejected. */
#define SPGEMM_MAX_BINS 12
#define SPGEMM_NUM_VARIANTS 20
enum { SPGEMM_ACC_SORT = 0 };

typedef struct {
    int32_t num_bins;                      /* 1..SPGEMM_MAX_BINS */
    int32_t bin_upper[SPGEMM_MAX_BINS];    /* increasing product-count bounds */
    int32_t bin_kernel[SPGEMM_MAX_BINS];   /* variant per bin */
    int32_t accumulator;                   /* SPGEMM_ACC_SORT */
    int32_t warps_per_block;               /* blocks of warp-team variants: 1..32 (clamped per
                                              variant to what its shared memory allows) */
    int32_t validate;                      /* nonzero: check inputs on the device */
    int32_t sym_warps_per_block;           /* symbolic pass; 0 = warps_per_block (clamped to 8 for
                                              warp variants up to 384, 16 above) */
} spgemm_tune;

typedef struct spgemm_handle spgemm_handle;

/* ---------------------------------------------------------------- handles */

/* Static string for a status code (never NULL). */
const char* spgemm_status_str(spgemm_status s);

/* Library version string. */
const char* spgemm_version(void);

/* Create a handle bound to the CUDA device current on the calling thread.
 * *out receives the handle; SPGEMM_ERR_CUDA if no device is usable. */
spgemm_status spgemm_create(spgemm_handle** out);

/* Free the handle's workspace and the handle (NULL is a no-op).  Waits for
 * the handle's outstanding work on every stream it used. */
spgemm_status spgemm_destroy(spgemm_handle* h);

/* Fill *t with the library's default tuning (no handle needed). */
spgemm_status spgemm_default_tune(spgemm_tune* t);

/* Set the tuning used by later calls (NULL restores the defaults).  Checked:
 * bounds increasing, variants known and large enough. */
spgemm_status spgemm_set_tune(spgemm_handle* h, const spgemm_tune* t);
spgemm_status spgemm_get_tune(const spgemm_handle* h, spgemm_tune* t);

/* ------------------------------------------------------- the product (Sec. 2)
 *
 * spgemm_symbolic: row sizes of C = A B.  Writes c_row_ptr (device, m+1,
 * int32) as the exclusive scan of the per-row distinct-column counts and
 * *c_nnz (host) = nnz(C).  B.val / A.val are not read.  Synchronises the
 * stream once (to return nnz).  SPGEMM_ERR_SHAPE if A.ncols != B.nrows,
 * SPGEMM_ERR_INDEX_OVERFLOW if nnz(C) > INT32_MAX (c_row_ptr then unspecified).
 */
spgemm_status spgemm_symbolic(spgemm_handle* h, const spgemm_csr_in* A, const spgemm_csr_in* B,
                              int32_t* c_row_ptr, int64_t* c_nnz, spgemm_stream_t stream);

/* spgemm_numeric: fills C->col_idx and C->val (device, nnz(C) each) of
 * C = A B, reading C->row_ptr as written by spgemm_symbolic for the same
 * A and B patterns.  Rows are written sorted.  Asynchronous (no host sync). */
spgemm_status spgemm_numeric(spgemm_handle* h, spgemm_dtype dtype, const spgemm_csr_in* A,
                             const spgemm_csr_in* B, spgemm_csr_out* C, spgemm_stream_t stream);

/* spgemm_products: *total (host) = sum over rows of the intermediate-product
 * count u_i = sum_{k in A_i} |B_k| (2 x total = the product's flop count),
 * an upper bound of nnz(C).  Synchronises once. */
spgemm_status spgemm_products(spgemm_handle* h, const spgemm_csr_in* A, const spgemm_csr_in* B, int64_t* total,
                              spgemm_stream_t stream);

/* spgemm_fused: C = A B in a single pass, without a separate symbolic pass,
 * into caller buffers of `capacity` entries (C->col_idx, C->val; C->row_ptr
 * of A.nrows + 1 entries is written; spgemm_products gives a capacity that
 * always suffices).  When every row fits the warp-team variants, tiles of
 * consecutive rows (one per warp of a block) are handed out in order, each
 * row is sorted and reduced on chip, and a tile's output offset is the sum of
 * the earlier tiles' counts (decoupled look-back, with a bounded wait that
 * reports SPGEMM_ERR_DEVICE_TIMEOUT instead of stalling).
 * Otherwise the call runs the symbolic and numeric passes.  Values and
 * pattern are identical to spgemm_symbolic + spgemm_numeric.  *c_nnz (host)
 * receives nnz(C); SPGEMM_ERR_CAPACITY if it exceeds capacity (outputs then
 * unspecified).  Synchronises once (twice on the two-pass route). */
spgemm_status spgemm_fused(spgemm_handle* h, spgemm_dtype dtype, const spgemm_csr_in* A, const spgemm_csr_in* B,
                           spgemm_csr_out* C, int64_t capacity, int64_t* c_nnz, spgemm_stream_t stream);

/* ------------------------------------------- product from host memory
 *
 * The same product as spgemm_symbolic + spgemm_numeric (Sec. 2), for inputs
 * and outputs in host memory, with the transfers overlapped: the output
 * rows are computed in `panels` row panels, and each panel's columns and
 * values travel to the host on a second stream of the handle while the
 * next panels are computed.  Host arrays in page-locked memory get the full
 * link bandwidth (pageable memory works, at the driver's staging speed).
 *
 * spgemm_host_symbolic: A, B are host CSR arrays (row_ptr, col_idx; val may
 *   be NULL); copies them into device buffers the handle owns (grown on
 *   demand, kept), sizes C and writes its row_ptr to c_row_ptr (host,
 *   A.nrows + 1 entries) and its nnz to *c_nnz.  Synchronises on `stream`.
 *   value_dtype: SPGEMM_F32 / SPGEMM_F64 when A->val and B->val hold values
 *   of that type: their upload starts on the handle's second stream and runs
 *   while the sizing does (it may still be running when the call returns);
 *   -1: the values are not touched.
 * spgemm_host_numeric: A, B the same host arrays, now with values of
 *   `dtype`; C->row_ptr the host row_ptr from the sizing call, C->col_idx
 *   and C->val host arrays of *c_nnz entries.  A call right after the sizing
 *   call with the same A and B pointers reuses the device copies of the
 *   indices (and of the values, when the sizing call uploaded them with this
 *   dtype); the host arrays must not change in between.  A later call with
 *   the same pointers copies everything again.  C is computed in `panels`
 *   row panels (1..1024, 0 = 8; the first half the size of the others); the
 *   columns and values of each finished panel are copied out while the next
 *   ones run.  Synchronises before returning.
 * Errors as the device calls; SPGEMM_ERR_OOM when the handle's buffers
 * cannot grow.
 */
spgemm_status spgemm_host_symbolic(spgemm_handle* h, int32_t value_dtype, const spgemm_csr_in* A,
                                   const spgemm_csr_in* B, int32_t* c_row_ptr, int64_t* c_nnz,
                                   spgemm_stream_t stream);
spgemm_status spgemm_host_numeric(spgemm_handle* h, spgemm_dtype dtype, const spgemm_csr_in* A,
                                  const spgemm_csr_in* B, spgemm_csr_out* C, int32_t panels,
                                  spgemm_stream_t stream);

/* ------------------------------------ ordered sum of partials (Sec. 4.4, Alg. 1)
 *
 * spgemm_merge: C = parts[0] + parts[1] + ... + parts[nparts-1] for CSR
 * matrices of one shape (the accumulation C_ijk += C_ijk^(r) of Alg. 1 over
 * the rounds r, done by cuSPARSE spgeam in the paper).  Row i of C is the
 * union of the row-i patterns; equal columns are added in part order.
 * Sizing call: C->col_idx == NULL -> writes C->row_ptr and *c_nnz (host),
 * synchronising once.  Fill call: C->col_idx != NULL -> fills col/val using
 * C->row_ptr from the sizing call; c_nnz may be NULL; asynchronous.
 * 1 <= nparts <= 64.
 */
spgemm_status spgemm_merge(spgemm_handle* h, spgemm_dtype dtype, int32_t nparts,
                           const spgemm_csr_in* parts, spgemm_csr_out* C, int64_t* c_nnz,
                           spgemm_stream_t stream);

/* ------------------------------- batched instances (Alg. 1 + Alg. 2, Sec. 3.3)
 *
 * spgemm_batched: many products in one pass.  Instance t is A[t] B[t].
 * Instances are grouped: group g owns instances [group_ptr[g],
 * group_ptr[g+1]) (host array, ngroups+1 entries; NULL means one instance
 * per group) and its output C[g] = sum over its instances, in that order, of
 * A[t] B[t] -- the trident output block C_ijk = sum_r A_{i r' k} B_{r' j}
 * with the rounds listed in stagger order.  All instances of a group must
 * have the same A.nrows and B.ncols (= C[g] shape).  B[t] of different
 * instances may alias the same device arrays (a shared tile is read in
 * place; on one device this is the allgathered tile of Alg. 2).
 * The partials are never materialised: each output row accumulates all its
 * instances at once, adding each instance's products first and then the
 * instance sums in group order (the same sums spgemm_merge of the partials
 * would give).
 * Sizing call: c_nnz != NULL -> writes every C[g].row_ptr and c_nnz[g]
 * (host, ngroups entries), synchronising once; col_idx/val are not read.
 * Fill call: c_nnz == NULL -> fills every C[g].col_idx / val (NULL allowed
 * only for a group whose nnz is 0), asynchronous.
 * tune: NULL uses the handle's tuning.  ninst <= 2^20, group sizes <= 64.
 */
spgemm_status spgemm_batched(spgemm_handle* h, spgemm_dtype dtype, int32_t ninst,
                             const spgemm_csr_in* A, const spgemm_csr_in* B, int32_t ngroups,
                             const int32_t* group_ptr, spgemm_csr_out* C, int64_t* c_nnz,
                             const spgemm_tune* tune, spgemm_stream_t stream);

/* ------------------------------------------------ persistent batched plan
 *
 * A plan is one batched problem (the arguments of spgemm_batched) sized once
 * and executed many times.  It owns a private workspace (bin lists,
 * descriptors, accumulators), so executing it is independent of other calls.
 *
 * spgemm_plan_create: runs the sizing pass: writes c_row_ptr[g] (host array
 * of ngroups device pointers, each nrows+1 int32) and c_nnz[g] (host),
 * synchronising once.  The inputs must stay allocated and unchanged for the
 * plan's lifetime.  tune NULL = library defaults.
 * spgemm_plan_execute: the numeric pass into C[g] (row_ptr as sized,
 * col_idx / val of c_nnz[g] entries).  use_graph != 0: the first execution
 * for a given set of output pointers runs the kernels directly and also
 * captures them into a CUDA graph owned by the plan; later executions with
 * the same outputs are one cudaGraphLaunch.  Asynchronous.
 * spgemm_plan_autotune: times candidate bin layouts and warps-per-block
 * settings on this problem (each candidate sized and executed into C, which
 * must be allocated), keeps the fastest in the plan and writes it to *chosen
 * (may be NULL).  Results are cached per device, dtype and product-count
 * histogram.  Every candidate gives the same output bits.  Synchronises.
 */
typedef struct spgemm_plan spgemm_plan;
spgemm_status spgemm_plan_create(spgemm_dtype dtype, int32_t ninst, const spgemm_csr_in* A, const spgemm_csr_in* B,
                                 int32_t ngroups, const int32_t* group_ptr, int32_t* const* c_row_ptr,
                                 int64_t* c_nnz, const spgemm_tune* tune, spgemm_stream_t stream,
                                 spgemm_plan** out);
spgemm_status spgemm_plan_execute(spgemm_plan* p, const spgemm_csr_out* C, int32_t use_graph,
                                  spgemm_stream_t stream);
spgemm_status spgemm_plan_autotune(spgemm_plan* p, const spgemm_csr_out* C, spgemm_stream_t stream,
                                   spgemm_tune* chosen);
spgemm_status spgemm_plan_launch_count(const spgemm_plan* p, int64_t* count);
spgemm_status spgemm_plan_destroy(spgemm_plan* p);

/* Concurrent bins (Sec. 3.3's asynchronous C-stationary tiles: no global
 * barrier between independent pieces of work).  The rows of different bins
 * are disjoint, so by default every call forks its per-bin launches onto
 * private streams of the handle (each first waits for the work already on
 * the call's stream) and joins them back before anything that needs all
 * bins; in a plan's CUDA graph they are parallel nodes.  enable = 0 issues
 * them one after another on the call's stream instead (the same results).
 * The plan variant drops the plan's captured graph. */
spgemm_status spgemm_set_concurrent_bins(spgemm_handle* h, int32_t enable);
spgemm_status spgemm_plan_set_concurrent_bins(spgemm_plan* p, int32_t enable);

/* Persistent autotune cache (host only).  The layouts spgemm_plan_autotune
 * chooses are kept per process, keyed by the GPU model (compute capability
 * and SM count), the dtype and the shape of the product-count histogram
 * (log2 of every bin's row count).  A cache file makes them outlive the
 * process: a text file, one entry per line,
 *     tsg-tune-1 <key: 16 hex digits> <num_bins> <warps_per_block>
 *                <sym_warps_per_block> then <bin_upper bin_kernel> per bin
 * spgemm_tune_cache_open(path, *loaded): takes the file's entries into the
 * process's cache (a later line replaces an earlier one with the same key;
 * lines that do not parse or fail the spgemm_set_tune checks are skipped)
 * and appends every later choice to it (one write per line, so processes
 * may share the file).  path NULL: the file named by the environment
 * variable TRIDENT_SPGEMM_TUNE_CACHE, else none.  A missing file counts as
 * empty and is created on the first append.  Without an open call the first
 * spgemm_plan_autotune reads the environment variable itself.  *loaded (may
 * be NULL) receives the entries taken.  SPGEMM_ERR_INVALID_ARG if the file
 * exists but cannot be read; spgemm_plan_autotune returns the same code when
 * it cannot append (the plan keeps the layout it chose).
 * spgemm_tune_cache_clear: empties the process's cache and detaches the
 * file (the file is not changed).
 * spgemm_tune_cache_store: records a layout under a key (checked as by
 * spgemm_set_tune) and appends it to the file, if one is open.
 * spgemm_tune_cache_count / _entry: the number of entries, and entry
 * `index` (0 <= index < count, in key order). */
spgemm_status spgemm_tune_cache_open(const char* path, int64_t* loaded);
spgemm_status spgemm_tune_cache_clear(void);
spgemm_status spgemm_tune_cache_store(uint64_t key, const spgemm_tune* t);
spgemm_status spgemm_tune_cache_count(int64_t* n);
spgemm_status spgemm_tune_cache_entry(int64_t index, uint64_t* key, spgemm_tune* t);

/* ------------------------------------------ trident partition (Sec. 3.2)
 *
 * spgemm_tile_split: cut X into nrp x ncp tiles.  Tile (rp, cp) holds rows
 * [row_bounds[rp], row_bounds[rp+1]) and columns [col_bounds[cp],
 * col_bounds[cp+1]) of X, with columns re-based to the tile (j -> j -
 * col_bounds[cp]) and each row's entries in X's stored order.  row_bounds
 * (nrp+1) and col_bounds (ncp+1) are host arrays, non-decreasing, from 0 to
 * X.nrows / X.ncols; 1 <= nrp, ncp and ncp <= 64.  tiles[rp * ncp + cp]
 * describes tile (rp, cp): nrows/ncols must equal the bound differences.
 * Sizing call: tile_nnz != NULL -> writes every tile's row_ptr and
 * tile_nnz[rp * ncp + cp] (host), synchronising once.  Fill call: tile_nnz
 * == NULL -> writes col_idx / val of every tile (val skipped when X.val is
 * NULL), asynchronous.
 * The trident split of A (m x kk) for a grid q x q x lambda uses row bounds
 * (coarse tile t) floor(t m / q) refined into lambda slices
 * lo + floor(s (hi - lo) / lambda), and column bounds floor(t kk / q); the
 * split of B uses coarse bounds on both sides.
 */
spgemm_status spgemm_tile_split(spgemm_handle* h, spgemm_dtype dtype, const spgemm_csr_in* X, int32_t nrp,
                                const int32_t* row_bounds, int32_t ncp, const int32_t* col_bounds,
                                spgemm_csr_out* tiles, int64_t* tile_nnz, spgemm_stream_t stream);

/* spgemm_trident_bounds: the boundaries of the trident split of [0, n)
 * (Sec. 3.2) for a grid q x q x lambda: coarse tile t is [coarse[t],
 * coarse[t+1]) with coarse[t] = floor(t n / q), t = 0..q; each coarse tile
 * [lo, hi) is cut into lambda contiguous slices, slice s of tile t starting
 * at fine[t lambda + s] = lo + floor(s (hi - lo) / lambda), and
 * fine[q lambda] = n.  Host arrays of q + 1 (coarse) and q lambda + 1 (fine)
 * entries; either may be NULL.  n >= 0, q >= 1, lambda >= 1 (products
 * computed in 64 bits); otherwise SPGEMM_ERR_INVALID_ARG.  Host-only: needs
 * no handle and no device.  These are the row bounds (fine) and column
 * bounds (coarse) spgemm_tile_split takes for A, and the coarse bounds on
 * both sides for B. */
spgemm_status spgemm_trident_bounds(int32_t n, int32_t q, int32_t lambda, int32_t* coarse, int32_t* fine);

/* ------------------------------------ static-Cannon rounds (Alg. 1, Eq. 2)
 *
 * spgemm_trident_schedule: the instance list of the trident grid q x q x
 * lambda in the layout spgemm_batched takes.  Output block (i, j, k) is group
 * g = (i q + j) lambda + k; its q instances are the rounds r = 0..q-1 in
 * order, round r multiplying A slice (i, r', k) by B tile (r', j) with the
 * stagger r' = (r + i + j) mod q.  a_tile[t] = (i lambda + k) q + r' indexes
 * the tiles of spgemm_tile_split on A (row slices x column tiles) and
 * b_tile[t] = r' q + j those of B; group_ptr[g] = g q.  Host arrays of
 * q*q*lambda*q (a_tile, b_tile) and q*q*lambda + 1 (group_ptr) entries.
 * Host-only: needs no handle and no device.
 */
spgemm_status spgemm_trident_schedule(int32_t q, int32_t lambda, int32_t* a_tile, int32_t* b_tile,
                                      int32_t* group_ptr);

/* ------------------------------------------------------------ differentiation
 *
 * spgemm_backward: gradients of a scalar loss L through C = A B with the
 * sparsity patterns held fixed (chain rule on C_ij = sum_k a_ik b_kj, Sec. 2):
 *   dA_ik = sum_{j in B_k} G_ij b_kj       for (i,k) in pattern(A)
 *   dB_kj = sum_{i: k in A_i} a_ik G_ij    for (k,j) in pattern(B)
 * where G_ij = dL/dC_ij is given as C->val on the pattern of C (C->row_ptr
 * and C->col_idx as returned by the forward product of the same A, B).
 * dA (device, nnz(A) values) and dB (device, nnz(B) values) may each be
 * NULL to skip.  dA is summed over B row k in stored order (deterministic).
 * deterministic == 0: dB by atomic scatter (fast; summation order not
 * fixed).  deterministic != 0: dB from the transpose of A (built in the
 * handle's workspace), each entry summed over i ascending.  Asynchronous.
 * A column of B's row k that is missing from row i of C latches
 * SPGEMM_ERR_INTERNAL (C is not the product's pattern).
 */
spgemm_status spgemm_backward(spgemm_handle* h, spgemm_dtype dtype, const spgemm_csr_in* A,
                              const spgemm_csr_in* B, const spgemm_csr_in* C, void* dA, void* dB,
                              int32_t deterministic, spgemm_stream_t stream);

/* spgemm_csr_transpose: XT = X^T.  XT->nrows = X->ncols, XT->ncols =
 * X->nrows; XT->row_ptr (X->ncols + 1), XT->col_idx and XT->val (X->nnz
 * each; val skipped when X->val is NULL) are caller-allocated.  Rows of XT
 * come out sorted (X must have no repeated column within a row).
 * Asynchronous; workspace from the handle. */
spgemm_status spgemm_csr_transpose(spgemm_handle* h, spgemm_dtype dtype, const spgemm_csr_in* X,
                                   spgemm_csr_out* XT, spgemm_stream_t stream);

/* spgemm_csr_permute: Y = P X Q^T, i.e. Y[row_perm[i], col_perm[j]] =
 * X[i, j] -- the random relabelling of rows and columns that turns a
 * structured (banded) matrix into an unstructured one whose trident tiles
 * carry even shares of the nonzeros (Sec. 5, the permuted HV15R runs).
 * row_perm (X->nrows int32) and col_perm (X->ncols int32) are device
 * arrays; NULL means the identity.  Y has X's shape; Y->row_ptr (nrows + 1),
 * Y->col_idx and Y->val (X->nnz each; val skipped when X->val is NULL) are
 * caller-allocated.  Y's rows come out sorted (X must have no repeated
 * column within a row).  Both maps are checked on the device to be
 * permutations before any entry of Y is written: SPGEMM_ERR_INVALID_ARG
 * otherwise (Y's row_ptr, col_idx and val then unspecified).  With a column
 * map, rows longer than 65536 entries are not re-sorted:
 * SPGEMM_ERR_UNSUPPORTED (Y unspecified).  Synchronises once (the check's
 * result). */
spgemm_status spgemm_csr_permute(spgemm_handle* h, spgemm_dtype dtype, const spgemm_csr_in* X,
                                 const int32_t* row_perm, const int32_t* col_perm, spgemm_csr_out* Y,
                                 spgemm_stream_t stream);

/* ------------------------------------------- Markov clustering (Sec. 5.6)
 *
 * One iteration of Markov clustering with the expansion step done by this
 * library's product, fused with the column operations.  The column-
 * stochastic n x n matrix M is passed TRANSPOSED (Mt: row r = column r of
 * M, float values), so that (M M)^T = Mt Mt and every column operation is
 * row-local.  Per row r of the expansion E = Mt Mt:
 *   e_j accumulated in double from float products a * b (each rounded to
 *   float);  w_j = e_j^inflation (inflation 2: e_j * e_j);  v_j = w_j / sum w;
 *   keep v_j >= prune (none kept: keep the largest v_j);  more than topk kept:
 *   keep the topk largest v_j;  equal v_j: the smaller column first;
 *   out_j = (float)(v_j / sum of kept v_j).
 * All keep/drop decisions are taken in double.  1 <= topk <= 1024.
 * spgemm_mcl_expand: computes the next iterate's row_ptr (device, n+1 int32,
 * caller-allocated) and *out_nnz (host), keeping the entries in the handle's
 * workspace; synchronises.  spgemm_mcl_collect: copies them into out->col_idx
 * / out->val (caller-allocated, out_nnz each; out->row_ptr from expand),
 * asynchronous.  No other call on the handle may come between the two.
 * The full expansion E is never stored: a row's kept entries (at most
 * min(products of the row, topk)) are all that is written.  Workspace held
 * by the handle: per block (4 per SM) n doubles, n ints and n / 32 words of
 * accumulator, plus, for the window-summed rows (up to 6 blocks per SM, 5
 * with 4096-column windows), 12 bytes of staging per product of capacity
 * (2^21) per block (about 19 GB on 152 SMs), plus the batched rows' two
 * buffers of 48 MB.
 */
typedef struct {
    double inflation;  /* r of the inflation step (2) */
    double prune;      /* drop v_j below this (1e-4) */
    int32_t topk;      /* keep at most this many per row (1000) */
    int32_t heavy;     /* rows with at least this many products run in batches
                          of a few rows on dense accumulators resident in L2
                          (0: max(4096, 2 n); < 0: never; with prune 0 never).
                          With every value in [2^-63, FLT_MAX], rows from 4096
                          products up to min(this, 2^21) sum their products
                          window by window in shared memory */
    int32_t window;    /* those rows: 0 by the pilot (spgemm_mcl_paths),
                          1 always window-summed, -1 never */
} spgemm_mcl_params;

spgemm_status spgemm_mcl_expand(spgemm_handle* h, const spgemm_csr_in* Mt, const spgemm_mcl_params* prm,
                                int32_t* out_row_ptr, int64_t* out_nnz, spgemm_stream_t stream);
spgemm_status spgemm_mcl_collect(spgemm_handle* h, spgemm_csr_out* out, spgemm_stream_t stream);
/* spgemm_mcl_paths: rows of the last spgemm_mcl_expand on the handle per
 * path -- rows[0] the per-block kernel, rows[1] window-summed in shared
 * memory, rows[2] the L2-resident batches -- and *pilot_ratio the products
 * per distinct column measured on up to 32 rows of the window-summed range
 * (0 when no pilot ran; above 4 those rows were given back to the per-block
 * kernel, whose accumulators then stay in L2).  Host only, no GPU work. */
spgemm_status spgemm_mcl_paths(const spgemm_handle* h, int64_t* rows, double* pilot_ratio);

/* ------------------------------------------------ allocation-free variant
 *
 * spgemm_csr_transpose_noalloc: the same result as spgemm_csr_transpose
 * (XT = X^T, rows sorted, arguments and layout identical) for callers that
 * must not allocate device memory: code whose device memory is owned by an
 * outside pool or budget that forbids allocations behind its back, and paths
 * that cannot afford an allocation's implicit synchronisation.  It takes no
 * handle and calls no allocating routine: its working memory is one fixed
 * array of SPGEMM_NOALLOC_SCRATCH_BYTES compiled into the library, held by
 * every GPU that loads it until the process exits.  A request whose working
 * set (about 12 bytes per column of X plus 8 (float) or 12 (double) bytes
 * per nonzero, each part rounded up to 256 bytes) exceeds the array returns
 * SPGEMM_ERR_UNSUPPORTED without launching anything.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  The
 * address is kept for the life of the process: after cudaDeviceReset (or
 * any other loss of the device's primary context) it is stale, so do not
 * call this entry point again in that process.  All calls share the array:
 * calls whose GPU work overlaps (other streams, unordered host threads)
 * race.  Asynchronous on `stream`.
 * The paper has no counterpart: this entry point exists for callers of the
 * library, not for the method.
 */
#define SPGEMM_NOALLOC_SCRATCH_BYTES (25u << 20)
spgemm_status spgemm_csr_transpose_noalloc(spgemm_dtype dtype, const spgemm_csr_in* X, spgemm_csr_out* XT,
                                           spgemm_stream_t stream);

/* --------------------------------------------------------- instrumentation */

/* Number of kernels this handle has launched since creation (host counter). */
spgemm_status spgemm_launch_count(const spgemm_handle* h, int64_t* count);

/* Synchronise the handle's last stream and report a latched device-side
 * inconsistency (SPGEMM_ERR_INTERNAL / SPGEMM_ERR_HASH_OVERFLOW /
 * SPGEMM_ERR_DEVICE_TIMEOUT) or SPGEMM_OK; clears the latch. */
spgemm_status spgemm_device_status(spgemm_handle* h);

/* Per-phase CUDA-event timing.  enable != 0 starts recording events around
 * each phase on the call's stream; spgemm_read_timing synchronises, adds up
 * the completed intervals and returns milliseconds per phase and the number
 * of intervals (launch groups) per phase since the last read, then resets.
 * Phases: 0 analysis, 1 symbolic rows, 2 scan, 3 numeric rows, 4 heavy rows,
 * 5 partition, 6 backward, 7 mcl.  ms and count have SPGEMM_NUM_PHASES
 * entries (host). */
#define SPGEMM_NUM_PHASES 8
spgemm_status spgemm_set_timing(spgemm_handle* h, int32_t enable);

/* Workspace limit.  spgemm_set_workspace_limit caps the device bytes the
 * handle's own workspace buffers may hold (bytes < 0: no cap, the default;
 * a plan's private workspace is not counted).  A call whose workspace would
 * grow past the cap returns SPGEMM_ERR_OOM before it allocates, leaving the
 * buffers already held in place (the handle stays usable); a failing
 * cudaMalloc gives the same code.  spgemm_workspace_bytes writes the bytes
 * currently held (host int64).  Host only; SPGEMM_ERR_INVALID_ARG for a NULL
 * handle or pointer. */
spgemm_status spgemm_set_workspace_limit(spgemm_handle* h, int64_t bytes);
spgemm_status spgemm_workspace_bytes(const spgemm_handle* h, int64_t* bytes);

/* Fault injection for tests of the bounded device wait (the look-back of
 * spgemm_fused's single pass; no other kernel of the library waits on
 * another).  spin_limit > 0 caps the polls of one look-back wait (<= 0
 * restores the default, 2^22 polls, seconds of waiting); hold_tile >= 0 makes
 * that tile of rows (tile t = rows t*w .. t*w + w - 1, w the warps per block)
 * never publish its count, so the next tile's wait runs out: the call then
 * returns SPGEMM_ERR_DEVICE_TIMEOUT, the device stays usable and C is
 * unspecified (every write still stays within capacity).  hold_tile = -1
 * turns the injection off; a tile beyond the last one has no effect.
 * SPGEMM_ERR_INVALID_ARG for hold_tile < -1.  Host only; applies to later
 * calls on the handle. */
spgemm_status spgemm_set_wait_test(spgemm_handle* h, int32_t spin_limit, int32_t hold_tile);
spgemm_status spgemm_read_timing(spgemm_handle* h, double* ms, int64_t* count);

#ifdef __cplusplus
}
#endif

#endif /* TRIDENT_SPGEMM_H */
