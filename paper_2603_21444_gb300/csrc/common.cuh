// Shared device-side definitions of the trident SpGEMM library (sm_103a).
//
// Work model.  Every call is a set of GROUPS, each producing one output CSR.
// A group owns one or more INSTANCES; instance t contributes A_t B_t (product
// mode) or, in merge mode, is itself a partial C_t whose rows are taken as
// they are.  A WORK UNIT is one output row (group g, row rho); units of all
// groups are numbered consecutively (group g owns units
// [unit_base[g], unit_base[g+1])).  Units are binned by their
// intermediate-product count u and their A-row length, and each bin is run by
// a kernel variant whose team (a warp or a whole block) holds up to CAP
// products of a row on chip.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tsg {

// ---------------------------------------------------------------- descriptors

struct InstDev {
    const int* arp;     // A_t row_ptr (product mode); unused in merge mode
    const int* acol;    // A_t col_idx
    const void* aval;   // A_t values
    const int* brp;     // B_t row_ptr (merge mode: the partial's row_ptr)
    const int* bcol;    // B_t col_idx
    const void* bval;   // B_t values
    long long bnnz;     // entries of bcol / bval (bulk copies stay inside them)
};

struct GroupDev {
    int inst_begin;     // first instance of the group
    int inst_count;     // number of instances (>= 1)
    int nrows;          // output rows
    int ncols;          // output columns
    int* crp;           // output row_ptr (nrows + 1)
    int* ccol;          // output col_idx
    void* cval;         // output values
    unsigned long long ncols_inv;  // floor(2^63 / ncols), for bucket maps
};

// kernel variants: team size and capacity (products per team); variant 9,
// a warp holding 384, sits between 3 and 4, and variant 10, one thread per
// row holding 16, below 0 (appended to keep indices stable).  Variants 5-8
// are block teams with the rank-in-bucket accumulator (rows.cuh), variants
// 11-14 block teams of 4, 8, 16, 32 warps running the warp counting sort
// across the block (rows_team.cuh): a second accumulator kind for the same
// capacities, 1024 to 8192.  Variant 15, a warp holding 320 (10 per lane),
// sits between 3 and 9: rows just above 256 products (the trident grid's
// rows scatter around 256) without the 384 variant's register and shared
// memory cost.
// Variants 16-19 are the block teams 11-14 with their B rows staged in
// shared memory by TMA bulk copies (rows_team.cuh).
constexpr int kNumVariants = 20;
__host__ __device__ constexpr bool variant_is_staged(int v) { return v >= 16 && v <= 19; }
__host__ __device__ constexpr bool variant_is_team(int v) { return (v >= 11 && v <= 14) || variant_is_staged(v); }
__host__ __device__ constexpr int variant_team(int v) {
    return variant_is_team(v) ? (128 << (variant_is_staged(v) ? v - 16 : v - 11))
                              : (v == 10 ? 1 : ((v <= 4 || v == 9 || v == 15) ? 32
                                                                             : (v == 5 ? 128 : (v == 6 ? 256 : 512))));
}
__host__ __device__ constexpr int variant_per(int v) {
    return variant_is_team(v) ? 8
                              : (v == 15 ? 10 : (v == 10 ? 16 : (v <= 4 ? (1 << v) : (v == 9 ? 12 : (v == 8 ? 16 : 8)))));
}
constexpr int kThreadRows = 256;  // rows (threads) per block of the thread-per-row variant
// largest power of two <= x (x >= 1)
__host__ __device__ constexpr int pow2floor_c(int x) { return x <= 1 ? 1 : 2 * pow2floor_c(x / 2); }
__host__ __device__ constexpr int variant_cap(int v) { return variant_team(v) * variant_per(v); }
constexpr int kMaxCap = 8192;
constexpr int kMaxBins = 12;
constexpr int kMaxGroupInst = 64;

struct BinTable {
    int nbins;
    int upper[kMaxBins];   // product-count upper bound per bin
    int amax[kMaxBins];    // A-row length bound per bin (capacity / 2)
};
// bin ids: 0..nbins-1 regular, nbins = heavy, nbins + 1 = empty
// (heavy and empty always follow the regular bins)

// status bits latched by kernels
enum : unsigned {
    kStatusInternal = 1u,      // a row produced a different count than row_ptr says
    kStatusHashOverflow = 2u,  // a probe sequence ran past the table size
    kStatusNotCanonical = 4u,  // validation failed
    kStatusTimeout = 8u,       // a bounded device wait ran out
    kStatusCapacity = 16u,     // output capacity exceeded
    kStatusBadMap = 32u,       // a row or column map is not a permutation
};

// single-pass product: ticket counter and look-back state (rows.cuh)
constexpr int kLookbackSpinLimit = 1 << 22;  // default cap on the polls of one look-back wait

struct FusedCtl {
    int* ticket;                 // next tile of rows to hand out
    unsigned long long* lb;      // per tile: flag << 62 | value
    long long cap;               // entries the output can hold
    int nunits;                  // rows
    int* crp;                    // output row_ptr (nunits + 1)
    int spin_limit;              // polls a look-back makes before it reports a timeout
    int hold_tile;               // fault injection: this tile never publishes its entry (-1: none)
};

// ------------------------------------------------------------------- helpers

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int pow2ceil(int x) {
    return x <= 1 ? 1 : 1 << (32 - __clz(x - 1));
}

// group of a unit: last g with unit_base[g] <= unit
__device__ __forceinline__ int unit_group(const long long* __restrict__ unit_base, int ngroups,
                                          long long unit) {
    if (ngroups == 1) return 0;
    int lo = 0, hi = ngroups;  // unit_base[lo] <= unit < unit_base[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(unit_base + mid) <= unit) lo = mid; else hi = mid;
    }
    return lo;
}

// Team primitives.  TEAM == 32: one warp is a team (several teams per
// block); otherwise the whole block (blockDim.x == TEAM) is one team and
// `scratch` points at >= 33 ints of shared memory private to the team.
template <int TEAM>
struct Team {
    static __device__ __forceinline__ int rank() { return TEAM == 32 ? (threadIdx.x & 31) : threadIdx.x; }
    static __device__ __forceinline__ void sync() {
        if (TEAM == 32) __syncwarp(); else __syncthreads();
    }
    // exclusive prefix sum of v over the team; *total receives the sum
    static __device__ __forceinline__ int scan_excl(int v, int* total, int* scratch) {
        const int lane = threadIdx.x & 31;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (TEAM == 32) {
            *total = __shfl_sync(0xffffffffu, x, 31);
            return x - v;
        } else {
            const int warp = threadIdx.x >> 5;
            constexpr int NW = TEAM / 32;
            if (lane == 31) scratch[warp] = x;
            __syncthreads();
            if (warp == 0) {
                int w = lane < NW ? scratch[lane] : 0;
                int z = w;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int y = __shfl_up_sync(0xffffffffu, z, o);
                    if (lane >= o) z += y;
                }
                if (lane < NW) scratch[lane] = z - w;
                if (lane == 31) scratch[32] = z;
            }
            __syncthreads();
            int r = scratch[warp] + x - v;
            *total = scratch[32];
            __syncthreads();
            return r;
        }
    }
    static __device__ __forceinline__ int sum(int v, int* scratch) {
        int t;
        scan_excl(v, &t, scratch);
        return t;
    }
    // exclusive count of set flags and the total, for one flag per thread
    static __device__ __forceinline__ int count_excl(bool f, int* total, int* scratch) {
        if (TEAM == 32) {
            unsigned b = __ballot_sync(0xffffffffu, f);
            *total = __popc(b);
            return __popc(b & lanemask_lt());
        }
        return scan_excl(f ? 1 : 0, total, scratch);
    }
};

// Bucket of a column for a row with NB buckets: monotone in col, in [0, NB).
// With inv = floor(2^63 / ncols) and nb = 2^e <= 2^31, mul = floor(2^(32+e) /
// ncols) = inv >> (31 - e) exactly, and col -> floor(col * mul / 2^32) maps
// [0, ncols) monotonically onto [0, nb).
struct Bucketer {
    unsigned mul;
    bool direct;
    __device__ __forceinline__ void init(int ncols, unsigned long long inv, int nb) {
        direct = ncols <= nb;
        mul = direct ? 0u : (unsigned)(inv >> __clz(nb));  // shift 31 - e
    }
    __device__ __forceinline__ int operator()(int col) const {
        return direct ? col : (int)__umulhi((unsigned)col, mul);
    }
};

template <typename T> __device__ __forceinline__ T mul_rn(T a, T b);
template <> __device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }
template <> __device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <typename T> __device__ __forceinline__ T add_rn(T a, T b);
template <> __device__ __forceinline__ double add_rn<double>(double a, double b) { return __dadd_rn(a, b); }
template <> __device__ __forceinline__ float add_rn<float>(float a, float b) { return __fadd_rn(a, b); }

}  // namespace tsg
