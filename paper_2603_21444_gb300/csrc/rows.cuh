// Row kernels of the local product (paper Sec. 2, Sec. 4.4) for sm_103a.
//
// One team (a warp, or a block for the larger variants) owns one output row
// (a work unit) at a time and keeps the whole row on chip:
//
//   meta    for every entry k of the row's A rows (all instances of the
//           group, in order): a pointer to B row k, a_ik, and the exclusive
//           prefix of |B_k|; this flattens the row's u products; thread r
//           owns products [r*PER, r*PER + PER) and walks them in order.
//   symbolic  the product columns go into a shared-memory hash set (linear
//           probing, 4 * pow2ceil(u) slots); the count of first insertions
//           is nnz(C_i).
//   numeric   deterministic sort accumulator: each product is keyed by
//           (column, p); a counting sort over NB = 2 pow2ceil(u) buckets (the
//           bucket is a monotone function of the column) followed by a rank
//           inside each bucket gives the products in (column, p) order; each
//           run of equal columns is then added in p order, i.e. in ascending
//           (instance, k) order, each instance's products first.  No floating
//           point atomics; the result does not depend on the variant or the
//           launch shape.
//
// Rows whose products or A entries exceed the largest variant go to the
// heavy path: one block per row, a shared-memory bitmap over a column chunk
// and (numeric) a dense accumulator in global memory updated with atomic adds.
#pragma once

#include "common.cuh"

namespace tsg {

struct RowArgs {
    const InstDev* __restrict__ inst;
    const GroupDev* __restrict__ groups;
    const long long* __restrict__ unit_base;
    int ngroups;
    const int* __restrict__ list;     // unit ids, grouped by bin
    const int* __restrict__ bin_off;  // bin b owns list[bin_off[b] .. bin_off[b+1])
    int bin;
    int merge;                        // nonzero: instances are partials to add
    unsigned* status;
    int* counts;                      // symbolic: per-unit row nnz
    int* tick;                        // numeric warp teams: per-bin row tickets, zero at launch
    int* glist;                       // numeric: rows deferred to the grouped kernel (null: none)
    int* gcount;                      // their count, zero at launch
};

__device__ __forceinline__ int search_pre(const int* m_pre, int nA, int p) {
    int lo = 0, hi = nA;  // m_pre[lo] <= p < m_pre[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (m_pre[mid] <= p) lo = mid; else hi = mid;
    }
    return lo;
}

// Flatten the row's A entries (over the group's instances).  Team-uniform
// results nA, u.  Returns false if the row exceeds the team's capacity
// (which the binning rules out unless the inputs changed under it).
template <int TEAM, bool VALS, typename T>
__device__ __forceinline__ bool build_meta(const RowArgs& a, const GroupDev& G, int rho, int maxa, int cap,
                                           const int** m_bc, const T** m_bv, T* m_a, int* m_pre,
                                           unsigned char* m_inst, int* scratch, int& nA, int& u) {
    const int r = Team<TEAM>::rank();
    nA = 0;
    u = 0;
    for (int t = 0; t < G.inst_count; ++t) {
        const InstDev& I = a.inst[G.inst_begin + t];
        const int* brp = I.brp;
        int a0 = 0, a1 = 1;
        if (!a.merge) {
            a0 = __ldg(I.arp + rho);
            a1 = __ldg(I.arp + rho + 1);
        }
        for (int e0 = a0; e0 < a1; e0 += TEAM) {
            const int e = e0 + r;
            const bool valid = e < a1;
            int len = 0, bs = 0;
            T av = T(1);
            if (valid) {
                const int k = a.merge ? rho : __ldg(I.acol + e);
                bs = __ldg(brp + k);
                len = __ldg(brp + k + 1) - bs;
                if (VALS && !a.merge) av = __ldg(reinterpret_cast<const T*>(I.aval) + e);
            }
            int tot;
            const int ex = Team<TEAM>::scan_excl(len, &tot, scratch);
            const int idx = nA + (e - e0);
            if (valid && idx < maxa) {
                m_bc[idx] = I.bcol + bs;
                if (VALS) {
                    m_bv[idx] = reinterpret_cast<const T*>(I.bval) + bs;
                    m_a[idx] = av;
                    m_inst[idx] = (unsigned char)t;
                }
                m_pre[idx] = u + ex;
            }
            nA += min(TEAM, a1 - e0);
            u += tot;
        }
    }
    const bool ok = nA <= maxa && u <= cap;
    if (ok && r == 0) m_pre[nA] = u;
    Team<TEAM>::sync();
    return ok;
}

// ------------------------------------------------------------------ symbolic

template <int CAP>
struct SymLayout {
    static constexpr int MAXA = CAP / 2;
    static constexpr int TBL = 4 * CAP;                           // hash slots (load <= 1/4)
    static constexpr int table = 0;                               // int[TBL]
    static constexpr int m_bc = table + 4 * TBL;                  // const int*[MAXA]
    static constexpr int m_pre = m_bc + 8 * MAXA;                 // int[MAXA + 1]
    static constexpr int scratch = (m_pre + 4 * (MAXA + 1) + 15) & ~15;  // int[34]
    static constexpr int bytes = (scratch + 34 * 4 + 15) & ~15;
    static_assert(bytes <= 227 * 1024, "team layout exceeds shared memory");
};

template <int TEAM, int PER>
__device__ __forceinline__ void sym_row(const RowArgs& a, int unit, char* sm) {
    constexpr int CAP = TEAM * PER;
    using L = SymLayout<CAP>;
    int* table = reinterpret_cast<int*>(sm + L::table);
    const int** m_bc = reinterpret_cast<const int**>(sm + L::m_bc);
    int* m_pre = reinterpret_cast<int*>(sm + L::m_pre);
    int* scratch = reinterpret_cast<int*>(sm + L::scratch);
    const int r = Team<TEAM>::rank();
    const int g = unit_group(a.unit_base, a.ngroups, unit);
    const GroupDev& G = a.groups[g];
    const int rho = (int)(unit - a.unit_base[g]);
    int nA, u;
    if (!build_meta<TEAM, false, float>(a, G, rho, L::MAXA, CAP, m_bc, nullptr, nullptr, m_pre, nullptr,
                                        scratch, nA, u)) {
        if (r == 0) {
            atomicOr(a.status, kStatusInternal);
            a.counts[unit] = 0;
        }
        return;
    }
    const int T2 = 4 * pow2ceil(u);
    const int shift = 32 - (31 - __clz(T2));
    for (int i = 4 * r; i < T2; i += 4 * TEAM) *reinterpret_cast<int4*>(table + i) = make_int4(-1, -1, -1, -1);
    // thread r owns products [r*PER, r*PER + PER): one search, then walk
    int cols[PER];
    {
        const int p0 = r * PER;
        int t = 0, tb = 0, te = 0;
        const int* bc = nullptr;
        if (p0 < u) {
            t = search_pre(m_pre, nA, p0);
            tb = m_pre[t];
            te = m_pre[t + 1];
            bc = m_bc[t];
        }
#pragma unroll
        for (int s = 0; s < PER; ++s) {
            const int p = p0 + s;
            cols[s] = -1;
            if (p < u) {
                while (p >= te) {
                    ++t;
                    tb = te;
                    te = m_pre[t + 1];
                    bc = m_bc[t];
                }
                cols[s] = __ldg(bc + (p - tb));
            }
        }
    }
    Team<TEAM>::sync();
    int fresh = 0;
    bool overflow = false;
#pragma unroll
    for (int s = 0; s < PER; ++s) {
        const int c = cols[s];
        if (c >= 0) {
            unsigned h = ((unsigned)c * 0x9E3779B1u) >> shift;
            int probe = 0;
            for (; probe < T2; ++probe) {
                const int old = atomicCAS(&table[h], -1, c);
                if (old == -1) { ++fresh; break; }
                if (old == c) break;
                h = (h + 1) & (T2 - 1);
            }
            overflow |= probe == T2;
        }
    }
    if (overflow) atomicOr(a.status, kStatusHashOverflow);
    const int total = Team<TEAM>::sum(fresh, scratch);
    if (r == 0) a.counts[unit] = total;
    Team<TEAM>::sync();
}

// ------------------------------------------------- coalesced warp gather
//
// A warp team's products are read in chunks of 4: lane L takes chunk
// s*32 + L (s = 0 .. PER/4 - 1), i.e. products [4(s*32+L), 4(s*32+L) + 4), so
// one warp instruction covers 128 consecutive products.  A chunk that lies in
// one B row and starts on a 16-byte boundary is read with 16-byte loads;
// otherwise element by element.  Product slot e of the lane holds product
// p = 4 (32 (e / 4) + L) + e % 4.

// When PER is not a multiple of 4 (the 320-product variant, PER = 10) the
// last PER % 4 slots form a narrower tail chunk after the 4-wide ones: lane L
// takes products 128 (PER / 4) + R L + v, v < R = PER % 4.
template <int PER>
__device__ __forceinline__ int chunk_product(int lane, int e) {
    constexpr int W = PER < 4 ? PER : 4;
    constexpr int NC = PER / W, R = PER - NC * W;
    if (R > 0 && e >= NC * W) return 32 * W * NC + R * lane + (e - NC * W);
    return W * (32 * (e / W) + lane) + e % W;
}

template <typename T>
struct Vec2 {};
template <>
struct Vec2<double> {
    // p is 16-byte aligned.  At a 32-byte boundary one 256-bit load takes the
    // lane's whole sector; two 128-bit loads would request it twice.
    static __device__ __forceinline__ void load4(const double* p, double* out) {
        if ((reinterpret_cast<uintptr_t>(p) & 31) == 0) {
            asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
                : "=d"(out[0]), "=d"(out[1]), "=d"(out[2]), "=d"(out[3])
                : "l"(p));
        } else {
            const double2 a = __ldg(reinterpret_cast<const double2*>(p));
            const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
            out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
        }
    }
};
template <>
struct Vec2<float> {
    static __device__ __forceinline__ void load4(const float* p, float* out) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p));
        out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
    }
};

// Owner entry of product p: the last t with m_pre[t] <= p.
__device__ __forceinline__ int owner_of(const int* m_pre, int nA, int p) {
    int lo = 0, hi = nA;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (m_pre[mid] <= p) lo = mid; else hi = mid;
    }
    return lo;
}

// col[e] = column of the lane's e-th product (-1 past u); with VALS,
// val[e] = a_ik * b_kj (merge: b_kj) and ins[e] = its instance.  The warp
// covers products [pbase, pbase + 32 PER) of the row (pbase = 0 for a warp
// team; warp w of a block team takes pbase = 32 PER w).
template <int PER, bool VALS, typename T>
__device__ __forceinline__ void gather_chunks(const RowArgs& a, int ib, int nA, int u, const int* m_pre,
                                              const int* m_bs, const T* m_a, const unsigned char* m_inst, int lane,
                                              int (&col)[PER], T (&val)[PER], int (&ins)[PER], int pbase = 0) {
    constexpr int W = PER < 4 ? PER : 4;  // chunk width
    constexpr int NC = PER / W, R = PER - NC * W;
    if constexpr (R > 0) {
        // tail chunk (PER % 4 products per lane), element by element
        const int pt = pbase + 32 * W * NC + R * lane;
#pragma unroll
        for (int v = 0; v < R; ++v) {
            const int e = NC * W + v;
            col[e] = -1;
            if (VALS) val[e] = T(0);
            ins[e] = 0;
            const int p = pt + v;
            if (p < u) {
                const int t = owner_of(m_pre, nA, p);
                const int ti = m_inst[t];
                const InstDev* I = a.inst + ib + ti;
                const int f = m_bs[t] + (p - m_pre[t]);
                col[e] = __ldg(I->bcol + f);
                if (VALS) {
                    const T bv = __ldg(reinterpret_cast<const T*>(I->bval) + f);
                    val[e] = a.merge ? bv : mul_rn(m_a[t], bv);
                }
                ins[e] = ti;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int p0 = pbase + W * (32 * c + lane);
#pragma unroll
        for (int v = 0; v < W; ++v) {
            col[W * c + v] = -1;
            if (VALS) val[W * c + v] = T(0);
            ins[W * c + v] = 0;
        }
        if (p0 >= u) continue;
        int t = owner_of(m_pre, nA, p0);
        int tb = m_pre[t], te = m_pre[t + 1];
        int ti = m_inst[t];
        const InstDev* I = a.inst + ib + ti;
        const int* bcol = I->bcol;
        const T* bval = reinterpret_cast<const T*>(I->bval);
        const int f0 = m_bs[t] + (p0 - tb);
        T av = VALS ? m_a[t] : T(1);
        if (W == 4 && p0 + 4 <= te && ((reinterpret_cast<uintptr_t>(bcol + f0) & 15) == 0) &&
            (!VALS || (reinterpret_cast<uintptr_t>(bval + f0) & 15) == 0)) {
            const int4 cc = __ldg(reinterpret_cast<const int4*>(bcol + f0));
            col[W * c + 0] = cc.x;
            col[W * c + (W > 1 ? 1 : 0)] = W > 1 ? cc.y : cc.x;
            col[W * c + (W > 2 ? 2 : 0)] = W > 2 ? cc.z : cc.x;
            col[W * c + (W > 3 ? 3 : 0)] = W > 3 ? cc.w : cc.x;
            if (VALS) {
                T bv[4];
                Vec2<T>::load4(bval + f0, bv);
#pragma unroll
                for (int v = 0; v < W; ++v) val[W * c + v] = a.merge ? bv[v] : mul_rn(av, bv[v]);
            }
#pragma unroll
            for (int v = 0; v < W; ++v) ins[W * c + v] = ti;
        } else if (W == 4 && p0 + 4 <= te) {
            // one B row, not 16-byte aligned: four independent element loads
#pragma unroll
            for (int v = 0; v < W; ++v) {
                col[W * c + v] = __ldg(bcol + f0 + v);
                if (VALS) {
                    const T bv = __ldg(bval + f0 + v);
                    val[W * c + v] = a.merge ? bv : mul_rn(av, bv);
                }
                ins[W * c + v] = ti;
            }
        } else {
#pragma unroll
            for (int v = 0; v < W; ++v) {
                const int p = p0 + v;
                if (p < u) {
                    while (p >= te) {
                        ++t;
                        tb = te;
                        te = m_pre[t + 1];
                        if (VALS) av = m_a[t];
                        const int tn = m_inst[t];
                        if (tn != ti) {
                            ti = tn;
                            I = a.inst + ib + ti;
                            bcol = I->bcol;
                            bval = reinterpret_cast<const T*>(I->bval);
                        }
                    }
                    const int f = m_bs[t] + (p - tb);
                    col[W * c + v] = __ldg(bcol + f);
                    if (VALS) {
                        const T bv = __ldg(bval + f);
                        val[W * c + v] = a.merge ? bv : mul_rn(av, bv);
                    }
                    ins[W * c + v] = ti;
                }
            }
        }
    }
}

// ------------------------------------------------- warp-team row meta
//
// Per A entry of the row (over the group's instances, instance by instance,
// entries in stored order): its first product (prefix of the B-row
// lengths), its B-row offset, a_ik (VALS) and its instance; nA and u for the
// row.  Entries beyond MAXA are counted but not stored (the caller rejects
// the row).  A row of several instances with at most 32 A entries in all
// takes one round of loads -- lane t reads instance t's bounds, then lane L
// its own A entry -- instead of one round of dependent loads per instance;
// the entries keep the same order, so nothing downstream changes.
template <bool VALS, typename T, int MAXA>
__device__ __forceinline__ void warp_meta(const RowArgs& a, int ib, int icount, int rho, int lane, int* m_pre,
                                          int* m_bs, T* m_a, unsigned char* m_inst, int& nA, int& u) {
    nA = 0;
    u = 0;
    if (icount > 1 && icount <= 32) {
        int ia0 = 0, ilen = 0;
        if (lane < icount) {
            const InstDev& I = a.inst[ib + lane];
            if (a.merge) {
                ilen = 1;
            } else {
                ia0 = __ldg(I.arp + rho);
                ilen = __ldg(I.arp + rho + 1) - ia0;
            }
        }
        int ix = ilen;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, ix, o);
            if (lane >= o) ix += y;
        }
        const int total = __shfl_sync(0xffffffffu, ix, 31);
        if (total <= 32) {
            int t = 0, e = 0;
            for (int q = 0; q < icount; ++q) {
                const int st = __shfl_sync(0xffffffffu, ix - ilen, q);
                const int ln = __shfl_sync(0xffffffffu, ilen, q);
                const int b0 = __shfl_sync(0xffffffffu, ia0, q);
                if (lane >= st && lane < st + ln) {
                    t = q;
                    e = b0 + (lane - st);
                }
            }
            const bool valid = lane < total;
            int len = 0, bs = 0;
            T av = T(1);
            if (valid) {
                const InstDev& I = a.inst[ib + t];
                const int k = a.merge ? rho : __ldg(I.acol + e);
                bs = __ldg(I.brp + k);
                len = __ldg(I.brp + k + 1) - bs;
                if (VALS && !a.merge) av = __ldg(reinterpret_cast<const T*>(I.aval) + e);
            }
            int x = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (valid && lane < MAXA) {
                m_pre[lane] = x - len;
                m_bs[lane] = bs;
                if (VALS) m_a[lane] = av;
                m_inst[lane] = (unsigned char)t;
            }
            nA = total;
            u = __shfl_sync(0xffffffffu, x, 31);
            return;
        }
    }
    for (int t = 0; t < icount; ++t) {
        const InstDev& I = a.inst[ib + t];
        int a0 = 0, a1 = 1;
        if (!a.merge) {
            a0 = __ldg(I.arp + rho);
            a1 = __ldg(I.arp + rho + 1);
        }
        for (int e0 = a0; e0 < a1; e0 += 32) {
            const int e = e0 + lane;
            const bool valid = e < a1;
            int len = 0, bs = 0;
            T av = T(1);
            if (valid) {
                const int k = a.merge ? rho : __ldg(I.acol + e);
                bs = __ldg(I.brp + k);
                len = __ldg(I.brp + k + 1) - bs;
                if (VALS && !a.merge) av = __ldg(reinterpret_cast<const T*>(I.aval) + e);
            }
            int x = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            const int idx = nA + lane;
            if (valid && idx < MAXA) {
                m_pre[idx] = u + x - len;
                m_bs[idx] = bs;
                if (VALS) m_a[idx] = av;
                m_inst[idx] = (unsigned char)t;
            }
            nA += min(32, a1 - e0);
            u += __shfl_sync(0xffffffffu, x, 31);
        }
    }
}

// ------------------------------------------------- strided warp gather
//
// For rows of at most 32 A entries whose B rows are short, a chunk of 4
// would often straddle two B rows or start off a 16-byte boundary and fall
// back to element loads.  There lane L takes product p = 32 s + L in slot s
// instead: one warp instruction reads 32 consecutive products, i.e. whole
// B rows, coalesced whatever their lengths and alignment.  Lane t holds A
// entry t (first product, B-row pointers, a value, instance) in registers.
// In each round of 32 products the entries starting inside the round set
// one bit each of a mask; the owner of product p is the entry with the
// highest start at or below p, else the owner carried over from the
// previous round, and its fields come from lane t by shuffles.

constexpr int kStridedMaxAvg = 16;  // strided when the mean B-row length is below this

template <int PER>
__device__ __forceinline__ bool use_strided(int nA, int u) {
    return PER >= 4 && nA <= 32 && u < kStridedMaxAvg * nA;
}

// owner_at: 32 ints of the warp's shared memory, free during the gather.
template <int PER, bool VALS, typename T>
__device__ __forceinline__ void gather_strided(const RowArgs& a, int ib, int nA, int u, const int* m_pre,
                                               const int* m_bs, const T* m_a, const unsigned char* m_inst,
                                               int* owner_at, int lane, int (&col)[PER], T (&val)[PER],
                                               int (&ins)[PER]) {
    constexpr int kNone = 0x7fffffff;  // start of an entry that owns no product
    int e_start = kNone, e_ins = 0;
    unsigned long long e_col = 0, e_val = 0;
    T e_av = T(0);
    if (lane < nA) {
        const int s0 = m_pre[lane];
        if (m_pre[lane + 1] > s0) e_start = s0;
        e_ins = m_inst[lane];
        const InstDev& I = a.inst[ib + e_ins];
        const int bs = m_bs[lane];
        e_col = reinterpret_cast<unsigned long long>(I.bcol + bs);
        if (VALS) {
            e_val = reinterpret_cast<unsigned long long>(reinterpret_cast<const T*>(I.bval) + bs);
            e_av = m_a[lane];
        }
    }
    int carry = 0;
#pragma unroll
    for (int s = 0; s < PER; ++s) {
        col[s] = -1;
        if (VALS) val[s] = T(0);
        ins[s] = 0;
        const int base = 32 * s;
        if (base >= u) continue;
        const int rel = e_start - base;
        const bool head = rel >= 0 && rel < 32;
        const unsigned heads = __reduce_or_sync(0xffffffffu, head ? 1u << rel : 0u);
        if (head) owner_at[rel] = lane;
        __syncwarp();
        const unsigned below = heads & (0xffffffffu >> (31 - lane));
        const int t = below ? owner_at[31 - __clz(below)] : carry;
        __syncwarp();
        carry = __shfl_sync(0xffffffffu, t, 31);
        const int ts = __shfl_sync(0xffffffffu, e_start, t);
        const unsigned long long cp = __shfl_sync(0xffffffffu, e_col, t);
        const int ti = __shfl_sync(0xffffffffu, e_ins, t);
        unsigned long long vp = 0;
        T av = T(0);
        if (VALS) {
            vp = __shfl_sync(0xffffffffu, e_val, t);
            av = __shfl_sync(0xffffffffu, e_av, t);
        }
        const int p = base + lane;
        if (p < u) {
            const int off = p - ts;
            col[s] = __ldg(reinterpret_cast<const int*>(cp) + off);
            if (VALS) {
                const T bv = __ldg(reinterpret_cast<const T*>(vp) + off);
                val[s] = a.merge ? bv : mul_rn(av, bv);
            }
            ins[s] = ti;
        }
    }
}

// ------------------------------------------------ symbolic, warp-team variant
//
// nnz(C_i) = u - (products whose column an earlier product already has).
// Every product sets one bit, chosen by a multiplicative hash of its column,
// of a shared-memory bitmap of 64 pow2ceil(u) bits (at most kSymBitsMax); a
// product that finds its bit already set is FLAGGED.  The first product to
// reach a bit is never flagged, so unflagged products have pairwise distinct
// columns (two of them would have met on one bit).  A flagged product f
// repeats an earlier column exactly when some other product g has f's
// column and g is unflagged, or flagged with a smaller index: in a column
// group of m products that counts m - 1 whether or not one of them is
// unflagged, and 0 for a lone product flagged by another column's bit.  The
// warp checks each flagged product -- about u / 128 per row besides true
// repeats -- against all u products with one ballot.  Exact for any hash.
// The meta keeps B-row offsets (4 B) instead of pointers and shares the
// bitmap's storage while the products are gathered.

constexpr int kSymBitsMax = 32768;
constexpr int kSymMaxFlagged = 32;  // more flagged products in a row: count with a hash set

template <int CAP>
struct WSymLayout {
    static constexpr int MAXA = CAP / 2;
    static constexpr int BITS = 64 * pow2floor_c(2 * CAP - 1) < kSymBitsMax ? 64 * pow2floor_c(2 * CAP - 1)
                                                                          : kSymBitsMax;  // 64 pow2ceil(CAP)
    static constexpr int bm = 0;                                   // u32[BITS / 32]
    static constexpr int m_pre = 0;                                // int[MAXA + 1] (aliases the bitmap)
    static constexpr int m_bs = m_pre + 4 * (MAXA + 1);            // int[MAXA]
    static constexpr int m_inst = m_bs + 4 * MAXA;                 // u8[MAXA]
    static constexpr int alias_end = (m_inst + MAXA) > BITS / 8 ? (m_inst + MAXA) : BITS / 8;
    static constexpr int owner = (alias_end + 15) & ~15;           // int[32] strided-gather scratch
    static constexpr int bytes = owner + 4 * 32;
    static_assert(BITS % 128 == 0, "bitmap cleared in 16-byte stores");
};

template <int PER>
__device__ __forceinline__ void sym_row_warp(const RowArgs& a, int unit, char* sm) {
    constexpr int CAP = 32 * PER;
    using L = WSymLayout<CAP>;
    static_assert(L::BITS >= 64 * pow2floor_c(2 * CAP - 1), "the fallback hash set needs 2 slots per product");
    unsigned* bm = reinterpret_cast<unsigned*>(sm + L::bm);
    int* m_pre = reinterpret_cast<int*>(sm + L::m_pre);
    int* m_bs = reinterpret_cast<int*>(sm + L::m_bs);
    unsigned char* m_inst = reinterpret_cast<unsigned char*>(sm + L::m_inst);
    const int lane = threadIdx.x & 31;
    const int g = unit_group(a.unit_base, a.ngroups, unit);
    const GroupDev& G = a.groups[g];
    const int rho = (int)(unit - a.unit_base[g]);
    const int ib = G.inst_begin, icount = G.inst_count;

    int nA, u;
    warp_meta<false, float, L::MAXA>(a, ib, icount, rho, lane, m_pre, m_bs, nullptr, m_inst, nA, u);
    if (nA > L::MAXA || u > CAP) {
        if (lane == 0) {
            atomicOr(a.status, kStatusInternal);
            a.counts[unit] = 0;
        }
        __syncwarp();
        return;
    }
    if (lane == 0) m_pre[nA] = u;
    __syncwarp();

    int col[PER];
    {
        float unused_val[PER];
        int unused_ins[PER];
        if (use_strided<PER>(nA, u))
            gather_strided<PER, false, float>(a, ib, nA, u, m_pre, m_bs, nullptr, m_inst,
                                              reinterpret_cast<int*>(sm + L::owner), lane, col, unused_val,
                                              unused_ins);
        else
            gather_chunks<PER, false, float>(a, ib, nA, u, m_pre, m_bs, nullptr, m_inst, lane, col, unused_val,
                                             unused_ins);
    }
    __syncwarp();  // the meta is dead: the bitmap takes its place
    const int nbits = min(64 * pow2ceil(u), L::BITS);
    const int shift = 32 - (31 - __clz(nbits));
    for (int i = 4 * lane; i < nbits / 32; i += 128) *reinterpret_cast<int4*>(bm + i) = make_int4(0, 0, 0, 0);
    __syncwarp();
    unsigned flagged = 0;  // bit s: the lane's product in slot s found its bit set
#pragma unroll
    for (int s = 0; s < PER; ++s)
        if (col[s] >= 0) {
            const unsigned h = ((unsigned)col[s] * 0x9E3779B1u) >> shift;
            const unsigned bit = 1u << (h & 31);
            if (atomicOr(bm + (h >> 5), bit) & bit) flagged |= 1u << s;
        }
    // A row that repeats its columns heavily flags most of its products; past
    // kSymMaxFlagged the warp counts the distinct columns with a hash set
    // instead (linear probing over 2 pow2ceil(u) slots, in the bitmap's
    // storage: 64 bits per product leave room for two 32-bit slots).
    int nflag = __popc(flagged);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nflag += __shfl_xor_sync(0xffffffffu, nflag, o);
    if (nflag > kSymMaxFlagged) {
        int* table = reinterpret_cast<int*>(bm);
        const int T2 = 2 * pow2ceil(u);
        const int tshift = 32 - (31 - __clz(T2));
        __syncwarp();
        for (int i = lane; i < T2; i += 32) table[i] = -1;
        __syncwarp();
        int fresh = 0;
        bool overflow = false;
#pragma unroll
        for (int s = 0; s < PER; ++s) {
            const int c = col[s];
            if (c >= 0) {
                unsigned h = ((unsigned)c * 0x9E3779B1u) >> tshift;
                int probe = 0;
                for (; probe < T2; ++probe) {
                    const int old = atomicCAS(&table[h], -1, c);
                    if (old == -1) {
                        ++fresh;
                        break;
                    }
                    if (old == c) break;
                    h = (h + 1) & (unsigned)(T2 - 1);
                }
                overflow |= probe == T2;
            }
        }
        if (overflow) atomicOr(a.status, kStatusHashOverflow);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fresh += __shfl_xor_sync(0xffffffffu, fresh, o);
        if (lane == 0) a.counts[unit] = fresh;
        __syncwarp();
        return;
    }
    // each flagged product against every product of the row (index s * 32 + lane)
    int dup = 0;
#pragma unroll
    for (int s = 0; s < PER; ++s) {
        unsigned m = __ballot_sync(0xffffffffu, (flagged >> s) & 1u);
        while (m) {
            const int fl = __ffs(m) - 1;
            m &= m - 1;
            const int cf = __shfl_sync(0xffffffffu, col[s], fl);
            const int idf = 32 * s + fl;
            bool hit = false;
#pragma unroll
            for (int t = 0; t < PER; ++t) {
                const int id = 32 * t + lane;
                hit |= col[t] == cf && id != idf && (((flagged >> t) & 1u) == 0 || id < idf);
            }
            dup += __any_sync(0xffffffffu, hit) ? 1 : 0;
        }
    }
    if (lane == 0) a.counts[unit] = u - dup;
    __syncwarp();
}

template <int TEAM, int PER>
__global__ void __launch_bounds__(TEAM == 32 ? (PER <= 12 ? 256 : 512) : TEAM,
                                    TEAM == 32 && PER <= 12 ? (PER == 12 ? 3 : 5) : 1) k_sym_rows(RowArgs a) {
    extern __shared__ __align__(16) char smem[];
    constexpr int CAP = TEAM * PER;
    const int begin = a.bin_off[a.bin], end = a.bin_off[a.bin + 1];
    int team, nteams;
    char* sm;
    if (TEAM == 32) {
        const int w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
        team = blockIdx.x * wpb + w;
        nteams = gridDim.x * wpb;
        sm = smem + w * WSymLayout<CAP>::bytes;
    } else {
        team = blockIdx.x;
        nteams = gridDim.x;
        sm = smem;
    }
    if constexpr (TEAM == 32) {
        // the next row's id is loaded before the current row starts
        int i = begin + team;
        int unit = i < end ? __ldg(a.list + i) : 0;
        for (; i < end; i += nteams) {
            const int next = i + nteams < end ? __ldg(a.list + i + nteams) : 0;
            sym_row_warp<PER>(a, unit, sm);
            unit = next;
        }
    } else {
        for (int i = begin + team; i < end; i += nteams) sym_row<TEAM, PER>(a, __ldg(a.list + i), sm);
    }
}

// ------------------------------------------------------------------- numeric

// ------------------------------------------------ thread-per-row variant
//
// Rows of at most 16 products (short A rows over short B rows: a
// restriction operator, ER with a handful of entries per row) leave most of
// a warp idle.  Here one thread takes a whole row: its products, in p order,
// go to its own column of a shared array (entry i of thread t at
// i * kThreadRows + t, so a warp's accesses never share a bank), an
// insertion sort by column that moves only strictly larger columns keeps
// equal columns in p order, and each run is summed in that order (each
// instance's products, then the instance sums in order): the same values
// as every other variant, bit for bit.

constexpr int kThreadCap = 16;

// The row's products in p order into slots i * kThreadRows (col always,
// value and instance with VALS); returns u, or -1 past kThreadCap.  A
// entries are taken 8 at a time with independent loads in three rounds
// (A entries, B-row bounds, every B row's first entry), so a row waits for
// a few memory round trips instead of three per A entry.
constexpr int kThreadBatch = 8;
static_assert(kThreadBatch == 8, "the vector path below loads a batch as two groups of four");

template <bool VALS, typename T>
__device__ __forceinline__ int thread_gather(const RowArgs& a, const GroupDev& G, int rho, int* sc, T* sv,
                                             unsigned char* si) {
    int n = 0;
    for (int q = 0; q < G.inst_count; ++q) {
        const InstDev& I = a.inst[G.inst_begin + q];
        const T* aval = reinterpret_cast<const T*>(I.aval);
        const T* bval = reinterpret_cast<const T*>(I.bval);
        int a0 = 0, a1 = 1;
        if (!a.merge) {
            a0 = __ldg(I.arp + rho);
            a1 = __ldg(I.arp + rho + 1);
        }
        for (int e0 = a0; e0 < a1; e0 += kThreadBatch) {
            int kk[kThreadBatch], b0[kThreadBatch], len[kThreadBatch], c0[kThreadBatch];
            T av[kThreadBatch], v0[kThreadBatch];
            // a whole batch at 16-byte boundaries: vector loads (a thread's
            // entries are contiguous, so this cuts its L1 requests 4 x)
            const bool vec = !a.merge && e0 + kThreadBatch <= a1 &&
                             ((reinterpret_cast<uintptr_t>(I.acol + e0) & 15) == 0) &&
                             (!VALS || (reinterpret_cast<uintptr_t>(aval + e0) & (4 * sizeof(T) - 1)) == 0);
            if (vec) {
                const int4 x0 = __ldg(reinterpret_cast<const int4*>(I.acol + e0));
                const int4 x1 = __ldg(reinterpret_cast<const int4*>(I.acol + e0 + 4));
                kk[0] = x0.x; kk[1] = x0.y; kk[2] = x0.z; kk[3] = x0.w;
                kk[4] = x1.x; kk[5] = x1.y; kk[6] = x1.z; kk[7] = x1.w;
                if (VALS) {
                    Vec2<T>::load4(aval + e0, av);
                    Vec2<T>::load4(aval + e0 + 4, av + 4);
                } else {
#pragma unroll
                    for (int e = 0; e < kThreadBatch; ++e) av[e] = T(1);
                }
            } else {
#pragma unroll
                for (int e = 0; e < kThreadBatch; ++e) {
                    kk[e] = 0;
                    av[e] = T(1);
                    if (e0 + e < a1) {
                        kk[e] = a.merge ? rho : __ldg(I.acol + e0 + e);
                        if (VALS && !a.merge) av[e] = __ldg(aval + e0 + e);
                    }
                }
            }
            int tot = 0;
#pragma unroll
            for (int e = 0; e < kThreadBatch; ++e) {
                b0[e] = 0;
                len[e] = 0;
                if (e0 + e < a1) {
                    b0[e] = __ldg(I.brp + kk[e]);
                    len[e] = __ldg(I.brp + kk[e] + 1) - b0[e];
                }
                tot += len[e];
            }
            if (n + tot > kThreadCap) return -1;
#pragma unroll
            for (int e = 0; e < kThreadBatch; ++e) {
                c0[e] = 0;
                v0[e] = T(0);
                if (len[e] > 0) {
                    c0[e] = __ldg(I.bcol + b0[e]);
                    if (VALS) v0[e] = __ldg(bval + b0[e]);
                }
            }
#pragma unroll
            for (int e = 0; e < kThreadBatch; ++e) {
                if (len[e] == 0) continue;
                sc[n * kThreadRows] = c0[e];
                if (VALS) {
                    sv[n * kThreadRows] = a.merge ? v0[e] : mul_rn(av[e], v0[e]);
                    si[n * kThreadRows] = (unsigned char)q;
                }
                ++n;
                for (int j = 1; j < len[e]; ++j, ++n) {
                    sc[n * kThreadRows] = __ldg(I.bcol + b0[e] + j);
                    if (VALS) {
                        const T bv = __ldg(bval + b0[e] + j);
                        sv[n * kThreadRows] = a.merge ? bv : mul_rn(av[e], bv);
                        si[n * kThreadRows] = (unsigned char)q;
                    }
                }
            }
        }
    }
    return n;
}

// symbolic counts of thread-per-row rows (defined in rows_sym.cu)
__global__ void __launch_bounds__(kThreadRows) k_sym_thread(RowArgs a);

template <typename T>
struct ThreadNumLayout {
    static constexpr int cols = 0;                                          // int[CAP * ROWS]
    static constexpr int vals = 4 * kThreadCap * kThreadRows;               // T[CAP * ROWS]
    static constexpr int inst = vals + (int)sizeof(T) * kThreadCap * kThreadRows;  // u8[CAP * ROWS]
    static constexpr int bytes = inst + kThreadCap * kThreadRows;
};

template <typename T>
__global__ void __launch_bounds__(kThreadRows) k_num_thread(RowArgs a) {
    extern __shared__ __align__(16) char smem[];
    using L = ThreadNumLayout<T>;
    int* sc = reinterpret_cast<int*>(smem + L::cols) + threadIdx.x;
    T* sv = reinterpret_cast<T*>(smem + L::vals) + threadIdx.x;
    unsigned char* si = reinterpret_cast<unsigned char*>(smem + L::inst) + threadIdx.x;
    const int begin = a.bin_off[a.bin], end = a.bin_off[a.bin + 1];
    for (int i = begin + blockIdx.x * kThreadRows + threadIdx.x; i < end; i += gridDim.x * kThreadRows) {
        const int unit = __ldg(a.list + i);
        const int g = unit_group(a.unit_base, a.ngroups, unit);
        const GroupDev& G = a.groups[g];
        const int rho = (int)(unit - a.unit_base[g]);
        const int row_begin = __ldg(G.crp + rho);
        const int row_len = __ldg(G.crp + rho + 1) - row_begin;
        const int n = thread_gather<true, T>(a, G, rho, sc, sv, si);
        if (n < 0) {
            atomicOr(a.status, kStatusInternal);
            continue;
        }
        for (int x = 1; x < n; ++x) {
            const int c = sc[x * kThreadRows];
            const T v = sv[x * kThreadRows];
            const unsigned char q = si[x * kThreadRows];
            int y = x - 1;
            while (y >= 0 && sc[y * kThreadRows] > c) {
                sc[(y + 1) * kThreadRows] = sc[y * kThreadRows];
                sv[(y + 1) * kThreadRows] = sv[y * kThreadRows];
                si[(y + 1) * kThreadRows] = si[y * kThreadRows];
                --y;
            }
            sc[(y + 1) * kThreadRows] = c;
            sv[(y + 1) * kThreadRows] = v;
            si[(y + 1) * kThreadRows] = q;
        }
        const bool multi = a.merge || G.inst_count > 1;
        int out = 0;
        int x = 0;
        while (x < n) {
            const int c = sc[x * kThreadRows];
            T sub = sv[x * kThreadRows], acc = T(0);
            bool have = false;
            int ci = si[x * kThreadRows];
            int y = x + 1;
            for (; y < n && sc[y * kThreadRows] == c; ++y) {
                const T v = sv[y * kThreadRows];
                const int iy = si[y * kThreadRows];
                if (multi && iy != ci) {
                    acc = have ? add_rn(acc, sub) : sub;
                    have = true;
                    sub = v;
                    ci = iy;
                } else {
                    sub = add_rn(sub, v);
                }
            }
            if (out < row_len) {
                __stcs(G.ccol + row_begin + out, c);
                __stcs(reinterpret_cast<T*>(G.cval) + row_begin + out, have ? add_rn(acc, sub) : sub);
            }
            ++out;
            x = y;
        }
        if (out != row_len) atomicOr(a.status, kStatusInternal);
    }
}

// ---------------------------------------------- grouped accumulation
//
// Rows whose products repeat their columns many times over (banded or
// stencil-like inputs: u products onto nnz(C_i) <= u / 4 columns that sit
// next to each other) defeat the bucket sort: a monotone bucket map puts a
// whole cluster of columns into one bucket, and sorting inside crowded
// buckets costs their size squared.  The numeric kernels defer such rows
// (known from the symbolic pass: u >= kGroupedDup nnz(C_i), with few
// columns and A entries) to k_num_grouped: one warp per row keeps one
// accumulator per distinct column in a shared-memory hash table and feeds
// it the products strictly in p order -- 32 at a time, the lanes of one
// column added by their lowest lane in lane (= p) order -- so every entry
// is summed in the same order as the bucket path (each instance's products,
// then the instance sums in order) and the result is identical bit for
// bit.  Only the distinct columns are sorted at the end (bitonic network).

constexpr int kGroupedDup = 4;      // deferred when u >= 4 nnz(C_i)
constexpr int kGroupedMaxD = 128;   // at most this many output columns
constexpr int kGroupedMaxA = 128;   // at most this many A entries (over the row's instances)
constexpr int kGroupedSlots = 2 * kGroupedMaxD;
constexpr int kGroupedWarps = 8;

__device__ __forceinline__ bool grouped_row(const RowArgs& a, int nA, int u, int row_len) {
    return a.glist != nullptr && row_len > 0 && row_len <= kGroupedMaxD && nA <= kGroupedMaxA &&
           u >= kGroupedDup * row_len;
}

template <typename T>
struct GroupedLayout {
    static constexpr int m_pre = 0;                                     // int[MAXA + 1]
    static constexpr int m_bs = m_pre + 4 * (kGroupedMaxA + 1);         // int[MAXA]
    static constexpr int m_a = (m_bs + 4 * kGroupedMaxA + 7) & ~7;      // T[MAXA]
    static constexpr int m_inst = m_a + (int)sizeof(T) * kGroupedMaxA;  // u8[MAXA]
    static constexpr int keys = 0;                                      // u64[MAXD], aliases the meta
    static constexpr int key = (m_inst + kGroupedMaxA + 15) & ~15;      // int[SLOTS] column per slot
    static constexpr int acc = key + 4 * kGroupedSlots;                 // T[SLOTS] sum of finished instances
    static constexpr int sub = acc + (int)sizeof(T) * kGroupedSlots;    // T[SLOTS] running sum of one instance
    static constexpr int st = sub + (int)sizeof(T) * kGroupedSlots;     // int[SLOTS] instance | 256 if acc set
    static constexpr int stage_v = st + 4 * kGroupedSlots;              // T[32] this round's values
    static constexpr int stage_i = stage_v + (int)sizeof(T) * 32;       // int[32] this round's instances
    static constexpr int bytes = (stage_i + 4 * 32 + 15) & ~15;
    static_assert(8 * kGroupedMaxD <= key, "sorted keys must fit the meta region");
    static_assert((acc & 7) == 0 && (stage_v & 7) == 0, "value arrays alignment");
};

template <typename T>
__device__ __forceinline__ void grouped_row_warp(const RowArgs& a, int unit, char* sm) {
    using L = GroupedLayout<T>;
    int* m_pre = reinterpret_cast<int*>(sm + L::m_pre);
    int* m_bs = reinterpret_cast<int*>(sm + L::m_bs);
    T* m_a = reinterpret_cast<T*>(sm + L::m_a);
    unsigned char* m_inst = reinterpret_cast<unsigned char*>(sm + L::m_inst);
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(sm + L::keys);
    int* skey = reinterpret_cast<int*>(sm + L::key);
    T* sacc = reinterpret_cast<T*>(sm + L::acc);
    T* ssub = reinterpret_cast<T*>(sm + L::sub);
    int* sst = reinterpret_cast<int*>(sm + L::st);
    T* stage_v = reinterpret_cast<T*>(sm + L::stage_v);
    int* stage_i = reinterpret_cast<int*>(sm + L::stage_i);

    const int lane = threadIdx.x & 31;
    const int g = unit_group(a.unit_base, a.ngroups, unit);
    const GroupDev& G = a.groups[g];
    const int rho = (int)(unit - a.unit_base[g]);
    const int row_begin = __ldg(G.crp + rho);
    const int row_len = __ldg(G.crp + rho + 1) - row_begin;
    const int ib = G.inst_begin, icount = G.inst_count;

    // meta: first product, B-row offset, a_ik, instance per A entry
    int nA, u;
    warp_meta<true, T, kGroupedMaxA>(a, ib, icount, rho, lane, m_pre, m_bs, m_a, m_inst, nA, u);
    if (nA > kGroupedMaxA || row_len > kGroupedMaxD || row_len <= 0) {
        if (lane == 0) atomicOr(a.status, kStatusInternal);
        __syncwarp();
        return;
    }
    if (lane == 0) m_pre[nA] = u;
    const int T2 = 2 * pow2ceil(row_len);  // <= kGroupedSlots
    const int shift = 32 - (31 - __clz(T2));
    for (int i = lane; i < T2; i += 32) {
        skey[i] = -1;
        sst[i] = -1;
    }
    __syncwarp();

    // products in p order, 32 per round (lane L: p = 32 s + L)
    bool overflow = false;
    int t = 0;
    for (int p0 = 0; p0 < u; p0 += 32) {
        const int p = p0 + lane;
        int slot = -1;
        if (p < u) {
            while (m_pre[t + 1] <= p) ++t;
            const int ti = m_inst[t];
            const InstDev& I = a.inst[ib + ti];
            const int f = m_bs[t] + (p - m_pre[t]);
            const int c = __ldg(I.bcol + f);
            const T bv = __ldg(reinterpret_cast<const T*>(I.bval) + f);
            stage_v[lane] = a.merge ? bv : mul_rn(m_a[t], bv);
            stage_i[lane] = ti;
            unsigned h = ((unsigned)c * 0x9E3779B1u) >> shift;
            for (int probe = 0; probe < T2; ++probe) {
                const int old = atomicCAS(&skey[h], -1, c);
                if (old == -1 || old == c) {
                    slot = (int)h;
                    break;
                }
                h = (h + 1) & (unsigned)(T2 - 1);
            }
            overflow |= slot < 0;
        }
        __syncwarp();
        // lanes of one column: the lowest adds them all, in lane order
        const unsigned peers = __match_any_sync(0xffffffffu, slot >= 0 ? slot : -1 - lane);
        if (slot >= 0 && (peers & lanemask_lt()) == 0) {
            int cur = sst[slot];
            T acc = sacc[slot], sub = ssub[slot];
            for (unsigned m = peers; m; m &= m - 1) {
                const int l = __ffs(m) - 1;
                const T v = stage_v[l];
                const int ins = stage_i[l];
                if (cur < 0) {
                    sub = v;
                    cur = ins;
                } else if ((cur & 255) != ins) {
                    acc = (cur & 256) ? add_rn(acc, sub) : sub;
                    sub = v;
                    cur = ins | 256;
                } else {
                    sub = add_rn(sub, v);
                }
            }
            sst[slot] = cur;
            sacc[slot] = acc;
            ssub[slot] = sub;
        }
        __syncwarp();
    }
    if (__any_sync(0xffffffffu, overflow)) {
        if (lane == 0) atomicOr(a.status, kStatusHashOverflow);
        __syncwarp();
        return;
    }

    // the distinct columns, sorted (the meta is dead: keys take its place)
    int D = 0;
    for (int i0 = 0; i0 < T2; i0 += 32) {
        const int i = i0 + lane;
        const int c = i < T2 ? skey[i] : -1;
        const unsigned m = __ballot_sync(0xffffffffu, c >= 0);
        if (c >= 0 && D + __popc(m & lanemask_lt()) < kGroupedMaxD)
            keys[D + __popc(m & lanemask_lt())] = ((unsigned long long)(unsigned)c << 32) | (unsigned)i;
        D += __popc(m);
    }
    if (D != row_len) {
        if (lane == 0) atomicOr(a.status, kStatusInternal);
        __syncwarp();
        return;
    }
    int Dp = 32;
    while (Dp < D) Dp <<= 1;
    for (int i = D + lane; i < Dp; i += 32) keys[i] = ~0ull;
    __syncwarp();
    for (int k = 2; k <= Dp; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int x = lane; x < Dp; x += 32) {
                const int y = x ^ j;
                if (y > x) {
                    const unsigned long long kx = keys[x], ky = keys[y];
                    if ((kx > ky) == ((x & k) == 0)) {
                        keys[x] = ky;
                        keys[y] = kx;
                    }
                }
            }
            __syncwarp();
        }
    }
    T* cval = reinterpret_cast<T*>(G.cval) + row_begin;
    int* ccol = G.ccol + row_begin;
    for (int d = lane; d < D; d += 32) {
        const unsigned long long kv = keys[d];
        const int sl = (int)(kv & 0xffffffffu);
        const int cur = sst[sl];
        const T res = (cur & 256) ? add_rn(sacc[sl], ssub[sl]) : ssub[sl];
        __stcs(ccol + d, (int)(kv >> 32));
        __stcs(cval + d, res);
    }
    __syncwarp();
}

template <typename T>
__global__ void __launch_bounds__(32 * kGroupedWarps) k_num_grouped(RowArgs a) {
    extern __shared__ __align__(16) char smem[];
    const int w = threadIdx.x >> 5;
    char* sm = smem + w * GroupedLayout<T>::bytes;
    const int n = *a.gcount;
    for (int i = blockIdx.x * kGroupedWarps + w; i < n; i += gridDim.x * kGroupedWarps)
        grouped_row_warp<T>(a, __ldg(a.glist + i), sm);
}

template <int CAP, typename T>
struct NumLayout {
    static constexpr int MAXA = CAP / 2;
    static constexpr int NBMAX = CAP >= 8192 ? CAP : 2 * CAP;         // most buckets
    static constexpr int cnt = 0;                                      // int[NBMAX + 4]
    static constexpr int skey = (NBMAX + 4) * 4;                       // u64[CAP]
    static constexpr int ocol = skey + 8 * CAP;                        // int[CAP]
    static constexpr int oval = ocol + 4 * CAP;                        // T[CAP]
    static constexpr int oinst = oval + (int)sizeof(T) * CAP;          // u8[CAP]
    static constexpr int scratch = (oinst + CAP + 15) & ~15;           // int[34]
    static constexpr int bytes = (scratch + 34 * 4 + 15) & ~15;
    // the meta arrays live in [skey, oinst) until the scatter overwrites them
    static constexpr int m_bc = skey;                                  // const int*[MAXA]
    static constexpr int m_bv = m_bc + 8 * MAXA;                       // const T*[MAXA]
    static constexpr int m_a = m_bv + 8 * MAXA;                        // T[MAXA]
    static constexpr int m_pre = m_a + (int)sizeof(T) * MAXA;          // int[MAXA + 1]
    static constexpr int m_inst = m_pre + 4 * (MAXA + 1);              // u8[MAXA]
    static_assert(m_inst + MAXA <= oinst, "meta does not fit its alias region");
    static_assert(bytes <= 227 * 1024, "team layout exceeds shared memory");
};

template <int TEAM, int PER, typename T>
__device__ __forceinline__ void num_row(const RowArgs& a, int unit, char* sm) {
    constexpr int CAP = TEAM * PER;
    using L = NumLayout<CAP, T>;
    int* cnt = reinterpret_cast<int*>(sm + L::cnt);
    unsigned long long* skey = reinterpret_cast<unsigned long long*>(sm + L::skey);
    int* ocol = reinterpret_cast<int*>(sm + L::ocol);
    T* oval = reinterpret_cast<T*>(sm + L::oval);
    unsigned char* oinst = reinterpret_cast<unsigned char*>(sm + L::oinst);
    int* scratch = reinterpret_cast<int*>(sm + L::scratch);
    const int** m_bc = reinterpret_cast<const int**>(sm + L::m_bc);
    const T** m_bv = reinterpret_cast<const T**>(sm + L::m_bv);
    T* m_a = reinterpret_cast<T*>(sm + L::m_a);
    int* m_pre = reinterpret_cast<int*>(sm + L::m_pre);
    unsigned char* m_inst = reinterpret_cast<unsigned char*>(sm + L::m_inst);

    const int r = Team<TEAM>::rank();
    const int g = unit_group(a.unit_base, a.ngroups, unit);
    const GroupDev& G = a.groups[g];
    const int rho = (int)(unit - a.unit_base[g]);
    const int row_begin = __ldg(G.crp + rho);
    const int row_len = __ldg(G.crp + rho + 1) - row_begin;
    int nA, u;
    if (!build_meta<TEAM, true, T>(a, G, rho, L::MAXA, CAP, m_bc, m_bv, m_a, m_pre, m_inst, scratch, nA, u)) {
        if (r == 0) atomicOr(a.status, kStatusInternal);
        return;
    }
    if (grouped_row(a, nA, u, row_len)) {
        if (r == 0) a.glist[atomicAdd(a.gcount, 1)] = unit;
        Team<TEAM>::sync();
        return;
    }
    // NB = 2 pow2ceil(u) buckets: most products sit alone in their bucket
    const int NB = min(2 * pow2ceil(u), L::NBMAX);
    Bucketer bk;
    bk.init(G.ncols, G.ncols_inv, NB);
    for (int i = 4 * r; i <= NB; i += 4 * TEAM) *reinterpret_cast<int4*>(cnt + i) = make_int4(0, 0, 0, 0);
    Team<TEAM>::sync();

    // gather: all loads first, then the bucket counts
    int col[PER];
    T val[PER];
    int hb[PER];  // low 16 bits: slot in bucket; high bits: instance
    {
        const int p0 = r * PER;
        int t = 0, tb = 0, te = 0, ti = 0;
        const int* bc = nullptr;
        const T* bvp = nullptr;
        T av = T(1);
        if (p0 < u) {
            t = search_pre(m_pre, nA, p0);
            tb = m_pre[t];
            te = m_pre[t + 1];
            bc = m_bc[t];
            bvp = m_bv[t];
            av = m_a[t];
            ti = m_inst[t];
        }
#pragma unroll
        for (int s = 0; s < PER; ++s) {
            const int p = p0 + s;
            col[s] = -1;
            val[s] = T(0);
            hb[s] = 0;
            if (p < u) {
                while (p >= te) {
                    ++t;
                    tb = te;
                    te = m_pre[t + 1];
                    bc = m_bc[t];
                    bvp = m_bv[t];
                    av = m_a[t];
                    ti = m_inst[t];
                }
                col[s] = __ldg(bc + (p - tb));
                const T bv = __ldg(bvp + (p - tb));
                val[s] = a.merge ? bv : mul_rn(av, bv);
                hb[s] = ti << 16;
            }
        }
    }
#pragma unroll
    for (int s = 0; s < PER; ++s)
        if (col[s] >= 0) hb[s] |= atomicAdd(&cnt[bk(col[s])], 1);
    Team<TEAM>::sync();

    // bucket starts: exclusive scan of cnt[0..NB), each thread a contiguous
    // slice (16-byte accesses when the slice allows)
    {
        const int per = NB >= TEAM ? NB / TEAM : 1;
        const int beg = r * per;
        int loc = 0;
        if (beg < NB) {
            if ((per & 3) == 0) {
                for (int i = 0; i < per; i += 4) {
                    const int4 v = *reinterpret_cast<const int4*>(cnt + beg + i);
                    loc += v.x + v.y + v.z + v.w;
                }
            } else {
                for (int i = 0; i < per; ++i) loc += cnt[beg + i];
            }
        }
        int tot;
        int ex = Team<TEAM>::scan_excl(loc, &tot, scratch);
        if (beg < NB) {
            if ((per & 3) == 0) {
                for (int i = 0; i < per; i += 4) {
                    int4 v = *reinterpret_cast<const int4*>(cnt + beg + i);
                    int4 o;
                    o.x = ex; ex += v.x;
                    o.y = ex; ex += v.y;
                    o.z = ex; ex += v.z;
                    o.w = ex; ex += v.w;
                    *reinterpret_cast<int4*>(cnt + beg + i) = o;
                }
            } else {
                for (int i = 0; i < per; ++i) {
                    const int c = cnt[beg + i];
                    cnt[beg + i] = ex;
                    ex += c;
                }
            }
        }
        if (r == 0) cnt[NB] = tot;
    }
    Team<TEAM>::sync();

    // a product alone in its bucket goes straight to its place; the others
    // scatter their (column, p) keys into bucket order
    const bool multi = a.merge || G.inst_count > 1;
#pragma unroll
    for (int s = 0; s < PER; ++s)
        if (col[s] >= 0) {
            const int b = bk(col[s]);
            const int lo = cnt[b];
            if (cnt[b + 1] - lo == 1) {
                ocol[lo] = col[s];
                oval[lo] = val[s];
                if (multi) oinst[lo] = (unsigned char)(hb[s] >> 16);
                col[s] = -1;
            } else {
                const unsigned p = (unsigned)(r * PER + s);
                skey[lo + (hb[s] & 0xffff)] = ((unsigned long long)(unsigned)col[s] << 32) | p;
            }
        }
    Team<TEAM>::sync();

    // rank inside a shared bucket -> position in (column, p) order
#pragma unroll
    for (int s = 0; s < PER; ++s)
        if (col[s] >= 0) {
            const unsigned p = (unsigned)(r * PER + s);
            const int b = bk(col[s]);
            const int lo = cnt[b], hi = cnt[b + 1];
            const unsigned long long key = ((unsigned long long)(unsigned)col[s] << 32) | p;
            int rank = 0;
            for (int q = lo; q < hi; ++q) rank += skey[q] < key;
            const int pos = lo + rank;
            ocol[pos] = col[s];
            oval[pos] = val[s];
            if (multi) oinst[pos] = (unsigned char)(hb[s] >> 16);
        }
    Team<TEAM>::sync();

    // one output entry per run of equal columns; add the run in p order,
    // each instance's products first, then the instance sums in order
    T* cval = reinterpret_cast<T*>(G.cval);
    int nout = 0;
    for (int q0 = 0; q0 < u; q0 += TEAM) {
        const int q = q0 + r;
        const bool valid = q < u;
        const int c = valid ? ocol[q] : -1;
        const bool head = valid && (q == 0 || ocol[q - 1] != c);
        int tot;
        const int idx = nout + Team<TEAM>::count_excl(head, &tot, scratch);
        if (head) {
            T sub = oval[q], acc = T(0);
            bool have = false;
            int ci = multi ? oinst[q] : 0;
            for (int e = q + 1; e < u && ocol[e] == c; ++e) {
                const T v = oval[e];
                if (multi && oinst[e] != ci) {
                    acc = have ? add_rn(acc, sub) : sub;
                    have = true;
                    sub = v;
                    ci = oinst[e];
                } else {
                    sub = add_rn(sub, v);
                }
            }
            const T res = have ? add_rn(acc, sub) : sub;
            if (idx < row_len) {
                G.ccol[row_begin + idx] = c;
                cval[row_begin + idx] = res;
            }
        }
        nout += tot;
    }
    if (r == 0 && nout != row_len) atomicOr(a.status, kStatusInternal);
    Team<TEAM>::sync();
}

// ------------------------------------------------ single-pass output offsets
//
// In the single-pass product a block takes tiles of consecutive rows in
// order (one row per warp) and each tile's output offset is the sum of the
// counts of all earlier tiles, found by a decoupled look-back: a tile first
// publishes its count (flag 1), walks back over earlier tiles adding their
// published values until it meets an inclusive prefix (flag 2), then
// publishes its own inclusive prefix.  Every earlier tile belongs to a
// running block (tickets go only to running blocks), so the walk ends; a
// bounded spin turns a stall into an error instead: after fc.spin_limit polls
// the wait sets kStatusTimeout and the tile publishes the partial sum it has,
// so later tiles do not wait on it in turn (their offsets are then wrong, but
// every write stays checked against the output's capacity).  One entry per tile
// rather than per row keeps the walks short: per-row entries arrive faster
// than a walk of 32 entries per memory round trip can follow.

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

constexpr int kLookbackPer = 4;  // entries read per lane and round: a window of 128 tiles

// Exclusive prefix of tile t's count c over tiles 0..t-1, called by a whole
// warp.  One round reads the 128 tiles before position j (lane l, slot k
// reads tile j - 32k - l; independent loads, one memory round trip): the
// tiles up to and including the nearest inclusive prefix are summed once all
// of them have published; otherwise the window moves 128 tiles back.
// Positions before tile 0 read as an inclusive prefix of 0.  Each entry is
// one 64-bit word carrying its flag with its value, so relaxed loads suffice.
__device__ __forceinline__ long long lookback_offset(const FusedCtl& fc, int t, long long c, unsigned* status) {
    const int lane = threadIdx.x & 31;
    const bool publish = t != fc.hold_tile;
    if (lane == 0 && publish) st_release_u64(fc.lb + t, (1ull << 62) | (unsigned long long)c);
    long long excl = 0;
    int j = t - 1, spins = 0;
    while (j >= 0) {
        unsigned long long w[kLookbackPer];
#pragma unroll
        for (int k = 0; k < kLookbackPer; ++k) {
            const int idx = j - 32 * k - lane;
            w[k] = idx >= 0 ? ld_relaxed_u64(fc.lb + idx) : (2ull << 62);
        }
        // need[k]: lanes of slot k up to and including the nearest inclusive prefix
        unsigned need[kLookbackPer];
        bool found = false, wait = false;
#pragma unroll
        for (int k = 0; k < kLookbackPer; ++k) {
            const unsigned incl = __ballot_sync(0xffffffffu, (w[k] >> 62) == 2);
            const unsigned none = __ballot_sync(0xffffffffu, (w[k] >> 62) == 0);
            need[k] = found ? 0u : (incl ? ((incl & (0u - incl)) << 1) - 1u : 0xffffffffu);
            found = found || incl != 0;
            wait = wait || (none & need[k]) != 0;
        }
        if (wait) {
            if (++spins > fc.spin_limit) {
                if (lane == 0) atomicOr(status, kStatusTimeout);
                break;
            }
            __nanosleep(64);
            continue;
        }
        long long v = 0;
#pragma unroll
        for (int k = 0; k < kLookbackPer; ++k)
            if ((need[k] >> lane) & 1u) v += (long long)(w[k] & ((1ull << 62) - 1));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (found) break;
        j -= 32 * kLookbackPer;
    }
    if (lane == 0 && publish) st_release_u64(fc.lb + t, (2ull << 62) | (unsigned long long)(excl + c));
    return excl;
}

// A warp's place in the current tile of the single-pass product.
struct FusedRow {
    const FusedCtl* fc;
    long long* sh;  // shared, one slot per warp of the block
    int tile, w, nw;
};

// Output offset of warp fr.w's row (count c) within the whole product.  Every
// warp of the block calls it exactly once per tile (c = 0 for a warp without
// a row): the counts are scanned in shared memory and warp 0 resolves the
// tile's offset by look-back.
__device__ __forceinline__ long long fused_offset(const FusedRow& fr, long long c, unsigned* status) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) fr.sh[fr.w] = c;
    __syncthreads();
    if (fr.w == 0) {
        const long long v = lane < fr.nw ? fr.sh[lane] : 0;
        long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const long long total = __shfl_sync(0xffffffffu, x, 31);
        const long long base = lookback_offset(*fr.fc, fr.tile, total, status);
        if (lane < fr.nw) fr.sh[lane] = base + x - v;
    }
    __syncthreads();
    return fr.sh[fr.w];
}

// ------------------------------------------------- numeric, warp-team variant
//
// The same accumulator as num_row, arranged for SIMT efficiency:
//   place     every product goes to its slot in its bucket (bucket start +
//             arrival order); for a bucket of one product that slot is final
//   sort      only buckets holding several products are sorted in place by
//             (column, p), one bucket per lane, from a compacted work list
//   compact   run heads found with shuffles; a head whose successor has
//             another column takes its value as is, otherwise adds its run
// The meta keeps B-row offsets instead of pointers (instance base pointers
// are looked up when the instance changes).

template <int CAP, typename T>
struct WNumLayout {
    static constexpr int MAXA = CAP / 2;
    static constexpr int NBMAX = 2 * pow2floor_c(CAP);             // most buckets (a power of two)
    static constexpr int cnt = 0;                                  // u16[NBMAX + 8] counts, then starts
    static constexpr int ocol = ((NBMAX + 8) * 2 + 15) & ~15;      // int[CAP]
    static constexpr int oval = ocol + 4 * CAP;                    // T[CAP]
    static constexpr int op = oval + (int)sizeof(T) * CAP;         // u16[CAP] product index
    static constexpr int oinst = op + 2 * CAP;                     // u8[CAP]
    static constexpr int wl = (oinst + CAP + 3) & ~3;              // u16[CAP / 2] buckets to sort
    static constexpr int bytes = (wl + CAP + 15) & ~15;
    // meta, aliased over [ocol, wl) while the products are gathered
    static constexpr int m_pre = ocol;                             // int[MAXA + 1]
    static constexpr int m_bs = m_pre + 4 * (MAXA + 1);            // int[MAXA]
    static constexpr int m_a = (m_bs + 4 * MAXA + 7) & ~7;         // T[MAXA]
    static constexpr int m_inst = m_a + (int)sizeof(T) * MAXA;     // u8[MAXA]
    static_assert(m_inst + MAXA <= wl, "meta does not fit its alias region");
    static_assert((oval & 7) == 0, "value array alignment");
};

template <int PER, typename T, bool FUSED = false>
__device__ __forceinline__ void num_row_warp(const RowArgs& a, int unit, char* sm, const FusedRow* fr = nullptr) {
    constexpr int CAP = 32 * PER;
    using L = WNumLayout<CAP, T>;
    // bucket counts and starts never exceed CAP <= 512: 16 bits each
    unsigned short* cnt = reinterpret_cast<unsigned short*>(sm + L::cnt);
    int* ocol = reinterpret_cast<int*>(sm + L::ocol);
    T* oval = reinterpret_cast<T*>(sm + L::oval);
    unsigned short* op = reinterpret_cast<unsigned short*>(sm + L::op);
    unsigned char* oinst = reinterpret_cast<unsigned char*>(sm + L::oinst);
    unsigned short* wl = reinterpret_cast<unsigned short*>(sm + L::wl);
    int* m_pre = reinterpret_cast<int*>(sm + L::m_pre);
    int* m_bs = reinterpret_cast<int*>(sm + L::m_bs);
    T* m_a = reinterpret_cast<T*>(sm + L::m_a);
    unsigned char* m_inst = reinterpret_cast<unsigned char*>(sm + L::m_inst);

    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const int g = unit_group(a.unit_base, a.ngroups, unit);
    const GroupDev& G = a.groups[g];
    const int rho = (int)(unit - a.unit_base[g]);
    // two-pass: the row's slot comes from the symbolic pass; single pass:
    // from the look-back once the row's count is known
    long long row_begin = FUSED ? 0 : __ldg(G.crp + rho);
    int row_len = FUSED ? -1 : __ldg(G.crp + rho + 1) - (int)row_begin;
    const int ncols = G.ncols;
    const unsigned long long ncols_inv = G.ncols_inv;
    const int ib = G.inst_begin, icount = G.inst_count;
    const bool multi = a.merge || icount > 1;

    // ---- meta: B-row offset, a_ik, instance and prefix per A entry
    int nA, u;
    warp_meta<true, T, L::MAXA>(a, ib, icount, rho, lane, m_pre, m_bs, m_a, m_inst, nA, u);
    if (nA > L::MAXA || u > CAP) {
        if (lane == 0) atomicOr(a.status, kStatusInternal);
        if (FUSED) fused_offset(*fr, 0, a.status);  // the block and later tiles must not wait
        __syncwarp();
        return;
    }
    if (!FUSED && grouped_row(a, nA, u, row_len)) {
        if (lane == 0) a.glist[atomicAdd(a.gcount, 1)] = unit;
        __syncwarp();
        return;
    }
    if (lane == 0) m_pre[nA] = u;
    const int NB = min(2 * pow2ceil(u), L::NBMAX);
    Bucketer bk;
    bk.init(ncols, ncols_inv, NB);
    for (int i = 8 * lane; i <= NB; i += 256) *reinterpret_cast<int4*>(cnt + i) = make_int4(0, 0, 0, 0);
    // a row whose nnz equals its product count has no repeated column: it
    // only needs sorting (no tie-break, no run compaction)
    bool distinct = !FUSED && row_len == u;
    __syncwarp();

    // ---- gather (chunked or strided product order; xp records p)
    int col[PER];
    T val[PER];
    int hh[PER];  // slot in bucket (low 16 bits) | instance << 16
    const bool strided = use_strided<PER>(nA, u);
    {
        int ins[PER];
        if (strided)
            gather_strided<PER, true, T>(a, ib, nA, u, m_pre, m_bs, m_a, m_inst, reinterpret_cast<int*>(wl), lane,
                                         col, val, ins);
        else
            gather_chunks<PER, true, T>(a, ib, nA, u, m_pre, m_bs, m_a, m_inst, lane, col, val, ins);
#pragma unroll
        for (int e = 0; e < PER; ++e) hh[e] = ins[e] << 16;
    }
    // bucket counts; the second arrival in a bucket lists it for sorting
    int nwl = 0;
#pragma unroll
    for (int s = 0; s < PER; ++s) {
        int h = -1, b = 0;
        if (col[s] >= 0) {
            b = bk(col[s]);
            // 32-bit atomic on the pair of 16-bit counters holding b
            const unsigned half = (unsigned)(b & 1) << 4;
            const unsigned old = atomicAdd(reinterpret_cast<unsigned*>(cnt) + (b >> 1), 1u << half);
            h = (int)((old >> half) & 0xffffu);
            hh[s] |= h;
        }
        const unsigned m = __ballot_sync(0xffffffffu, h == 1);
        if (h == 1) wl[nwl + __popc(m & lt)] = (unsigned short)b;
        nwl += __popc(m);
    }
    __syncwarp();

    // the meta is dead from here on: the remaining arrays never alias
    unsigned short* __restrict__ xcnt = cnt;
    int* __restrict__ xcol = ocol;
    T* __restrict__ xval = oval;
    unsigned short* __restrict__ xp = op;
    unsigned char* __restrict__ xinst = oinst;
    unsigned short* __restrict__ xwl = wl;
    // ---- bucket starts: exclusive scan in rounds of 32 x 8 counters
    {
        int base = 0;
        for (int i0 = 0; i0 < NB; i0 += 256) {
            const int i = i0 + 8 * lane;
            int4 v = make_int4(0, 0, 0, 0);
            if (i < NB) v = *reinterpret_cast<const int4*>(xcnt + i);
            const unsigned w[4] = {(unsigned)v.x, (unsigned)v.y, (unsigned)v.z, (unsigned)v.w};
            int loc = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) loc += (int)(w[k] & 0xffffu) + (int)(w[k] >> 16);
            int x = loc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            unsigned ex = (unsigned)(base + x - loc);
            if (i < NB) {
                unsigned o[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const unsigned lo = ex;
                    ex += w[k] & 0xffffu;
                    o[k] = lo | (ex << 16);
                    ex += w[k] >> 16;
                }
                *reinterpret_cast<int4*>(xcnt + i) = make_int4((int)o[0], (int)o[1], (int)o[2], (int)o[3]);
            }
            base += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) xcnt[NB] = (unsigned short)u;
    }
    __syncwarp();

    // ---- place every product at its bucket slot
#pragma unroll
    for (int s = 0; s < PER; ++s)
        if (col[s] >= 0) {
            const int pos = xcnt[bk(col[s])] + (hh[s] & 0xffff);
            xcol[pos] = col[s];
            xval[pos] = val[s];
            if (!distinct) {
                xp[pos] = (unsigned short)(strided ? 32 * s + lane : chunk_product<PER>(lane, s));
                if (multi) xinst[pos] = (unsigned char)(hh[s] >> 16);
            }
        }
    __syncwarp();

    bool repeated = false;
    // ---- sort each listed bucket in place: by column, ties by p
    for (int w = lane; w < nwl; w += 32) {
        const int b = xwl[w];
        const int lo = xcnt[b], hi = xcnt[b + 1];
        if (distinct) {
            for (int i = lo + 1; i < hi; ++i) {
                const int c = xcol[i];
                const T v = xval[i];
                int j = i - 1;
                while (j >= lo && xcol[j] > c) {
                    xcol[j + 1] = xcol[j];
                    xval[j + 1] = xval[j];
                    --j;
                }
                xcol[j + 1] = c;
                xval[j + 1] = v;
            }
        } else {
            for (int i = lo + 1; i < hi; ++i) {
                const int c = xcol[i];
                const int pp = xp[i];
                const T v = xval[i];
                const unsigned char ins = multi ? xinst[i] : 0;
                int j = i - 1;
                while (j >= lo && (xcol[j] > c || (xcol[j] == c && xp[j] > pp))) {
                    xcol[j + 1] = xcol[j];
                    xp[j + 1] = xp[j];
                    xval[j + 1] = xval[j];
                    if (multi) xinst[j + 1] = xinst[j];
                    --j;
                }
                xcol[j + 1] = c;
                xp[j + 1] = (unsigned short)pp;
                xval[j + 1] = v;
                if (multi) xinst[j + 1] = ins;
            }
            if (FUSED)
                for (int i = lo + 1; i < hi; ++i) repeated |= xcol[i] == xcol[i - 1];
        }
    }
    __syncwarp();
    if (FUSED) {
        // the row's count: u when no column repeats, else the number of runs
        distinct = !__any_sync(0xffffffffu, repeated);
        int cnt_out = u;
        if (!distinct) {
            cnt_out = 0;
            for (int q = lane; q < u; q += 32) cnt_out += q == 0 || xcol[q] != xcol[q - 1];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cnt_out += __shfl_xor_sync(0xffffffffu, cnt_out, o);
        }
        const long long off = fused_offset(*fr, cnt_out, a.status);
        const FusedCtl* fc = fr->fc;
        if (lane == 0) {
            fc->crp[unit] = (int)off;
            if (unit == fc->nunits - 1) fc->crp[fc->nunits] = (int)(off + cnt_out);
            if (off + cnt_out > fc->cap) atomicOr(a.status, kStatusCapacity);
        }
        if (off + cnt_out > fc->cap) {
            __syncwarp();
            return;
        }
        row_begin = off;
        row_len = cnt_out;
    }

    // output rows are stored evict-first: they are not read again here, and
    // the B rows that later rows gather should keep their place in L2
    T* cval = reinterpret_cast<T*>(G.cval) + row_begin;
    int* ccol = G.ccol + row_begin;
    if (distinct) {
        // ---- sorted products are the row: copy out
        for (int q = lane; q < u; q += 32) {
            __stcs(ccol + q, xcol[q]);
            __stcs(cval + q, xval[q]);
        }
        __syncwarp();
        return;
    }

    // ---- compact runs of equal columns and write the row
    int nout = 0, carry = -1;
    for (int q0 = 0; q0 < u; q0 += 32) {
        const int q = q0 + lane;
        const bool valid = q < u;
        const int c = valid ? xcol[q] : -2;
        int prev = __shfl_up_sync(0xffffffffu, c, 1);
        if (lane == 0) prev = carry;
        int next = __shfl_down_sync(0xffffffffu, c, 1);
        if (lane == 31) next = q + 1 < u ? xcol[q + 1] : -2;
        const bool head = valid && c != prev;
        const unsigned hm = __ballot_sync(0xffffffffu, head);
        if (head) {
            T res = xval[q];
            if (next == c) {
                // several products on this column: add them in p order (in
                // merge or multi-instance mode each instance's products first)
                T sub = res, acc = T(0);
                bool have = false;
                int ci = multi ? xinst[q] : 0;
                for (int e = q + 1; e < u && xcol[e] == c; ++e) {
                    const T v = xval[e];
                    if (multi && xinst[e] != ci) {
                        acc = have ? add_rn(acc, sub) : sub;
                        have = true;
                        sub = v;
                        ci = xinst[e];
                    } else {
                        sub = add_rn(sub, v);
                    }
                }
                res = have ? add_rn(acc, sub) : sub;
            }
            const int idx = nout + __popc(hm & lt);
            if (idx < row_len) {
                __stcs(ccol + idx, c);
                __stcs(cval + idx, res);
            }
        }
        nout += __popc(hm);
        carry = __shfl_sync(0xffffffffu, c, 31);
    }
    if (lane == 0 && nout != row_len) atomicOr(a.status, kStatusInternal);
    __syncwarp();
}

template <int TEAM, int PER, typename T>
__global__ void __launch_bounds__(TEAM == 32 ? (PER <= 8 ? 1024 : (PER == 12 ? 256 : 512)) : TEAM,
                                    TEAM == 32 && PER == 12 ? 3 : (TEAM == 32 && PER == 10 ? 2 : 1))
    k_num_rows(RowArgs a) {
    extern __shared__ __align__(16) char smem[];
    constexpr int CAP = TEAM * PER;
    const int begin = a.bin_off[a.bin], end = a.bin_off[a.bin + 1];
    int team, nteams;
    char* sm;
    if (TEAM == 32) {
        const int w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
        team = blockIdx.x * wpb + w;
        nteams = gridDim.x * wpb;
        sm = smem + w * WNumLayout<CAP, T>::bytes;
    } else {
        team = blockIdx.x;
        nteams = gridDim.x;
        sm = smem;
    }
    if constexpr (TEAM == 32) {
        // rows are handed out one at a time: the per-row cost varies (gather
        // latency, collisions, the SM's distance to the L2 slices), and a
        // static stride leaves the slowest warps to finish the bin alone.
        // The next ticket is drawn before the current row starts, so the
        // atomic's round trip overlaps the row.
        const int lane = threadIdx.x & 31;
        (void)team;
        (void)nteams;
        int nxt = lane == 0 ? atomicAdd(a.tick + a.bin, 1) : 0;
        for (;;) {
            const int i = begin + __shfl_sync(0xffffffffu, nxt, 0);
            if (i >= end) break;
            if (lane == 0) nxt = atomicAdd(a.tick + a.bin, 1);
            num_row_warp<PER, T>(a, __ldg(a.list + i), sm);
        }
    } else {
        for (int i = begin + team; i < end; i += nteams) num_row<TEAM, PER, T>(a, __ldg(a.list + i), sm);
    }
}

template <int PER, typename T>
__global__ void __launch_bounds__(PER <= 8 ? 1024 : (PER == 12 ? 256 : 512), PER == 12 ? 3 : (PER == 10 ? 2 : 1))
    k_num_fused(RowArgs a, FusedCtl fc) {
    extern __shared__ __align__(16) char smem[];
    __shared__ long long sh_off[32];
    __shared__ int sh_tile;
    constexpr int CAP = 32 * PER;
    const int w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    char* sm = smem + w * WNumLayout<CAP, T>::bytes;
    FusedRow fr{&fc, sh_off, 0, w, nw};
    // a tile is drawn only when the block can start it: a tile drawn ahead
    // would delay every later tile's offset by a whole tile of work
    for (;;) {
        if (threadIdx.x == 0) sh_tile = atomicAdd(fc.ticket, 1);
        __syncthreads();
        fr.tile = sh_tile;
        if ((long long)fr.tile * nw >= fc.nunits) break;  // the same for the whole block
        const int row = fr.tile * nw + w;
        if (row < fc.nunits)
            num_row_warp<PER, T, true>(a, row, sm, &fr);
        else
            fused_offset(fr, 0, a.status);
    }
}

// ---------------------------------------------------------------- heavy rows

constexpr int kHeavyThreads = 512;
constexpr int kHeavyChunk = 1 << 20;  // columns per pass (a 128 KB bitmap)

// Visit every product of a heavy row; fn(col, value) (value unused when !VALS).
template <bool VALS, typename T, typename F>
__device__ __forceinline__ void heavy_products(const RowArgs& a, const GroupDev& G, int rho, F&& fn) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = 0; t < G.inst_count; ++t) {
        const InstDev& I = a.inst[G.inst_begin + t];
        const T* bval = reinterpret_cast<const T*>(I.bval);
        if (a.merge) {
            const int bs = __ldg(I.brp + rho), be = __ldg(I.brp + rho + 1);
            for (int f = bs + (int)threadIdx.x; f < be; f += blockDim.x)
                fn(__ldg(I.bcol + f), VALS ? __ldg(bval + f) : T(0));
        } else {
            const int a0 = __ldg(I.arp + rho), a1 = __ldg(I.arp + rho + 1);
            const T* aval = reinterpret_cast<const T*>(I.aval);
            for (int e = a0 + warp; e < a1; e += nw) {
                const int k = __ldg(I.acol + e);
                const T av = VALS ? __ldg(aval + e) : T(0);
                const int bs = __ldg(I.brp + k), be = __ldg(I.brp + k + 1);
                for (int f = bs + lane; f < be; f += 32)
                    fn(__ldg(I.bcol + f), VALS ? mul_rn(av, __ldg(bval + f)) : T(0));
            }
        }
    }
}

__global__ void __launch_bounds__(kHeavyThreads, 1) k_sym_heavy(RowArgs a, int chunk);

template <typename T>
__global__ void __launch_bounds__(kHeavyThreads, 1) k_num_heavy(RowArgs a, T* dense, int chunk) {
    extern __shared__ __align__(16) unsigned bm[];
    __shared__ int scratch[34];
    T* D = dense + (size_t)blockIdx.x * chunk;
    const int words = chunk >> 5;
    const int begin = a.bin_off[a.bin], end = a.bin_off[a.bin + 1];
    for (int i = begin + blockIdx.x; i < end; i += gridDim.x) {
        const int unit = __ldg(a.list + i);
        const int g = unit_group(a.unit_base, a.ngroups, unit);
        const GroupDev& G = a.groups[g];
        const int rho = (int)(unit - a.unit_base[g]);
        const int row_begin = __ldg(G.crp + rho);
        const int row_len = __ldg(G.crp + rho + 1) - row_begin;
        T* cval = reinterpret_cast<T*>(G.cval);
        int out = 0;
        for (long long c0 = 0; c0 < G.ncols; c0 += chunk) {
            for (int w = threadIdx.x; w < words; w += blockDim.x) bm[w] = 0u;
            __syncthreads();
            heavy_products<true, T>(a, G, rho, [&](int col, T v) {
                const unsigned rel = (unsigned)((long long)col - c0);
                if (rel < (unsigned)chunk) {
                    atomicAdd(D + rel, v);
                    atomicOr(bm + (rel >> 5), 1u << (rel & 31));
                }
            });
            __threadfence();
            __syncthreads();
            const int per = (words + blockDim.x - 1) / blockDim.x;
            const int w0 = threadIdx.x * per;
            const int w1 = min(w0 + per, words);
            int loc = 0;
            for (int w = w0; w < w1; ++w) loc += __popc(bm[w]);
            int tot;
            int pos = out + Team<kHeavyThreads>::scan_excl(loc, &tot, scratch);
            for (int w = w0; w < w1; ++w) {
                unsigned m = bm[w];
                while (m) {
                    const int b = __ffs(m) - 1;
                    m &= m - 1;
                    const int rel = (w << 5) + b;
                    const T v = __ldcg(D + rel);
                    __stcg(D + rel, T(0));
                    if (pos < row_len) {
                        G.ccol[row_begin + pos] = (int)(c0 + rel);
                        cval[row_begin + pos] = v;
                    }
                    ++pos;
                }
            }
            out += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0 && out != row_len) atomicOr(a.status, kStatusInternal);
    }
}

}  // namespace tsg
