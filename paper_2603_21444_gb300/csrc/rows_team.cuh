// Numeric rows of 1k..8k products: a block team running the warp team's
// counting sort (Sec. 2's row-wise product, the accumulator of Sec. 4.4
// restated for one GB300 SM).
//
// A block of NW warps owns one output row at a time (rows handed out by a
// per-bin ticket).  Warp w gathers products [256 w, 256 w + 256) of the row
// with the coalesced chunked gather, 8 per lane, and keeps them in registers.
// Every product is counted into its bucket (NB = 2 pow2ceil(u) buckets, a
// monotone map of the column, or the column itself when the row's column
// range is smaller: then each bucket is one column, a dense accumulator);
// 16-bit counters updated in pairs by 32-bit shared atomics return each
// product's slot in its bucket.  One block-wide scan turns the counts into
// bucket starts, every product is stored at start + slot, buckets holding
// several products are sorted in place by (column, p) -- one thread per
// bucket, from a list built while counting -- and the sorted row is either
// copied out (no repeated column) or compacted run by run, each run added in
// p order (each instance's products first, then the instance sums in order).
// The summation order is the warp kernels' and the oracle's: results are
// bit-identical to every other on-chip variant.
//
// Compared with the block variants of rows.cuh (bucket sort with an
// in-bucket rank over 32-bit keys, per-thread sequential gathers, one block
// per SM at 4096 products), this keeps the products in registers, halves
// the counters and reads B rows coalesced, so two blocks of 512 threads fit
// an SM at 4096 products.
#pragma once

#include "rows.cuh"

namespace tsg {

constexpr int kTeamPer = 8;  // products per thread
constexpr int kStageMaxA = 128;  // staged rows: at most this many A entries

template <int CAP, typename T>
struct TNumLayout {
    static constexpr int MAXA = CAP / 2;
    static constexpr int NBMAX = 2 * CAP;                          // CAP is a power of two
    static constexpr int cnt = 0;                                  // u16[NBMAX + 8] counts, then starts
    static constexpr int ocol = ((NBMAX + 8) * 2 + 15) & ~15;      // int[CAP]
    static constexpr int oval = ocol + 4 * CAP;                    // T[CAP]
    static constexpr int op = oval + (int)sizeof(T) * CAP;         // u16[CAP] product index
    static constexpr int oinst = op + 2 * CAP;                     // u8[CAP]
    static constexpr int wl = (oinst + CAP + 3) & ~3;              // u16[CAP / 2] buckets to sort
    static constexpr int ctl = (wl + CAP + 15) & ~15;              // int[kCtl]
    static constexpr int kCtl = 128;
    static constexpr int bytes = ctl + 4 * kCtl;
    // staged variant only (after `bytes`): the meta of rows of at most
    // kStageMaxA A entries, their staging offsets, and the copy barrier; the
    // staged B rows themselves occupy [ocol, wl)
    static constexpr int s_a = (bytes + 15) & ~15;                 // T[kStageMaxA]
    static constexpr int s_pre = s_a + (int)sizeof(T) * kStageMaxA;  // int[kStageMaxA + 1]
    static constexpr int s_bs = s_pre + 4 * (kStageMaxA + 1);      // int[kStageMaxA]
    static constexpr int s_offc = s_bs + 4 * kStageMaxA;           // int[kStageMaxA] staged column offset
    static constexpr int s_offv = s_offc + 4 * kStageMaxA;         // int[kStageMaxA] staged value offset
    static constexpr int s_inst = s_offv + 4 * kStageMaxA;         // u8[kStageMaxA]
    static constexpr int s_bar = (s_inst + kStageMaxA + 15) & ~15; // u64 mbarrier
    static constexpr int bytes_staged = s_bar + 16;
    static constexpr int stage_bytes = wl - ocol;                  // room for the staged B rows
    // ctl words: [0, 32) and [96, 128) scan scratch (two slots used in
    // turn), 40 / 42 row tickets (used in turn), 41 listed buckets,
    // [48, 48 + 32) heads per warp
    static constexpr int c_ticket = 40, c_nwl = 41, c_heads = 48, c_scan2 = 96;
    // meta, aliased over [ocol, wl) while the products are gathered
    static constexpr int m_pre = ocol;                             // int[MAXA + 1]
    static constexpr int m_bs = m_pre + 4 * (MAXA + 1);            // int[MAXA]
    static constexpr int m_a = (m_bs + 4 * MAXA + 7) & ~7;         // T[MAXA]
    static constexpr int m_inst = m_a + (int)sizeof(T) * MAXA;     // u8[MAXA]
    static_assert((CAP & (CAP - 1)) == 0, "team capacity must be a power of two");
    static_assert(m_inst + MAXA <= wl, "meta does not fit its alias region");
    static_assert((oval & 7) == 0, "value array alignment");
    static_assert(bytes_staged <= 227 * 1024, "team layout exceeds shared memory");
};

// Exclusive prefix sum over the block with a single barrier: each warp's
// total goes to scratch[w], then every warp scans the NW totals itself.
// scratch is read after the barrier, so it must not be written again before
// every thread has passed a later block barrier: consecutive calls without
// one in between alternate between two scratch slots.
template <int NT>
__device__ __forceinline__ int team_scan1(int v, int* total, int* scratch) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) scratch[w] = x;
    __syncthreads();
    const int t = lane < NW ? scratch[lane] : 0;
    int z = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, z, o);
        if (lane >= o) z += y;
    }
    const int before = __shfl_sync(0xffffffffu, z - t, w);
    *total = __shfl_sync(0xffffffffu, z, NW - 1);
    return before + x - v;
}

// Row meta of a block team: per A entry (instances in order, entries in
// stored order) its first product, B-row offset, a_ik and instance; nA and
// u for the row (the same in every thread).  Entries beyond MAXA are counted
// but not stored (the caller rejects the row).  Ends with a block barrier.
template <int NT, typename T, int MAXA>
__device__ __forceinline__ void team_meta(const RowArgs& a, int ib, int icount, int rho, int* m_pre, int* m_bs,
                                          T* m_a, unsigned char* m_inst, int* scratch, int* scratch2, int& nA,
                                          int& u) {
    const int tid = threadIdx.x;
    nA = 0;
    u = 0;
    int calls = 0;
    for (int t = 0; t < icount; ++t) {
        const InstDev& I = a.inst[ib + t];
        int a0 = 0, a1 = 1;
        if (!a.merge) {
            a0 = __ldg(I.arp + rho);
            a1 = __ldg(I.arp + rho + 1);
        }
        for (int e0 = a0; e0 < a1; e0 += NT) {
            const int e = e0 + tid;
            const bool valid = e < a1;
            int len = 0, bs = 0;
            T av = T(1);
            if (valid) {
                const int k = a.merge ? rho : __ldg(I.acol + e);
                bs = __ldg(I.brp + k);
                len = __ldg(I.brp + k + 1) - bs;
                if (!a.merge) av = __ldg(reinterpret_cast<const T*>(I.aval) + e);
            }
            int tot;
            const int ex = team_scan1<NT>(len, &tot, (calls++ & 1) ? scratch2 : scratch);
            const int idx = nA + (e - e0);
            if (valid && idx < MAXA) {
                m_pre[idx] = u + ex;
                m_bs[idx] = bs;
                m_a[idx] = av;
                m_inst[idx] = (unsigned char)t;
            }
            nA += min(NT, a1 - e0);
            u += tot;
        }
    }
    __syncthreads();
}

// ------------------------------------------------ TMA staging of B rows
//
// The staged variant (STAGED) copies every B row segment a row reads into
// shared memory with one 1D bulk copy (cp.async.bulk, no multicast) per
// array and A entry, completing on an mbarrier, and gathers the products
// from shared memory.  A bulk copy moves 16-byte units between 16-byte
// aligned addresses, so each segment is copied from the 16-byte boundary at
// or below its start to the one at or above its end, into its own slot
// (16-byte aligned, 48 bytes of slack per entry keeps slots apart: slot t of
// the columns starts at align16(4 pre_t + 48 t), of the values at
// align16(size(T) pre_t + 48 t)), and read at the start's offset within its
// 16 bytes.  A row is staged when it has at most kStageMaxA A entries, its
// slots fit [ocol, wl), and every rounded segment lies inside its array;
// otherwise it is gathered from global memory as in the plain variant.  The
// barrier wait is bounded: past kStageSpinLimit polls the row is abandoned
// with kStatusTimeout latched (its products dropped, every write in bounds).

constexpr unsigned kStageSpinLimit = 1u << 26;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// one arrival that also expects `bytes` of bulk copies in the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The lane's products [pbase + 4 (32 c + lane), + 4) from the staged slots.
template <int PER, typename T>
__device__ __forceinline__ void gather_staged(const char* stage, const int* s_pre, const int* s_offc, const int* s_offv,
                                              const T* s_a, const unsigned char* s_inst, bool merge, int nA, int u,
                                              int lane, int pbase, int (&col)[PER], T (&val)[PER], int (&ins)[PER]) {
    static_assert(PER % 4 == 0, "chunks of four");
#pragma unroll
    for (int c = 0; c < PER / 4; ++c) {
        const int p0 = pbase + 4 * (32 * c + lane);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            col[4 * c + v] = -1;
            val[4 * c + v] = T(0);
            ins[4 * c + v] = 0;
        }
        if (p0 >= u) continue;
        int t = owner_of(s_pre, nA, p0);
        int tb = s_pre[t], te = s_pre[t + 1];
        int oc = s_offc[t], ov = s_offv[t];
        T av = s_a[t];
        int ti = s_inst[t];
        const int j0 = p0 - tb;
        if (p0 + 4 <= te && ((oc + 4 * j0) & 15) == 0 && ((ov + (int)sizeof(T) * j0) & 15) == 0) {
            const int4 cc = *reinterpret_cast<const int4*>(stage + oc + 4 * j0);
            T bv[4];
            if (sizeof(T) == 8) {
                const double2 x = *reinterpret_cast<const double2*>(stage + ov + 8 * j0);
                const double2 y = *reinterpret_cast<const double2*>(stage + ov + 8 * j0 + 16);
                bv[0] = (T)x.x; bv[1] = (T)x.y; bv[2] = (T)y.x; bv[3] = (T)y.y;
            } else {
                const float4 x = *reinterpret_cast<const float4*>(stage + ov + 4 * j0);
                bv[0] = (T)x.x; bv[1] = (T)x.y; bv[2] = (T)x.z; bv[3] = (T)x.w;
            }
            col[4 * c + 0] = cc.x;
            col[4 * c + 1] = cc.y;
            col[4 * c + 2] = cc.z;
            col[4 * c + 3] = cc.w;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                val[4 * c + v] = merge ? bv[v] : mul_rn(av, bv[v]);
                ins[4 * c + v] = ti;
            }
        } else {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int p = p0 + v;
                if (p < u) {
                    while (p >= te) {
                        ++t;
                        tb = te;
                        te = s_pre[t + 1];
                        oc = s_offc[t];
                        ov = s_offv[t];
                        av = s_a[t];
                        ti = s_inst[t];
                    }
                    const int j = p - tb;
                    col[4 * c + v] = *reinterpret_cast<const int*>(stage + oc + 4 * j);
                    const T bv = *reinterpret_cast<const T*>(stage + ov + (int)sizeof(T) * j);
                    val[4 * c + v] = merge ? bv : mul_rn(av, bv);
                    ins[4 * c + v] = ti;
                }
            }
        }
    }
}

template <int NW, typename T, bool STAGED = false>
__device__ __forceinline__ void num_row_team(const RowArgs& a, int unit, char* sm, unsigned* parity = nullptr) {
    constexpr int NT = 32 * NW;
    constexpr int PER = kTeamPer;
    constexpr int CAP = NT * PER;
    using L = TNumLayout<CAP, T>;
    unsigned short* cnt = reinterpret_cast<unsigned short*>(sm + L::cnt);
    int* xcol = reinterpret_cast<int*>(sm + L::ocol);
    T* xval = reinterpret_cast<T*>(sm + L::oval);
    unsigned short* xp = reinterpret_cast<unsigned short*>(sm + L::op);
    unsigned char* xinst = reinterpret_cast<unsigned char*>(sm + L::oinst);
    unsigned short* wl = reinterpret_cast<unsigned short*>(sm + L::wl);
    int* ctl = reinterpret_cast<int*>(sm + L::ctl);
    int* m_pre = reinterpret_cast<int*>(sm + L::m_pre);
    int* m_bs = reinterpret_cast<int*>(sm + L::m_bs);
    T* m_a = reinterpret_cast<T*>(sm + L::m_a);
    unsigned char* m_inst = reinterpret_cast<unsigned char*>(sm + L::m_inst);

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned lt = lanemask_lt();
    const int g = unit_group(a.unit_base, a.ngroups, unit);
    const GroupDev& G = a.groups[g];
    const int rho = (int)(unit - a.unit_base[g]);
    const int row_begin = __ldg(G.crp + rho);
    const int row_len = __ldg(G.crp + rho + 1) - row_begin;
    const int ib = G.inst_begin, icount = G.inst_count;
    const bool multi = a.merge || icount > 1;

    // staged variant: rows of few A entries keep their meta outside the
    // staging area
    bool small = false;
    if (STAGED) {
        int na = 0;
        for (int t = 0; t < icount; ++t) {
            if (a.merge) {
                ++na;
            } else {
                const InstDev& I = a.inst[ib + t];
                na += __ldg(I.arp + rho + 1) - __ldg(I.arp + rho);
            }
        }
        small = na <= kStageMaxA;
        if (small) {
            m_pre = reinterpret_cast<int*>(sm + L::s_pre);
            m_bs = reinterpret_cast<int*>(sm + L::s_bs);
            m_a = reinterpret_cast<T*>(sm + L::s_a);
            m_inst = reinterpret_cast<unsigned char*>(sm + L::s_inst);
        }
    }
    int nA, u;
    if (STAGED && small)
        team_meta<NT, T, kStageMaxA>(a, ib, icount, rho, m_pre, m_bs, m_a, m_inst, ctl, ctl + L::c_scan2, nA, u);
    else
        team_meta<NT, T, L::MAXA>(a, ib, icount, rho, m_pre, m_bs, m_a, m_inst, ctl, ctl + L::c_scan2, nA, u);
    if (STAGED && small && nA > kStageMaxA) {  // the inputs changed under us
        if (tid == 0) atomicOr(a.status, kStatusInternal);
        __syncthreads();
        return;
    }
    if (nA > L::MAXA || u > CAP) {  // the binning rules this out unless the inputs changed
        if (tid == 0) atomicOr(a.status, kStatusInternal);
        __syncthreads();
        return;
    }
    if (grouped_row(a, nA, u, row_len)) {
        if (tid == 0) a.glist[atomicAdd(a.gcount, 1)] = unit;
        __syncthreads();
        return;
    }
    // buckets: 2 pow2ceil(u), or one per column when the column range is smaller
    const int NB = min(min(2 * pow2ceil(u), L::NBMAX), pow2ceil(G.ncols));
    Bucketer bk;
    bk.init(G.ncols, G.ncols_inv, NB);
    if (tid == 0) {
        m_pre[nA] = u;
        ctl[L::c_nwl] = 0;
    }
    for (int i = 8 * tid; i <= NB; i += 8 * NT) *reinterpret_cast<int4*>(cnt + i) = make_int4(0, 0, 0, 0);
    const bool distinct = row_len == u;  // no repeated column: sort only
    __syncthreads();

    // ---- staging (staged variant): one bulk copy per A entry and array
    bool staged = false;
    if (STAGED && small) {
        int* s_offc = reinterpret_cast<int*>(sm + L::s_offc);
        int* s_offv = reinterpret_cast<int*>(sm + L::s_offv);
        unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm + L::s_bar);
        bool ok = true;
        uintptr_t csrc = 0, vsrc = 0;
        unsigned cbytes = 0, vbytes = 0;
        int oc = 0, ov = 0;
        if (tid < nA) {
            const InstDev& I = a.inst[ib + m_inst[tid]];
            const int len = m_pre[tid + 1] - m_pre[tid];
            const uintptr_t cb = reinterpret_cast<uintptr_t>(I.bcol), vb = reinterpret_cast<uintptr_t>(I.bval);
            const uintptr_t ca = cb + 4ull * (unsigned)m_bs[tid], va = vb + sizeof(T) * (unsigned)m_bs[tid];
            csrc = ca & ~uintptr_t(15);
            vsrc = va & ~uintptr_t(15);
            const uintptr_t cend = (ca + 4ull * len + 15) & ~uintptr_t(15);
            const uintptr_t vend = (va + sizeof(T) * len + 15) & ~uintptr_t(15);
            ok = csrc >= cb && vsrc >= vb && cend <= cb + 4ull * (unsigned long long)I.bnnz &&
                 vend <= vb + sizeof(T) * (unsigned long long)I.bnnz;
            cbytes = len > 0 ? (unsigned)(cend - csrc) : 0u;
            vbytes = len > 0 ? (unsigned)(vend - vsrc) : 0u;
            const int c0 = (4 * m_pre[tid] + 48 * tid + 15) & ~15;
            const int v0 = ((int)sizeof(T) * m_pre[tid] + 48 * tid + 15) & ~15;
            oc = c0 + (int)(ca - csrc);
            ov = v0 + (int)(va - vsrc);
            s_offc[tid] = oc;
            s_offv[tid] = ov;
        }
        // the column slots, then the value slots, inside [ocol, wl)
        const int cspan = (4 * u + 48 * nA + 15 + 15) & ~15;
        const int vspan = ((int)sizeof(T) * u + 48 * nA + 15 + 15) & ~15;
        staged = __syncthreads_and(ok) && cspan + vspan <= L::stage_bytes;
        int total = 0;
        if (staged) team_scan1<NT>((int)(cbytes + vbytes), &total, ctl);
        staged = staged && total > 0;
        if (staged) {
            char* stage = sm + L::ocol;
            // earlier generic accesses to the slots come before the copies;
            // the barrier expects every byte before any copy is issued
            fence_proxy_async_smem();
            if (tid == 0) mbar_arrive_expect_tx(bar, (unsigned)total);
            __syncthreads();
            if (tid < nA) {
                if (cbytes) bulk_g2s(stage + (oc & ~15), reinterpret_cast<const void*>(csrc), cbytes, bar);
                if (vbytes) bulk_g2s(stage + cspan + (ov & ~15), reinterpret_cast<const void*>(vsrc), vbytes, bar);
            }
            unsigned spins = 0;
            bool done = false;
            while (!(done = mbar_try_wait(bar, *parity)) && ++spins < kStageSpinLimit) {
            }
            done = __syncthreads_and(done);
            *parity ^= 1u;
            if (!done) {
                if (tid == 0) atomicOr(a.status, kStatusTimeout);
                staged = false;
                u = 0;  // abandon the row's products
            }
            // the value slots follow the column slots
            if (tid < nA) s_offv[tid] += cspan;
            __syncthreads();
        }
    }

    // ---- gather: warp w, products [256 w, 256 w + 256), chunked
    int col[PER];
    T val[PER];
    int hh[PER];  // slot in bucket (low 16 bits) | instance << 16
    {
        int ins[PER];
        if (STAGED && staged)
            gather_staged<PER, T>(sm + L::ocol, m_pre, reinterpret_cast<const int*>(sm + L::s_offc),
                                  reinterpret_cast<const int*>(sm + L::s_offv), m_a, m_inst, a.merge, nA, u, lane,
                                  32 * PER * w, col, val, ins);
        else
            gather_chunks<PER, true, T>(a, ib, nA, u, m_pre, m_bs, m_a, m_inst, lane, col, val, ins, 32 * PER * w);
#pragma unroll
        for (int e = 0; e < PER; ++e) hh[e] = ins[e] << 16;
    }
    // ---- bucket counts; the second arrival in a bucket lists it for sorting
#pragma unroll
    for (int s = 0; s < PER; ++s) {
        int h = -1, b = 0;
        if (col[s] >= 0) {
            b = bk(col[s]);
            const unsigned half = (unsigned)(b & 1) << 4;
            const unsigned old = atomicAdd(reinterpret_cast<unsigned*>(cnt) + (b >> 1), 1u << half);
            h = (int)((old >> half) & 0xffffu);
            hh[s] |= h;
        }
        const unsigned m = __ballot_sync(0xffffffffu, h == 1);
        if (m) {
            int base = 0;
            if (lane == 0) base = atomicAdd(ctl + L::c_nwl, __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (h == 1) wl[base + __popc(m & lt)] = (unsigned short)b;
        }
    }
    __syncthreads();  // the meta is dead from here on

    // ---- bucket starts: one block-wide exclusive scan, a contiguous slice
    // of the counters per thread (NB and NT are powers of two)
    {
        const int per = NB >= NT ? NB / NT : 1;
        const int beg = tid * per;
        const bool mine = beg < NB;
        int loc = 0;
        if (mine) {
            if (per >= 8) {
                for (int i = 0; i < per; i += 8) {
                    const int4 v = *reinterpret_cast<const int4*>(cnt + beg + i);
                    const unsigned x[4] = {(unsigned)v.x, (unsigned)v.y, (unsigned)v.z, (unsigned)v.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k) loc += (int)(x[k] & 0xffffu) + (int)(x[k] >> 16);
                }
            } else {
                for (int i = 0; i < per; ++i) loc += cnt[beg + i];
            }
        }
        int tot;
        unsigned ex = (unsigned)team_scan1<NT>(loc, &tot, ctl + L::c_scan2);
        if (mine) {
            if (per >= 8) {
                for (int i = 0; i < per; i += 8) {
                    const int4 v = *reinterpret_cast<const int4*>(cnt + beg + i);
                    const unsigned x[4] = {(unsigned)v.x, (unsigned)v.y, (unsigned)v.z, (unsigned)v.w};
                    unsigned o[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const unsigned lo = ex;
                        ex += x[k] & 0xffffu;
                        o[k] = lo | (ex << 16);
                        ex += x[k] >> 16;
                    }
                    *reinterpret_cast<int4*>(cnt + beg + i) = make_int4((int)o[0], (int)o[1], (int)o[2], (int)o[3]);
                }
            } else {
                for (int i = 0; i < per; ++i) {
                    const unsigned c = cnt[beg + i];
                    cnt[beg + i] = (unsigned short)ex;
                    ex += c;
                }
            }
        }
        if (tid == 0) cnt[NB] = (unsigned short)u;
    }
    __syncthreads();

    // ---- every product to its bucket slot
#pragma unroll
    for (int s = 0; s < PER; ++s)
        if (col[s] >= 0) {
            const int pos = cnt[bk(col[s])] + (hh[s] & 0xffff);
            xcol[pos] = col[s];
            xval[pos] = val[s];
            if (!distinct) {
                xp[pos] = (unsigned short)(32 * PER * w + chunk_product<PER>(lane, s));
                if (multi) xinst[pos] = (unsigned char)(hh[s] >> 16);
            }
        }
    __syncthreads();

    // ---- sort each listed bucket in place: by column, ties by p
    const int nwl = ctl[L::c_nwl];
    for (int x = tid; x < nwl; x += NT) {
        const int b = wl[x];
        const int lo = cnt[b], hi = cnt[b + 1];
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
        }
    }
    __syncthreads();

    // output rows are stored evict-first (not read again here)
    T* cval = reinterpret_cast<T*>(G.cval) + row_begin;
    int* ccol = G.ccol + row_begin;
    if (distinct) {
        for (int q = tid; q < u; q += NT) {
            __stcs(ccol + q, xcol[q]);
            __stcs(cval + q, xval[q]);
        }
        __syncthreads();
        return;
    }

    // ---- compact runs: warp w takes sorted positions [w seg, w seg + seg);
    // pass 1 counts its run heads, pass 2 writes them after the earlier warps'
    const int seg = ((u + NW - 1) / NW + 31) & ~31;
    const int q0 = w * seg, q1 = min(u, q0 + seg);
    int heads = 0;
    for (int q = q0 + lane; q - lane < q1; q += 32) {
        const bool head = q < q1 && (q == 0 || xcol[q - 1] != xcol[q]);
        heads += __popc(__ballot_sync(0xffffffffu, head));
    }
    if (lane == 0) ctl[L::c_heads + w] = heads;
    __syncthreads();
    int nout = 0;
    for (int x = 0; x < w; ++x) nout += ctl[L::c_heads + x];
    for (int q = q0 + lane; q - lane < q1; q += 32) {
        const bool valid = q < q1;
        const int c = valid ? xcol[q] : -1;
        const bool head = valid && (q == 0 || xcol[q - 1] != c);
        const unsigned hm = __ballot_sync(0xffffffffu, head);
        if (head) {
            T sub = xval[q], acc = T(0);
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
            const T res = have ? add_rn(acc, sub) : sub;
            const int idx = nout + __popc(hm & lt);
            if (idx < row_len) {
                __stcs(ccol + idx, c);
                __stcs(cval + idx, res);
            }
        }
        nout += __popc(hm);
    }
    if (w == NW - 1 && lane == 0 && nout != row_len) atomicOr(a.status, kStatusInternal);
    __syncthreads();
}

// at most 64 registers per thread: 1024 threads' worth of blocks per SM
template <int NW, typename T, bool STAGED = false>
__global__ void __launch_bounds__(32 * NW, (32 / NW) < 1 ? 1 : (32 / NW)) k_num_team(RowArgs a) {
    extern __shared__ __align__(16) char smem[];
    using L = TNumLayout<32 * NW * kTeamPer, T>;
    int* ctl = reinterpret_cast<int*>(smem + L::ctl);
    const int begin = a.bin_off[a.bin], end = a.bin_off[a.bin + 1];
    unsigned parity = 0;
    if (STAGED) {
        if (threadIdx.x == 0) mbar_init(reinterpret_cast<unsigned long long*>(smem + L::s_bar), 1);
        __syncthreads();
    }
    // rows by ticket; the next ticket is drawn while the current row runs,
    // into the other of two slots (the row's barriers publish it)
    int slot = 0;
    if (threadIdx.x == 0) ctl[L::c_ticket] = atomicAdd(a.tick + a.bin, 1);
    __syncthreads();
    for (;;) {
        const int i = begin + ctl[L::c_ticket + 2 * slot];
        if (i >= end) break;  // the same in every thread
        if (threadIdx.x == 0) ctl[L::c_ticket + 2 * (slot ^ 1)] = atomicAdd(a.tick + a.bin, 1);
        slot ^= 1;
        num_row_team<NW, T, STAGED>(a, __ldg(a.list + i), smem, &parity);  // ends with a block barrier
    }
}

}  // namespace tsg
