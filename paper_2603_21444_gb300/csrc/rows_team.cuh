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
    static constexpr int kCtl = 96;
    static constexpr int bytes = ctl + 4 * kCtl;
    // ctl words: [0, 34) scan scratch, 40 row ticket, 41 listed buckets,
    // [48, 48 + 32) heads per warp
    static constexpr int c_ticket = 40, c_nwl = 41, c_heads = 48;
    // meta, aliased over [ocol, wl) while the products are gathered
    static constexpr int m_pre = ocol;                             // int[MAXA + 1]
    static constexpr int m_bs = m_pre + 4 * (MAXA + 1);            // int[MAXA]
    static constexpr int m_a = (m_bs + 4 * MAXA + 7) & ~7;         // T[MAXA]
    static constexpr int m_inst = m_a + (int)sizeof(T) * MAXA;     // u8[MAXA]
    static_assert((CAP & (CAP - 1)) == 0, "team capacity must be a power of two");
    static_assert(m_inst + MAXA <= wl, "meta does not fit its alias region");
    static_assert((oval & 7) == 0, "value array alignment");
    static_assert(bytes <= 227 * 1024, "team layout exceeds shared memory");
};

// Row meta of a block team: per A entry (instances in order, entries in
// stored order) its first product, B-row offset, a_ik and instance; nA and
// u for the row (the same in every thread).  Entries beyond MAXA are counted
// but not stored (the caller rejects the row).  Ends with a block barrier.
template <int NT, typename T, int MAXA>
__device__ __forceinline__ void team_meta(const RowArgs& a, int ib, int icount, int rho, int* m_pre, int* m_bs,
                                          T* m_a, unsigned char* m_inst, int* scratch, int& nA, int& u) {
    const int tid = threadIdx.x;
    nA = 0;
    u = 0;
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
            const int ex = Team<NT>::scan_excl(len, &tot, scratch);
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

template <int NW, typename T>
__device__ __forceinline__ void num_row_team(const RowArgs& a, int unit, char* sm) {
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

    int nA, u;
    team_meta<NT, T, L::MAXA>(a, ib, icount, rho, m_pre, m_bs, m_a, m_inst, ctl, nA, u);
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

    // ---- gather: warp w, products [256 w, 256 w + 256), chunked
    int col[PER];
    T val[PER];
    int hh[PER];  // slot in bucket (low 16 bits) | instance << 16
    {
        int ins[PER];
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
        unsigned ex = (unsigned)Team<NT>::scan_excl(loc, &tot, ctl);
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
template <int NW, typename T>
__global__ void __launch_bounds__(32 * NW, (32 / NW) < 1 ? 1 : (32 / NW)) k_num_team(RowArgs a) {
    extern __shared__ __align__(16) char smem[];
    using L = TNumLayout<32 * NW * kTeamPer, T>;
    int* ctl = reinterpret_cast<int*>(smem + L::ctl);
    const int begin = a.bin_off[a.bin], end = a.bin_off[a.bin + 1];
    // rows by ticket; the next ticket is drawn while the current row runs
    if (threadIdx.x == 0) ctl[L::c_ticket] = atomicAdd(a.tick + a.bin, 1);
    __syncthreads();
    for (;;) {
        const int i = begin + ctl[L::c_ticket];
        if (i >= end) break;  // the same in every thread
        __syncthreads();      // everyone has read the ticket
        if (threadIdx.x == 0) ctl[L::c_ticket] = atomicAdd(a.tick + a.bin, 1);
        num_row_team<NW, T>(a, __ldg(a.list + i), smem);  // ends with a block barrier
    }
}

}  // namespace tsg
