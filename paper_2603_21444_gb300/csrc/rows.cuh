// Row kernels of the local product (paper Sec. 2, Sec. 4.4) for sm_103a.
//
// One team (a warp, or a block for the larger variants) owns one output row
// (a work unit) at a time and keeps the whole row on chip:
//
//   meta    for every entry k of the row's A rows (all instances of the
//           group, in order): a pointer to B row k, a_ik, and the exclusive
//           prefix of |B_k|; this flattens the row's u products so product p
//           is read by thread p mod TEAM (coalesced reads of each B row).
//   symbolic  the product columns go into a shared-memory hash set (linear
//           probing, 2 * pow2ceil(u) slots); the count of first insertions
//           is nnz(C_i).
//   numeric   deterministic sort accumulator: each product is keyed by
//           (column, p); a counting sort over NB = pow2ceil(u) buckets (the
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
    static constexpr int table = 0;                               // int[2 CAP]
    static constexpr int m_bc = table + 8 * CAP;                  // const int*[MAXA]
    static constexpr int m_pre = m_bc + 8 * MAXA;                 // int[MAXA + 1]
    static constexpr int scratch = (m_pre + 4 * (MAXA + 1) + 15) & ~15;  // int[34]
    static constexpr int bytes = (scratch + 34 * 4 + 15) & ~15;
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
    const int T2 = 2 * pow2ceil(u);
    const int shift = 32 - (31 - __clz(T2));
    for (int i = r; i < T2; i += TEAM) table[i] = -1;
    int cols[PER];
#pragma unroll
    for (int s = 0; s < PER; ++s) {
        const int p = s * TEAM + r;
        cols[s] = -1;
        if (p < u) {
            const int t = search_pre(m_pre, nA, p);
            cols[s] = __ldg(m_bc[t] + (p - m_pre[t]));
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

template <int TEAM, int PER>
__global__ void __launch_bounds__(TEAM == 32 ? 512 : TEAM, 1) k_sym_rows(RowArgs a) {
    extern __shared__ __align__(16) char smem[];
    constexpr int CAP = TEAM * PER;
    const int begin = a.bin_off[a.bin], end = a.bin_off[a.bin + 1];
    int team, nteams;
    char* sm;
    if (TEAM == 32) {
        const int w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
        team = blockIdx.x * wpb + w;
        nteams = gridDim.x * wpb;
        sm = smem + w * SymLayout<CAP>::bytes;
    } else {
        team = blockIdx.x;
        nteams = gridDim.x;
        sm = smem;
    }
    for (int i = begin + team; i < end; i += nteams) sym_row<TEAM, PER>(a, __ldg(a.list + i), sm);
}

// ------------------------------------------------------------------- numeric

template <int CAP, typename T>
struct NumLayout {
    static constexpr int MAXA = CAP / 2;
    static constexpr int cnt = 0;                                      // int[CAP + 1]
    static constexpr int skey = ((CAP + 1) * 4 + 15) & ~15;           // u64[CAP]
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
    const int NB = pow2ceil(u);
    Bucketer bk;
    bk.init(G.ncols, NB);
    for (int i = r; i <= NB; i += TEAM) cnt[i] = 0;
    Team<TEAM>::sync();

    // gather: all loads first, then the bucket counts
    int col[PER];
    T val[PER];
    int hb[PER];  // low 16 bits: slot in bucket; high bits: instance
#pragma unroll
    for (int s = 0; s < PER; ++s) {
        const int p = s * TEAM + r;
        col[s] = -1;
        val[s] = T(0);
        hb[s] = 0;
        if (p < u) {
            const int t = search_pre(m_pre, nA, p);
            const int j = p - m_pre[t];
            col[s] = __ldg(m_bc[t] + j);
            const T bv = __ldg(m_bv[t] + j);
            val[s] = a.merge ? bv : mul_rn(m_a[t], bv);
            hb[s] = (int)m_inst[t] << 16;
        }
    }
#pragma unroll
    for (int s = 0; s < PER; ++s)
        if (col[s] >= 0) hb[s] |= atomicAdd(&cnt[bk(col[s])], 1);
    Team<TEAM>::sync();

    // bucket starts: exclusive scan of cnt[0..NB)
    {
        const int per = NB >= TEAM ? NB / TEAM : 1;
        const int beg = r * per;
        int loc = 0;
        if (beg < NB)
            for (int i = 0; i < per; ++i) loc += cnt[beg + i];
        int tot;
        int ex = Team<TEAM>::scan_excl(loc, &tot, scratch);
        if (beg < NB)
            for (int i = 0; i < per; ++i) {
                const int c = cnt[beg + i];
                cnt[beg + i] = ex;
                ex += c;
            }
        if (r == 0) cnt[NB] = tot;
    }
    Team<TEAM>::sync();

    // scatter the (column, p) keys into bucket order
#pragma unroll
    for (int s = 0; s < PER; ++s)
        if (col[s] >= 0) {
            const unsigned p = (unsigned)(s * TEAM + r);
            skey[cnt[bk(col[s])] + (hb[s] & 0xffff)] = ((unsigned long long)(unsigned)col[s] << 32) | p;
        }
    Team<TEAM>::sync();

    // rank inside the bucket -> position in (column, p) order
#pragma unroll
    for (int s = 0; s < PER; ++s)
        if (col[s] >= 0) {
            const unsigned p = (unsigned)(s * TEAM + r);
            const int b = bk(col[s]);
            const int lo = cnt[b], hi = cnt[b + 1];
            const unsigned long long key = ((unsigned long long)(unsigned)col[s] << 32) | p;
            int rank = 0;
            for (int q = lo; q < hi; ++q) rank += skey[q] < key;
            const int pos = lo + rank;
            ocol[pos] = col[s];
            oval[pos] = val[s];
            oinst[pos] = (unsigned char)(hb[s] >> 16);
        }
    Team<TEAM>::sync();

    // one output entry per run of equal columns; add the run in p order,
    // each instance's products first, then the instance sums in order
    const bool multi = a.merge || G.inst_count > 1;
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
            int ci = oinst[q];
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

template <int TEAM, int PER, typename T>
__global__ void __launch_bounds__(TEAM == 32 ? 512 : TEAM, 1) k_num_rows(RowArgs a) {
    extern __shared__ __align__(16) char smem[];
    constexpr int CAP = TEAM * PER;
    const int begin = a.bin_off[a.bin], end = a.bin_off[a.bin + 1];
    int team, nteams;
    char* sm;
    if (TEAM == 32) {
        const int w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
        team = blockIdx.x * wpb + w;
        nteams = gridDim.x * wpb;
        sm = smem + w * NumLayout<CAP, T>::bytes;
    } else {
        team = blockIdx.x;
        nteams = gridDim.x;
        sm = smem;
    }
    for (int i = begin + team; i < end; i += nteams) num_row<TEAM, PER, T>(a, __ldg(a.list + i), sm);
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
