// qm_community.cuh -- community-major scoring of one community by a thread group.
//
// Sec. III-A observes that the contribution of a community to the metrics
// without ground truth needs only the edges inside it, the edges on its
// boundary, the edge counts to each neighbouring community and the sizes of it
// and its neighbours, with no dependency between communities.  The kernels
// below take that decomposition literally: a thread group (one warp, or a whole
// block for a large community) owns community c, walks the CSR rows of its
// members, gathers each neighbour's label, counts neighbours inside c
// (2|E_c^in|) and counts every other neighbouring community c_j in a
// shared-memory hash table (|E_c,cj|).  The group then evaluates community c's
// bracketed term of Eq. (9), its six measures (Sec. II-B.3) and its share of
// Eq. (8), with no global atomics and no materialised pair list.
//
// The same walk over the members of a detected community c' with the ground
// truth labels as keys yields the contingency cells |c n c'| of Eqs. (1)-(4).
#pragma once

#include "qm_device.cuh"

namespace qmk {

// Inputs of one partition on one graph.  The batched kernel writes `members`
// and `start` earlier in the same launch, so they are always read through L2
// (__ldcg) after the writer's fence and barrier, never through L1 or the
// read-only path.
struct ScoreCtx {
    const long long *row_ptr;
    const int *col;
    const int *labels;
    const int *members;   // node ids grouped by label: members[start[c] .. start[c+1])
    const int *start;     // int[K + 1]
    const Rcp *recip;     // per community: rcp_of(|c|)
    long long E;          // |E|
    long long n, n_arcs;  // graph size (bounds of the arrays above)
    int K;
    int *err;             // set to 2 when a community cannot be counted (see score_community)
    // optional per-community outputs (device pointers or null)
    long long *pc_size, *pc_ein, *pc_eout;
    double *pc_dens, *pc_contr, *pc_expn, *pc_cond, *pc_qds;
};

struct CompareCtx {
    const int *truth;        // labels of C (ground truth)
    const int *tl;           // truth label of each member position, or null: truth[members[i]]
    const int *members;      // nodes grouped by found label (used when tl is null)
    const int *start;        // int[k_found + 1]
    const int *size_a;       // |c| for c in C
    unsigned *rowmax_n;      // per truth community: max_c' |c n c'|
    unsigned long long *rowmax_r; // per truth community: bits of max 2|c n c'| / (|c|+|c'|)
    long long N;
    int ka, kb;
    int *err;
    const double *logt = nullptr;  // plain comparison: log(N / n), then n / N, 1 <= n <= LOGT_MAX; or null
    int *size_a_acc = nullptr;     // plain comparison: |c| summed from the cells (zeroed), or null
};


// Upper bound of the number of hash classes a block splits one community's
// neighbour ids into.  A community with more than R_MAX * max_used distinct
// neighbouring communities is reported as an error instead of being counted.
constexpr unsigned R_MAX = 1u << 10;

// Group-wide helpers.  A group is either one warp (gsize = 32) or the whole
// block (gsize = blockDim.x).  `red` is block-shared scratch of >= 33 words
// (used only by block groups).
__device__ __forceinline__ unsigned long long group_sum_u64(unsigned long long v, int gsize,
                                                            unsigned long long *red)
{
    v = warp_sum_u64(v);
    if (gsize == 32) return __shfl_sync(0xffffffffu, v, 0);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    block_sync();
    if (lane == 0) red[wid] = v;
    block_sync();
    if (wid == 0) {
        unsigned long long t = lane < nw ? red[lane] : 0ull;
        t = warp_sum_u64(t);
        if (lane == 0) red[32] = t;
    }
    block_sync();
    return red[32];
}

__device__ __forceinline__ unsigned group_max_u32(unsigned v, int gsize, unsigned long long *red)
{
    for (int d = 16; d > 0; d >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, d));
    v = __shfl_sync(0xffffffffu, v, 0);
    if (gsize == 32) return v;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    block_sync();
    if (lane == 0) red[wid] = v;
    block_sync();
    if (wid == 0) {
        unsigned t = lane < nw ? (unsigned)red[lane] : 0u;
        for (int d = 16; d > 0; d >>= 1) t = max(t, __shfl_down_sync(0xffffffffu, t, d));
        if (lane == 0) red[32] = t;
    }
    block_sync();
    return (unsigned)red[32];
}

__device__ __forceinline__ i128 group_sum_i128(i128 v, int gsize, unsigned long long *red)
{
    v = warp_sum_i128(v);
    const int lane = threadIdx.x & 31;
    if (gsize == 32) {
        unsigned long long lo = __shfl_sync(0xffffffffu, (unsigned long long)(u128)v, 0);
        unsigned long long hi = __shfl_sync(0xffffffffu, (unsigned long long)((u128)v >> 64), 0);
        return (i128)(((u128)hi << 64) | lo);
    }
    const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    block_sync();
    if (lane == 0) { red[2 * wid] = (unsigned long long)(u128)v; red[2 * wid + 1] = (unsigned long long)((u128)v >> 64); }
    block_sync();
    if (threadIdx.x == 0) {
        i128 t = 0;
        for (int w = 0; w < nw; ++w) t += (i128)(((u128)red[2 * w + 1] << 64) | red[2 * w]);
        red[64] = (unsigned long long)(u128)t;
        red[65] = (unsigned long long)((u128)t >> 64);
    }
    block_sync();
    return (i128)(((u128)red[65] << 64) | red[64]);
}

// Exclusive scan of one value per group thread; returns the group total.
__device__ __forceinline__ unsigned group_exclusive_scan(unsigned v, unsigned &excl, int gsize,
                                                         unsigned long long *red)
{
    const int lane = threadIdx.x & 31;
    unsigned inc = v;
    for (int d = 1; d < 32; d <<= 1) {
        unsigned t = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += t;
    }
    if (gsize == 32) {
        excl = inc - v;
        return __shfl_sync(0xffffffffu, inc, 31);
    }
    const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    block_sync();
    if (lane == 31) red[wid] = inc;
    block_sync();
    if (wid == 0) {
        unsigned t = lane < nw ? (unsigned)red[lane] : 0u, s = t;
        for (int d = 1; d < 32; d <<= 1) {
            unsigned u = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += u;
        }
        if (lane < nw) red[lane] = s - t;  // exclusive warp offsets
        if (lane == 31) red[32] = s;
    }
    block_sync();
    excl = (unsigned)red[wid] + inc - v;
    return (unsigned)red[32];
}

// Reads out the table: calls f(key, count) for every occupied slot and clears it.
template <typename F>
__device__ __forceinline__ void tab_drain(const SmemTable &t, int gtid, int gsize, F f)
{
    const int n = min(*t.n_used, t.max_used);
    for (int i = gtid; i < n; i += gsize) {
        const int h = t.used[i];
        if (!QM_CHK(h, t.cap, 9)) continue;
        const unsigned long long s = t.slot[h];
        f((int)(s >> 32) - 1, (long long)(s & 0xFFFFFFFFull));
        t.slot[h] = 0ull;
    }
}

// Clears every slot (after an overflow, when `used` is incomplete).
__device__ __forceinline__ void tab_wipe(const SmemTable &t, int gtid, int gsize)
{
    for (int i = gtid; i < t.cap; i += gsize) t.slot[i] = 0ull;
}

__device__ __forceinline__ u128 shfl_down_u128(u128 v, int d)
{
    unsigned long long lo = __shfl_down_sync(0xffffffffu, (unsigned long long)v, d);
    unsigned long long hi = __shfl_down_sync(0xffffffffu, (unsigned long long)(v >> 64), d);
    return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ double u128_to_double(u128 v)
{
    return __dadd_rn(__dmul_rn((double)(unsigned long long)(v >> 64), 18446744073709551616.0),
                     (double)(unsigned long long)v);
}

// Community c's share of the Eq. (9) split penalty when each unordered pair
// of communities is charged once, to its smaller id: T_c / (|E| |c|), T_c in
// 64.64 fixed point (see score_community).
__device__ __forceinline__ double pair_penalty_once(u128 t, long long size, long long E)
{
    return __ddiv_rn(ldexp(u128_to_double(t), -64), __dmul_rn((double)E, (double)size));
}

// Community c's own split penalty of Eq. (9), S_c / (2|E| |c|) (the
// per-community Qds term), S_c in 64.64 fixed point.
__device__ __forceinline__ double pair_penalty_own(u128 s, long long size, long long E)
{
    return __ddiv_rn(ldexp(u128_to_double(s), -64), __dmul_rn(__dmul_rn(2.0, (double)E), (double)size));
}


// Group totals of NW 64-bit words per thread, delivered to the group leader
// (group thread 0): a warp reduction, then for a block group one exchange
// through `red` (>= 32 * NW words) and one barrier.  Only the leader's result
// is meaningful.  Words are added as unsigned integers, so a 128-bit value can
// travel as two words and be recombined with carry by the caller (see sum128).
template <int NW>
__device__ __forceinline__ void group_words_to_leader(unsigned long long (&v)[NW], int gsize,
                                                      unsigned long long *red)
{
#pragma unroll
    for (int k = 0; k < NW; ++k) v[k] = warp_sum_u64(v[k]);
    if (gsize == 32) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NW; ++k) red[wid * NW + k] = v[k];
    block_sync();
    if (threadIdx.x == 0)
        for (int w = 1; w < nw; ++w)
#pragma unroll
            for (int k = 0; k < NW; ++k) v[k] += red[w * NW + k];
}

// A 128-bit group total, summed exactly (warp shuffles of both halves, then the
// warps' totals through `red` at word offset `at`).  Valid in the leader only.
__device__ __forceinline__ u128 group_u128_to_leader(u128 v, int gsize, unsigned long long *red, int at)
{
    for (int d = 16; d > 0; d >>= 1) v += shfl_down_u128(v, d);
    if (gsize == 32) return v;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        red[at + 2 * wid] = (unsigned long long)v;
        red[at + 2 * wid + 1] = (unsigned long long)(v >> 64);
    }
    block_sync();
    if (threadIdx.x == 0)
        for (int w = 1; w < nw; ++w) v += ((u128)red[at + 2 * w + 1] << 64) | red[at + 2 * w];
    return v;
}


// A 192-bit group total (valid in the leader only); the warps' totals travel
// through `red` at word offset `at` (3 words per warp).
__device__ __forceinline__ U192 group_u192_to_leader(U192 v, int gsize, unsigned long long *red, int at)
{
    v = u192_warp_sum(v);
    if (gsize == 32) return v;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        red[at + 3 * wid] = v.w0;
        red[at + 3 * wid + 1] = v.w1;
        red[at + 3 * wid + 2] = v.w2;
    }
    block_sync();
    if (threadIdx.x == 0)
        for (int w = 1; w < nw; ++w) {
            const U192 o{red[at + 3 * w], red[at + 3 * w + 1], red[at + 3 * w + 2]};
            u192_add(v, o);
        }
    return v;
}

// Score community c with a group (one warp, or a whole block).  Returns false
// only for a warp whose table overflowed (nothing was accumulated; the caller
// re-queues c for a block).  A block handles overflow itself by splitting the
// neighbour ids into R hash classes and walking the rows once per class.
//
// Each warp of the group takes its own chunks of 32 members (a warp-local
// prefix sum of their degrees in `offs`/`rs`, the warp's slices of shared
// staging), so the arc walk needs no block-wide barrier; all warps insert into
// the group's shared table.  The split penalty of Eq. (9) summed over all
// communities is
//   sum_i sum_{j != i} |E_ij|^2 / (2|E| |c_i| |c_j|) = sum_i T_i / (|E| |c_i|)
// with T_i = sum_{j > i} |E_ij|^2 / |c_j|: the ordered sum counts every
// unordered pair twice with the same value, so each pair is charged once, to
// its smaller id, and only neighbour ids above i are counted.  T_i is summed
// exactly with 128-bit reciprocals (x.recip, see rcp_of): one division per
// community is done in FP64.  A per-community Qds term needs i's own penalty
// S_i / (2|E| |c_i|) with S_i = sum_{j != i} |E_ij|^2 / |c_j|, which is then
// summed as well.
__device__ __forceinline__ bool score_community(const ScoreCtx &x, int c, const SmemTable &tab,
                                                unsigned *offs, long long *rs, ScoreAcc *acc,
                                                int gtid, int gsize, unsigned long long *red)
{
    const int lane = threadIdx.x & 31;
    const int wrank = gtid >> 5;
    unsigned *offw = offs + (threadIdx.x >> 5) * 33;
    long long *rsw = rs + (threadIdx.x >> 5) * 32;
    const int mb = __ldcg(&x.start[c]), me = __ldcg(&x.start[c + 1]);
    const long long size = me - mb;
    unsigned R = 1;
    const bool full = x.pc_qds != nullptr;
    for (;;) {
        unsigned long long same = 0, vol = 0, slots = 0, cnt2 = 0;
        U192 inner, inner_full;
        u192_zero(inner);
        u192_zero(inner_full);
        bool ok = true;
        for (unsigned r = 0; r < R && ok; ++r) {
            for (int cb = mb + wrank * 32; cb < me; cb += gsize) {
                const int i = cb + lane;
                unsigned d = 0;
                long long rsi = 0;
                if (i < me && QM_CHK(i, x.n, 1)) {
                    const int u = __ldcg(&x.members[i]);
                    if (QM_CHK(u, x.n, 2)) {
                        rsi = __ldg(&x.row_ptr[u]);
                        d = (unsigned)(__ldg(&x.row_ptr[u + 1]) - rsi);
                    }
                }
                if (r == 0) vol += d;
                unsigned inc = d;
#pragma unroll
                for (int s2 = 1; s2 < 32; s2 <<= 1) {
                    const unsigned t = __shfl_up_sync(0xffffffffu, inc, s2);
                    if (lane >= s2) inc += t;
                }
                const unsigned total = __shfl_sync(0xffffffffu, inc, 31);
                const int nm = min(32, me - cb);
                if (lane < nm) { offw[lane] = inc - d; rsw[lane] = rsi; }
                __syncwarp();
                for (unsigned e0 = lane; e0 < total; e0 += 128u) {
                    int v[4], lv[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const unsigned e = e0 + 32u * k;
                        v[k] = -1;
                        if (e < total) {
                            const int o = upper_bound_smem(offw, nm, e) - 1;
                            if (QM_CHK(o, nm, 4) && QM_CHK(rsw[o] + (e - offw[o]), x.n_arcs, 3))
                                v[k] = __ldg(&x.col[rsw[o] + (e - offw[o])]);
                            if (!QM_CHK(v[k], x.n, 5)) v[k] = -1;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) lv[k] = v[k] >= 0 ? __ldg(&x.labels[v[k]]) : -1;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (v[k] < 0) continue;
                        if (!QM_CHK(lv[k], x.K, 6)) continue;
                        if (lv[k] == c) {
                            if (r == 0) ++same;
                        } else if ((full || lv[k] > c) && (R == 1 || tab_split((unsigned)lv[k], R) == r)) {
                            tab_insert(tab, (unsigned)lv[k]);
                        }
                    }
                }
                __syncwarp();
            }
            group_sync(gsize);
            if (*(volatile int *)tab.overflow) {
                ok = false;
                break;
            }
            tab_drain(tab, gtid, gsize, [&](int key, long long cnt) {
                if (!QM_CHK(key, x.K, 7)) return;
                const unsigned long long q = (unsigned long long)cnt * (unsigned long long)cnt;
                const Rcp rj = ld_rcp_cg(&x.recip[key]);
                if (full) u192_mac(inner_full, q, rj);
                if (key > c) {
                    u192_mac(inner, q, rj);
                    ++slots;
                    cnt2 += q;
                }
            });
            group_sync(gsize);
            if (gtid == 0) *tab.n_used = 0;
            group_sync(gsize);
        }
        if (!ok) {
            tab_wipe(tab, gtid, gsize);
            group_sync(gsize);
            if (gtid == 0) { *tab.n_used = 0; *tab.overflow = 0; }
            group_sync(gsize);
            if (gsize == 32) return false;
            // Pass 0 completed, so the exact boundary arc count E_out (an upper
            // bound of the distinct neighbour communities) sizes R.
            unsigned long long w2[2] = {vol, same};
            group_words_to_leader<2>(w2, gsize, red);
            if (gtid == 0) {
                const unsigned long long eout = w2[0] - w2[1];
                const unsigned long long need = (eout * 4 + 3ull * tab.max_used - 1) / (3ull * tab.max_used);
                red[255] = max((unsigned long long)R * 2ull, need);
            }
            group_sync(gsize);
            const unsigned long long nr = red[255];
            group_sync(gsize);
            if (nr > R_MAX) {
                if (gtid == 0) atomicOr(x.err, 2);
                return true;
            }
            R = (unsigned)nr;
            continue;
        }
        // commit: the group leader receives the totals and adds the community's
        // terms to the group's shared accumulator
        unsigned long long w4[4] = {same, vol, slots, cnt2};
        group_words_to_leader<4>(w4, gsize, red);
        const u128 inner_t = u192_shr64(group_u192_to_leader(inner, gsize, red, 128));
        u128 full_t = 0;
        if (full) {
            group_sync(gsize);  // the leader has read inner's words from `red` before they are reused
            full_t = u192_shr64(group_u192_to_leader(inner_full, gsize, red, 128));
        }
        if (gtid == 0) {
            same = w4[0];
            vol = w4[1];
            const long long ein = (long long)(same / 2), eout = (long long)(vol - same);
            double qs, dens, contr, expn, cond;
            community_terms(ein, eout, size, x.E, qs, dens, contr, expn, cond);
            const double pen = pair_penalty_once(inner_t, size, x.E);
            acc->qds_pair += fp_from_double(pen, SC_QDS);
            acc->slots += w4[2];
            acc->cnt2 += w4[3];
            acc->qds_self += fp_from_double(qs, SC_QDS);
            acc->dens += fp_from_double(dens, SC_MEAN);
            acc->contr += fp_from_double(contr, SC_MEAN);
            acc->expn += fp_from_double(expn, SC_MEAN);
            acc->cond += fp_from_double(cond, SC_MEAN);
            acc->vol2 += (u128)vol * (u128)vol;
            acc->ein += (unsigned long long)ein;
            acc->eout += (unsigned long long)eout;
            acc->nonempty += 1;
            if (x.pc_size) x.pc_size[c] = size;
            if (x.pc_ein) x.pc_ein[c] = ein;
            if (x.pc_eout) x.pc_eout[c] = eout;
            if (x.pc_dens) x.pc_dens[c] = dens;
            if (x.pc_contr) x.pc_contr[c] = contr;
            if (x.pc_expn) x.pc_expn[c] = expn;
            if (x.pc_cond) x.pc_cond[c] = cond;
            if (x.pc_qds) x.pc_qds[c] = __dsub_rn(qs, pair_penalty_own(full_t, size, x.E));
        }
        return true;
    }
}

// Contingency cells of one detected community b: hash the ground-truth labels
// of its members.  A warp group is only given communities whose size fits its
// table (the number of distinct keys never exceeds the member count), so only
// a block group can overflow; it then splits the keys into R classes.
__device__ __forceinline__ void compare_community(const CompareCtx &x, int b, const SmemTable &tab,
                                                  CompareAcc *acc, int gtid, int gsize,
                                                  unsigned long long *red)
{
    const int mb = __ldcg(&x.start[b]), me = __ldcg(&x.start[b + 1]);
    const long long nb = me - mb;
    unsigned R = 1;
    if (nb > tab.max_used) R = (unsigned)((nb * 4 + 3LL * tab.max_used - 1) / (3LL * tab.max_used));
    for (;;) {
        if (R > R_MAX) {
            if (gtid == 0) atomicOr(x.err, 2);
            return;
        }
        unsigned colmax = 0;
        unsigned long long a11 = 0, cells = 0;
        i128 vi = 0, hn = 0;
        bool ok = true;
        for (unsigned r = 0; r < R; ++r) {
            for (int i0 = mb + (gtid & ~31); i0 < me; i0 += gsize) {  // warp-uniform trips
                const int i = i0 + (gtid & 31);
                const int a = i < me ? (x.tl ? __ldcg(&x.tl[i]) : __ldg(&x.truth[__ldcg(&x.members[i])])) : 0;
                tab_insert_warp(tab, (unsigned)a, i < me && (R == 1 || tab_split((unsigned)a, R) == r));
            }
            group_sync(gsize);
            if (*(volatile int *)tab.overflow) { ok = false; break; }
            tab_drain(tab, gtid, gsize, [&](int a, long long n) {
                const long long na = __ldcg(&x.size_a[a]);
                a11 += (unsigned long long)(n * (n - 1) / 2);
                ++cells;
                colmax = max(colmax, (unsigned)n);
                atomicMax(&x.rowmax_n[a], (unsigned)n);
                atomicMax(&x.rowmax_r[a], (unsigned long long)__double_as_longlong(f_ratio(n, na, nb)));
                const double l1 = cell_log(n, na, nb);
                vi += fp_from_double(vi_term_l(n, l1), SC_VI);
                hn += fp_from_double(nmi_num_term_l(n, x.N, l1, log_ratio(x.N, n)), SC_H);
            });
            group_sync(gsize);
            if (gtid == 0) *tab.n_used = 0;
            group_sync(gsize);
        }
        if (!ok) {
            tab_wipe(tab, gtid, gsize);
            group_sync(gsize);
            if (gtid == 0) { *tab.n_used = 0; *tab.overflow = 0; }
            group_sync(gsize);
            R *= 2;
            continue;
        }
        for (int d = 16; d > 0; d >>= 1) colmax = max(colmax, __shfl_down_sync(0xffffffffu, colmax, d));
        unsigned long long w[3] = {a11, cells, 0ull};
        // the column maximum travels through the same exchange: the warps'
        // maxima are combined by the leader below
        if (gsize != 32) {
            if ((threadIdx.x & 31) == 0) red[96 + (threadIdx.x >> 5)] = colmax;
        }
        group_words_to_leader<3>(w, gsize, red);
        const u128 vi_t = group_u128_to_leader((u128)vi, gsize, red, 128);
        const u128 hn_t = group_u128_to_leader((u128)hn, gsize, red, 192);
        if (gtid == 0) {
            if (gsize != 32)
                for (int k = 1; k < (int)(blockDim.x >> 5); ++k) colmax = max(colmax, (unsigned)red[96 + k]);
            acc->a11 += w[0];
            acc->cells += w[1];
            acc->vi += (i128)vi_t;
            acc->hnum += (i128)hn_t;
            acc->nvd += colmax;
            acc->sb += (unsigned long long)(nb * (nb - 1) / 2);
            acc->hden += fp_from_double(entropy_term(nb, x.N), SC_H);
            acc->kb += 1;
        }
        return;
    }
}

// One contingency cell |c_a n c'_b| = n (Eqs. 1-4), written by the counting
// pass of the comparison and turned into terms by a parallel pass.
struct __align__(16) Cell {
    int a, b;
    unsigned n, pad;
};

// Counts the truth labels of found community b's members (x.tl, in member
// order) and appends one Cell per distinct truth label to cells[*ncells ..].
// Only the integer column maximum (NVD, Eq. 4) and the cell count are kept
// here; every term that needs the cell sizes is formed later, in parallel.
// The hash classes are chosen up front with room to spare (distinct labels
// are at most min(|b|, ka)), because cells of a finished class are already
// out; a class that still overflows is reported, never silently dropped.
__device__ __forceinline__ void compare_cells_community(const CompareCtx &x, int b, const SmemTable &tab,
                                                        CompareAcc *acc, int gtid, int gsize,
                                                        unsigned long long *red, Cell *cells, int *ncells)
{
    const int mb = __ldcg(&x.start[b]), me = __ldcg(&x.start[b + 1]);
    const long long nb = me - mb;
    const long long distinct = min(nb, (long long)x.ka);
    unsigned R = 1;
    if (distinct > tab.max_used) R = (unsigned)((2 * distinct + tab.max_used - 1) / tab.max_used);
    if (R > R_MAX) {
        if (gtid == 0) atomicOr(x.err, 2);
        return;
    }
    unsigned colmax = 0;
    unsigned long long ncell = 0;
    for (unsigned r = 0; r < R; ++r) {
        for (int i0 = mb + (gtid & ~31); i0 < me; i0 += gsize) {  // warp-uniform trips
            const int i = i0 + (gtid & 31);
            const int a = i < me ? (x.tl ? __ldcg(&x.tl[i]) : __ldg(&x.truth[__ldcg(&x.members[i])])) : 0;
            tab_insert_warp(tab, (unsigned)a, i < me && (R == 1 || tab_split((unsigned)a, R) == r));
        }
        group_sync(gsize);
        if (*(volatile int *)tab.overflow) {
            if (gtid == 0) atomicOr(x.err, 2);
            return;
        }
        const int nu = min(*tab.n_used, tab.max_used);
        int base = 0;
        if (gtid == 0 && nu > 0) base = atomicAdd(ncells, nu);
        if (gsize == 32) {
            base = __shfl_sync(0xffffffffu, base, 0);
        } else {
            if (gtid == 0) red[255] = (unsigned long long)base;
            group_sync(gsize);
            base = (int)red[255];
        }
        for (int i = gtid; i < nu; i += gsize) {
            const int h = tab.used[i];
            if (!QM_CHK(h, tab.cap, 9)) continue;
            const unsigned long long sv = tab.slot[h];
            const unsigned n = (unsigned)(sv & 0xFFFFFFFFull);
            cells[base + i] = Cell{(int)(sv >> 32) - 1, b, n, 0u};
            if (x.size_a_acc) atomicAdd(&x.size_a_acc[(int)(sv >> 32) - 1], (int)n);
            colmax = max(colmax, n);
            tab.slot[h] = 0ull;
        }
        ncell += (unsigned long long)nu;
        group_sync(gsize);
        if (gtid == 0) *tab.n_used = 0;
        group_sync(gsize);
    }
    colmax = (unsigned)group_max_u32(colmax, gsize, red);
    if (gtid == 0) {
        acc->nvd += colmax;
        acc->cells += ncell;
    }
    if (gsize != 32) group_sync(gsize);
}

// ---------------------------------------------------------------- two-phase scoring
//
// Phase A (k_expand) visits every member of every community in member order
// and looks up the labels of its neighbours.  Arcs to the member's own
// community are only counted; the labels of the other arcs are packed densely
// at the front of the community's arc segment, nbr[aoff[start[c]] ..
// aoff[start[c]] + inter[c]), in no particular order.  Phase B
// (count_community) reads that packed run with coalesced loads and counts
// |E_cj| for every j != c in a shared-memory table.  Phase B leaves one
// integer record per community; the FP64 terms are formed afterwards for all
// communities in parallel (k_score_terms).

// Per-community record written by phase B (unsigned 64-bit words).  INNER is
// T_c = sum_{j > c} |E_cj|^2 / |c_j| (64.64 fixed point), the community's share
// of the Eq. (9) split penalty when every unordered pair {c, j} is charged once
// (to its smaller id); SLOTS and CNT2 count those pairs and sum |E_cj|^2.  FULL
// is S_c = sum_{j != c} |E_cj|^2 / |c_j|, the community's own penalty sum,
// formed only when the per-community Qds terms are asked for.
enum { REC_SAME = 0, REC_VOL = 1, REC_SLOTS = 2, REC_CNT2 = 3, REC_INNER_LO = 4, REC_INNER_HI = 5,
       REC_FULL_LO = 6, REC_FULL_HI = 7, REC_WORDS = 8 };

struct CountCtx {
    const int *nbr;                   // packed inter-community neighbour labels
    const unsigned *aoff;             // [n + 1] arc offset of each member position
    const int *start;                 // [K + 1] member offsets
    const int *inter;                 // [K] cut arcs of each community (its packed run may hold only part)
    const Rcp *recip;                 // rcp_of(|c|)
    unsigned long long *rec;          // [K][REC_WORDS]
    int K;
    int *err;
    int full;                         // also form S_c (per-community Qds terms asked for)
};

// L2 eviction-priority hints (PTX createpolicy / ld.global.L2::cache_hint):
// the label array is gathered at random and should stay resident, while the
// adjacency and the packed labels stream through once.
__device__ __forceinline__ unsigned long long l2_policy_evict_last()
{
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ int ld_hint(const int *ptr, unsigned long long pol)
{
    int v;
    asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(ptr), "l"(pol));
    return v;
}

// Largest load of a phase-B counting table: a run is given to a table that
// it fills to at most COUNT_FILL_NUM / COUNT_FILL_DEN of its slots (beyond
// that, the probe chains of linear probing grow, and a warp waits for its
// longest).
constexpr int COUNT_FILL_NUM = 3, COUNT_FILL_DEN = 4;
__host__ __device__ constexpr long long count_fill(long long cap) { return cap * COUNT_FILL_NUM / COUNT_FILL_DEN; }

// Epoch-tagged counting tables (phase B).  A group's table is reused for
// community after community: every slot carries the epoch it was written in
// and counts as empty unless that is the group's current epoch, so a new
// community (or hash class) only advances the epoch instead of clearing the
// table; epoch 0 marks a slot never used.  After 255 epochs the group wipes
// its table and starts again at 1.  Both layouts take `bytes_per_slot` = 8
// bytes of shared memory per slot and expose the same calls:
//   add(key, epoch)  adds one occurrence and returns how many came before it
//                    in this epoch, or -1 when the table is full;
//   wipe(gtid, gsize).
// Runs never exceed 2^24 entries here (longer ones take the general path), so
// every count fits the fields below.
constexpr unsigned ET_MAX_RUN = 1u << 24;

// 64-bit slots [63:56] epoch [55:25] key + 1 [24:0] occurrences, for any K.
struct EpochTable {
    unsigned long long *slot;
    int cap;
    int *overflow;   // shared flag: a key found no free slot

    static constexpr int CNT_BITS = 25;
    static constexpr unsigned long long CNT_MASK = (1ull << CNT_BITS) - 1ull;

    __device__ __forceinline__ int add(unsigned key, unsigned epoch) const
    {
        const unsigned long long tag = ((unsigned long long)epoch << 56) | ((unsigned long long)(key + 1u) << CNT_BITS);
        unsigned h = tab_hash(key, cap);
        unsigned long long cur = ((volatile unsigned long long *)slot)[h];
        const int limit = 2 * cap + 64;
        for (int step = 0; step < limit; ++step) {
            if (!QM_CHK(h, cap, 8)) return -1;
            if ((unsigned)(cur >> 56) != epoch) {
                const unsigned long long prev = atomicCAS(&slot[h], cur, tag | 1ull);
                if (prev == cur) return 0;
                cur = prev;  // the slot changed under us: look at it again
                continue;
            }
            if ((cur & ~CNT_MASK) == tag) return (int)(atomicAdd(&slot[h], 1ull) & CNT_MASK);
            if ((step & 15) == 15 && *(volatile int *)overflow) return -1;
            h = (h + 1u == (unsigned)cap) ? 0u : h + 1u;
            cur = ((volatile unsigned long long *)slot)[h];
        }
        *overflow = 1;
        return -1;
    }

    __device__ __forceinline__ void wipe(int gtid, int gsize) const
    {
        for (int i = gtid; i < cap; i += gsize) slot[i] = 0ull;
    }
};

// Two 32-bit words per slot, for K < 2^24: key[h] = [31:24] epoch [23:0]
// key + 1, claimed with a 32-bit CAS (half the shared-memory atomic work of
// a 64-bit one), and rep[h] = [31:24] epoch [23:0] repeats, touched only by
// second and later occurrences of a key.  The first occurrence leaves rep[h]
// alone: a word of an older epoch reads as no repeats.
struct EpochTable32 {
    unsigned *key;   // [cap]
    unsigned *rep;   // [cap], right after key
    int cap;
    int *overflow;

    __device__ __forceinline__ int add(unsigned k, unsigned epoch) const
    {
        const unsigned tag = (epoch << 24) | (k + 1u);
        unsigned h = tab_hash(k, cap);
        unsigned cur = ((volatile unsigned *)key)[h];
        const int limit = 2 * cap + 64;
        for (int step = 0; step < limit; ++step) {
            if (!QM_CHK(h, cap, 8)) return -1;
            if ((cur >> 24) != epoch) {
                const unsigned prev = atomicCAS(&key[h], cur, tag);
                if (prev == cur) return 0;
                cur = prev;  // the slot changed under us: look at it again
                continue;
            }
            if (cur == tag) {
                unsigned w = ((volatile unsigned *)rep)[h];
                for (int r = 0; r < limit; ++r) {
                    const bool same = (w >> 24) == epoch;
                    const unsigned prev = atomicCAS(&rep[h], w, same ? w + 1u : ((epoch << 24) | 1u));
                    if (prev == w) return 1 + (same ? (int)(w & 0xFFFFFFu) : 0);
                    w = prev;
                }
                break;
            }
            if ((step & 15) == 15 && *(volatile int *)overflow) return -1;
            h = (h + 1u == (unsigned)cap) ? 0u : h + 1u;
            cur = ((volatile unsigned *)key)[h];
        }
        *overflow = 1;
        return -1;
    }

    __device__ __forceinline__ void wipe(int gtid, int gsize) const
    {
        for (int i = gtid; i < 2 * cap; i += gsize) key[i] = 0u;  // key and rep are contiguous
    }
};

// Four consecutive words of shared memory in one load, read afresh.
__device__ __forceinline__ uint4 ld_shared_v4_volatile(const unsigned *p)
{
    uint4 v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(a));
    return v;
}

// The words of EpochTable32, probed four slots at a time: a key's probe
// sequence starts at the aligned group of four slots that holds
// tab_hash(k, cap), and one 16-byte load reads a whole group, so the longest
// chain of probes in a warp (which the warp waits for) is about a quarter as
// long.  The table lives in shared memory, 16-byte aligned, with cap a
// multiple of 4.
struct EpochTable32V {
    unsigned *key;   // [cap]
    unsigned *rep;   // [cap], right after key
    int cap;
    int *overflow;

    // a later occurrence of the key in slot h: its repeat count
    __device__ __forceinline__ int repeat(unsigned h, unsigned epoch) const
    {
        unsigned w = ((volatile unsigned *)rep)[h];
        for (int r = 0; r < 2 * cap + 64; ++r) {
            const bool same = (w >> 24) == epoch;
            const unsigned prev = atomicCAS(&rep[h], w, same ? w + 1u : ((epoch << 24) | 1u));
            if (prev == w) return 1 + (same ? (int)(w & 0xFFFFFFu) : 0);
            w = prev;
        }
        *overflow = 1;
        return -1;
    }

    __device__ __forceinline__ int add(unsigned k, unsigned epoch) const
    {
        const unsigned tag = (epoch << 24) | (k + 1u);
        unsigned g = tab_hash(k, cap) & ~3u;
        const int limit = cap / 4 + 16;
        for (int step = 0; step < limit; ++step) {
            if (!QM_CHK(g + 3u, cap, 8)) return -1;
            const uint4 w = ld_shared_v4_volatile(key + g);
            const unsigned c4[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                unsigned cur = c4[s];
                if (cur != tag && (cur >> 24) != epoch) {  // a slot free in this epoch: claim it
                    cur = atomicCAS(&key[g + s], cur, tag);
                    if (cur == c4[s]) return 0;
                    // taken meanwhile (by this key, or another one)
                }
                if (cur == tag) return repeat(g + s, epoch);
            }
            if ((step & 3) == 3 && *(volatile int *)overflow) return -1;
            g = (g + 4u >= (unsigned)cap) ? 0u : g + 4u;
        }
        *overflow = 1;
        return -1;
    }

    __device__ __forceinline__ void wipe(int gtid, int gsize) const
    {
        for (int i = gtid; i < 2 * cap; i += gsize) key[i] = 0u;  // key and rep are contiguous
    }
};

// Table over `cap` slots at `base` (8 bytes each).
template <class TAB>
__device__ __forceinline__ TAB make_table(unsigned long long *base, int cap, int *overflow);
template <>
__device__ __forceinline__ EpochTable make_table<EpochTable>(unsigned long long *base, int cap, int *overflow)
{
    return EpochTable{base, cap, overflow};
}
template <>
__device__ __forceinline__ EpochTable32 make_table<EpochTable32>(unsigned long long *base, int cap, int *overflow)
{
    return EpochTable32{(unsigned *)base, (unsigned *)base + cap, cap, overflow};
}
template <>
__device__ __forceinline__ EpochTable32V make_table<EpochTable32V>(unsigned long long *base, int cap, int *overflow)
{
    return EpochTable32V{(unsigned *)base, (unsigned *)base + cap, cap, overflow};
}

// Next epoch of a group (all its threads hold the same value); wipes the
// table when the 8-bit epoch wraps.  The caller has passed a group barrier
// since the table's last use.
template <class TAB>
__device__ __forceinline__ unsigned etab_next_epoch(const TAB &t, unsigned epoch, int gtid, int gsize)
{
    if (epoch < 255u) return epoch + 1u;
    t.wipe(gtid, gsize);
    group_sync_n(gsize);
    return 1u;
}

// Writes community c's record from the group totals (leader only).
__device__ __forceinline__ void put_record(const CountCtx &x, int c, unsigned vol, unsigned m,
                                           unsigned long long slots, unsigned long long cnt2, const U192 &inner,
                                           const U192 &inner_full)
{
    const u128 in = u192_shr64(inner), fu = u192_shr64(inner_full);
    unsigned long long *rc = x.rec + (size_t)c * REC_WORDS;
    // |E_c^out| is the cut-arc count (the packed run may hold only part of it)
    (void)m;
    rc[REC_SAME] = (unsigned long long)(vol - (unsigned)x.inter[c]);
    rc[REC_VOL] = (unsigned long long)vol;
    rc[REC_SLOTS] = slots;
    rc[REC_CNT2] = cnt2;
    rc[REC_INNER_LO] = (unsigned long long)in;
    rc[REC_INNER_HI] = (unsigned long long)(in >> 64);
    rc[REC_FULL_LO] = (unsigned long long)fu;
    rc[REC_FULL_HI] = (unsigned long long)(fu >> 64);
}

// Group totals of (slots, cnt2, inner[, inner_full]) delivered to the leader
// with one exchange (5 or 8 words per warp in `red`); for a block its barrier
// also orders this community's inserts before the next community's.
template <bool FULL>
__device__ __forceinline__ void group_totals(unsigned long long &slots, unsigned long long &cnt2, U192 &inner,
                                             U192 &inner_full, int gsize, unsigned long long *red)
{
    slots = warp_sum_u64(slots);
    cnt2 = warp_sum_u64(cnt2);
    inner = u192_warp_sum(inner);
    if (FULL) inner_full = u192_warp_sum(inner_full);
    if (gsize == 32) return;
    constexpr int WW = FULL ? 8 : 5;
    // the group's warps are w0 .. w0 + nw - 1; its leader is its first thread
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = gsize >> 5;
    const int w0 = ((int)threadIdx.x / gsize) * nw;
    if (lane == 0) {
        red[WW * wid] = slots;
        red[WW * wid + 1] = cnt2;
        red[WW * wid + 2] = inner.w0;
        red[WW * wid + 3] = inner.w1;
        red[WW * wid + 4] = inner.w2;
        if (FULL) {
            red[WW * wid + 5] = inner_full.w0;
            red[WW * wid + 6] = inner_full.w1;
            red[WW * wid + 7] = inner_full.w2;
        }
    }
    group_sync_n(gsize);
    if ((int)threadIdx.x % gsize == 0)
        for (int w = w0 + 1; w < w0 + nw; ++w) {
            slots += red[WW * w];
            cnt2 += red[WW * w + 1];
            const U192 o{red[WW * w + 2], red[WW * w + 3], red[WW * w + 4]};
            u192_add(inner, o);
            if (FULL) {
                const U192 f{red[WW * w + 5], red[WW * w + 6], red[WW * w + 7]};
                u192_add(inner_full, f);
            }
        }
}

// Header of one community's packed run, written by k_classify: the run is
// nbr[a0 .. a0 + m), the community's volume is vol (2|E_c^in| + |E_c^out|).
struct __align__(16) RunHdr {
    int c;
    unsigned a0, m, vol;
};

// Adds one entry's share of the pair sum: the k-th occurrence (prev = k - 1)
// of a key with reciprocal r adds (2k - 1) r.
__device__ __forceinline__ void add_share(U192 &inner, unsigned long long &slots, unsigned long long &cnt2, int prev,
                                          const Rcp &r)
{
    if (prev == 0) {  // first occurrence (the common case): q = 1
        u192_add_rcp(inner, r);
        cnt2 += 1ull;
        slots += 1ull;
    } else {
        const unsigned long long q = 2ull * (unsigned long long)prev + 1ull;
        u192_mac(inner, q, r);
        cnt2 += q;
    }
}

// Counts the m entries of community h.c's run, read from `src` (shared-memory
// staging when SMEM, else the packed array in global memory), with a group (a
// warp, or the whole block).  Every entry is a label j != c, so m bounds the
// distinct keys.  Only labels j > c are counted (each unordered pair is
// charged to its smaller id, see score_community), unless FULL, when every
// label is counted and S_c formed too.  Each counted entry adds its own share
// of the Eq. (9) pair sum: the k-th occurrence of key j adds (2k - 1) Rcp_j, so
// no pass over the table is needed afterwards.  When m exceeds what the table
// holds at 3/4 load the keys are split into R hash classes and the run is read
// once per class.  `epoch` is the group's table epoch (updated).
template <bool SMEM, bool FULL, class TAB>
__device__ __forceinline__ void count_run(const CountCtx &x, const RunHdr &h, const int *src, const TAB &tab,
                                          unsigned &epoch, int gtid, int gsize, unsigned long long *red)
{
    const unsigned m = h.m;
    const unsigned fill = (unsigned)count_fill(tab.cap);
    unsigned R = m <= fill ? 1u : (unsigned)min((unsigned long long)R_MAX, ((unsigned long long)m + fill - 1) / fill);
    const int c = h.c;
    for (;;) {
        unsigned long long slots = 0, cnt2 = 0, s_dummy = 0, c_dummy = 0;
        U192 inner, inner_full;
        u192_zero(inner);
        u192_zero(inner_full);
        bool ok = true;
        for (unsigned r = 0; r < R && ok; ++r) {
            epoch = etab_next_epoch(tab, epoch, gtid, gsize);
            // one entry per thread per step (several table probes in flight per
            // thread serialise worse than more warps do); the next entry's label
            // and reciprocal are fetched before this entry's table update
            auto fetch = [&](unsigned e, int &lv, Rcp &rj) {
                lv = -1;
                if (e < m) lv = SMEM ? src[e] : __ldcs(&src[e]);
                if (lv >= 0 && (!QM_CHK(lv, x.K, 6) || (!FULL && lv < c) ||
                                (R > 1 && tab_split((unsigned)lv, R) != r)))
                    lv = -1;
                if (lv >= 0) rj = ld_rcp(&x.recip[lv]);
            };
            int lv_n;
            Rcp rj_n;
            fetch((unsigned)gtid, lv_n, rj_n);
            for (unsigned e = gtid; e < m; e += gsize) {
                const int lv = lv_n;
                const Rcp rj = rj_n;
                fetch(e + gsize, lv_n, rj_n);
                if (lv < 0) continue;
                const int prev = tab.add((unsigned)lv, epoch);
                if (prev < 0) continue;  // overflow: this pass is discarded
                if (!FULL || lv > c) add_share(inner, slots, cnt2, prev, rj);
                if (FULL) add_share(inner_full, s_dummy, c_dummy, prev, rj);
            }
            group_sync_n(gsize);
            if (*(volatile int *)tab.overflow) ok = false;
        }
        if (!ok) {
            group_sync_n(gsize);
            if (gtid == 0) *tab.overflow = 0;
            group_sync_n(gsize);
            const unsigned nr = R * 2u;
            if (nr > R_MAX) {
                if (gtid == 0) atomicOr(x.err, 2);
                return;
            }
            R = nr;
            continue;
        }
        group_totals<FULL>(slots, cnt2, inner, inner_full, gsize, red);
        if (gtid == 0) put_record(x, h.c, h.vol, m, slots, cnt2, inner, inner_full);
        if (gsize == 32) __syncwarp();
        return;
    }
}

// The same count for runs too long for the staged block path, including runs
// of 2^24 entries or more (a key may then occur 2^25 times or more): 64-bit
// counts in the tab_insert table, one pass over the used slots per class.
// Block groups only; the table must be empty on entry and is left empty.
__device__ __forceinline__ void count_run_general(const CountCtx &x, const RunHdr &h, const SmemTable &tab, int gtid,
                                                  int gsize, unsigned long long *red)
{
    const unsigned m = h.m;
    const int c = h.c;
    const bool full = x.full != 0;
    const int *src = x.nbr + h.a0;
    const unsigned cap_keys = (unsigned)tab.max_used;
    unsigned R = m <= cap_keys ? 1u : (unsigned)min((unsigned long long)R_MAX, (5ull * m + 4ull * cap_keys - 1) / (4ull * cap_keys));
    for (;;) {
        unsigned long long slots = 0, cnt2 = 0;
        U192 inner, inner_full;
        u192_zero(inner);
        u192_zero(inner_full);
        bool ok = true;
        for (unsigned r = 0; r < R && ok; ++r) {
            for (unsigned e = gtid; e < m; e += gsize) {
                const int lv = __ldcs(&src[e]);
                if (!QM_CHK(lv, x.K, 6) || (!full && lv < c)) continue;
                if (R == 1 || tab_split((unsigned)lv, R) == r) tab_insert(tab, (unsigned)lv);
            }
            group_sync(gsize);
            if (*(volatile int *)tab.overflow) {
                ok = false;
                break;
            }
            tab_drain(tab, gtid, gsize, [&](int key, long long cnt) {
                if (!QM_CHK(key, x.K, 7)) return;
                const unsigned long long q = (unsigned long long)cnt * (unsigned long long)cnt;
                const Rcp rj = ld_rcp(&x.recip[key]);
                if (full) u192_mac(inner_full, q, rj);
                if (key > c) {
                    u192_mac(inner, q, rj);
                    ++slots;
                    cnt2 += q;
                }
            });
            group_sync(gsize);
            if (gtid == 0) *tab.n_used = 0;
            group_sync(gsize);
        }
        if (!ok) {
            tab_wipe(tab, gtid, gsize);
            group_sync(gsize);
            if (gtid == 0) { *tab.n_used = 0; *tab.overflow = 0; }
            group_sync(gsize);
            const unsigned nr = R * 2u;
            if (nr > R_MAX) {
                if (gtid == 0) atomicOr(x.err, 2);
                return;
            }
            R = nr;
            continue;
        }
        group_totals<true>(slots, cnt2, inner, inner_full, gsize, red);
        if (gtid == 0) put_record(x, h.c, h.vol, m, slots, cnt2, inner, inner_full);
        group_sync(gsize);
        return;
    }
}

// Eq. (9), Sec. II-B.3 and the Eq. (8) integers of community c from its
// record.  pen_out receives c's own split penalty (valid when the record holds
// S_c, i.e. the count ran with per-community terms asked for).
__device__ __forceinline__ void terms_from_record(const unsigned long long *rc, long long size, long long E,
                                                  ScoreAcc &acc, double *pen_out, double *qs_out,
                                                  double *dens_o, double *contr_o, double *expn_o,
                                                  double *cond_o)
{
    const unsigned long long same = rc[REC_SAME], vol = rc[REC_VOL];
    const long long ein = (long long)(same / 2), eout = (long long)(vol - same);
    double qs, dens, contr, expn, cond;
    community_terms(ein, eout, size, E, qs, dens, contr, expn, cond);
    const u128 inner = ((u128)rc[REC_INNER_HI] << 64) | rc[REC_INNER_LO];
    const u128 full = ((u128)rc[REC_FULL_HI] << 64) | rc[REC_FULL_LO];
    const double pen = pair_penalty_once(inner, size, E);
    acc.qds_pair += fp_from_double(pen, SC_QDS);
    acc.slots += rc[REC_SLOTS];
    acc.cnt2 += rc[REC_CNT2];
    acc.qds_self += fp_from_double(qs, SC_QDS);
    acc.dens += fp_from_double(dens, SC_MEAN);
    acc.contr += fp_from_double(contr, SC_MEAN);
    acc.expn += fp_from_double(expn, SC_MEAN);
    acc.cond += fp_from_double(cond, SC_MEAN);
    acc.vol2 += (u128)vol * (u128)vol;
    acc.ein += (unsigned long long)ein;
    acc.eout += (unsigned long long)eout;
    acc.nonempty += 1;
    *pen_out = pair_penalty_own(full, size, E);
    *qs_out = qs;
    *dens_o = dens;
    *contr_o = contr;
    *expn_o = expn;
    *cond_o = cond;
}

// Row maximum of the Eq. (3) ratio 2 n / (n_a + n_b) over a truth community's
// cells, for the passes that form all cells before the rows: kept as the exact
// fraction (n << 32 | n_a + n_b) of the largest n / (n_a + n_b), compared by
// cross-multiplication (both below 2^31, so the products fit 64 bits), and
// turned into the ratio's double once per row (rowmax_ratio_settle) instead of
// dividing for every cell.  Rounding is monotone, so the largest correctly
// rounded ratio is the rounded largest ratio: the same bits.
__device__ __forceinline__ void rowmax_ratio_update(unsigned long long *slot, unsigned long long n,
                                                    unsigned long long d)
{
    const unsigned long long key = (n << 32) | d;
    unsigned long long cur = *(volatile unsigned long long *)slot;
    while (cur == 0ull || n * (cur & 0xFFFFFFFFull) > (cur >> 32) * d) {
        const unsigned long long prev = atomicCAS(slot, cur, key);
        if (prev == cur) return;
        cur = prev;
    }
}

// The row's fraction (rowmax_ratio_update) as the bits of its f_ratio double.
__device__ __forceinline__ void rowmax_ratio_settle(unsigned long long *slot, long long na)
{
    const unsigned long long key = __ldcg(slot);
    if (!key) return;
    const long long n = (long long)(key >> 32), d = (long long)(key & 0xFFFFFFFFull);
    *slot = (unsigned long long)__double_as_longlong(f_ratio(n, na, d - na));
}

// Row side of the contingency table for truth community a (Eqs. 2-4).
__device__ __forceinline__ void compare_row(const CompareCtx &x, int a, CompareAcc &acc)
{
    const long long na = __ldcg(&x.size_a[a]);
    if (na == 0) return;
    acc.sa += (unsigned long long)(na * (na - 1) / 2);
    acc.nvd += __ldcg(&x.rowmax_n[a]);
    const double r = __longlong_as_double((long long)__ldcg(&x.rowmax_r[a]));
    acc.f += fp_from_double(__dmul_rn((double)na, r), SC_F);
    acc.hden += fp_from_double(entropy_term(na, x.N), SC_H);
    acc.ka += 1;
}

}  // namespace qmk
