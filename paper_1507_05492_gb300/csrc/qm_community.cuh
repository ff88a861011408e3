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
    const int *members;      // nodes grouped by found label
    const int *start;        // int[k_found + 1]
    const int *size_a;       // |c| for c in C
    unsigned *rowmax_n;      // per truth community: max_c' |c n c'|
    unsigned long long *rowmax_r; // per truth community: bits of max 2|c n c'| / (|c|+|c'|)
    long long N;
    int ka, kb;
    int *err;
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

// Score community c with a group.  Returns false only for a warp group whose
// table overflowed (nothing was accumulated; the caller re-queues c for a block).
// A block group handles overflow itself by splitting the neighbour ids into R
// hash classes and walking the rows once per class.
//   offs: group-shared unsigned[gsize + 1]; rs: group-shared long long[gsize]
//   ctl:  group-shared int[2] (n_used, overflow) already wired into `tab`
__device__ __forceinline__ bool score_community(const ScoreCtx &x, int c, const SmemTable &tab,
                                                unsigned *offs, long long *rs, ScoreAcc *acc,
                                                int gtid, int gsize, unsigned long long *red)
{
    const int mb = __ldcg(&x.start[c]), me = __ldcg(&x.start[c + 1]);
    const long long size = me - mb;
#ifdef QM_DBG_VERIFY_AGREE
    if (gsize == 32) {
        QM_CHK(c == __shfl_sync(0xffffffffu, c, 0) && mb == __shfl_sync(0xffffffffu, mb, 0) &&
               me == __shfl_sync(0xffffffffu, me, 0) ? 0 : 1, 1, 28);
    } else {
        __shared__ int dbg_agree[3];
        block_sync();
        if (gtid == 0) { dbg_agree[0] = c; dbg_agree[1] = mb; dbg_agree[2] = me; }
        block_sync();
        QM_CHK(c == dbg_agree[0] && mb == dbg_agree[1] && me == dbg_agree[2] ? 0 : 1, 1, 27);
        block_sync();
    }
#endif
    unsigned R = 1;
    for (;;) {
        unsigned long long same = 0, vol = 0;
        i128 pair_fp = 0;
        unsigned long long slots = 0, cnt2 = 0;
        bool ok = true;
        for (unsigned r = 0; r < R && ok; ++r) {
            for (int cb = mb; cb < me; cb += gsize) {
                const int i = cb + gtid;
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
                unsigned excl;
                const int nm = min(gsize, me - cb);
                const unsigned total = group_exclusive_scan(d, excl, gsize, red);
                if (gtid < nm) { offs[gtid] = excl; rs[gtid] = rsi; }
                group_sync(gsize);
#ifdef QM_DBG_VERIFY_OFFS
                if (gtid < nm)
                    QM_CHKX(offs[gtid] + d == (gtid + 1 < nm ? offs[gtid + 1] : total) ? 0 : 1, 1,
                            23 + 100 * (gsize == 32 ? 1 : 2) + 1000 * (gtid + 1 < nm ? 1 : 2),
                            c, gtid, ((long long)nm << 32) | (unsigned)(me - mb),
                            ((long long)total << 32) | (unsigned)(offs[gtid] + d));
                if (gtid == 0) QM_CHK(gsize == 32 || gsize == (int)blockDim.x ? 0 : 1, 1, 26);
#endif
                for (unsigned e0 = gtid; e0 < total; e0 += 4u * gsize) {
                    int v[4], lv[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const unsigned e = e0 + k * gsize;
                        v[k] = -1;
                        if (e < total) {
                            const int o = upper_bound_smem(offs, nm, e) - 1;
                            if (QM_CHK(o, nm, 4) && QM_CHK(rs[o] + (e - offs[o]), x.n_arcs, 3))
                                v[k] = __ldg(&x.col[rs[o] + (e - offs[o])]);
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
                        } else if (R == 1 || tab_split((unsigned)lv[k], R) == r) {
                            tab_insert(tab, (unsigned)lv[k]);
                        }
                    }
                }
                group_sync(gsize);
            }
            if (*tab.overflow) {
                ok = false;
                break;
            }
            tab_drain(tab, gtid, gsize, [&](int key, long long cnt) {
                if (!QM_CHK(key, x.K, 7)) return;
                const long long sj = __ldcg(&x.start[key + 1]) - __ldcg(&x.start[key]);
                pair_fp += fp_from_double(pair_term(cnt, size, sj, x.E), SC_QDS);
                ++slots;
                cnt2 += (unsigned long long)(cnt * cnt);
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
            // Pass 0 completed, so the boundary arc count E_out (an upper bound of
            // the distinct neighbour communities) is known: size R from it.
            const unsigned long long eout = group_sum_u64(vol, gsize, red) - group_sum_u64(same, gsize, red);
            const unsigned long long need = (eout * 4 + 3ull * tab.max_used - 1) / (3ull * tab.max_used);
            unsigned long long nr = max((unsigned long long)R * 2ull, need);
            if (nr > R_MAX) {
                if (gtid == 0) atomicOr(x.err, 2);
                return true;
            }
            R = (unsigned)nr;
            continue;
        }
        // commit: group totals, then the group leader adds them to the group's
        // shared accumulator
        same = group_sum_u64(same, gsize, red);
        vol = group_sum_u64(vol, gsize, red);
        slots = group_sum_u64(slots, gsize, red);
        cnt2 = group_sum_u64(cnt2, gsize, red);
        const i128 pc_pair = group_sum_i128(pair_fp, gsize, red);
        if (gtid == 0) {
            const long long ein = (long long)(same / 2), eout = (long long)(vol - same);
            double qs, dens, contr, expn, cond;
            community_terms(ein, eout, size, x.E, qs, dens, contr, expn, cond);
            acc->qds_pair += pc_pair;
            acc->slots += slots;
            acc->cnt2 += cnt2;
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
            if (x.pc_qds) x.pc_qds[c] = __dsub_rn(qs, fp_to_double(pc_pair, SC_QDS));
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
            for (int i = mb + gtid; i < me; i += gsize) {
                const int a = __ldg(&x.truth[__ldcg(&x.members[i])]);
                if (R == 1 || tab_split((unsigned)a, R) == r) tab_insert(tab, (unsigned)a);
            }
            group_sync(gsize);
            if (*tab.overflow) { ok = false; break; }
            tab_drain(tab, gtid, gsize, [&](int a, long long n) {
                const long long na = __ldcg(&x.size_a[a]);
                a11 += (unsigned long long)(n * (n - 1) / 2);
                ++cells;
                colmax = max(colmax, (unsigned)n);
                atomicMax(&x.rowmax_n[a], (unsigned)n);
                atomicMax(&x.rowmax_r[a], (unsigned long long)__double_as_longlong(f_ratio(n, na, nb)));
                vi += fp_from_double(vi_term(n, na, nb), SC_VI);
                hn += fp_from_double(nmi_num_term(n, na, nb, x.N), SC_H);
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
        colmax = group_max_u32(colmax, gsize, red);
        a11 = group_sum_u64(a11, gsize, red);
        cells = group_sum_u64(cells, gsize, red);
        vi = group_sum_i128(vi, gsize, red);
        hn = group_sum_i128(hn, gsize, red);
        if (gtid == 0) {
            acc->a11 += a11;
            acc->cells += cells;
            acc->vi += vi;
            acc->hnum += hn;
            acc->nvd += colmax;
            acc->sb += (unsigned long long)(nb * (nb - 1) / 2);
            acc->hden += fp_from_double(entropy_term(nb, x.N), SC_H);
            acc->kb += 1;
        }
        return;
    }
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
