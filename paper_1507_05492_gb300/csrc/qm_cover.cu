// qm_cover.cu -- the metrics of a cover (overlapping communities).
//
// The paper leaves overlapping communities to future work (Sec. VI); its
// formulas are written with node sets, and a cover is scored by reading them
// literally: |c| its members, |E_c^in| the edges with both ends in c,
// |E_c^out| those with exactly one end in c, |E_ci,cj| those that leave c_i
// and enter c_j (u in c_i \ c_j, v in c_j \ c_i), |c n c'| the nodes in both,
// and a pair of nodes "in the same community" when the two share one.
//
// Scoring (Eqs. 8-9, Sec. II-B.3): the cover is brought to the graph's stored
// order, transposed into member lists, and one block per community walks its
// members' arcs, testing the far end's list for c, counting the boundary arcs,
// and counting in a shared-memory table the communities j > c of the far end
// that the near end is not in (each unordered pair is charged to its smaller
// id, as in the partition path).  The terms are formed and summed exactly as
// there (qm_finalize.cuh), so a cover with one community per node gives the
// partition's bits.
//
// Comparison (Eqs. 1-7): one block per truth community counts the cells
// |a n b| over its members' found lists; rows and columns add the entropy, F
// and NVD terms.  The pair counts come from the cells and sizes as for a
// partition (sum C(|a n b|, 2) counts a pair once per cell holding both), less
// a correction over pairs of nodes that share two or more communities on one
// side: such pairs can only be formed by nodes with two or more memberships,
// which each block lists and pairs up.
#include <algorithm>
#include <climits>

#include "qm_cover.h"
#include "qm_community.cuh"
#include "qm_finalize.cuh"

namespace qm {
using namespace qmk;

namespace {

constexpr int COVER_THREADS = 256;
constexpr int COVER_SMEM = 48 * 1024;
constexpr int OVL_CAP = 2048;  // overlapping members of one community paired in shared memory

// extra accumulator words after the GC_* words of a comparison
enum { GC_SAME_A_CORR = GC_COUNT, GC_SAME_B_CORR = GC_COUNT + 1, GC_A11_CORR = GC_COUNT + 2, GC_WORDS = GC_COUNT + 3 };
enum { CC_NEXT_A = 0, CC_NEXT_B = 1, CC_NEXT_C = 2, CC_SCAN = 8 };

size_t al(size_t x) { return (x + 255) / 256 * 256; }

void carve_side(char *&p, CoverSide &c, long long n, long long m, int K)
{
    c.off = (int *)p;
    p += al(((size_t)n + 1) * 4);
    c.memb = (int *)p;
    p += al((size_t)std::max(m, 1LL) * 4);
    c.len = (int *)p;
    p += al(((size_t)n + 1) * 4);
    c.cstart = (int *)p;
    p += al(((size_t)K + 1) * 4);
    c.cmem = (int *)p;
    p += al((size_t)std::max(m, 1LL) * 4);
    c.K = K;
}

}  // namespace

size_t cover_score_ws_bytes(long long n, long long m, int K)
{
    return carve_cover_score_ws(reinterpret_cast<void *>(4096), n, m, K).bytes;
}

CoverWs carve_cover_score_ws(void *base, long long n, long long m, int K)
{
    CoverWs w{};
    char *p = (char *)base;
    w.status = (int *)p;
    w.counters = (int *)(p + 16);
    p += 256;
    w.gacc = (unsigned long long *)p;
    p += al(64 * 8);
    w.result = p;
    p += al(sizeof(qm_quality));
    w.a.size = (int *)p;
    p += al((size_t)K * 4);
    w.a.cur = (int *)p;
    p += al((size_t)K * 4);
    w.zero_bytes = (size_t)(p - (char *)base);
    carve_side(p, w.a, n, m, K);
    w.recip = (Rcp *)p;
    p += al((size_t)K * 16);
    w.scan_tmp = (int *)p;
    p += al((scan_tmp_elems(std::max<long long>(n + 1, K)) + 64) * 4);
    w.bytes = (size_t)(p - (char *)base);
    return w;
}

size_t cover_compare_ws_bytes(long long n, long long ma, int ka, long long mb, int kb)
{
    return carve_cover_compare_ws(reinterpret_cast<void *>(4096), n, ma, ka, mb, kb).bytes;
}

CoverWs carve_cover_compare_ws(void *base, long long n, long long ma, int ka, long long mb, int kb)
{
    CoverWs w{};
    char *p = (char *)base;
    w.status = (int *)p;
    w.counters = (int *)(p + 16);
    p += 256;
    w.gacc = (unsigned long long *)p;
    p += al(64 * 8);
    w.result = p;
    p += al(sizeof(qm_compare));
    w.a.size = (int *)p;
    p += al((size_t)ka * 4);
    w.a.cur = (int *)p;
    p += al((size_t)ka * 4);
    w.b.size = (int *)p;
    p += al((size_t)kb * 4);
    w.b.cur = (int *)p;
    p += al((size_t)kb * 4);
    w.colmax = (unsigned *)p;
    p += al((size_t)kb * 4);
    w.zero_bytes = (size_t)(p - (char *)base);
    carve_side(p, w.a, n, ma, ka);
    carve_side(p, w.b, n, mb, kb);
    w.rowmax = (unsigned *)p;
    p += al((size_t)ka * 4);
    w.rowbest = (unsigned long long *)p;
    p += al((size_t)ka * 8);
    w.scan_tmp = (int *)p;
    p += al((scan_tmp_elems(std::max<long long>(n + 1, std::max(ka, kb))) + 64) * 4);
    w.bytes = (size_t)(p - (char *)base);
    return w;
}

// ------------------------------------------------------------------ bringing a cover to the stored order

// List length of every stored node (its caller node's list when the graph is
// renumbered), with the offsets' checks (non-decreasing from 0 to m).
__global__ void k_cover_len(const long long *mptr, long long n, long long m, const int *inv, int *len, int *status)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    bool bad = false;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const long long u = inv ? (long long)__ldg(&inv[j]) : j;
        const long long b = __ldg(&mptr[u]), e = __ldg(&mptr[u + 1]);
        if (b < 0 || e < b || e > m || e - b > INT_MAX) {
            bad = true;
            len[j] = 0;
        } else {
            len[j] = (int)(e - b);
        }
        if (j == 0 && (__ldg(&mptr[0]) != 0 || __ldg(&mptr[n]) != m)) bad = true;
    }
    if (bad) atomicOr(status, 1);
}

// Copies every stored node's list to its new offset, checks it (ids in [0, K),
// strictly increasing) and counts the community sizes.
__global__ void k_cover_copy(const long long *mptr, const int *memb, long long n, const int *inv, int K,
                             const int *off, int *out, int *size, int *status)
{
    if (*(volatile int *)status) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    bool bad = false;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const long long u = inv ? (long long)__ldg(&inv[j]) : j;
        const long long b = __ldg(&mptr[u]);
        const int o = __ldg(&off[j]), len = __ldg(&off[j + 1]) - o;
        int prev = -1;
        for (int k = 0; k < len; ++k) {
            const int c = __ldg(&memb[b + k]);
            if (c < 0 || c >= K || c <= prev) {
                bad = true;
                break;
            }
            prev = c;
            out[o + k] = c;
            atomicAdd(&size[c], 1);
        }
    }
    if (bad) atomicOr(status, 1);
}

// Members of every community: node j into its communities' lists.
__global__ void k_cover_scatter(const int *off, const int *memb, long long n, const int *cstart, int *cur, int *cmem,
                                const int *status)
{
    if (*status) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride)
        for (int k = __ldg(&off[j]); k < __ldg(&off[j + 1]); ++k) {
            const int c = __ldg(&memb[k]);
            cmem[__ldg(&cstart[c]) + atomicAdd(&cur[c], 1)] = (int)j;
        }
}

__global__ void k_cover_rcp(const int *size, int K, Rcp *recip, const int *status)
{
    if (*status) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < K; c += gridDim.x * blockDim.x)
        recip[c] = size[c] > 0 ? rcp_of(size[c]) : Rcp{0ull, 0ull};
}

// ------------------------------------------------------------------ device helpers

__device__ __forceinline__ bool list_has(const int *l, int len, int c)
{
    for (int k = 0; k < len; ++k) {
        const int x = __ldg(&l[k]);
        if (x == c) return true;
        if (x > c) return false;
    }
    return false;
}

// |x n y| of two sorted lists, and their smallest common id (INT_MAX if none).
__device__ __forceinline__ int list_meet(const int *x, int lx, const int *y, int ly, int *first)
{
    int i = 0, j = 0, k = 0;
    *first = INT_MAX;
    while (i < lx && j < ly) {
        const int a = __ldg(&x[i]), b = __ldg(&y[j]);
        if (a == b) {
            if (k == 0) *first = a;
            ++k;
            ++i;
            ++j;
        } else if (a < b) {
            ++i;
        } else {
            ++j;
        }
    }
    return k;
}

// The block's next community from a shared claim counter (every thread gets it).
__device__ __forceinline__ int claim_next(int *counter, int *slot)
{
    block_sync();
    if (threadIdx.x == 0) *slot = atomicAdd(counter, 1);
    block_sync();
    return *slot;
}

// ------------------------------------------------------------------ scoring

struct CoverScoreArgs {
    const long long *row_ptr;
    const int *col;
    const int *off, *memb;     // stored-order lists
    const int *cstart, *cmem;  // members of each community
    const Rcp *recip;
    int K;
    long long E;
    int *next;                 // claim counter
    unsigned long long *g;     // GS_* accumulators
    int *status;
    SmemPlan plan;             // shared-memory layout of the block
};

__global__ void __launch_bounds__(COVER_THREADS) k_cover_score(CoverScoreArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_c;
    if (*a.status) return;
    const SmemPlan &p = a.plan;
    unsigned long long *red = (unsigned long long *)(sm + p.red_off);
    int *ctl = (int *)(sm + p.ctl_off);
    unsigned long long *slot = (unsigned long long *)(sm + p.slot_off);
    int *used = (int *)(sm + p.used_off);
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, wid = tid >> 5, W = T >> 5;
    for (int i = tid; i < p.cap; i += T) slot[i] = 0ull;
    if (tid < 2) ctl[tid] = 0;
    block_sync();
    const SmemTable tab{slot, used, &ctl[0], &ctl[1], p.cap, p.max_used};
    ScoreAcc acc;
    score_acc_zero(acc);
    for (;;) {
        const int c = claim_next(a.next, &s_c);
        if (c >= a.K) break;
        const int mb = __ldg(&a.cstart[c]), me = __ldg(&a.cstart[c + 1]);
        const long long size = me - mb;
        if (size == 0) continue;
        unsigned R = 1;
        for (;;) {
            unsigned long long same = 0, out = 0, slots = 0, cnt2 = 0;
            U192 pair;
            u192_zero(pair);
            bool ok = true;
            for (unsigned r = 0; r < R && ok; ++r) {
                for (int idx = mb + wid; idx < me; idx += W) {
                    const int u = __ldg(&a.cmem[idx]);
                    const int *A = a.memb + __ldg(&a.off[u]);
                    const int la = __ldg(&a.off[u + 1]) - __ldg(&a.off[u]);
                    const long long rb = __ldg(&a.row_ptr[u]), re = __ldg(&a.row_ptr[u + 1]);
                    for (long long e = rb + lane; e < re; e += 32) {
                        const int v = __ldg(&a.col[e]);
                        const int *B = a.memb + __ldg(&a.off[v]);
                        const int lb = __ldg(&a.off[v + 1]) - __ldg(&a.off[v]);
                        if (list_has(B, lb, c)) {
                            if (r == 0) ++same;
                            continue;
                        }
                        if (r == 0) ++out;
                        for (int y = 0; y < lb; ++y) {  // communities j > c that v is in and u is not
                            const int j = __ldg(&B[y]);
                            if (j <= c || list_has(A, la, j)) continue;
                            if (R == 1 || tab_split((unsigned)j, R) == r) tab_insert(tab, (unsigned)j);
                        }
                    }
                }
                block_sync();
                if (*(volatile int *)tab.overflow) {
                    ok = false;
                    break;
                }
                tab_drain(tab, tid, T, [&](int key, long long cnt) {
                    if (!QM_CHK(key, a.K, 40)) return;
                    const unsigned long long q = (unsigned long long)cnt * (unsigned long long)cnt;
                    u192_mac(pair, q, ld_rcp_cg(&a.recip[key]));
                    ++slots;
                    cnt2 += q;
                });
                block_sync();
                if (tid == 0) *tab.n_used = 0;
                block_sync();
            }
            if (!ok) {
                tab_wipe(tab, tid, T);
                block_sync();
                if (tid == 0) {
                    *tab.n_used = 0;
                    *tab.overflow = 0;
                }
                block_sync();
                if (R * 2u > R_MAX) {
                    if (tid == 0) atomicOr(a.status, 2);
                    break;
                }
                R *= 2u;
                continue;
            }
            unsigned long long w4[4] = {same, out, slots, cnt2};
            group_words_to_leader<4>(w4, T, red);
            const u128 pair_t = u192_shr64(group_u192_to_leader(pair, T, red, 128));
            if (tid == 0) {
                const long long ein = (long long)(w4[0] / 2), eout = (long long)w4[1];
                double qs, dens, contr, expn, cond;
                community_terms(ein, eout, size, a.E, qs, dens, contr, expn, cond);
                const double pen = pair_penalty_once(pair_t, size, a.E);
                const unsigned long long vol = 2ull * (unsigned long long)ein + (unsigned long long)eout;
                acc.qds_pair += fp_from_double(pen, SC_QDS);
                acc.qds_self += fp_from_double(qs, SC_QDS);
                acc.dens += fp_from_double(dens, SC_MEAN);
                acc.contr += fp_from_double(contr, SC_MEAN);
                acc.expn += fp_from_double(expn, SC_MEAN);
                acc.cond += fp_from_double(cond, SC_MEAN);
                acc.vol2 += (u128)vol * (u128)vol;
                acc.ein += (unsigned long long)ein;
                acc.eout += (unsigned long long)eout;
                acc.nonempty += 1;
                acc.slots += w4[2];
                acc.cnt2 += w4[3];
            }
            break;
        }
    }
    if (tid == 0) {  // only the leader holds sums
        limbs_add(a.g + GS_QDS_SELF, acc.qds_self);
        limbs_add(a.g + GS_QDS_PAIR, acc.qds_pair);
        limbs_add(a.g + GS_DENS, acc.dens);
        limbs_add(a.g + GS_CONTR, acc.contr);
        limbs_add(a.g + GS_EXPN, acc.expn);
        limbs_add(a.g + GS_COND, acc.cond);
        limbs_add(a.g + GS_VOL2, (i128)acc.vol2);
        const unsigned long long u[5] = {acc.ein, acc.eout, acc.nonempty, acc.slots, acc.cnt2};
        const int at[5] = {GS_EIN, GS_EOUT, GS_NONEMPTY, GS_SLOTS, GS_CNT2};
        for (int k = 0; k < 5; ++k)
            if (u[k]) atomicAdd(a.g + at[k], u[k]);
    }
}

// Eqs. (8)-(9) and the means from the sums; cut_edges_total of a cover is the
// sum over communities of |E_c^out| (an edge may leave several communities).
__global__ void k_cover_score_fin(const unsigned long long *g, const int *status, long long n, long long E,
                                  qm_quality *out)
{
    if (threadIdx.x != 0 || *status) return;
    ScoreTotals t;
    t.qds_self = limbs_get(g + GS_QDS_SELF);
    t.qds_pair = limbs_get(g + GS_QDS_PAIR);
    t.dens = limbs_get(g + GS_DENS);
    t.contr = limbs_get(g + GS_CONTR);
    t.expn = limbs_get(g + GS_EXPN);
    t.cond = limbs_get(g + GS_COND);
    t.vol2 = limbs_get(g + GS_VOL2);
    t.ein = g[GS_EIN];
    t.eout = g[GS_EOUT];
    t.nonempty = g[GS_NONEMPTY];
    t.slots = g[GS_SLOTS];
    t.cnt2 = g[GS_CNT2];
    qm_quality r;
    make_quality(t, n, E, &r);
    r.cut_edges_total = (long long)t.eout;
    *out = r;
}

// ------------------------------------------------------------------ comparison

struct CoverCmpArgs {
    const int *aoff, *amemb, *acstart, *acmem;  // truth side
    const int *boff, *bmemb, *bcstart, *bcmem;  // found side
    const int *size_a, *size_b;
    int ka, kb;
    long long N;
    unsigned *rowmax;
    unsigned long long *rowbest;
    unsigned *colmax;
    int *next_a, *next_b, *next_c;
    unsigned long long *g;
    int *status;
    SmemPlan plan;
};

__device__ __forceinline__ void flush_compare_acc(const CompareAcc &acc, unsigned long long *g, unsigned long long *red)
{
    const int T = blockDim.x;
    i128 v = group_sum_i128(acc.vi, T, red);
    if (threadIdx.x == 0) limbs_add(g + GC_VI, v);
    v = group_sum_i128(acc.hnum, T, red);
    if (threadIdx.x == 0) limbs_add(g + GC_HNUM, v);
    v = group_sum_i128(acc.hden, T, red);
    if (threadIdx.x == 0) limbs_add(g + GC_HDEN, v);
    v = group_sum_i128(acc.f, T, red);
    if (threadIdx.x == 0) limbs_add(g + GC_F, v);
    const unsigned long long *src[7] = {&acc.a11, &acc.sa, &acc.sb, &acc.nvd, &acc.cells, &acc.ka, &acc.kb};
    const int dst[7] = {GC_A11, GC_SA, GC_SB, GC_NVD, GC_CELLS, GC_KA, GC_KB};
    for (int k = 0; k < 7; ++k) {
        const unsigned long long u = group_sum_u64(*src[k], T, red);
        if (threadIdx.x == 0 && u) atomicAdd(g + dst[k], u);
    }
}

// The cells of every truth community a: counts |a n b| over a's members' found
// lists, then per cell the Eq. (1)-(2) terms, C(|a n b|, 2), the row's largest
// cell and F ratio (Eqs. 3-4), and each column's largest cell.
__global__ void __launch_bounds__(COVER_THREADS) k_cover_cells(CoverCmpArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_c;
    if (*a.status) return;
    const SmemPlan &p = a.plan;
    unsigned long long *red = (unsigned long long *)(sm + p.red_off);
    int *ctl = (int *)(sm + p.ctl_off);
    unsigned long long *slot = (unsigned long long *)(sm + p.slot_off);
    int *used = (int *)(sm + p.used_off);
    const int tid = threadIdx.x, T = blockDim.x;
    for (int i = tid; i < p.cap; i += T) slot[i] = 0ull;
    if (tid < 2) ctl[tid] = 0;
    block_sync();
    const SmemTable tab{slot, used, &ctl[0], &ctl[1], p.cap, p.max_used};
    CompareAcc acc;
    compare_acc_zero(acc);
    for (;;) {
        const int c = claim_next(a.next_c, &s_c);
        if (c >= a.ka) break;
        const int mb = __ldg(&a.acstart[c]), me = __ldg(&a.acstart[c + 1]);
        const long long na = me - mb;
        if (na == 0) continue;
        unsigned R = 1;
        for (;;) {
            unsigned rmax = 0;
            unsigned long long rbest = 0;
            CompareAcc part;
            compare_acc_zero(part);
            bool ok = true;
            for (unsigned r = 0; r < R && ok; ++r) {
                for (int idx = mb + tid; idx < me; idx += T) {
                    const int i = __ldg(&a.acmem[idx]);
                    for (int k = __ldg(&a.boff[i]); k < __ldg(&a.boff[i + 1]); ++k) {
                        const int b = __ldg(&a.bmemb[k]);
                        if (R == 1 || tab_split((unsigned)b, R) == r) tab_insert(tab, (unsigned)b);
                    }
                }
                block_sync();
                if (*(volatile int *)tab.overflow) {
                    ok = false;
                    break;
                }
                tab_drain(tab, tid, T, [&](int b, long long n) {
                    if (!QM_CHK(b, a.kb, 41)) return;
                    const long long nb = __ldg(&a.size_b[b]);
                    part.a11 += (unsigned long long)(n * (n - 1) / 2);
                    part.cells += 1;
                    const double l1 = cell_log(n, na, nb);
                    part.vi += fp_from_double(vi_term_l(n, l1), SC_VI);
                    part.hnum += fp_from_double(nmi_num_term_l(n, a.N, l1, log_ratio(a.N, n)), SC_H);
                    rmax = max(rmax, (unsigned)n);
                    rbest = max(rbest, (unsigned long long)__double_as_longlong(f_ratio(n, na, nb)));
                    atomicMax(&a.colmax[b], (unsigned)n);
                });
                block_sync();
                if (tid == 0) *tab.n_used = 0;
                block_sync();
            }
            if (!ok) {
                tab_wipe(tab, tid, T);
                block_sync();
                if (tid == 0) {
                    *tab.n_used = 0;
                    *tab.overflow = 0;
                }
                block_sync();
                if (R * 2u > R_MAX) {
                    if (tid == 0) atomicOr(a.status, 2);
                    break;
                }
                R *= 2u;
                continue;
            }
            compare_acc_add(acc, part);
            // the row's largest cell and ratio (non-negative doubles order as their bits)
            const unsigned m = group_max_u32(rmax, T, red);
            unsigned long long bb = rbest;
            for (int d = 16; d > 0; d >>= 1) bb = max(bb, __shfl_down_sync(0xffffffffu, bb, d));
            block_sync();
            if ((tid & 31) == 0) red[tid >> 5] = bb;
            block_sync();
            if (tid == 0) {
                unsigned long long best = 0;
                for (int w = 0; w < (T >> 5); ++w) best = max(best, red[w]);
                a.rowmax[c] = m;
                a.rowbest[c] = best;
            }
            break;
        }
    }
    flush_compare_acc(acc, a.g, red);
}

// Row side (truth communities): C(|a|, 2), the entropy term, F, NVD row maxima.
__global__ void k_cover_rows(CoverCmpArgs a)
{
    __shared__ unsigned long long red[72];
    if (*a.status) return;
    CompareAcc acc;
    compare_acc_zero(acc);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.ka; c += gridDim.x * blockDim.x) {
        const long long na = a.size_a[c];
        if (na == 0) continue;
        acc.sa += (unsigned long long)(na * (na - 1) / 2);
        acc.nvd += a.rowmax[c];
        acc.f += fp_from_double(__dmul_rn((double)na, __longlong_as_double((long long)a.rowbest[c])), SC_F);
        acc.hden += fp_from_double(entropy_term(na, a.N), SC_H);
        acc.ka += 1;
    }
    flush_compare_acc(acc, a.g, red);
}

// Column side (found communities): C(|b|, 2), the entropy term, NVD column maxima.
__global__ void k_cover_cols(CoverCmpArgs a)
{
    __shared__ unsigned long long red[72];
    if (*a.status) return;
    CompareAcc acc;
    compare_acc_zero(acc);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.kb; c += gridDim.x * blockDim.x) {
        const long long nb = a.size_b[c];
        if (nb == 0) continue;
        acc.sb += (unsigned long long)(nb * (nb - 1) / 2);
        acc.nvd += a.colmax[c];
        acc.hden += fp_from_double(entropy_term(nb, a.N), SC_H);
        acc.kb += 1;
    }
    flush_compare_acc(acc, a.g, red);
}

// Pair index k < L(L-1)/2 -> (p, q), p < q < L.
__device__ __forceinline__ void pair_of(long long k, long long *p, long long *q)
{
    long long b = (long long)((1.0 + sqrt(1.0 + 8.0 * (double)k)) * 0.5);
    while (b * (b - 1) / 2 > k) --b;
    while ((b + 1) * b / 2 <= k) ++b;
    *q = b;
    *p = k - b * (b - 1) / 2;
}

// Pair-count corrections for pairs of nodes sharing two or more communities on
// side X (the other side is Y).  For community c of X, its members with two or
// more memberships are paired up; a pair is taken by the smallest community
// the two share in X, so once.  With k = |X(i) n X(j)| and k' = |Y(i) n Y(j)|:
//   same_X correction  k - 1                      (when k >= 2)
//   a11 correction     k k' - 1 (side A, k >= 2, k k' >= 1), or k' - 1 (side B,
//                      k' >= 2 and k = 1, the pairs side A did not take)
template <bool SIDE_A>
__global__ void __launch_bounds__(COVER_THREADS) k_cover_pairs(CoverCmpArgs a)
{
    __shared__ int s_c, s_n;
    __shared__ int ovl[OVL_CAP];
    __shared__ unsigned long long red[72];
    if (*a.status) return;
    const int *xoff = SIDE_A ? a.aoff : a.boff, *xmemb = SIDE_A ? a.amemb : a.bmemb;
    const int *yoff = SIDE_A ? a.boff : a.aoff, *ymemb = SIDE_A ? a.bmemb : a.amemb;
    const int *xcstart = SIDE_A ? a.acstart : a.bcstart, *xcmem = SIDE_A ? a.acmem : a.bcmem;
    const int kx = SIDE_A ? a.ka : a.kb;
    const int tid = threadIdx.x, T = blockDim.x;
    unsigned long long same_corr = 0, a11_corr = 0;
    for (;;) {
        const int c = claim_next(SIDE_A ? a.next_a : a.next_b, &s_c);
        if (c >= kx) break;
        const int mb = __ldg(&xcstart[c]), me = __ldg(&xcstart[c + 1]);
        if (me - mb < 2) continue;
        // members with two or more memberships on this side
        if (tid == 0) s_n = 0;
        block_sync();
        for (int idx = mb + tid; idx < me; idx += T) {
            const int i = __ldg(&xcmem[idx]);
            if (__ldg(&xoff[i + 1]) - __ldg(&xoff[i]) >= 2) {
                const int at = atomicAdd(&s_n, 1);
                if (at < OVL_CAP) ovl[at] = i;
            }
        }
        block_sync();
        const int L = s_n;
        if (L < 2) continue;
        const bool in_smem = L <= OVL_CAP;
        // pairs of overlapping members (from shared memory, or the whole member
        // list filtered again when there are too many to hold)
        const long long Lp = in_smem ? L : (long long)(me - mb);
        const long long npairs = Lp * (Lp - 1) / 2;
        for (long long k = tid; k < npairs; k += T) {
            long long pp, qq;
            pair_of(k, &pp, &qq);
            const int i = in_smem ? ovl[pp] : __ldg(&xcmem[mb + pp]);
            const int j = in_smem ? ovl[qq] : __ldg(&xcmem[mb + qq]);
            const int li = __ldg(&xoff[i + 1]) - __ldg(&xoff[i]), lj = __ldg(&xoff[j + 1]) - __ldg(&xoff[j]);
            if (li < 2 || lj < 2) continue;
            int first = 0, dummy = 0;
            const int kxx = list_meet(xmemb + __ldg(&xoff[i]), li, xmemb + __ldg(&xoff[j]), lj, &first);
            if (first != c || kxx < 2) continue;
            const int kyy = list_meet(ymemb + __ldg(&yoff[i]), __ldg(&yoff[i + 1]) - __ldg(&yoff[i]),
                                      ymemb + __ldg(&yoff[j]), __ldg(&yoff[j + 1]) - __ldg(&yoff[j]), &dummy);
            same_corr += (unsigned long long)(kxx - 1);
            if (SIDE_A) {
                if (kyy >= 1) a11_corr += (unsigned long long)(kxx * kyy - 1);
            } else {
                if (kyy == 1) a11_corr += (unsigned long long)(kxx - 1);
            }
        }
    }
    const unsigned long long s = group_sum_u64(same_corr, T, red);
    const unsigned long long q = group_sum_u64(a11_corr, T, red);
    if (tid == 0) {
        if (s) atomicAdd(a.g + (SIDE_A ? GC_SAME_A_CORR : GC_SAME_B_CORR), s);
        if (q) atomicAdd(a.g + GC_A11_CORR, q);
    }
}

__global__ void k_cover_compare_fin(const unsigned long long *g, const int *status, long long n, qm_compare *out)
{
    if (threadIdx.x != 0 || *status) return;
    CompareTotals t;
    t.vi = limbs_get(g + GC_VI);
    t.hnum = limbs_get(g + GC_HNUM);
    t.hden = limbs_get(g + GC_HDEN);
    t.f = limbs_get(g + GC_F);
    t.a11 = g[GC_A11] - g[GC_A11_CORR];
    t.sa = g[GC_SA] - g[GC_SAME_A_CORR];
    t.sb = g[GC_SB] - g[GC_SAME_B_CORR];
    t.nvd = g[GC_NVD];
    t.cells = g[GC_CELLS];
    t.ka = g[GC_KA];
    t.kb = g[GC_KB];
    make_compare(t, n, out);
}

// ------------------------------------------------------------------ launchers

namespace {

int grid_of(long long n, int threads, int num_sms, int per_sm)
{
    long long g = (n + threads - 1) / threads;
    g = std::min<long long>(g, (long long)num_sms * per_sm);
    return (int)std::max<long long>(g, 1);
}

// Brings one cover to the stored order and builds its member lists.
int prepare_side(const long long *mptr, const int *memb, long long m, long long n, const int *inv,
                 const CoverSide &c, const CoverWs &w, int num_sms, cudaStream_t s)
{
    int L = 0;
    k_cover_len<<<grid_of(n, 256, num_sms, 8), 256, 0, s>>>(mptr, n, m, inv, c.len, w.status);
    ++L;
    const int l1 = scan_offsets(c.len, (int)n, c.off, w.scan_tmp, w.counters + CC_SCAN, w.status, s);
    if (l1 < 0) return -1;
    L += l1;
    k_cover_copy<<<grid_of(n, 256, num_sms, 8), 256, 0, s>>>(mptr, memb, n, inv, c.K, c.off, c.memb, c.size,
                                                            w.status);
    ++L;
    const int l2 = scan_offsets(c.size, c.K, c.cstart, w.scan_tmp, w.counters + CC_SCAN, w.status, s);
    if (l2 < 0) return -1;
    L += l2;
    k_cover_scatter<<<grid_of(n, 256, num_sms, 8), 256, 0, s>>>(c.off, c.memb, n, c.cstart, c.cur, c.cmem,
                                                               w.status);
    ++L;
    return L;
}

}  // namespace

void prepare_cover_kernels()
{
    cudaFuncSetAttribute(k_cover_score, cudaFuncAttributeMaxDynamicSharedMemorySize, COVER_SMEM);
    cudaFuncSetAttribute(k_cover_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, COVER_SMEM);
    k_fill_log_int<<<(LOGT_MAX + 256) / 256, 256>>>();  // this unit's copy of the log(i) table
    cudaDeviceSynchronize();
}

int launch_cover_score(const GraphDev &g, const long long *mptr, const int *memb, long long m, int K,
                       const CoverWs &w, int num_sms, cudaStream_t s)
{
    const long long n = g.n;
    int L = prepare_side(mptr, memb, m, n, g.inv, w.a, w, num_sms, s);
    if (L < 0) return -1;
    k_cover_rcp<<<grid_of(K, 256, num_sms, 4), 256, 0, s>>>(w.a.size, K, w.recip, w.status);
    CoverScoreArgs a;
    a.row_ptr = g.row_ptr;
    a.col = g.col;
    a.off = w.a.off;
    a.memb = w.a.memb;
    a.cstart = w.a.cstart;
    a.cmem = w.a.cmem;
    a.recip = w.recip;
    a.K = K;
    a.E = g.n_arcs / 2;
    a.next = w.counters + CC_NEXT_C;
    a.g = w.gacc;
    a.status = w.status;
    a.plan = plan_smem(COVER_THREADS, COVER_SMEM);
    k_cover_score<<<std::min(num_sms * 4, std::max(K, 1)), COVER_THREADS, COVER_SMEM, s>>>(a);
    k_cover_score_fin<<<1, 32, 0, s>>>(w.gacc, w.status, n, g.n_arcs / 2, (qm_quality *)w.result);
    L += 3;
    return cudaGetLastError() == cudaSuccess ? L : -1;
}

int launch_cover_compare(const long long *aptr, const int *amemb, long long ma, int ka, const long long *bptr,
                         const int *bmemb, long long mb, int kb, long long n, const CoverWs &w, int num_sms,
                         cudaStream_t s)
{
    int L1 = prepare_side(aptr, amemb, ma, n, nullptr, w.a, w, num_sms, s);
    if (L1 < 0) return -1;
    int L2 = prepare_side(bptr, bmemb, mb, n, nullptr, w.b, w, num_sms, s);
    if (L2 < 0) return -1;
    CoverCmpArgs a;
    a.aoff = w.a.off;
    a.amemb = w.a.memb;
    a.acstart = w.a.cstart;
    a.acmem = w.a.cmem;
    a.boff = w.b.off;
    a.bmemb = w.b.memb;
    a.bcstart = w.b.cstart;
    a.bcmem = w.b.cmem;
    a.size_a = w.a.size;
    a.size_b = w.b.size;
    a.ka = ka;
    a.kb = kb;
    a.N = n;
    a.rowmax = w.rowmax;
    a.rowbest = w.rowbest;
    a.colmax = w.colmax;
    a.next_a = w.counters + CC_NEXT_A;
    a.next_b = w.counters + CC_NEXT_B;
    a.next_c = w.counters + CC_NEXT_C;
    a.g = w.gacc;
    a.status = w.status;
    a.plan = plan_smem(COVER_THREADS, COVER_SMEM);
    k_cover_cells<<<std::min(num_sms * 4, std::max(ka, 1)), COVER_THREADS, COVER_SMEM, s>>>(a);
    k_cover_rows<<<grid_of(ka, 256, num_sms, 2), 256, 0, s>>>(a);
    k_cover_cols<<<grid_of(kb, 256, num_sms, 2), 256, 0, s>>>(a);
    k_cover_pairs<true><<<std::min(num_sms * 4, std::max(ka, 1)), COVER_THREADS, 0, s>>>(a);
    k_cover_pairs<false><<<std::min(num_sms * 4, std::max(kb, 1)), COVER_THREADS, 0, s>>>(a);
    k_cover_compare_fin<<<1, 32, 0, s>>>(w.gacc, w.status, n, (qm_compare *)w.result);
    return cudaGetLastError() == cudaSuccess ? L1 + L2 + 6 : -1;
}

}  // namespace qm
