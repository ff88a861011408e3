// qm_batched.cu -- scoring and comparing many partitions in one launch.
//
// Two implementations.  The default is the two-phase pipeline of qm_batched.h:
// the kernels of the plain two-phase path, each run over all candidates of a
// wave at once (label histograms and counting sort, far-end label gathers into
// packed runs, one integer record per community, contingency cells, then the
// FP64 terms of every community and cell with all lanes busy).  Items with
// more arcs than that pipeline's runs hold take k_batched: a persistent kernel
// in which a block takes the next item from a global queue and runs the
// one-kernel path for it on its own (histogram, prefix sum, counting sort, the
// community-major pass of Sec. III-A, cells and row maxima of Eqs. (1)-(7),
// final reduction), with no grid-wide barrier and no inter-block wait.  Both
// use the per-term formulas, fixed-point sums and final arithmetic of the plain
// path, so every result is bit-identical to scoring that partition alone.
#include <algorithm>

#include "qm_internal.h"
#include "qm_batched.h"
#include "qm_community.cuh"
#include "qm_expand.cuh"
#include "qm_finalize.cuh"

namespace qm {
using namespace qmk;

__host__ __device__ static inline size_t al(size_t x) { return (x + 255) / 256 * 256; }

size_t batch_scratch_bytes(long long n_max, int k_max, int kt_max, int slots)
{
    const size_t per = al((size_t)n_max * 4) + al((size_t)(k_max + 1) * 4) + al((size_t)kt_max * 4) * 2 +
                       al((size_t)kt_max * 8) + al((size_t)k_max * 4) * 3 + al((size_t)k_max * 4) +
                       al((size_t)k_max * 16);
    return per * (size_t)slots;
}

BatchScratch carve_batch_scratch(void *base, long long n_max, int k_max, int kt_max, int slots)
{
    BatchScratch b;
    char *p = (char *)base;
    b.n_max = n_max;
    b.k_max = k_max;
    b.kt_max = kt_max;
    b.slots = slots;
    b.members = (int *)p;
    p += al((size_t)n_max * 4) * slots;
    b.start = (int *)p;
    p += al((size_t)(k_max + 1) * 4) * slots;
    b.size_a = (int *)p;
    p += al((size_t)kt_max * 4) * slots;
    b.rowmax_n = (unsigned *)p;
    p += al((size_t)kt_max * 4) * slots;
    b.rowmax_r = (unsigned long long *)p;
    p += al((size_t)kt_max * 8) * slots;
    b.big_list = (int *)p;          // three lists of k_max per slot
    p += al((size_t)k_max * 4) * 3 * slots;
    b.size = (int *)p;
    p += al((size_t)k_max * 4) * slots;
    b.recip = (Rcp *)p;
    return b;
}

struct BatchKArgs {
    const BatchItem *items;
    int count;
    int *queue;
    BatchScratch bs;
    SmemPlan plan;
    int big_thr;
};

__global__ void __launch_bounds__(BATCH_MAX_THREADS) k_batched(BatchKArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_item, s_bad, s_nbig, s_ncmp, s_next, s_novf, s_next2;
    const SmemPlan &p = a.plan;
    unsigned long long *red = (unsigned long long *)(sm + p.red_off);
    int *ctl = (int *)(sm + p.ctl_off);
    unsigned *offs = (unsigned *)(sm + p.offs_off);
    long long *rs = (long long *)(sm + p.rs_off);
    unsigned long long *slot = (unsigned long long *)(sm + p.slot_off);
    int *used = (int *)(sm + p.used_off);
    const int T = blockDim.x, W = T >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;

    const BatchScratch &bs = a.bs;
    const size_t sl = blockIdx.x;
    int *members = (int *)((char *)bs.members + sl * al((size_t)bs.n_max * 4));
    int *start = (int *)((char *)bs.start + sl * al((size_t)(bs.k_max + 1) * 4));
    int *size_a = (int *)((char *)bs.size_a + sl * al((size_t)bs.kt_max * 4));
    unsigned *rowmax_n = (unsigned *)((char *)bs.rowmax_n + sl * al((size_t)bs.kt_max * 4));
    unsigned long long *rowmax_r = (unsigned long long *)((char *)bs.rowmax_r + sl * al((size_t)bs.kt_max * 8));
    int *big_score = (int *)((char *)bs.big_list + sl * al((size_t)bs.k_max * 4) * 3);
    int *big_cmp = big_score + al((size_t)bs.k_max * 4) / 4;
    int *ovf = big_cmp + al((size_t)bs.k_max * 4) / 4;
    int *gsize = (int *)((char *)bs.size + sl * al((size_t)bs.k_max * 4));
    Rcp *recip = (Rcp *)((char *)bs.recip + sl * al((size_t)bs.k_max * 16));

    for (int i = tid; i < p.cap; i += T) slot[i] = 0ull;
    for (int i = tid; i < 2 * (W + 1); i += T) ctl[i] = 0;
    block_sync();
    const SmemTable tb{slot, used, &ctl[0], &ctl[1], p.cap, p.max_used};
    const SmemTable tw{slot + wid * p.cap_w, used + wid * p.max_used_w, &ctl[2 + 2 * wid], &ctl[3 + 2 * wid],
                       p.cap_w, p.max_used_w};

    for (;;) {
        if (tid == 0) s_item = atomicAdd(a.queue, 1);
        block_sync();
        const int it = s_item;
        if (it >= a.count) break;
        const BatchItem I = a.items[it];
        const long long n = I.n;
        const int K = I.K;
        const bool do_score = (I.flags & 1) != 0;
        const bool do_cmp = (I.flags & 2) != 0 && I.truth != nullptr;
        const int kt = do_cmp ? I.k_truth : 0;
        const bool smem_hist = (long long)K + kt <= 2LL * p.cap;
        int *cnt = smem_hist ? (int *)slot : gsize;       // label counts, then cursors
        int *cnt_a = smem_hist ? (int *)slot + K : size_a;
        if (tid == 0) { s_bad = 0; s_nbig = 0; s_ncmp = 0; s_next = 0; s_novf = 0; s_next2 = 0; }
        if (!smem_hist) {
            for (int i = tid; i < K; i += T) gsize[i] = 0;
            for (int i = tid; i < kt; i += T) size_a[i] = 0;
        }
        for (int i = tid; i < kt; i += T) { rowmax_n[i] = 0u; rowmax_r[i] = 0ull; }
        block_sync();

        // 1. label histograms (with range checks)
        bool bad = false;
        for (long long u = tid; u < n; u += T) {
            const int l = __ldg(&I.labels[u]);
            if ((unsigned)l >= (unsigned)K) bad = true;
            else atomicAdd(&cnt[l], 1);
            if (do_cmp) {
                const int t = __ldg(&I.truth[u]);
                if ((unsigned)t >= (unsigned)kt) bad = true;
                else atomicAdd(&cnt_a[t], 1);
            }
        }
        if (bad) s_bad = 1;
        block_sync();
        if (s_bad) {
            if (tid == 0) *I.status = 1;
            if (smem_hist) for (int i = tid; i < K + kt; i += T) ((int *)slot)[i] = 0;
            block_sync();
            continue;
        }
        if (smem_hist)
            for (int i = tid; i < kt; i += T) size_a[i] = cnt_a[i];
        // rowmax arrays and size_a written above are read later in this launch
        __threadfence();

        // 2. exclusive prefix of the community sizes; lists of large communities;
        //    cnt[] becomes the scatter cursor
        unsigned carry = 0;
        for (int c0 = 0; c0 < K; c0 += T) {
            const int c = c0 + tid;
            const int s = c < K ? cnt[c] : 0;
            unsigned excl;
            const unsigned tot = group_exclusive_scan((unsigned)s, excl, T, red);
            if (c < K) {
                start[c] = (int)(carry + excl);
                cnt[c] = (int)(carry + excl);
                if (s > 0) recip[c] = rcp_of(s);
                if (do_score && s > a.big_thr) {
                    const int k = atomicAdd(&s_nbig, 1);
                    if (QM_CHK(k, bs.k_max, 12)) big_score[k] = c;
                }
                if (do_cmp && s > p.max_used_w) {
                    const int k = atomicAdd(&s_ncmp, 1);
                    if (QM_CHK(k, bs.k_max, 12)) big_cmp[k] = c;
                }
            }
            carry += tot;
        }
        if (tid == 0) start[K] = (int)carry;
        __threadfence();  // start[] and the lists are read by other warps below
        block_sync();

        // 3. counting sort of the nodes by label
        for (long long u = tid; u < n; u += T) {
            const int l = __ldg(&I.labels[u]);
            if (!QM_CHK(l, K, 11)) continue;
            const int pos = atomicAdd(&cnt[l], 1);
            if (QM_CHK(pos, n, 10) && QM_CHK(pos, bs.n_max, 15)) members[pos] = (int)u;
        }
        __threadfence();  // members[] is read by every warp below
        block_sync();
        if (smem_hist) {
            for (int i = tid; i < K + kt; i += T) ((int *)slot)[i] = 0;
            block_sync();
        }

        // 4. metrics without ground truth
        if (do_score) {
            ScoreCtx x;
            x.row_ptr = I.row_ptr;
            x.col = I.col;
            x.labels = I.labels;
            x.members = members;
            x.start = start;
            x.recip = recip;
            x.E = I.n_arcs / 2;
            x.n = n;
            x.n_arcs = I.n_arcs;
            x.K = K;
            x.err = I.status;
            x.pc_size = x.pc_ein = x.pc_eout = nullptr;
            x.pc_dens = x.pc_contr = x.pc_expn = x.pc_cond = x.pc_qds = nullptr;
            ScoreAcc *sacc = (ScoreAcc *)(sm + p.acc_off);
            for (int i = tid; i < W; i += T) score_acc_zero(sacc[i]);
            block_sync();
            const int nbig = s_nbig;
            for (int i = 0; i < nbig; ++i) {
                score_community(x, __ldcg(&big_score[i]), tb, offs, rs, &sacc[0], tid, T, red);
            }
            const int chunk = claim_chunk(K, W);
            for (;;) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&s_next, chunk);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (base >= K) break;
                const int c = base + lane;
                const int sz = lane < chunk && c < K ? __ldcg(&start[c + 1]) - __ldcg(&start[c]) : 0;
                unsigned mask = __ballot_sync(0xffffffffu, sz > 0 && sz <= a.big_thr);
                while (mask) {
                    const int j = __ffs(mask) - 1;
                    mask &= mask - 1;
                    if (!score_community(x, base + j, tw, offs, rs, &sacc[wid], lane, 32, red))
                        if (lane == 0) {
                            const int k = atomicAdd(&s_novf, 1);
                            if (QM_CHK(k, bs.k_max, 13)) ovf[k] = base + j;
                        }
                }
            }
            __threadfence();
            block_sync();
            const int novf = s_novf;
            for (int i = 0; i < novf; ++i) score_community(x, __ldcg(&ovf[i]), tb, offs, rs, &sacc[0], tid, T, red);
            block_sync();
            if (tid == 0) {
                ScoreAcc t = sacc[0];
                for (int w = 1; w < W; ++w) score_acc_add(t, sacc[w]);
                ScoreTotals tt;
                tt.qds_self = t.qds_self;
                tt.qds_pair = t.qds_pair;
                tt.dens = t.dens;
                tt.contr = t.contr;
                tt.expn = t.expn;
                tt.cond = t.cond;
                tt.vol2 = (i128)t.vol2;
                tt.ein = t.ein;
                tt.eout = t.eout;
                tt.nonempty = t.nonempty;
                tt.slots = t.slots;
                tt.cnt2 = t.cnt2;
                make_quality(tt, n, I.n_arcs / 2, I.out_q);
            }
        }

        // 5. metrics with ground truth
        if (do_cmp) {
            CompareCtx x;
            x.truth = I.truth;
            x.tl = nullptr;
            x.members = members;
            x.start = start;
            x.size_a = size_a;
            x.rowmax_n = rowmax_n;
            x.rowmax_r = rowmax_r;
            x.N = n;
            x.ka = kt;
            x.kb = K;
            x.err = I.status;
            CompareAcc *cacc = (CompareAcc *)(sm + p.acc_off);
            block_sync();
            for (int i = tid; i < W; i += T) compare_acc_zero(cacc[i]);
            block_sync();
            const int ncmp = s_ncmp;
            for (int i = 0; i < ncmp; ++i) compare_community(x, __ldcg(&big_cmp[i]), tb, &cacc[0], tid, T, red);
            const int chunk2 = claim_chunk(K, W);
            for (;;) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&s_next2, chunk2);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (base >= K) break;
                const int b = base + lane;
                const int sz = lane < chunk2 && b < K ? __ldcg(&start[b + 1]) - __ldcg(&start[b]) : 0;
                unsigned mask = __ballot_sync(0xffffffffu, sz > 0 && sz <= p.max_used_w);
                while (mask) {
                    const int j = __ffs(mask) - 1;
                    mask &= mask - 1;
                    compare_community(x, base + j, tw, &cacc[wid], lane, 32, red);
                }
            }
            __threadfence();
            block_sync();  // row maxima complete
            CompareAcc racc;
            compare_acc_zero(racc);
            for (int r = tid; r < kt; r += T) compare_row(x, r, racc);
            CompareTotals t;
            t.hden = group_sum_i128(racc.hden, T, red);
            t.f = group_sum_i128(racc.f, T, red);
            t.sa = group_sum_u64(racc.sa, T, red);
            t.nvd = group_sum_u64(racc.nvd, T, red);
            t.ka = group_sum_u64(racc.ka, T, red);
            if (tid == 0) {
                CompareAcc c = cacc[0];
                for (int w = 1; w < W; ++w) compare_acc_add(c, cacc[w]);
                t.vi = c.vi;
                t.hnum = c.hnum;
                t.hden += c.hden;
                t.f += c.f;
                t.a11 = c.a11;
                t.sa += c.sa;
                t.sb = c.sb;
                t.nvd += c.nvd;
                t.cells = c.cells;
                t.ka += c.ka;
                t.kb = c.kb;
                make_compare(t, n, I.out_c);
            }
        }
        block_sync();
    }
}

// ------------------------------------------------------------------ the two-phase pipeline over all candidates

enum { BU_NBIG_S = 0, BU_NBIG_C = 1, BU_NEXT_BIG_S = 2, BU_NEXT_BIG_C = 3, BU_NEXT_UNIT_S = 4,
       BU_NEXT_UNIT_C = 5, BU_CTR = 16 };

size_t batch_units_bytes(int count, long long n_max, long long a_max, int k_max, int kt_max, bool cells)
{
    return carve_batch_units(reinterpret_cast<void *>(4096), count, n_max, a_max, k_max, kt_max, cells).bytes;
}

BatchUnits carve_batch_units(void *base, int count, long long n_max, long long a_max, int k_max, int kt_max,
                             bool cells)
{
    BatchUnits b{};
    char *p = (char *)base;
    const size_t C = (size_t)count, N = (size_t)n_max, A = (size_t)std::max(a_max, 1LL);
    const size_t Kx = (size_t)k_max, Kt = (size_t)kt_max;
    auto take = [&](size_t bytes) {
        char *q = p;
        p += al(bytes);
        return (void *)q;
    };
    b.n_max = n_max;
    b.a_max = a_max;
    b.k_max = k_max;
    b.kt_max = kt_max;
    b.count = count;
    b.tpre = (int *)take((C + 1) * 4);
    b.cpre = (int *)take((C + 1) * 4);
    b.kpre = (int *)take((C + 1) * 4);
    b.logt = (double *)take(LOGT_WORDS * 8);
    b.zero = p;
    b.cv = (unsigned long long *)take(C * Kx * 8);
    b.inter = (int *)take(C * Kx * 4);
    b.inter_hi = (int *)take(C * Kx * 4);
    b.size_a = (int *)take(C * Kt * 4);
    b.rowmax_n = (unsigned *)take(C * Kt * 4);
    b.rowmax_r = (unsigned long long *)take(C * Kt * 8);
    b.ncells = (int *)take(C * 4);
    b.gcell = (unsigned long long *)take(C * 2 * 8);
    b.ctr = (int *)take(BU_CTR * 4);
    b.zero_bytes = (size_t)(p - (char *)b.zero);
    b.members = (int *)take(C * N * 4);
    b.aoff = (unsigned *)take(C * (N + 1) * 4);
    b.start = (int *)take(C * (Kx + 1) * 4);
    b.recip = (Rcp *)take(C * Kx * sizeof(Rcp));
    b.rec = (unsigned long long *)take(C * Kx * REC_WORDS * 8);
    b.nbr = (int *)take(C * A * 4);
    b.cells = cells ? take(C * N * sizeof(Cell)) : nullptr;
    const size_t U = std::max<size_t>(C * Kx, 1);
    b.big_s = (unsigned long long *)take(U * 8);
    b.big_c = (unsigned long long *)take(U * 8);
    b.bytes = (size_t)(p - (char *)base);
    return b;
}

// One candidate's slices of the scratch.
struct BuSlice {
    int *members, *start, *inter, *inter_hi, *nbr, *size_a;
    unsigned long long *cv;
    unsigned *aoff, *rowmax_n;
    Rcp *recip;
    unsigned long long *rec, *rowmax_r;
    Cell *cells;
};

__device__ __forceinline__ BuSlice bu_slice(const BatchUnits &b, int it)
{
    const size_t i = (size_t)it, N = (size_t)b.n_max, Kx = (size_t)b.k_max, Kt = (size_t)b.kt_max;
    BuSlice s;
    s.members = b.members + i * N;
    s.aoff = b.aoff + i * (N + 1);
    s.start = b.start + i * (Kx + 1);
    s.cv = b.cv + i * Kx;
    s.recip = b.recip + i * Kx;
    s.inter = b.inter + i * Kx;
    s.inter_hi = b.inter_hi + i * Kx;
    s.rec = b.rec + i * Kx * REC_WORDS;
    s.nbr = b.nbr + i * (size_t)std::max(b.a_max, 1LL);
    s.cells = b.cells ? (Cell *)b.cells + i * N : nullptr;
    s.size_a = b.size_a + i * Kt;
    s.rowmax_n = b.rowmax_n + i * Kt;
    s.rowmax_r = b.rowmax_r + i * Kt;
    return s;
}

__device__ __forceinline__ unsigned long long bu_key(int it, int c)
{
    return ((unsigned long long)(unsigned)it << 32) | (unsigned)c;
}

__device__ __forceinline__ bool bu_dead(const BatchItem &I) { return *(volatile int *)I.status != 0; }

// log(N / i) and i / N for i = 1 .. LOGT_MAX (the same expressions as the
// plain comparison's tables, so the same bits).
__global__ void k_bu_logt(double *logt, long long N)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= LOGT_MAX; i += gridDim.x * blockDim.x) {
        logt[i] = i == 0 ? 0.0 : log_ratio(N, i);
        logt[LOGT_MAX + 1 + i] = nmi_over(i, N);
    }
}

// The candidate holding unit u of a prefix (pre[p] <= u < pre[p + 1]), cur a guess.
__device__ __forceinline__ int bu_item(const int *pre, int count, int u, int cur)
{
    if (cur >= 0 && u >= __ldg(&pre[cur]) && u < __ldg(&pre[cur + 1])) return cur;
    int lo = 0, hi = count;  // largest p with pre[p] <= u
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&pre[mid]) <= u) lo = mid; else hi = mid;
    }
    return lo;
}

// A community's histogram word: members in the high bits, the volume (the
// degree sum, 2|E_c^in| + |E_c^out|) in the low BU_ARC_BITS bits.  The counting
// sort adds (1, deg u) to the community's cursor word, so the one atomic
// returns both the member position of u and the arc offset of that position.
constexpr int BU_ARC_BITS = 40;
constexpr unsigned long long BU_ARC_MASK = (1ull << BU_ARC_BITS) - 1ull;

__device__ __forceinline__ unsigned long long bu_degree(const BatchItem &I, long long v)
{
    return (I.flags & 1) ? (unsigned long long)(__ldg(&I.row_ptr[v + 1]) - __ldg(&I.row_ptr[v])) : 0ull;
}

// Label histograms with range checks over (candidate, node tile) units; a
// candidate with an id out of range gets status bit 0 and no further work.
__global__ void __launch_bounds__(256) k_bu_hist(const BatchItem *items, int count, BatchUnits b)
{
    const int units = __ldg(&b.tpre[count]);
    int cur = -1;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
        const int it = cur = bu_item(b.tpre, count, u, cur);
        const BatchItem &I = items[it];
        const BuSlice S = bu_slice(b, it);
        const long long v0 = (long long)(u - __ldg(&b.tpre[it])) * BATCH_UNITS_TILE;
        const long long v1 = min(I.n, v0 + BATCH_UNITS_TILE);
        const bool do_cmp = (I.flags & 2) != 0 && I.truth != nullptr;
        const int K = I.K, kt = I.k_truth;
        bool bad = false;
        for (long long v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
            const int l = __ldg(&I.labels[v]);
            if ((unsigned)l >= (unsigned)K) bad = true;
            else atomicAdd(&S.cv[l], (1ull << BU_ARC_BITS) | bu_degree(I, v));
            if (do_cmp) {
                const int t = __ldg(&I.truth[v]);
                if ((unsigned)t >= (unsigned)kt) bad = true;
                else atomicAdd(&S.size_a[t], 1);
            }
        }
        if (bad) atomicOr(I.status, 1);
    }
}

// One block per candidate: community offsets and volumes (exclusive scans of
// the histogram words), reciprocals of the sizes, and the cursor words of the
// counting sort.
__global__ void __launch_bounds__(BATCH_MAX_THREADS) k_bu_scan(const BatchItem *items, int count, BatchUnits b)
{
    __shared__ unsigned long long red[72];
    const int tid = threadIdx.x, T = blockDim.x;
    for (int it = blockIdx.x; it < count; it += gridDim.x) {
        const BatchItem I = items[it];
        if (bu_dead(I)) continue;
        const BuSlice S = bu_slice(b, it);
        const int K = I.K;
        unsigned carry_m = 0, carry_a = 0;
        for (int c0 = 0; c0 < K; c0 += T) {
            const int c = c0 + tid;
            const unsigned long long w = c < K ? __ldcg(&S.cv[c]) : 0ull;
            const unsigned m = (unsigned)(w >> BU_ARC_BITS), vol = (unsigned)(w & BU_ARC_MASK);
            unsigned ex_m, ex_a;
            const unsigned tot_m = group_exclusive_scan(m, ex_m, T, red);
            const unsigned tot_a = group_exclusive_scan(vol, ex_a, T, red);
            if (c < K) {
                S.start[c] = (int)(carry_m + ex_m);
                S.cv[c] = ((unsigned long long)(carry_m + ex_m) << BU_ARC_BITS) | (carry_a + ex_a);
                if (m > 0) S.recip[c] = rcp_of(m);
            }
            carry_m += tot_m;
            carry_a += tot_a;
        }
        if (tid == 0) {
            S.start[K] = (int)carry_m;
            S.aoff[I.n] = carry_a;
        }
        block_sync();
    }
}

// The counting sort over (candidate, node tile) units: each node takes its
// member position and that position's arc offset from one atomic.
__global__ void __launch_bounds__(256) k_bu_scatter(const BatchItem *items, int count, BatchUnits b)
{
    const int units = __ldg(&b.tpre[count]);
    int cur = -1;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
        const int it = cur = bu_item(b.tpre, count, u, cur);
        const BatchItem &I = items[it];
        if (bu_dead(I)) continue;
        const BuSlice S = bu_slice(b, it);
        const long long v0 = (long long)(u - __ldg(&b.tpre[it])) * BATCH_UNITS_TILE;
        const long long v1 = min(I.n, v0 + BATCH_UNITS_TILE);
        for (long long v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
            const int l = __ldg(&I.labels[v]);
            const unsigned long long old = atomicAdd(&S.cv[l], (1ull << BU_ARC_BITS) | bu_degree(I, v));
            const long long pos = (long long)(old >> BU_ARC_BITS);
            if (QM_CHK(pos, I.n, 10)) {
                S.members[pos] = (int)v;
                S.aoff[pos] = (unsigned)(old & BU_ARC_MASK);
            }
        }
    }
}

// A warp's share of phase A for the batched pipeline: expand_chunk, except
// that when the chunk's members are not a few runs of consecutive node ids
// (the usual case for candidate partitions), the owner of each arc of the
// chunk is tabulated once (each lane writes its member's index over its arc
// range, up to BU_OWN_CAP arcs) instead of searched for arc by arc.
constexpr int BU_OWN_CAP = 2048;

__device__ __forceinline__ void bu_expand_chunk(long long p0, long long n, const long long *__restrict__ row_ptr,
                                                const int *__restrict__ col, const int *__restrict__ labels,
                                                const int *__restrict__ members, const unsigned *__restrict__ aoff,
                                                const int *__restrict__ start, int *inter, int *inter_hi,
                                                int *__restrict__ nbr, unsigned *offw, long long *rsw, int *cw,
                                                unsigned char *own, unsigned long long keep, int lane)
{
    const int nm = (int)min(32LL, n - p0);
    const unsigned base = __ldg(&aoff[p0]);
    int u = -2;
    if (lane < nm) {
        u = __ldcs(&members[p0 + lane]);
        offw[lane] = __ldg(&aoff[p0 + lane]) - base;
        rsw[lane] = __ldg(&row_ptr[u]);
        cw[lane] = ld_hint(&labels[u], keep);
    }
    if (lane == 0) offw[nm] = __ldg(&aoff[p0 + nm]) - base;
    __syncwarp();
    const int u_prev = __shfl_up_sync(0xffffffffu, u, 1);
    const bool valid = lane < nm;
    const bool newrun = valid && (lane == 0 || cw[lane] != cw[lane - 1]);
    unsigned runs = __ballot_sync(0xffffffffu, newrun);
    const unsigned segs = __ballot_sync(0xffffffffu, newrun || (valid && u != u_prev + 1));
    u128 w_in = 0, w_out = 0;
    if (__popc(segs) <= EXPAND_MAX_SEGS) {
        unsigned rem = segs;
        while (rem) {
            const int lo = __ffs(rem) - 1;
            rem &= rem - 1;
            const int hi = rem ? __ffs(rem) - 1 : nm;
            const unsigned e_lo = offw[lo], e_hi = offw[hi];
            if (e_lo == e_hi) continue;
            const int c = cw[lo];
            const unsigned cbase = __ldg(&aoff[__ldg(&start[c])]);
            const long long cs = rsw[lo] - (long long)e_lo;  // CSR index of arc e is cs + e
            expand_range<false, false, true>(e_lo, e_hi, c, cbase, [cs](unsigned e) { return cs + (long long)e; },
                                             col, labels, nullptr, inter, inter_hi, nbr, keep, lane, nullptr, nullptr,
                                             w_in, w_out);
        }
    } else {
        const bool tab = offw[nm] <= (unsigned)BU_OWN_CAP;
        if (tab) {
            const unsigned a = lane < nm ? offw[lane] : 0u, z = lane < nm ? offw[lane + 1] : 0u;
            for (unsigned e = a; e < z; ++e) own[e] = (unsigned char)lane;
            __syncwarp();
        }
        while (runs) {
            const int m_lo = __ffs(runs) - 1;
            runs &= runs - 1;
            const int m_hi = runs ? __ffs(runs) - 1 : nm;
            const unsigned e_lo = offw[m_lo], e_hi = offw[m_hi];
            if (e_lo == e_hi) continue;
            const int c = cw[m_lo];
            const unsigned cbase = __ldg(&aoff[__ldg(&start[c])]);
            if (tab)
                expand_range<false, false, true>(
                    e_lo, e_hi, c, cbase,
                    [=](unsigned e) {
                        const int o = own[e];
                        return rsw[o] + (long long)(e - offw[o]);
                    },
                    col, labels, nullptr, inter, inter_hi, nbr, keep, lane, nullptr, nullptr, w_in, w_out);
            else
                expand_range<false, false, true>(
                    e_lo, e_hi, c, cbase,
                    [=](unsigned e) {
                        const int o = m_lo + upper_bound_smem(offw + m_lo, m_hi - m_lo, e) - 1;
                        return rsw[o] + (long long)(e - offw[o]);
                    },
                    col, labels, nullptr, inter, inter_hi, nbr, keep, lane, nullptr, nullptr, w_in, w_out);
        }
    }
    __syncwarp();
}

// Phase A over every scored candidate: warp by warp over (candidate, 32
// member positions) units, in unit order, so the warps in flight share a few
// candidates' label arrays in L2.
__global__ void __launch_bounds__(EXPAND_THREADS) k_bu_expand(const BatchItem *items, int count, BatchUnits b)
{
    __shared__ unsigned offs_s[EXPAND_THREADS / 32][33];
    __shared__ long long rs_s[EXPAND_THREADS / 32][32];
    __shared__ int cw_s[EXPAND_THREADS / 32][32];
    __shared__ unsigned char own_s[EXPAND_THREADS / 32][BU_OWN_CAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned long long keep = l2_policy_evict_last();
    const int units = __ldg(&b.cpre[count]);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    int cur = -1;
    for (int u = blockIdx.x * (blockDim.x >> 5) + w; u < units; u += nwarps) {
        const int it = cur = bu_item(b.cpre, count, u, cur);
        const BatchItem &I = items[it];
        if (!(I.flags & 1) || bu_dead(I)) continue;
        const BuSlice S = bu_slice(b, it);
        const long long p0 = (long long)(u - __ldg(&b.cpre[it])) * 32;
        bu_expand_chunk(p0, I.n, I.row_ptr, I.col, I.labels, S.members, S.aoff, S.start, S.inter, S.inter_hi, S.nbr,
                        offs_s[w], rs_s[w], cw_s[w], own_s[w], keep, lane);
    }
}

// Warp-aggregated table updates for phase B.  Candidate partitions send many
// arcs of a community to the same few neighbours, so the lanes of a warp
// often hold the same key; they are merged (__match_any_sync) and one lane
// adds all q occurrences.  The k-th occurrence of a key adds (2k - 1) Rcp_j to
// the pair sum (see count_run), so q occurrences numbered lo+1 .. lo+q add
// ((lo + q)^2 - lo^2) Rcp_j: the same exact integer total as one at a time.
__device__ __forceinline__ unsigned long long sq_diff(unsigned long long lo, unsigned long long q)
{
    return q * (2ull * lo + q);  // (lo + q)^2 - lo^2
}

// Adds q occurrences of key k in `epoch`; returns their share multiplier
// (sum of 2k - 1 over the occurrences taken) and whether the key is new, or 0
// when the table is full (the pass is then discarded).
__device__ __forceinline__ unsigned long long bu_add_n(const EpochTable32 &t, unsigned k, unsigned q, unsigned epoch,
                                                       bool &first)
{
    const unsigned tag = (epoch << 24) | (k + 1u);
    // repeats beyond a key's first occurrence, in rep[h]; returns those before
    auto rep_add = [&](unsigned h, unsigned r) -> unsigned {
        unsigned w = ((volatile unsigned *)t.rep)[h];
        for (;;) {
            const bool same = (w >> 24) == epoch;
            const unsigned prev = atomicCAS(&t.rep[h], w, same ? w + r : ((epoch << 24) | r));
            if (prev == w) return same ? (w & 0xFFFFFFu) : 0u;
            w = prev;
        }
    };
    unsigned h = tab_hash(k, t.cap);
    unsigned cur = ((volatile unsigned *)t.key)[h];
    const int limit = 2 * t.cap + 64;
    for (int step = 0; step < limit; ++step) {
        if ((cur >> 24) != epoch) {
            const unsigned prev = atomicCAS(&t.key[h], cur, tag);
            if (prev == cur) {
                // occurrence 1, then q - 1 repeats numbered after those already counted
                first = true;
                if (q == 1) return 1ull;
                const unsigned w0 = rep_add(h, q - 1);
                return 1ull + sq_diff(1ull + w0, q - 1);
            }
            cur = prev;
            continue;
        }
        if (cur == tag) {
            first = false;
            const unsigned w0 = rep_add(h, q);
            return sq_diff(1ull + w0, q);
        }
        if ((step & 15) == 15 && *(volatile int *)t.overflow) return 0ull;
        h = (h + 1u == (unsigned)t.cap) ? 0u : h + 1u;
        cur = ((volatile unsigned *)t.key)[h];
    }
    *t.overflow = 1;
    return 0ull;
}

__device__ __forceinline__ unsigned long long bu_add_n(const EpochTable &t, unsigned k, unsigned q, unsigned epoch,
                                                       bool &first)
{
    const unsigned long long tag =
        ((unsigned long long)epoch << 56) | ((unsigned long long)(k + 1u) << EpochTable::CNT_BITS);
    unsigned h = tab_hash(k, t.cap);
    unsigned long long cur = ((volatile unsigned long long *)t.slot)[h];
    const int limit = 2 * t.cap + 64;
    for (int step = 0; step < limit; ++step) {
        if ((unsigned)(cur >> 56) != epoch) {
            const unsigned long long prev = atomicCAS(&t.slot[h], cur, tag | (unsigned long long)q);
            if (prev == cur) {
                first = true;
                return sq_diff(0ull, q);
            }
            cur = prev;
            continue;
        }
        if ((cur & ~EpochTable::CNT_MASK) == tag) {
            first = false;
            const unsigned long long lo = atomicAdd(&t.slot[h], (unsigned long long)q) & EpochTable::CNT_MASK;
            return sq_diff(lo, q);
        }
        if ((step & 15) == 15 && *(volatile int *)t.overflow) return 0ull;
        h = (h + 1u == (unsigned)t.cap) ? 0u : h + 1u;
        cur = ((volatile unsigned long long *)t.slot)[h];
    }
    *t.overflow = 1;
    return 0ull;
}

// count_run (phase B of the plain path) with warp-aggregated updates: the same
// record, the same bits.  Every warp of the group walks the run in
// warp-uniform steps of BU_CU entries a lane, all loaded (with their
// reciprocals) before the table updates, so that its lanes can merge equal
// keys and several loads are in flight.
constexpr int BU_CU = 4;

template <class TAB>
__device__ __forceinline__ void count_run_agg(const CountCtx &x, const RunHdr &h, const int *src, const TAB &tab,
                                              unsigned &epoch, int gtid, int gsize, unsigned long long *red)
{
    const unsigned m = h.m;
    const unsigned fill = (unsigned)(3 * tab.cap / 4);
    unsigned R = m <= fill ? 1u : (unsigned)min((unsigned long long)R_MAX, ((unsigned long long)m + fill - 1) / fill);
    const int c = h.c, lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long slots = 0, cnt2 = 0;
        U192 inner, inner_full;
        u192_zero(inner);
        u192_zero(inner_full);
        bool ok = true;
        for (unsigned r = 0; r < R && ok; ++r) {
            epoch = etab_next_epoch(tab, epoch, gtid, gsize);
            for (unsigned e0 = (unsigned)(gtid & ~31) * BU_CU; e0 < m; e0 += (unsigned)gsize * BU_CU) {
                int lv[BU_CU];
                Rcp rj[BU_CU];
#pragma unroll
                for (int k = 0; k < BU_CU; ++k) {
                    const unsigned e = e0 + (unsigned)lane + 32u * k;
                    lv[k] = e < m ? __ldcs(&src[e]) : -1;
                    if (lv[k] >= 0 &&
                        (!QM_CHK(lv[k], x.K, 6) || lv[k] < c || (R > 1 && tab_split((unsigned)lv[k], R) != r)))
                        lv[k] = -1;
                }
#pragma unroll
                for (int k = 0; k < BU_CU; ++k)
                    if (lv[k] >= 0) rj[k] = ld_rcp(&x.recip[lv[k]]);
#pragma unroll
                for (int k = 0; k < BU_CU; ++k) {
                    const unsigned act = __ballot_sync(0xffffffffu, lv[k] >= 0);
                    if (lv[k] < 0) continue;
                    const unsigned peers = __match_any_sync(act, lv[k]);
                    if (lane != __ffs(peers) - 1) continue;
                    bool first = false;
                    const unsigned long long q2 = bu_add_n(tab, (unsigned)lv[k], (unsigned)__popc(peers), epoch, first);
                    if (q2 == 0ull) continue;  // overflow: this pass is discarded
                    if (q2 == 1ull) u192_add_rcp(inner, rj[k]);
                    else u192_mac(inner, q2, rj[k]);
                    cnt2 += q2;
                    slots += first ? 1ull : 0ull;
                }
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
        group_totals<false>(slots, cnt2, inner, inner_full, gsize, red);
        if (gtid == 0) put_record(x, h.c, h.vol, m, slots, cnt2, inner, inner_full);
        if (gsize == 32) __syncwarp();
        return;
    }
}

// Phase B with a direct-mapped 16-bit counter per label id (two to a 32-bit
// word of shared memory), for candidates whose K ids all fit: a first pass
// adds each entry to its key's counter; a second pass takes each key's count
// at its first visit (an atomic AND that also clears the counter) and adds
// |E_cj|^2 Rcp_j for it, so the counters are back at zero for the next run.
// The record is the same as count_run's: the same exact integer sums.  Runs
// must be shorter than 2^16 entries.
__device__ __forceinline__ void count_run_direct(const CountCtx &x, const RunHdr &h, const int *src, unsigned *w16,
                                                 int gtid, int gsize, unsigned long long *red)
{
    const unsigned m = h.m;
    const int c = h.c;
    for (unsigned e0 = (unsigned)gtid; e0 < m; e0 += (unsigned)gsize * BU_CU) {
        int lv[BU_CU];
#pragma unroll
        for (int k = 0; k < BU_CU; ++k) {
            const unsigned e = e0 + (unsigned)gsize * k;
            lv[k] = e < m ? __ldg(&src[e]) : -1;
        }
#pragma unroll
        for (int k = 0; k < BU_CU; ++k)
            if (lv[k] > c && QM_CHK(lv[k], x.K, 6)) atomicAdd(&w16[lv[k] >> 1], 1u << ((lv[k] & 1) << 4));
    }
    group_sync_n(gsize);
    unsigned long long slots = 0, cnt2 = 0;
    U192 inner, inner_full;
    u192_zero(inner);
    u192_zero(inner_full);
    for (unsigned e0 = (unsigned)gtid; e0 < m; e0 += (unsigned)gsize * BU_CU) {
        int lv[BU_CU];
        unsigned cnt[BU_CU];
        Rcp rj[BU_CU];
#pragma unroll
        for (int k = 0; k < BU_CU; ++k) {
            const unsigned e = e0 + (unsigned)gsize * k;
            lv[k] = e < m ? __ldg(&src[e]) : -1;
            if (lv[k] <= c || !QM_CHK(lv[k], x.K, 6)) lv[k] = -1;
        }
#pragma unroll
        for (int k = 0; k < BU_CU; ++k) {
            cnt[k] = 0u;
            if (lv[k] >= 0) {
                const unsigned sh = ((unsigned)lv[k] & 1u) << 4;
                cnt[k] = (atomicAnd(&w16[lv[k] >> 1], ~(0xFFFFu << sh)) >> sh) & 0xFFFFu;
            }
        }
#pragma unroll
        for (int k = 0; k < BU_CU; ++k)
            if (cnt[k]) rj[k] = ld_rcp(&x.recip[lv[k]]);
#pragma unroll
        for (int k = 0; k < BU_CU; ++k) {
            if (!cnt[k]) continue;
            const unsigned long long q = (unsigned long long)cnt[k] * cnt[k];
            if (q == 1ull) u192_add_rcp(inner, rj[k]);
            else u192_mac(inner, q, rj[k]);
            cnt2 += q;
            slots += 1ull;
        }
    }
    group_totals<false>(slots, cnt2, inner, inner_full, gsize, red);
    if (gtid == 0) put_record(x, h.c, h.vol, m, slots, cnt2, inner, inner_full);
    if (gsize == 32) __syncwarp();
}

// The run header of community c of one candidate: its packed run and volume.
__device__ __forceinline__ RunHdr bu_run(const BuSlice &S, int c)
{
    const unsigned a0 = __ldcg(&S.aoff[__ldcg(&S.start[c])]), a1 = __ldcg(&S.aoff[__ldcg(&S.start[c + 1])]);
    return RunHdr{c, a0, (unsigned)__ldcg(&S.inter_hi[c]), a1 - a0};
}

// A group's shared-memory counting region: `words` 32-bit words that serve
// either as direct 16-bit counters (count_run_direct, left all zero) or as an
// epoch-tagged hash table (count_run_agg, left tagged: `dirty`).
struct BuRegion {
    unsigned *w;
    int words;
    bool dirty;
    unsigned epoch;
};

// Phase B of one community of one candidate with a group: its record.
template <class TAB>
__device__ __forceinline__ void bu_count_one(const BatchItem &I, const BuSlice &S, const RunHdr &h, const TAB &tab,
                                             BuRegion &rg, int gtid, int gsize, unsigned long long *red)
{
    CountCtx x;
    x.nbr = S.nbr;
    x.aoff = S.aoff;
    x.start = S.start;
    x.inter = S.inter;
    x.recip = S.recip;
    x.rec = S.rec;
    x.K = I.K;
    x.err = I.status;
    x.full = 0;
    if ((long long)I.K <= 2LL * rg.words && h.m < (1u << 16)) {
        if (rg.dirty) {  // a hash pass left tagged slots: clear them once
            for (int i = gtid; i < rg.words; i += gsize) rg.w[i] = 0u;
            group_sync_n(gsize);
            rg.dirty = false;
            rg.epoch = 0;
        }
        count_run_direct(x, h, S.nbr + h.a0, rg.w, gtid, gsize, red);
        return;
    }
    rg.dirty = true;
    count_run_agg<TAB>(x, h, S.nbr + h.a0, tab, rg.epoch, gtid, gsize, red);
}

struct BuArgs {
    const BatchItem *items;
    int count;
    BatchUnits b;
    int smem_bytes;
    SmemPlan plan;  // comparison tables
    int phase;      // 0: single warps over all units (larger ones are listed), 1: whole blocks over the list
};

// Shared-memory carving of k_bu_count: the group-total exchange (256 words),
// overflow flags, then the counting table (W warp slices, or one block table).
constexpr int BU_COUNT_SLOT_OFF = 256 * 8 + 256;

// Phase B over every scored candidate's communities: runs a warp's table holds
// at 3/4 load are counted by single warps (phase 0), the others by whole blocks
// (phase 1), with direct counters when the candidate's ids fit the group's
// region, else with the epoch-tagged tables of the plain path.
template <class TAB>
__global__ void __launch_bounds__(BATCH_MAX_THREADS, 1) k_bu_count(BuArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_i;
    const BatchUnits &b = a.b;
    const int T = blockDim.x, W = T >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    unsigned long long *red = (unsigned long long *)sm;
    int *ovf = (int *)(sm + 256 * 8);
    unsigned long long *slot = (unsigned long long *)(sm + BU_COUNT_SLOT_OFF);
    const int cap_w = (a.smem_bytes - BU_COUNT_SLOT_OFF) / 8 / W;
    for (int i = tid; i < cap_w * W; i += T) slot[i] = 0ull;
    for (int i = tid; i <= W; i += T) ovf[i] = 0;
    block_sync();
    if (a.phase == 0) {
        const TAB tab = make_table<TAB>(slot + (size_t)wid * cap_w, cap_w, &ovf[wid]);
        BuRegion rg{(unsigned *)(slot + (size_t)wid * cap_w), 2 * cap_w, false, 0u};
        const unsigned fill_w = (unsigned)(3 * cap_w / 4);
        const int units = __ldg(&b.kpre[a.count]);
        const int chunk = claim_chunk(units, (long long)gridDim.x * W);
        int look = -1;
        for (;;) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&b.ctr[BU_NEXT_UNIT_S], chunk);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= units) break;
            // each lane sizes one unit of the chunk; the warp then counts the
            // small runs in order and lists the others
            int it = -1;
            RunHdr h{0, 0u, 0u, 0u};
            bool small = false;
            if (lane < chunk && base + lane < units) {
                it = look = bu_item(b.kpre, a.count, base + lane, look);
                const int c = base + lane - __ldg(&b.kpre[it]);
                const BatchItem &I = a.items[it];
                if ((I.flags & 1) && !bu_dead(I)) {
                    const BuSlice S = bu_slice(b, it);
                    if (__ldcg(&S.start[c + 1]) > __ldcg(&S.start[c])) {
                        h = bu_run(S, c);
                        small = h.m <= fill_w;
                        if (!small) b.big_s[atomicAdd(&b.ctr[BU_NBIG_S], 1)] = bu_key(it, c);
                    }
                }
            }
            unsigned mask = __ballot_sync(0xffffffffu, small);
            while (mask) {
                const int j = __ffs(mask) - 1;
                mask &= mask - 1;
                const int itj = __shfl_sync(0xffffffffu, it, j);
                const RunHdr hj{__shfl_sync(0xffffffffu, h.c, j), __shfl_sync(0xffffffffu, h.a0, j),
                                __shfl_sync(0xffffffffu, h.m, j), __shfl_sync(0xffffffffu, h.vol, j)};
                bu_count_one<TAB>(a.items[itj], bu_slice(b, itj), hj, tab, rg, lane, 32, red);
            }
        }
        return;
    }
    const TAB tab = make_table<TAB>(slot, cap_w * W, &ovf[W]);
    BuRegion rg{(unsigned *)slot, 2 * cap_w * W, false, 0u};
    const int nbig = *(volatile int *)&b.ctr[BU_NBIG_S];
    for (;;) {
        if (tid == 0) s_i = atomicAdd(&b.ctr[BU_NEXT_BIG_S], 1);
        block_sync();
        const int i = s_i;
        block_sync();
        if (i >= nbig) break;
        const unsigned long long key = __ldcg(&b.big_s[i]);
        const int it = (int)(key >> 32), c = (int)(key & 0xFFFFFFFFull);
        const BuSlice S = bu_slice(b, it);
        bu_count_one<TAB>(a.items[it], S, bu_run(S, c), tab, rg, tid, T, red);
    }
}

// Contingency cells of found community c of one candidate with a group; its
// column maximum and cell count go to the candidate's accumulators.
__device__ __forceinline__ void bu_cells_one(const BatchItem &I, const BuSlice &S, unsigned long long *gcell, int c,
                                             int *ncells, const SmemTable &tab, int gtid, int gsize,
                                             unsigned long long *red)
{
    CompareCtx x;
    x.truth = I.truth;
    x.tl = nullptr;
    x.members = S.members;
    x.start = S.start;
    x.size_a = S.size_a;
    x.rowmax_n = S.rowmax_n;
    x.rowmax_r = S.rowmax_r;
    x.N = I.n;
    x.ka = I.k_truth;
    x.kb = I.K;
    x.err = I.status;
    CompareAcc acc;
    compare_acc_zero(acc);
    compare_cells_community(x, c, tab, &acc, gtid, gsize, red, S.cells, ncells);
    if (gtid == 0) {
        if (acc.nvd) atomicAdd(&gcell[0], acc.nvd);
        if (acc.cells) atomicAdd(&gcell[1], acc.cells);
    }
}

// Cells of every compared candidate's found communities: single warps take
// the communities whose members fit a warp's table (phase 0), whole blocks the
// others (phase 1).
__global__ void __launch_bounds__(BATCH_MAX_THREADS, 1) k_bu_cells(BuArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_i;
    const SmemPlan &p = a.plan;
    const BatchUnits &b = a.b;
    unsigned long long *red = (unsigned long long *)(sm + p.red_off);
    int *ctl = (int *)(sm + p.ctl_off);
    unsigned long long *slot = (unsigned long long *)(sm + p.slot_off);
    int *used = (int *)(sm + p.used_off);
    const int T = blockDim.x, W = T >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    for (int i = tid; i < p.cap; i += T) slot[i] = 0ull;
    for (int i = tid; i < 2 * (W + 1); i += T) ctl[i] = 0;
    block_sync();
    if (a.phase == 0) {
        const SmemTable tw{slot + wid * p.cap_w, used + wid * p.max_used_w, &ctl[2 + 2 * wid], &ctl[3 + 2 * wid],
                           p.cap_w, p.max_used_w};
        const int units = __ldg(&b.kpre[a.count]);
        const int chunk = claim_chunk(units, (long long)gridDim.x * W);
        int look = -1;
        for (;;) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&b.ctr[BU_NEXT_UNIT_C], chunk);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= units) break;
            int it = -1, c = 0;
            bool small = false;
            if (lane < chunk && base + lane < units) {
                it = look = bu_item(b.kpre, a.count, base + lane, look);
                c = base + lane - __ldg(&b.kpre[it]);
                const BatchItem &I = a.items[it];
                if ((I.flags & 2) && I.truth && !bu_dead(I)) {
                    const int *st = b.start + (size_t)it * ((size_t)b.k_max + 1);
                    const int sz = __ldcg(&st[c + 1]) - __ldcg(&st[c]);
                    small = sz > 0 && sz <= p.max_used_w;
                    if (sz > p.max_used_w) b.big_c[atomicAdd(&b.ctr[BU_NBIG_C], 1)] = bu_key(it, c);
                }
            }
            unsigned mask = __ballot_sync(0xffffffffu, small);
            while (mask) {
                const int j = __ffs(mask) - 1;
                mask &= mask - 1;
                const int itj = __shfl_sync(0xffffffffu, it, j), cj = __shfl_sync(0xffffffffu, c, j);
                bu_cells_one(a.items[itj], bu_slice(b, itj), b.gcell + 2 * (size_t)itj, cj, b.ncells + itj, tw,
                             lane, 32, red);
            }
        }
        return;
    }
    const SmemTable tb{slot, used, &ctl[0], &ctl[1], p.cap, p.max_used};
    const int nbig = *(volatile int *)&b.ctr[BU_NBIG_C];
    for (;;) {
        if (tid == 0) s_i = atomicAdd(&b.ctr[BU_NEXT_BIG_C], 1);
        block_sync();
        const int i = s_i;
        block_sync();
        if (i >= nbig) break;
        const unsigned long long key = __ldcg(&b.big_c[i]);
        const int it = (int)(key >> 32), c = (int)(key & 0xFFFFFFFFull);
        bu_cells_one(a.items[it], bu_slice(b, it), b.gcell + 2 * (size_t)it, c, b.ncells + it, tb, tid, T, red);
    }
}

constexpr int BU_FIN_THREADS = 256;
constexpr int BU_CELLS_SMEM = 48 * 1024;  // shared memory of a k_bu_cells block at most

// One block per candidate: the FP64 terms of every community record (Eq. (9),
// Sec. II-B.3) and of every contingency cell, column and row (Eqs. 1-7), all
// lanes busy, summed in fixed point; then the final results.
__global__ void __launch_bounds__(BU_FIN_THREADS) k_bu_fin(const BatchItem *items, int count, BatchUnits b)
{
    __shared__ unsigned long long red[72];
    const int tid = threadIdx.x, T = blockDim.x;
    for (int it = blockIdx.x; it < count; it += gridDim.x) {
        const BatchItem I = items[it];
        if (bu_dead(I)) continue;
        const BuSlice S = bu_slice(b, it);
        const long long E = I.n_arcs / 2;
        if (I.flags & 1) {
            ScoreAcc acc;
            score_acc_zero(acc);
            for (int c = tid; c < I.K; c += T) {
                const long long size = __ldcg(&S.start[c + 1]) - __ldcg(&S.start[c]);
                if (size <= 0) continue;
                double pen, qs, dens, contr, expn, cond;
                terms_from_record(S.rec + (size_t)c * REC_WORDS, size, E, acc, &pen, &qs, &dens, &contr, &expn, &cond);
            }
            ScoreTotals t;
            t.qds_self = group_sum_i128(acc.qds_self, T, red);
            t.qds_pair = group_sum_i128(acc.qds_pair, T, red);
            t.dens = group_sum_i128(acc.dens, T, red);
            t.contr = group_sum_i128(acc.contr, T, red);
            t.expn = group_sum_i128(acc.expn, T, red);
            t.cond = group_sum_i128(acc.cond, T, red);
            t.vol2 = group_sum_i128((i128)acc.vol2, T, red);
            t.ein = group_sum_u64(acc.ein, T, red);
            t.eout = group_sum_u64(acc.eout, T, red);
            t.nonempty = group_sum_u64(acc.nonempty, T, red);
            t.slots = group_sum_u64(acc.slots, T, red);
            t.cnt2 = group_sum_u64(acc.cnt2, T, red);
            if (tid == 0) make_quality(t, I.n, E, I.out_q);
        }
        if ((I.flags & 2) && I.truth && S.cells) {
            CompareCtx x;
            x.truth = I.truth;
            x.tl = nullptr;
            x.members = S.members;
            x.start = S.start;
            x.size_a = S.size_a;
            x.rowmax_n = S.rowmax_n;
            x.rowmax_r = S.rowmax_r;
            x.N = I.n;
            x.ka = I.k_truth;
            x.kb = I.K;
            x.err = I.status;
            const double *logt = I.n == b.logt_n ? b.logt : nullptr;
            CompareAcc acc;
            compare_acc_zero(acc);
            const int nc = __ldcg(&b.ncells[it]);
            for (int i = tid; i < nc; i += T) {
                const Cell cl = S.cells[i];
                if (!QM_CHK(cl.a, x.ka, 30) || !QM_CHK(cl.b, x.kb, 31)) continue;
                const long long n = cl.n, na = __ldcg(&S.size_a[cl.a]);
                const long long nb = __ldcg(&S.start[cl.b + 1]) - __ldcg(&S.start[cl.b]);
                acc.a11 += (unsigned long long)(n * (n - 1) / 2);
                atomicMax(&S.rowmax_n[cl.a], (unsigned)n);
                rowmax_ratio_update(&S.rowmax_r[cl.a], (unsigned long long)n, (unsigned long long)(na + nb));
                const double l1 = cell_log(n, na, nb);
                acc.vi += fp_from_double(vi_term_l(n, l1), SC_VI);
                const bool tab = logt && n <= LOGT_MAX;
                const double lr = tab ? __ldg(&logt[n]) : log_ratio(x.N, n);
                const double q = tab ? __ldg(&logt[LOGT_MAX + 1 + n]) : nmi_over(n, x.N);
                acc.hnum += fp_from_double(nmi_num_term_q(q, l1, lr), SC_H);
            }
            for (int c = tid; c < I.K; c += T) {
                const long long nb = __ldcg(&S.start[c + 1]) - __ldcg(&S.start[c]);
                if (nb == 0) continue;
                acc.sb += (unsigned long long)(nb * (nb - 1) / 2);
                acc.hden += fp_from_double(entropy_term(nb, x.N), SC_H);
                acc.kb += 1;
            }
            __threadfence();
            block_sync();  // this candidate's row maxima are complete
            for (int r = tid; r < x.ka; r += T) {
                rowmax_ratio_settle(&S.rowmax_r[r], __ldcg(&S.size_a[r]));
                compare_row(x, r, acc);
            }
            CompareTotals t;
            t.vi = group_sum_i128(acc.vi, T, red);
            t.hnum = group_sum_i128(acc.hnum, T, red);
            t.hden = group_sum_i128(acc.hden, T, red);
            t.f = group_sum_i128(acc.f, T, red);
            t.a11 = group_sum_u64(acc.a11, T, red);
            t.sa = group_sum_u64(acc.sa, T, red);
            t.sb = group_sum_u64(acc.sb, T, red);
            t.nvd = group_sum_u64(acc.nvd, T, red);
            t.ka = group_sum_u64(acc.ka, T, red);
            t.kb = group_sum_u64(acc.kb, T, red);
            if (tid == 0) {
                t.nvd += __ldcg(&b.gcell[2 * (size_t)it]);
                t.cells = __ldcg(&b.gcell[2 * (size_t)it + 1]);
                make_compare(t, x.N, I.out_c);
            }
        }
        block_sync();
    }
}

int batch_units_blocks_per_sm(const Shape &sh)
{
    int a = 0, c = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_bu_count<EpochTable32>, sh.threads, sh.smem_bytes);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_bu_cells, sh.threads, sh.smem_bytes);
    return std::max(1, std::min(a, c));
}

int launch_batch_units(const BatchItem *items_dev, int count, const BatchUnits &b, long long logt_n,
                       const Shape &sh, int num_sms, cudaStream_t s)
{
    BatchUnits bb = b;
    bb.logt_n = logt_n;
    BuArgs a;
    a.items = items_dev;
    a.count = count;
    a.b = bb;
    a.smem_bytes = sh.smem_bytes;
    a.plan = plan_smem(sh.threads, sh.smem_bytes);
    const int grid = num_sms * std::max(1, sh.blocks_per_sm);
    static const int expand_per_sm = [] {
        int e = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&e, k_bu_expand, EXPAND_THREADS, 0);
        return std::max(1, e);
    }();
    int L = 0;
    k_bu_hist<<<num_sms * 8, 256, 0, s>>>(items_dev, count, bb);
    k_bu_scan<<<std::min(count, num_sms * 4), BATCH_MAX_THREADS, 0, s>>>(items_dev, count, bb);
    k_bu_scatter<<<num_sms * 8, 256, 0, s>>>(items_dev, count, bb);
    k_bu_expand<<<num_sms * expand_per_sm, EXPAND_THREADS, 0, s>>>(items_dev, count, bb);
    L += 4;
    const bool k32 = bb.k_max < (1 << 24) - 1;
    for (int ph = 0; ph < 2; ++ph) {
        a.phase = ph;
        if (k32) k_bu_count<EpochTable32><<<grid, sh.threads, sh.smem_bytes, s>>>(a);
        else k_bu_count<EpochTable><<<grid, sh.threads, sh.smem_bytes, s>>>(a);
        ++L;
    }
    if (bb.cells) {
        // a found community's distinct truth labels are at most its members,
        // so the cells need smaller tables than the counts: more blocks per SM
        const int smem_c = std::min(sh.smem_bytes, BU_CELLS_SMEM);
        a.plan = plan_smem(sh.threads, smem_c);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bu_cells, sh.threads, smem_c);
        const int grid_c = num_sms * std::max(1, per_sm);
        for (int ph = 0; ph < 2; ++ph) {
            a.phase = ph;
            k_bu_cells<<<grid_c, sh.threads, smem_c, s>>>(a);
            ++L;
        }
    }
    k_bu_fin<<<std::min(count, num_sms * 8), BU_FIN_THREADS, 0, s>>>(items_dev, count, bb);
    ++L;
    return cudaGetLastError() == cudaSuccess ? L : -1;
}

void launch_batch_logt(double *logt, long long N, cudaStream_t s)
{
    k_bu_logt<<<(LOGT_MAX + 256) / 256, 256, 0, s>>>(logt, N);
}

void prepare_batched_kernel()
{
    cudaFuncSetAttribute(k_bu_count<EpochTable32>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    cudaFuncSetAttribute(k_bu_count<EpochTable>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    cudaFuncSetAttribute(k_bu_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    k_fill_log_int<<<(LOGT_MAX + 256) / 256, 256>>>();  // this unit's copy of the log table
    cudaDeviceSynchronize();
}

int batched_blocks_per_sm(const Shape &sh)
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched, sh.threads, sh.smem_bytes);
    return nb;
}

int launch_batched(const BatchItem *items_dev, int count, int *queue, const BatchScratch &bs,
                   const Shape &sh, int num_sms, cudaStream_t s, TraceFn tr)
{
    (void)num_sms;
    BatchKArgs a;
    a.items = items_dev;
    a.count = count;
    a.queue = queue;
    a.bs = bs;
    a.plan = plan_smem(sh.threads, sh.smem_bytes);
    a.big_thr = sh.big_community;
    if (tr) tr("k_batched", s);
    k_batched<<<bs.slots, sh.threads, sh.smem_bytes, s>>>(a);
    if (tr) tr(nullptr, s);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace qm

#ifdef QM_BOUNDS_CHECK
// Diagnostic build only: (site, index, bound, violations) of the first bad index.
extern "C" int qm_debug_read(unsigned long long *rec4)
{
    return (int)cudaMemcpyFromSymbol(rec4, qmk::qm_dbg_rec, sizeof(unsigned long long) * 8);
}
#endif
