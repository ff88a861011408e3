// qm_batched.cu -- one persistent launch that scores many partitions.
//
// Work items are (graph, partition[, ground truth]) triples.  A block takes the
// next item from a global queue and runs the whole pipeline of the plain path
// for it on its own: label histogram (in shared memory when the ids fit),
// prefix sum, counting sort of the nodes by label, the community-major pass of
// Sec. III-A (large communities by the whole block, the rest by single warps),
// the contingency cells and row maxima of Eqs. (1)-(7), and the final
// reduction.  No item needs another block, so there is no grid-wide barrier and
// no inter-block wait.  The per-term formulas, the fixed-point sums and the
// final arithmetic are the same device functions as in the plain path, so every
// result is bit-identical to scoring that partition alone.
#include "qm_internal.h"
#include "qm_community.cuh"
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

void prepare_batched_kernel()
{
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
