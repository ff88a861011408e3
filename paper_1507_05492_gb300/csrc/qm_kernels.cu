// qm_kernels.cu -- the plain (one partition per call) scoring path.
//
// Pipeline of qm_score_partition, all on one stream:
//   k_hist      |c| for every label id, with the label range check
//   k_scan_*    exclusive prefix of |c| -> member offsets; list of large communities
//   k_scatter   node ids grouped by community (a counting sort)
//   k_score_cm  community-major pass (Sec. III-A decomposition): large communities
//               by whole blocks, the rest by single warps
//   k_score_cm  again over the communities whose warp table overflowed
//   k_score_fin exact sums -> qm_quality
// qm_compare_partitions runs the same counting sort on the detected labels,
// hashes the ground-truth labels of each detected community's members into the
// contingency cells, then walks the ground-truth communities for the row maxima.
#include <atomic>
#include <climits>

#include "qm_internal.h"
#include "qm_community.cuh"
#include "qm_expand.cuh"
#include "qm_finalize.cuh"

namespace qm {
using namespace qmk;

enum { C_BIG_COUNT = 0, C_BIG_NEXT = 1, C_SMALL_NEXT = 2, C_OVF_COUNT = 3, C_OVF_NEXT = 4, C_SMALL_COUNT = 5,
       C_LONG_COUNT = 6, C_NCELLS = 7, C_MID_COUNT = 8, C_BX_COUNT = 9, C_BX_BAD = 10 };

constexpr int SCAN_TILE = 4096;   // elements per block in the multi-block scan
constexpr int SCAN_SINGLE_MAX = 1 << 16;

SmemPlan plan_smem(int T, int S)
{
    SmemPlan p;
    const int W = T / 32;
    int off = 0;
    p.red_off = off;
    off += 256 * 8;   // reduction exchange: 32 warps x 4 words, two 128-bit slots, a broadcast word
    p.ctl_off = off;
    off += ((2 * (W + 1) * 4 + 15) / 16) * 16;
    p.acc_off = off;    // one ScoreAcc / CompareAcc per warp
    off += W * 160;
    p.offs_off = off;
    off += (((T + W) * 4 + 15) / 16) * 16;
    p.rs_off = off;
    off += T * 8;
    const int rest = S - off;
    int cap = rest / 11;
    cap = (cap / W) * W;
    int mu = (cap * 3) / 4;
    mu = (mu / W) * W;
    p.slot_off = off;
    off += cap * 8;
    p.used_off = off;
    off += mu * 4;
    p.cap = cap;
    p.max_used = mu;
    p.cap_w = cap / W;
    p.max_used_w = mu / W;
    p.bytes = off;
    return p;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

CountPlan plan_count(int T, int S)
{
    CountPlan p;
    const int W = T / 32;
    int off = 0;
    p.red_off = off;
    off += 256 * 8;
    p.ctl_off = off;
    off += ((2 * (W + 1) * 4 + 15) / 16) * 16;
    p.bar_off = off;
    off += 16;
    p.stage_off = off;
    // 8 bytes per slot plus two staging buffers of the largest load (4 bytes an
    // entry, + 8 entries of slack)
    const int rest = S - off;
    int cap = (int)((long long)(rest - 2 * 4 * 12) * COUNT_FILL_DEN / (8 * COUNT_FILL_DEN + 8 * COUNT_FILL_NUM));
    cap = (cap / (4 * W)) * (4 * W);  // the warps' and groups' tables: multiples of 4 slots (EpochTable32V)
    p.cap = cap;
    p.fill = (int)count_fill(cap);
    p.stage_elems = (p.fill + 8 + 3) & ~3;
    off += 2 * p.stage_elems * 4;
    p.slot_off = off;
    off += cap * 8;
    p.cap_w = cap / W;
    p.fill_w = (int)count_fill(p.cap_w);
    // four groups of W/4 warps, each with a quarter of the table, take the
    // runs between a warp's and the block's reach
    p.ng = (W >= 8 && W % 4 == 0) ? 4 : 1;
    p.cap_g = cap / p.ng;
    p.fill_g = p.ng > 1 ? (int)count_fill(p.cap_g) : p.fill_w;
    p.bytes = off;
    return p;
}

static int scan_tiles(int K) { return (K + SCAN_TILE - 1) / SCAN_TILE; }

size_t score_ws_bytes(long long n, int K) { return carve_score_ws(reinterpret_cast<void *>(4096), n, K).bytes; }

ScoreWs carve_score_ws(void *base, long long n, int K)
{
    ScoreWs w{};
    char *p = (char *)base;
    w.status = (int *)p;
    w.counters = (int *)(p + 16);
    p += 256;
    w.gacc = (unsigned long long *)p;
    p += align_up(32 * 8, 256);
    w.result = (qm_quality *)p;
    p += align_up(sizeof(qm_quality), 256);
    w.size = (int *)p;
    p += align_up((size_t)K * 4, 256);
    w.zero_bytes = (size_t)(p - (char *)base);
    w.start = (int *)p;
    p += align_up(((size_t)K + 1) * 4, 256);
    w.recip = (Rcp *)p;
    p += align_up((size_t)K * 16, 256);
    w.cursor = (int *)p;
    p += align_up((size_t)K * 4, 256);
    w.big_list = (int *)p;
    p += align_up((size_t)K * 4, 256);
    w.ovf_list = (int *)p;
    p += align_up((size_t)K * 4, 256);
    w.members = (int *)p;
    p += align_up((size_t)n * 4, 256);
    w.scan_tmp = (int *)p;
    p += align_up((size_t)(scan_tiles(K) + 1) * 4, 256);
    w.bytes = (size_t)(p - (char *)base);
    return w;
}

size_t compare_ws_bytes(long long n, int ka, int kb)
{
    return carve_compare_ws(reinterpret_cast<void *>(4096), n, ka, kb).bytes;
}

CompareWs carve_compare_ws(void *base, long long n, int ka, int kb)
{
    CompareWs w{};
    char *p = (char *)base;
    w.status = (int *)p;
    w.counters = (int *)(p + 16);
    p += 256;
    w.gacc = (unsigned long long *)p;
    p += align_up(32 * 8, 256);
    w.result = (qm_compare *)p;
    p += align_up(sizeof(qm_compare), 256);
    w.size_a = (int *)p;
    p += align_up((size_t)ka * 4, 256);
    w.rowmax_n = (unsigned *)p;
    p += align_up((size_t)ka * 4, 256);
    w.size_b = (int *)p;
    p += align_up((size_t)kb * 4, 256);
    w.rowmax_r = (unsigned long long *)p;
    p += align_up((size_t)ka * 8, 256);
    w.zero_bytes = (size_t)(p - (char *)base);
    w.start = (int *)p;
    p += align_up(((size_t)kb + 1) * 4, 256);
    w.cursor = (int *)p;
    p += align_up((size_t)kb * 4, 256);
    w.big_list = (int *)p;
    p += align_up((size_t)kb * 4, 256);
    w.members = (int *)p;
    p += align_up((size_t)n * 4, 256);
    w.cells = (Cell *)p;  // at most one new cell per node
    p += align_up((size_t)n * sizeof(Cell), 256);
    w.scan_tmp = (int *)p;
    p += align_up((size_t)(scan_tiles(kb) + 1) * 4, 256);
    w.logt = (double *)p;
    p += align_up((size_t)LOGT_WORDS * 8, 256);
    w.bytes = (size_t)(p - (char *)base);
    return w;
}

// ------------------------------------------------------------------ histogram

// |c| for every label id (and the ground-truth sizes when `b` is given).
// Labels outside [0, K) set bit 0 of *status and are skipped.  When the ids fit,
// each block counts in shared memory first and adds its non-zero bins once.
// Community sizes of one or two labellings.  With few label ids the counts
// are privatised in shared memory; otherwise the lanes of a warp that share a
// label add their count with one global atomic.
__device__ __forceinline__ void hist_add_warp(int *size, int l, unsigned act)
{
    const unsigned peers = __match_any_sync(act, l);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&size[l], __popc(peers));
}

constexpr int HIST_UNROLL = 4;

__global__ void k_hist(const int *__restrict__ a, int ka, int *size_a, const int *__restrict__ b,
                       int kb, int *size_b, long long n, int *status, int use_smem)
{
    extern __shared__ int sh[];
    if (use_smem) {
        for (int i = threadIdx.x; i < ka + kb; i += blockDim.x) sh[i] = 0;
        block_sync();
    }
    bool bad = false;
    const int lane = threadIdx.x & 31;
    // each warp takes HIST_UNROLL * 32 consecutive labels a step, all loads
    // issued before the first count
    const long long wg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long step = ((long long)gridDim.x * blockDim.x >> 5) * (32 * HIST_UNROLL);
    for (long long i0 = wg * (32 * HIST_UNROLL); i0 < n; i0 += step) {
        int va[HIST_UNROLL], vb[HIST_UNROLL];
#pragma unroll
        for (int q = 0; q < HIST_UNROLL; ++q) {
            const long long i = i0 + q * 32 + lane;
            va[q] = i < n ? __ldcs(&a[i]) : 0;
            vb[q] = (b && i < n) ? __ldcs(&b[i]) : 0;
        }
#pragma unroll
        for (int q = 0; q < HIST_UNROLL; ++q) {
            const bool in = i0 + q * 32 + lane < n;
            const int la = va[q];
            const bool oka = in && (unsigned)la < (unsigned)ka;
            if (in && !oka) bad = true;
            if (use_smem) {
                if (oka) atomicAdd(&sh[la], 1);
            } else {
                const unsigned act = __ballot_sync(0xffffffffu, oka);
                if (oka) hist_add_warp(size_a, la, act);
            }
            if (b) {
                const int lb = vb[q];
                const bool okb = in && (unsigned)lb < (unsigned)kb;
                if (in && !okb) bad = true;
                if (use_smem) {
                    if (okb) atomicAdd(&sh[ka + lb], 1);
                } else {
                    const unsigned act = __ballot_sync(0xffffffffu, okb);
                    if (okb) hist_add_warp(size_b, lb, act);
                }
            }
        }
    }
    if (bad) atomicOr(status, 1);
    if (use_smem) {
        block_sync();
        for (int i = threadIdx.x; i < ka; i += blockDim.x)
            if (sh[i]) atomicAdd(&size_a[i], sh[i]);
        for (int i = threadIdx.x; i < kb; i += blockDim.x)
            if (sh[ka + i]) atomicAdd(&size_b[i], sh[ka + i]);
    }
}

// Labels of a graph stored renumbered (QM_REORDER) gathered into its order,
// out[j] = labels[inv[j]], with the community sizes of k_hist counted on the
// way (the histogram does not depend on the order; in the new order a warp's
// labels mostly agree, so the warp-aggregated atomics merge well).
__global__ void k_permute_hist(const int *__restrict__ labels, const int *__restrict__ inv, long long n,
                               int *__restrict__ out, int K, int *size, int *status, int use_smem)
{
    extern __shared__ int sh[];
    if (use_smem) {
        for (int i = threadIdx.x; i < K; i += blockDim.x) sh[i] = 0;
        block_sync();
    }
    bool bad = false;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); j0 < n; j0 += stride) {
        const long long j = j0 + lane;
        const bool in = j < n;
        const int l = in ? __ldg(&labels[__ldg(&inv[j])]) : 0;
        if (in) out[j] = l;
        const bool ok = in && (unsigned)l < (unsigned)K;
        if (in && !ok) bad = true;
        if (use_smem) {
            if (ok) atomicAdd(&sh[l], 1);
        } else {
            const unsigned act = __ballot_sync(0xffffffffu, ok);
            if (ok) hist_add_warp(size, l, act);
        }
    }
    if (bad) atomicOr(status, 1);
    if (use_smem) {
        block_sync();
        for (int i = threadIdx.x; i < K; i += blockDim.x)
            if (sh[i]) atomicAdd(&size[i], sh[i]);
    }
}


// ------------------------------------------------------------------ scan

// Exclusive prefix of size[0..K) by one block.  Writes start[0..K], optionally
// cursor = start, and appends ids with size > big_thr to big_list.
__global__ void k_scan_single(const int *size, int K, int *start, int *cursor, Rcp *recip,
                              int big_thr, int *big_list, int *counters, const int *status)
{
    __shared__ unsigned long long red[72];
    if (*status) return;
    const int T = blockDim.x;
    const long long per = ((long long)K + T - 1) / T;
    const long long b = (long long)threadIdx.x * per, e = min(b + per, (long long)K);
    unsigned sum = 0;
    for (long long i = b; i < e; ++i) sum += (unsigned)size[i];
    unsigned excl;
    const unsigned total = group_exclusive_scan(sum, excl, T, red);
    unsigned run = excl;
    for (long long i = b; i < e; ++i) {
        const int s = size[i];
        start[i] = (int)run;
        if (cursor) cursor[i] = (int)run;
        if (recip && s > 0) recip[i] = rcp_of(s);
        if (s > big_thr) big_list[atomicAdd(&counters[C_BIG_COUNT], 1)] = (int)i;
        run += (unsigned)s;
    }
    if (threadIdx.x == 0) start[K] = (int)total;
}

__global__ void k_scan_tiles(const int *size, int K, int *tile_sum, const int *status)
{
    __shared__ unsigned long long red[72];
    if (*status) return;
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    unsigned s = 0;
    for (int j = threadIdx.x; j < SCAN_TILE; j += blockDim.x) {
        const long long i = base + j;
        if (i < K) s += (unsigned)size[i];
    }
    s = (unsigned)group_sum_u64(s, blockDim.x, red);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = (int)s;
}

__global__ void k_scan_apply(const int *size, int K, const int *tile_off, int *start, int *cursor,
                             Rcp *recip, int big_thr, int *big_list, int *counters,
                             const int *status)
{
    __shared__ unsigned long long red[72];
    if (*status) return;
    const int per = SCAN_TILE / blockDim.x;
    const long long b = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * per;
    unsigned sum = 0;
    for (int j = 0; j < per; ++j)
        if (b + j < K) sum += (unsigned)size[b + j];
    unsigned excl;
    group_exclusive_scan(sum, excl, blockDim.x, red);
    unsigned run = (unsigned)tile_off[blockIdx.x] + excl;
    for (int j = 0; j < per; ++j) {
        const long long i = b + j;
        if (i >= K) break;
        const int s = size[i];
        start[i] = (int)run;
        if (cursor) cursor[i] = (int)run;
        if (recip && s > 0) recip[i] = rcp_of(s);
        if (s > big_thr) big_list[atomicAdd(&counters[C_BIG_COUNT], 1)] = (int)i;
        run += (unsigned)s;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) start[K] = tile_off[gridDim.x];
}

// ------------------------------------------------------------------ scatter

// Counting sort of the nodes by label: members[pos] receives the node id, or
// vals[node] when vals is given (the comparison places each node's truth
// label straight into its detected community's run, read in node order).
// (When vals are given and kv > 0, a value outside [0, kv) sets bit 0 of
// *status, as a label outside its range does in k_hist.)
__global__ void k_scatter(const int *__restrict__ labels, const int *__restrict__ vals, long long n, int *cursor,
                          int *members, int *status, int kv)
{
    if (*status) return;
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int l = __ldg(&labels[i]);
        const int pos = atomicAdd(&cursor[l], 1);
        const int v = vals ? __ldcs(&vals[i]) : (int)i;
        if (vals && kv > 0 && (unsigned)v >= (unsigned)kv) bad = true;
        members[pos] = v;
    }
    if (bad) atomicOr(status, 1);
}

// ------------------------------------------------------------------ community pass

struct ScoreKArgs {
    ScoreCtx x;
    const int *big_list;
    const int *ovf_in;
    int *ovf_out;
    int *counters;
    unsigned long long *gacc;
    const int *status;
    int big_thr;
    int phase;   // 0: large communities then warps over all ids; 1: overflow list
    SmemPlan plan;
};

// Adds the block's per-warp accumulators to the partition's global sums
// (called by thread 0 after a barrier).
__device__ __forceinline__ void flush_score(const ScoreAcc *sacc, int W, unsigned long long *g)
{
    ScoreAcc t = sacc[0];
    for (int w = 1; w < W; ++w) score_acc_add(t, sacc[w]);
    limbs_add(g + GS_QDS_SELF, t.qds_self);
    limbs_add(g + GS_QDS_PAIR, t.qds_pair);
    limbs_add(g + GS_DENS, t.dens);
    limbs_add(g + GS_CONTR, t.contr);
    limbs_add(g + GS_EXPN, t.expn);
    limbs_add(g + GS_COND, t.cond);
    limbs_add(g + GS_VOL2, (i128)t.vol2);
    if (t.ein) atomicAdd(g + GS_EIN, t.ein);
    if (t.eout) atomicAdd(g + GS_EOUT, t.eout);
    if (t.nonempty) atomicAdd(g + GS_NONEMPTY, t.nonempty);
    if (t.slots) atomicAdd(g + GS_SLOTS, t.slots);
    if (t.cnt2) atomicAdd(g + GS_CNT2, t.cnt2);
}

__global__ void __launch_bounds__(1024) k_score_cm(ScoreKArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_item;
    if (*a.status) return;
    const SmemPlan &p = a.plan;
    unsigned long long *red = (unsigned long long *)(sm + p.red_off);
    int *ctl = (int *)(sm + p.ctl_off);
    unsigned *offs = (unsigned *)(sm + p.offs_off);
    long long *rs = (long long *)(sm + p.rs_off);
    unsigned long long *slot = (unsigned long long *)(sm + p.slot_off);
    int *used = (int *)(sm + p.used_off);
    const int T = blockDim.x, W = T >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    ScoreAcc *sacc = (ScoreAcc *)(sm + p.acc_off);
    for (int i = threadIdx.x; i < p.cap; i += T) slot[i] = 0ull;
    for (int i = threadIdx.x; i < 2 * (W + 1); i += T) ctl[i] = 0;
    for (int i = threadIdx.x; i < W; i += T) score_acc_zero(sacc[i]);
    block_sync();

    const SmemTable tb{slot, used, &ctl[0], &ctl[1], p.cap, p.max_used};
    const int *list = a.phase == 0 ? a.big_list : a.ovf_in;
    int *next = &a.counters[a.phase == 0 ? C_BIG_NEXT : C_OVF_NEXT];
    const int count = a.counters[a.phase == 0 ? C_BIG_COUNT : C_OVF_COUNT];
    for (;;) {
        if (threadIdx.x == 0) {
            const int i = atomicAdd(next, 1);
            s_item = i < count ? list[i] : -1;
        }
        block_sync();
        const int c = s_item;
        block_sync();
        if (c < 0) break;
        score_community(a.x, c, tb, offs, rs, &sacc[0], threadIdx.x, T, red);
    }
    if (a.phase == 0) {
        const SmemTable tw{slot + wid * p.cap_w, used + wid * p.max_used_w, &ctl[2 + 2 * wid],
                           &ctl[3 + 2 * wid], p.cap_w, p.max_used_w};
        const int chunk = claim_chunk(a.x.K, (long long)gridDim.x * W);
        for (;;) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&a.counters[C_SMALL_NEXT], chunk);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= a.x.K) break;
            const int c = base + lane;
            int sz = 0;
            if (lane < chunk && c < a.x.K) sz = a.x.start[c + 1] - a.x.start[c];
            unsigned mask = __ballot_sync(0xffffffffu, sz > 0 && sz <= a.big_thr);
            while (mask) {
                const int j = __ffs(mask) - 1;
                mask &= mask - 1;
                if (!score_community(a.x, base + j, tw, offs, rs, &sacc[wid], lane, 32, red)) {
                    if (lane == 0) a.ovf_out[atomicAdd(&a.counters[C_OVF_COUNT], 1)] = base + j;
                }
            }
        }
    }
    block_sync();
    if (threadIdx.x == 0) flush_score(sacc, W, a.gacc);
}

__global__ void k_score_fin(const unsigned long long *g, const int *status, long long n, long long E,
                            qm_quality *out, int weighted)
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
    make_quality(t, n, E, out);
    if (weighted) out->modularity = fp_to_double(limbs_get(g + GS_QW), SC_QDS);
}

// ------------------------------------------------------------------ compare

struct CompareKArgs {
    CompareCtx x;
    const int *big_list;
    int *counters;
    Cell *cells;
    unsigned long long *gacc;
    const int *status;
    SmemPlan plan;
};

__device__ __forceinline__ void flush_compare(const CompareAcc &acc, unsigned long long *g,
                                              unsigned long long *red)
{
    const int T = blockDim.x;
    i128 v;
    v = group_sum_i128(acc.vi, T, red);
    if (threadIdx.x == 0) limbs_add(g + GC_VI, v);
    v = group_sum_i128(acc.hnum, T, red);
    if (threadIdx.x == 0) limbs_add(g + GC_HNUM, v);
    v = group_sum_i128(acc.hden, T, red);
    if (threadIdx.x == 0) limbs_add(g + GC_HDEN, v);
    v = group_sum_i128(acc.f, T, red);
    if (threadIdx.x == 0) limbs_add(g + GC_F, v);
    const unsigned long long *src[7] = {&acc.a11, &acc.sa, &acc.sb, &acc.nvd, &acc.cells, &acc.ka, &acc.kb};
    const int dst[7] = {GC_A11, GC_SA, GC_SB, GC_NVD, GC_CELLS, GC_KA, GC_KB};
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const unsigned long long u = group_sum_u64(*src[k], T, red);
        if (threadIdx.x == 0 && u) atomicAdd(g + dst[k], u);
    }
}

__device__ __forceinline__ void flush_compare_one(const CompareAcc &t, unsigned long long *g)
{
    limbs_add(g + GC_VI, t.vi);
    limbs_add(g + GC_HNUM, t.hnum);
    limbs_add(g + GC_HDEN, t.hden);
    limbs_add(g + GC_F, t.f);
    if (t.a11) atomicAdd(g + GC_A11, t.a11);
    if (t.sa) atomicAdd(g + GC_SA, t.sa);
    if (t.sb) atomicAdd(g + GC_SB, t.sb);
    if (t.nvd) atomicAdd(g + GC_NVD, t.nvd);
    if (t.cells) atomicAdd(g + GC_CELLS, t.cells);
    if (t.ka) atomicAdd(g + GC_KA, t.ka);
    if (t.kb) atomicAdd(g + GC_KB, t.kb);
}

__global__ void __launch_bounds__(1024) k_compare_cm(CompareKArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_item;
    if (*a.status) return;
    const SmemPlan &p = a.plan;
    unsigned long long *red = (unsigned long long *)(sm + p.red_off);
    int *ctl = (int *)(sm + p.ctl_off);
    unsigned long long *slot = (unsigned long long *)(sm + p.slot_off);
    int *used = (int *)(sm + p.used_off);
    const int T = blockDim.x, W = T >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    CompareAcc *cacc = (CompareAcc *)(sm + p.acc_off);
    for (int i = threadIdx.x; i < p.cap; i += T) slot[i] = 0ull;
    for (int i = threadIdx.x; i < 2 * (W + 1); i += T) ctl[i] = 0;
    for (int i = threadIdx.x; i < W; i += T) compare_acc_zero(cacc[i]);
    block_sync();
    const SmemTable tb{slot, used, &ctl[0], &ctl[1], p.cap, p.max_used};
    const int count = a.counters[C_BIG_COUNT];
    for (;;) {
        if (threadIdx.x == 0) {
            const int i = atomicAdd(&a.counters[C_BIG_NEXT], 1);
            s_item = i < count ? a.big_list[i] : -1;
        }
        block_sync();
        const int b = s_item;
        block_sync();
        if (b < 0) break;
        compare_cells_community(a.x, b, tb, &cacc[0], threadIdx.x, T, red, a.cells, &a.counters[C_NCELLS]);
    }
    const SmemTable tw{slot + wid * p.cap_w, used + wid * p.max_used_w, &ctl[2 + 2 * wid],
                       &ctl[3 + 2 * wid], p.cap_w, p.max_used_w};
    const int chunk = claim_chunk(a.x.kb, (long long)gridDim.x * W);
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&a.counters[C_SMALL_NEXT], chunk);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= a.x.kb) break;
        const int b = base + lane;
        int sz = 0;
        if (lane < chunk && b < a.x.kb) sz = a.x.start[b + 1] - a.x.start[b];
        unsigned mask = __ballot_sync(0xffffffffu, sz > 0 && sz <= p.max_used_w);
        while (mask) {
            const int j = __ffs(mask) - 1;
            mask &= mask - 1;
            compare_cells_community(a.x, base + j, tw, &cacc[wid], lane, 32, red, a.cells,
                                    &a.counters[C_NCELLS]);
        }
    }
    block_sync();
    if (threadIdx.x == 0) {
        CompareAcc t = cacc[0];
        for (int w = 1; w < W; ++w) compare_acc_add(t, cacc[w]);
        flush_compare_one(t, a.gacc);
    }
}

__global__ void k_compare_rows(CompareCtx x, unsigned long long *g, const int *status)
{
    __shared__ unsigned long long red[72];
    if (*status) return;
    CompareAcc acc;
    compare_acc_zero(acc);
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < x.ka; a += gridDim.x * blockDim.x) {
        rowmax_ratio_settle(&x.rowmax_r[a], __ldcg(&x.size_a[a]));
        compare_row(x, a, acc);
    }
    flush_compare(acc, g, red);
}

// Terms of every contingency cell (Eqs. 1-4), in parallel over the cell list:
// the pair count, the VI and NMI-numerator terms, and the row maxima of the
// F-measure and NVD (Eqs. 3-4) per truth community (NVD's by atomicMax, F's as
// an exact fraction that k_compare_rows turns into its ratio).
__global__ void k_compare_cells(CompareCtx x, const Cell *cells, const int *counters, const int *size_b,
                                unsigned long long *g, const int *status)
{
    __shared__ unsigned long long red[72];
    if (*status) return;
    CompareAcc acc;
    compare_acc_zero(acc);
    const int nc = counters[C_NCELLS];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
        const Cell c = cells[i];
        if (!QM_CHK(c.a, x.ka, 30) || !QM_CHK(c.b, x.kb, 31)) continue;
        const long long n = c.n, na = __ldg(&x.size_a[c.a]), nb = __ldg(&size_b[c.b]);
        acc.a11 += (unsigned long long)(n * (n - 1) / 2);
        atomicMax(&x.rowmax_n[c.a], (unsigned)n);
        rowmax_ratio_update(&x.rowmax_r[c.a], (unsigned long long)n, (unsigned long long)(na + nb));
        const double l1 = cell_log(n, na, nb);
        acc.vi += fp_from_double(vi_term_l(n, l1), SC_VI);
        const bool tab = n <= LOGT_MAX;
        acc.hnum += fp_from_double(nmi_num_term_q(tab ? __ldg(&x.logt[LOGT_MAX + 1 + n]) : nmi_over(n, x.N), l1,
                                                  tab ? __ldg(&x.logt[n]) : log_ratio(x.N, n)),
                                   SC_H);
    }
    flush_compare(acc, g, red);
}

// log(N / n) and n / N for n = 1 .. LOGT_MAX (contingency cells and community
// sizes are mostly small, so k_compare_cells then takes one logarithm and no
// division per cell at most).
__global__ void k_log_table(double *logt, long long N)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= LOGT_MAX; i += gridDim.x * blockDim.x) {
        logt[i] = i == 0 ? 0.0 : log_ratio(N, i);
        logt[LOGT_MAX + 1 + i] = nmi_over(i, N);
    }
}

// Column side of every found community b: C(|b|, 2), its entropy term, the count.
__global__ void k_compare_cols(const int *size_b, int kb, long long N, unsigned long long *g, const int *status)
{
    __shared__ unsigned long long red[72];
    if (*status) return;
    CompareAcc acc;
    compare_acc_zero(acc);
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < kb; b += gridDim.x * blockDim.x) {
        const long long nb = size_b[b];
        if (nb == 0) continue;
        acc.sb += (unsigned long long)(nb * (nb - 1) / 2);
        acc.hden += fp_from_double(entropy_term(nb, N), SC_H);
        acc.kb += 1;
    }
    flush_compare(acc, g, red);
}

__global__ void k_compare_fin(const unsigned long long *g, const int *status, long long n, qm_compare *out)
{
    if (threadIdx.x != 0 || *status) return;
    CompareTotals t;
    t.vi = limbs_get(g + GC_VI);
    t.hnum = limbs_get(g + GC_HNUM);
    t.hden = limbs_get(g + GC_HDEN);
    t.f = limbs_get(g + GC_F);
    t.a11 = g[GC_A11];
    t.sa = g[GC_SA];
    t.sb = g[GC_SB];
    t.nvd = g[GC_NVD];
    t.cells = g[GC_CELLS];
    t.ka = g[GC_KA];
    t.kb = g[GC_KB];
    make_compare(t, n, out);
}

// ------------------------------------------------------------------ graph validation

// Always: row offsets non-decreasing from 0 to n_arcs, column ids in [0, n),
// maximum degree.  With `full`: rows strictly increasing (no repeated arcs), no
// self-loops, and the reverse arc (v, u) present (binary search in the sorted
// row of v).
__global__ void k_validate(const long long *row_ptr, const int *col, long long n, long long n_arcs,
                           int full, int *status, unsigned long long *max_deg)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    bool bad = false;
    unsigned long long md = 0;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const long long b = row_ptr[u], e = row_ptr[u + 1];
        if (u == 0 && b != 0) bad = true;
        if (u == n - 1 && e != n_arcs) bad = true;
        if (e < b || b < 0 || e > n_arcs) { bad = true; continue; }
        md = max(md, (unsigned long long)(e - b));
        for (long long k = b; k < e; ++k) {
            const int v = col[k];
            if (v < 0 || v >= n) { bad = true; break; }
            if (!full) continue;
            if (v == u || (k > b && col[k - 1] >= v)) { bad = true; break; }
            long long lo = row_ptr[v], hi = row_ptr[v + 1];
            if (lo < 0 || hi > n_arcs || hi < lo) { bad = true; break; }
            bool found = false;
            while (lo < hi) {
                const long long mid = (lo + hi) >> 1;
                const int w = col[mid];
                if (w == (int)u) { found = true; break; }
                if (w < (int)u) lo = mid + 1; else hi = mid;
            }
            if (!found) { bad = true; break; }
        }
    }
    if (bad) atomicOr(status, 1);
    for (int d = 16; d > 0; d >>= 1) md = max(md, __shfl_down_sync(0xffffffffu, md, d));
    if ((threadIdx.x & 31) == 0) atomicMax(max_deg, md);
}

// ------------------------------------------------------------------ launchers

// Grid of a community-major kernel: one block per SM and resident slot, but
// no more blocks than there are communities (any of which may need a whole
// block), so that a small graph does not start blocks that find no work.
struct Shape;
static int community_grid(long long K, int num_sms, const Shape &sh);

static int grid_for(long long n, int threads, int num_sms, int per_sm)
{
    long long g = (n + threads - 1) / threads;
    const long long cap = (long long)num_sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// ------------------------------------------------------------------ two-phase scoring

// Counting sort of the nodes by label (as k_scatter) that also records the
// degree of the node placed at each member position (read in node order, so
// the row-offset reads are coalesced).  The lanes of a warp that hold one label
// take their places with a single atomic, in node order: on a graph whose nodes
// are numbered cluster by cluster (QM_REORDER) consecutive member positions
// are then mostly consecutive nodes, whose rows are adjacent (see k_expand).
__global__ void k_scatter_deg(const int *__restrict__ labels, const long long *__restrict__ row_ptr, long long n,
                              int *cursor, int *members, int *degm, const int *status)
{
    if (*status) return;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < n; i0 += stride) {
        const long long i = i0 + lane;
        const unsigned act = __ballot_sync(0xffffffffu, i < n);
        if (i >= n) continue;
        const int l = __ldg(&labels[i]);
        const unsigned peers = __match_any_sync(act, l);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&cursor[l], __popc(peers));
        base = __shfl_sync(peers, base, leader);
        const int pos = base + __popc(peers & ((1u << lane) - 1u));
        members[pos] = (int)i;
        degm[pos] = (int)(__ldg(&row_ptr[i + 1]) - __ldg(&row_ptr[i]));
    }
}

// The packed label copy read by the far-end gathers (PACK_BITS-bit ids, three
// to a word; see qm_expand.cuh).  After k_pack_blocks (bx_bad set) only when
// the block encoding did not fit.
__global__ void k_pack3(const int *__restrict__ labels, long long n, unsigned long long *__restrict__ plab,
                        const int *status, const int *bx_bad)
{
    if (*status || (bx_bad && !*bx_bad)) return;
    const long long words = (n + 2) / 3;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < words;
         t += (long long)gridDim.x * blockDim.x) {
        const long long i = 3 * t;
        unsigned long long w = (unsigned long long)(__ldcs(&labels[i]) & 0x1FFFFF);
        if (i + 1 < n) w |= (unsigned long long)(__ldcs(&labels[i + 1]) & 0x1FFFFF) << PACK_BITS;
        if (i + 2 < n) w |= (unsigned long long)(__ldcs(&labels[i + 2]) & 0x1FFFFF) << (2 * PACK_BITS);
        plab[t] = w;
    }
}

// The block encoding of the labels (ld_label_blk in qm_expand.cuh) in the
// buffer of the packed copy, which is larger: a half-warp per block of 16
// nodes, each warp taking PACKB_UNROLL pairs of blocks a step with all their
// loads issued first.  Blocks of three or more labels take exception slots
// (one atomic per warp and block pair; the order is whatever the atomics give)
// while fewer than xcap are taken; a warp that finds them gone sets *bad and
// stops (as does every later one that needs a slot), and the packed copy
// replaces the encoding.
constexpr int PACKB_UNROLL = 4;

__global__ void k_pack_blocks(const int *__restrict__ labels, long long n, unsigned long long *__restrict__ blab,
                              long long xcap, int *xcount, int *bad, const int *status)
{
    if (*status) return;
    const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const unsigned hmask = 0xFFFFu << (16 * half);
    const long long nb = (n + BLK_NODES - 1) / BLK_NODES;
    const unsigned xbase = (unsigned)(2 * nb);  // first word of the exception area
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (long long b0 = wg * 2 * PACKB_UNROLL; b0 < nb; b0 += 2 * PACKB_UNROLL * nwarps) {
        int lv[PACKB_UNROLL];
#pragma unroll
        for (int q = 0; q < PACKB_UNROLL; ++q) {
            const long long i = (b0 + 2 * q + half) * BLK_NODES + hl;
            lv[q] = i < n ? __ldcs(&labels[i]) : 0;
        }
#pragma unroll
        for (int q = 0; q < PACKB_UNROLL; ++q) {
            const long long b = b0 + 2 * q + half;
            const bool inb = b < nb, real = inb && b * BLK_NODES + hl < n;
            int l = lv[q];
            const int A = __shfl_sync(0xffffffffu, l, 16 * half);
            if (!real) l = A;  // nodes past the end take the block's first label
            const unsigned notA = __ballot_sync(0xffffffffu, l != A) & hmask;
            const int B = __shfl_sync(0xffffffffu, l, notA ? __ffs(notA) - 1 : 16 * half);
            const bool exc = (__ballot_sync(0xffffffffu, l != A && l != B) & hmask) != 0;
            const unsigned isB = (__ballot_sync(0xffffffffu, l == B && B != A) & hmask) >> (16 * half);
            const unsigned need = __ballot_sync(0xffffffffu, hl == 0 && inb && exc);
            int x0 = 0;
            if (lane == 0 && need) x0 = atomicAdd(xcount, __popc(need));
            x0 = __shfl_sync(0xffffffffu, x0, 0);
            if (need && x0 >= xcap) {  // the slots ran out (here or in another warp): give up the encoding
                if (lane == 0) atomicExch(bad, 1);
                return;
            }
            const int x = x0 + __popc(need & ((1u << (16 * half)) - 1u));
            unsigned long long word;
            if (!exc) {
                word = (unsigned long long)(A & 0x1FFFFF) | ((unsigned long long)(B & 0x1FFFFF) << PACK_BITS) |
                       ((unsigned long long)isB << 42);
            } else {
                if (x < xcap) {
                    if (inb) ((int *)blab)[xbase + (unsigned)x * BLK_NODES + hl] = l;
                } else if (hl == 0 && inb) {
                    atomicExch(bad, 1);
                }
                word = (1ull << 63) | (unsigned long long)(xbase + (unsigned)min((long long)x, xcap) * BLK_NODES);
            }
            if (inb && hl == 0) blab[b] = word;
        }
    }
}

// Exception slots of the block encoding: a sixteenth of the blocks, and what
// the packed copy's buffer leaves after the block words.
static long long blocks_xcap(long long n)
{
    const long long nb = (n + BLK_NODES - 1) / BLK_NODES, words = (n + 2) / 3;
    return std::max(0LL, std::min(nb / 16, (2 * words - 2 * nb) / BLK_NODES));
}

// Phase A (the far-end label gathers) lives in qm_expand.cuh: expand_chunk is one
// warp's share of it.  LAB is the label source of the gathers; with bx_bad (the
// block encoding was tried) the LAB_BLOCKS launch runs when it fits and the
// LAB_PACK3 launch when it does not.  Register budgets: 40 for the block
// encoding (six resident blocks; its gathers hit L2 and wait on latency), 48
// for the others (64 with weights).

template <bool WT, int LAB, bool HI>
__global__ void __launch_bounds__(EXPAND_THREADS, LAB == LAB_BLOCKS ? 6 : WT ? 4 : 5) k_expand(const long long *__restrict__ row_ptr,
                                                           const int *__restrict__ col,
                                                           const int *__restrict__ labels,
                                                           const unsigned long long *__restrict__ plab,
                                                           const int *__restrict__ members,
                                                           const unsigned *__restrict__ aoff,
                                                           const int *__restrict__ start, long long n,
                                                           int *inter, int *inter_hi, int *__restrict__ nbr,
                                                           const int *status,
                                                           Shard own, const float *__restrict__ wt,
                                                           float *__restrict__ nbrw, unsigned long long *wl,
                                                           const int *bx_bad = nullptr)
{
    __shared__ unsigned offs_s[EXPAND_THREADS / 32][33];
    __shared__ long long rs_s[EXPAND_THREADS / 32][32];
    __shared__ int cw_s[EXPAND_THREADS / 32][32];
    if (*status) return;
    if (bx_bad && (LAB == LAB_BLOCKS) == (*bx_bad != 0)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned long long keep = l2_policy_evict_last();
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long p0 = ((long long)blockIdx.x * (blockDim.x >> 5) + w) * 32; p0 < n; p0 += nwarps * 32)
        expand_chunk<WT, LAB, HI>(p0, n, row_ptr, col, labels, plab, members, aoff, start, inter, inter_hi, nbr,
                                   own, wt, nbrw, wl, offs_s[w], rs_s[w], cw_s[w], keep, lane);
}

// Half-edge phase A (ALGO_HALF): as k_expand over the upper rows; same2 (the
// `inter` array) receives 2|E_c^in| and cursor (`inter_hi`) the run lengths.
template <bool PACK, bool FULL>
__global__ void __launch_bounds__(EXPAND_THREADS) k_expand_half(const long long *__restrict__ up_ptr,
                                                                const int *__restrict__ up_col,
                                                                const int *__restrict__ labels,
                                                                const unsigned long long *__restrict__ plab,
                                                                const int *__restrict__ members,
                                                                const unsigned *__restrict__ cbase, long long n,
                                                                int *same2, int *cursor, int *__restrict__ nbr,
                                                                const int *status)
{
    __shared__ unsigned offs_s[EXPAND_THREADS / 32][33];
    __shared__ long long rs_s[EXPAND_THREADS / 32][32];
    __shared__ int cw_s[EXPAND_THREADS / 32][32];
    if (*status) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned long long keep = l2_policy_evict_last();
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long p0 = ((long long)blockIdx.x * (blockDim.x >> 5) + w) * 32; p0 < n; p0 += nwarps * 32)
        expand_chunk_half<PACK, FULL>(p0, n, up_ptr, up_col, labels, plab, members, cbase, same2, cursor, nbr,
                                      offs_s[w], rs_s[w], cw_s[w], keep, lane);
}

// Each community's segment base, cbase[c] = aoff[start[c]] (for the appends
// of the half-edge phase A into other communities' runs).
__global__ void k_cbase(const int *start, const unsigned *aoff, int K, unsigned *cbase, const int *status)
{
    if (*status) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < K; c += gridDim.x * blockDim.x)
        cbase[c] = aoff[start[c]];
}

#include "qm_binned.cuh"

// One header per non-empty community, sorted into four lists by run length
// m (the community's packed entries, an upper bound on the distinct keys its
// count will see): m <= warp_fill for single warps, up to group_fill for groups
// of warps, up to block_fill for whole blocks of k_count, longer runs for
// k_count_long.  Appends are warp-aggregated.  After the half-edge phase A,
// cut_from_intra (the `inter` array) turns from 2|E_c^in| into the cut arcs.
__global__ void k_classify(const int *start, const unsigned *aoff, const int *mlen, int K, int warp_fill,
                           int group_fill, int block_fill, RunHdr *big, RunHdr *small, RunHdr *lng, RunHdr *mid,
                           int *counters, const int *status, Shard own, int *cut_from_intra)
{
    if (*status) return;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (long long c0 = (long long)blockIdx.x * blockDim.x; c0 < K; c0 += (long long)gridDim.x * blockDim.x) {
        const long long cl = c0 + threadIdx.x;
        int cls = -1;
        RunHdr h{-1, 0u, 0u, 0u};
        if (cl < K) {
            const int c = (int)cl;
            const int s0 = start[c], s1 = start[c + 1];
            if (s1 > s0 && own.owns(c)) {
                const unsigned a0 = aoff[s0];
                h = RunHdr{c, a0, (unsigned)mlen[c], aoff[s1] - a0};
                // half-edge phase A left 2|E_c^in| there: the cut arcs are the rest of the volume
                if (cut_from_intra) cut_from_intra[c] = (int)(h.vol - (unsigned)cut_from_intra[c]);
                cls = h.m > (unsigned)block_fill ? 2
                      : h.m > (unsigned)group_fill ? 0
                      : h.m > (unsigned)warp_fill ? 3 : 1;
            }
        }
        const int ctr[4] = {C_BIG_COUNT, C_SMALL_COUNT, C_LONG_COUNT, C_MID_COUNT};
        RunHdr *const lists[4] = {big, small, lng, mid};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned mask = __ballot_sync(0xffffffffu, cls == k);
            if (!mask) continue;
            const int leader = __ffs(mask) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(&counters[ctr[k]], __popc(mask));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (cls == k) lists[k][base + __popc(mask & lt)] = h;
        }
    }
}

struct CountKArgs {
    CountCtx x;
    const RunHdr *big;
    const RunHdr *small;
    const RunHdr *mid;
    int *counters;
    const int *status;
    CountPlan plan;
    unsigned stage_wait;  // polls of each pipelined staging wait before the block gives up
};

constexpr unsigned STAGE_WAIT_LIMIT = 1u << 22;

// Poll limit of the pipelined staging wait of k_count for later launches
// (qm_debug_set_stage_wait).  The wait that drains a block's copies after an
// expiry always keeps STAGE_WAIT_LIMIT.
static std::atomic<unsigned> g_stage_wait{STAGE_WAIT_LIMIT};

void set_stage_wait_polls(long long polls)
{
    g_stage_wait.store(polls < 0 ? STAGE_WAIT_LIMIT : (unsigned)std::min(polls, (long long)INT_MAX));
}

// Phase B.  Runs longer than a warp table takes go to whole blocks in a static
// round-robin; while a block counts one run, the next run is already on its
// way into shared memory (a TMA bulk copy into the other of two staging
// buffers, completing on an mbarrier) and the header after that is being
// loaded.  Short runs then go to single warps, claim_chunk headers at a time.  Each
// group has its own epoch-tagged table (see count_run).  Runs longer than the
// staging buffers go to k_count_long.
template <class TAB, bool FULL>
__global__ void __launch_bounds__(1024) k_count(CountKArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ RunHdr ring[3];
    __shared__ int s_timeout;
    if (*a.status) return;
    const CountPlan &p = a.plan;
    unsigned long long *red = (unsigned long long *)(sm + p.red_off);
    int *ctl = (int *)(sm + p.ctl_off);
    unsigned long long *bars = (unsigned long long *)(sm + p.bar_off);
    int *stage = (int *)(sm + p.stage_off);
    unsigned long long *slot = (unsigned long long *)(sm + p.slot_off);
    const int T = blockDim.x, tid = threadIdx.x, wid = tid >> 5, lane = tid & 31, W = T >> 5;
    for (int i = tid; i < p.cap; i += T) slot[i] = 0ull;
    for (int i = tid; i < 2 * (W + 1); i += T) ctl[i] = 0;
    const int nbig = a.counters[C_BIG_COUNT];
    const long long G = gridDim.x, b = blockIdx.x;
    const RunHdr none{-1, 0u, 0u, 0u};
    // thread 0's bookkeeping of the staging buffers: copies issued and
    // consumed per buffer, packed as issued0 | issued1 << 16 ... (wrapping
    // 16-bit counters; only their difference and low bit are used)
    unsigned issued = 0u, used = 0u;
    auto cnt_of = [](unsigned v, int k) { return (v >> (16 * k)) & 0xFFFFu; };
    auto issue = [&](const RunHdr &h, int k) {
        const unsigned lo = h.a0 & ~3u;
        const unsigned bytes = ((h.a0 - lo) + h.m + 3u) / 4u * 16u;
        bulk_load_smem(stage + k * p.stage_elems, a.x.nbr + lo, bytes, &bars[k]);
        issued = (issued & ~(0xFFFFu << (16 * k))) | (((cnt_of(issued, k) + 1u) & 0xFFFFu) << (16 * k));
    };
    auto consume = [&](int k) {
        used = (used & ~(0xFFFFu << (16 * k))) | (((cnt_of(used, k) + 1u) & 0xFFFFu) << (16 * k));
    };
    if (tid == 0) {
        s_timeout = 0;
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_proxy_async_smem();
        ring[0] = b < nbig ? a.big[b] : none;
        ring[1] = b + G < nbig ? a.big[b + G] : none;
        if (ring[0].c >= 0) issue(ring[0], 0);
    }
    block_sync();
    const TAB eb = make_table<TAB>(slot, p.cap, &ctl[1]);
    unsigned epoch = 0;
    bool aborted = false;
    for (int it = 0;; ++it) {
        const RunHdr h = ring[it % 3];
        if (h.c < 0) break;
        const int k = it & 1;
        RunHdr nn = none;
        if (tid == 0) {
            // wait for this run's copy first and issue the next one only then, so
            // that at most one copy is in flight whenever a wait can expire
            if (mbar_wait(&bars[k], cnt_of(used, k) & 1u, a.stage_wait)) {
                consume(k);
                const RunHdr hn = ring[(it + 1) % 3];
                if (hn.c >= 0) {
                    fence_proxy_async_smem();
                    issue(hn, k ^ 1);
                }
                const long long idx = b + (long long)(it + 2) * G;
                if (idx < nbig) nn = a.big[idx];
            } else {
                s_timeout = 1;
            }
        }
        block_sync();
        if (s_timeout) {
            aborted = true;
            break;
        }
        count_run<true, FULL>(a.x, h, stage + k * p.stage_elems + (h.a0 & 3u), eb, epoch, tid, T, red);
        if (tid == 0) ring[(it + 2) % 3] = nn;
    }
    if (aborted) {
        // report, and let the one copy still in flight land before the block
        // exits (thread 0 keeps the block, and so its shared memory, alive
        // while it waits; the wait is bounded like every other)
        if (tid == 0) {
            atomicOr(a.x.err, 4);
            for (int q = 0; q < 2; ++q)
                while (cnt_of(used, q) != cnt_of(issued, q) && mbar_wait(&bars[q], cnt_of(used, q) & 1u, STAGE_WAIT_LIMIT))
                    consume(q);
        }
        return;
    }
    // runs between a warp's and the block's reach: groups of warps, each with
    // a quarter of the table (started empty) and its own named barrier, take
    // runs in a static round-robin
    if (p.ng > 1) {
        block_sync();
        for (int i = tid; i < p.cap; i += T) slot[i] = 0ull;
        block_sync();
        const int GS = T / p.ng, g = tid / GS, gtid = tid % GS;
        const TAB eg = make_table<TAB>(slot + (size_t)g * p.cap_g, p.cap_g, &ctl[3 + 2 * (g * (GS >> 5))]);
        unsigned gepoch = 0;
        const int nmid = a.counters[C_MID_COUNT];
        for (long long i = b * p.ng + g; i < nmid; i += G * p.ng) {
            const RunHdr h = a.mid[i];
            count_run<false, FULL>(a.x, h, a.x.nbr + h.a0, eg, gepoch, gtid, GS, red);
        }
    }
    // the warps' tables are slices of the block's: start them empty
    block_sync();
    for (int i = tid; i < p.cap; i += T) slot[i] = 0ull;
    block_sync();
    const TAB ew = make_table<TAB>(slot + wid * p.cap_w, p.cap_w, &ctl[3 + 2 * wid]);
    unsigned wepoch = 0;
    const int nsmall = a.counters[C_SMALL_COUNT];
    const int chunk = claim_chunk(nsmall, G * W);
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&a.counters[C_SMALL_NEXT], chunk);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= nsmall) break;
        const RunHdr mine = lane < chunk && base + lane < nsmall ? a.small[base + lane] : none;
        const int cnt = min(chunk, nsmall - base);
        for (int j = 0; j < cnt; ++j) {
            RunHdr h;
            h.c = __shfl_sync(0xffffffffu, mine.c, j);
            h.a0 = __shfl_sync(0xffffffffu, mine.a0, j);
            h.m = __shfl_sync(0xffffffffu, mine.m, j);
            h.vol = __shfl_sync(0xffffffffu, mine.vol, j);
            count_run<false, FULL>(a.x, h, a.x.nbr + h.a0, ew, wepoch, lane, 32, red);
        }
    }
}

// Runs longer than the block tables of k_count hold at 3/4 load (and any run
// of 2^24 entries or more), one block each, with 64-bit counts
// (count_run_general).
__global__ void __launch_bounds__(1024) k_count_long(CountCtx x, const RunHdr *lng, const int *counters,
                                                      SmemPlan p, const int *status)
{
    extern __shared__ __align__(16) unsigned char sm[];
    if (*status) return;
    const int n = counters[C_LONG_COUNT];
    if ((int)blockIdx.x >= n) return;
    unsigned long long *red = (unsigned long long *)(sm + p.red_off);
    int *ctl = (int *)(sm + p.ctl_off);
    unsigned long long *slot = (unsigned long long *)(sm + p.slot_off);
    int *used = (int *)(sm + p.used_off);
    for (int i = threadIdx.x; i < p.cap; i += blockDim.x) slot[i] = 0ull;
    if (threadIdx.x < 2) ctl[threadIdx.x] = 0;
    block_sync();
    const SmemTable tb{slot, used, &ctl[0], &ctl[1], p.cap, p.max_used};
    for (int i = blockIdx.x; i < n; i += gridDim.x) count_run_general(x, lng[i], tb, threadIdx.x, blockDim.x, red);
}

// ------------------------------------------------------------------ phase B by sorting (algorithm 6)
//
// The same per-community records as k_count, from sorted runs instead of hash
// tables (Eq. (9)'s |E_cj| are the lengths of the equal-label stretches of
// c's run once it is sorted).  A group stages the run in shared memory, sorts
// it by label with a least-significant-digit radix sort (8-bit digits; each
// warp histograms a contiguous tile, the digit offsets are scanned over warps
// and digits, and each warp scatters its tile in order, lanes ranked among
// equal digits by __match_any_sync, so every pass is stable), then each
// stretch's first entry finds its end by binary search and adds
// |E_cj|^2 Rcp_j.  Runs of up to SORT_WARP_CAP entries are sorted by single
// warps, longer ones up to the block's buffers by whole blocks; longer runs
// take k_count_long.
constexpr int SORT_BINS = 256;
constexpr int SORT_WARP_CAP = 256;

struct SortPlan {
    int red_off, hist_off, buf_off;
    int cap;  // entries of each of the block's two buffers
    int bytes;
};

static SortPlan plan_sort(int T, int S)
{
    SortPlan p;
    const int W = T / 32;
    int off = 0;
    p.red_off = off;
    off += 256 * 8;
    p.hist_off = off;
    off += W * SORT_BINS * 4;
    p.buf_off = off;
    p.cap = std::max(0, (S - off) / 8) / 32 * 32;
    p.bytes = off + p.cap * 8;
    return p;
}

// Sorts run h (entries nbr[a0 .. a0 + m)) with a group and writes its record.
// A and B are the group's buffers (at least m entries each), hist its
// per-warp digit counters (SORT_BINS per warp); `passes` covers the bits of
// the largest label id.
template <bool FULL>
__device__ __forceinline__ void sort_count_run(const CountCtx &x, const RunHdr &h, int *A, int *B, unsigned *hist,
                                               int passes, int gtid, int gsize, unsigned long long *red)
{
    const int m = (int)h.m, c = h.c, lane = threadIdx.x & 31, wl = gtid >> 5, nw = gsize >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int i = gtid; i < m; i += gsize) A[i] = __ldcs(&x.nbr[h.a0 + i]);
    group_sync_n(gsize);
    const int per = (m + nw - 1) / nw, t0 = min(m, wl * per), t1 = min(m, t0 + per);
    unsigned *hw = hist + wl * SORT_BINS;
    const int dpt = max(1, SORT_BINS / gsize), d0 = gtid * dpt;  // digits whose offsets this thread forms
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        for (int d = lane; d < SORT_BINS; d += 32) hw[d] = 0u;
        __syncwarp();
        for (int i = t0 + lane; i < t1; i += 32) atomicAdd(&hw[((unsigned)A[i] >> shift) & 255u], 1u);
        group_sync_n(gsize);
        // offset of (warp w, digit d): all entries of smaller digits, then those
        // of digit d in warps before w
        unsigned tot[8], sum = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            tot[k] = 0u;
            const int d = d0 + k;
            if (k < dpt && d < SORT_BINS) {
                unsigned t = 0;
                for (int w = 0; w < nw; ++w) {
                    const unsigned v = hist[w * SORT_BINS + d];
                    hist[w * SORT_BINS + d] = t;
                    t += v;
                }
                tot[k] = t;
                sum += t;
            }
        }
        unsigned excl;
        group_exclusive_scan(sum, excl, gsize, red);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int d = d0 + k;
            if (k < dpt && d < SORT_BINS) {
                for (int w = 0; w < nw; ++w) hist[w * SORT_BINS + d] += excl;
                excl += tot[k];
            }
        }
        group_sync_n(gsize);
        for (int i0 = t0; i0 < t1; i0 += 32) {
            const int i = i0 + lane;
            const bool valid = i < t1;
            const unsigned act = __ballot_sync(0xffffffffu, valid);
            int key = 0, pos = 0;
            unsigned d = 0u, peers = 0u;
            if (valid) {
                key = A[i];
                d = ((unsigned)key >> shift) & 255u;
                peers = __match_any_sync(act, d);
                pos = (int)hw[d] + __popc(peers & lt);
            }
            __syncwarp();
            if (valid) {
                B[pos] = key;
                if (lane == __ffs(peers) - 1) hw[d] += (unsigned)__popc(peers);
            }
            __syncwarp();
        }
        group_sync_n(gsize);
        int *t = A;
        A = B;
        B = t;
    }
    unsigned long long slots = 0, cnt2 = 0;
    U192 inner, inner_full;
    u192_zero(inner);
    u192_zero(inner_full);
    for (int i = gtid; i < m; i += gsize) {
        const int key = A[i];
        if (i > 0 && A[i - 1] == key) continue;  // not the first of its stretch
        int lo = i + 1, hi = m;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (A[mid] == key) lo = mid + 1; else hi = mid;
        }
        if (!QM_CHK(key, x.K, 7)) continue;
        const unsigned long long cnt = (unsigned long long)(lo - i), q = cnt * cnt;
        const Rcp rj = ld_rcp(&x.recip[key]);
        if (FULL) u192_mac(inner_full, q, rj);
        if (!FULL || key > c) {
            u192_mac(inner, q, rj);
            ++slots;
            cnt2 += q;
        }
    }
    group_totals<FULL>(slots, cnt2, inner, inner_full, gsize, red);
    if (gtid == 0) put_record(x, h.c, h.vol, (unsigned)m, slots, cnt2, inner, inner_full);
    group_sync_n(gsize);  // the buffers are reused by the next run
}

struct CountSortArgs {
    CountCtx x;
    const RunHdr *big;    // runs for whole blocks
    const RunHdr *small;  // runs for single warps
    int *counters;
    const int *status;
    SortPlan plan;
    int passes;
};

template <bool FULL>
__global__ void __launch_bounds__(1024) k_count_sort(CountSortArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_i;
    if (*a.status) return;
    const SortPlan &p = a.plan;
    unsigned long long *red = (unsigned long long *)(sm + p.red_off);
    unsigned *hist = (unsigned *)(sm + p.hist_off);
    int *buf = (int *)(sm + p.buf_off);
    const int T = blockDim.x, W = T >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int nbig = a.counters[C_BIG_COUNT];
    for (;;) {
        if (tid == 0) s_i = atomicAdd(&a.counters[C_BIG_NEXT], 1);
        block_sync();
        const int i = s_i;
        block_sync();
        if (i >= nbig) break;
        sort_count_run<FULL>(a.x, a.big[i], buf, buf + p.cap, hist, a.passes, tid, T, red);
    }
    int *wa = buf + wid * 2 * SORT_WARP_CAP;
    const int nsmall = a.counters[C_SMALL_COUNT];
    const int chunk = claim_chunk(nsmall, (long long)gridDim.x * W);
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&a.counters[C_SMALL_NEXT], chunk);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= nsmall) break;
        const int top = min(nsmall, base + chunk);
        for (int i = base; i < top; ++i)
            sort_count_run<FULL>(a.x, a.small[i], wa, wa + SORT_WARP_CAP, hist + wid * SORT_BINS, a.passes, lane, 32,
                                 red);
    }
}

bool sort_shape_ok(int threads, int smem_bytes)
{
    const SortPlan p = plan_sort(threads, smem_bytes);
    return p.cap >= (threads / 32) * SORT_WARP_CAP && p.bytes <= smem_bytes;
}

int sort_blocks_per_sm(const Shape &sh)
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_count_sort<false>, sh.threads, sh.smem_bytes);
    return nb;
}

// Block reduction of per-thread sums into the partition's global limbs.
__device__ __forceinline__ void flush_score_threads(const ScoreAcc &acc, unsigned long long *g,
                                                    unsigned long long *red)
{
    const int T = blockDim.x;
    const i128 v[7] = {acc.qds_self, acc.qds_pair, acc.dens, acc.contr, acc.expn, acc.cond, (i128)acc.vol2};
    const int at[7] = {GS_QDS_SELF, GS_QDS_PAIR, GS_DENS, GS_CONTR, GS_EXPN, GS_COND, GS_VOL2};
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const i128 t = group_sum_i128(v[k], T, red);
        if (threadIdx.x == 0) limbs_add(g + at[k], t);
    }
    const unsigned long long u[5] = {acc.ein, acc.eout, acc.nonempty, acc.slots, acc.cnt2};
    const int au[5] = {GS_EIN, GS_EOUT, GS_NONEMPTY, GS_SLOTS, GS_CNT2};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const unsigned long long t = group_sum_u64(u[k], T, red);
        if (threadIdx.x == 0 && t) atomicAdd(g + au[k], t);
    }
}

// FP64 terms of every community from the phase-B records, all in parallel.
__global__ void k_score_terms(const int *start, const unsigned long long *rec, int K, long long E, PerCommDev pc,
                              unsigned long long *g, const int *status, Shard own)
{
    __shared__ unsigned long long red[72];
    if (*status) return;
    ScoreAcc acc;
    score_acc_zero(acc);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < K; c += gridDim.x * blockDim.x) {
        const long long size = start[c + 1] - start[c];
        if (size == 0 || !own.owns(c)) continue;
        double pen, qs, dens, contr, expn, cond;
        const unsigned long long *rc = rec + (size_t)c * REC_WORDS;
        terms_from_record(rc, size, E, acc, &pen, &qs, &dens, &contr, &expn, &cond);
        if (pc.size) pc.size[c] = size;
        if (pc.ein) pc.ein[c] = (long long)(rc[REC_SAME] / 2);
        if (pc.eout) pc.eout[c] = (long long)(rc[REC_VOL] - rc[REC_SAME]);
        if (pc.dens) pc.dens[c] = dens;
        if (pc.contr) pc.contr[c] = contr;
        if (pc.expn) pc.expn[c] = expn;
        if (pc.cond) pc.cond[c] = cond;
        if (pc.qds) pc.qds[c] = __dsub_rn(qs, pen);
    }
    flush_score_threads(acc, g, red);
}

#include "qm_weighted.cuh"

// Launch shape of k_count_w (weighted graphs) and its occupancy.
constexpr int COUNT_W_THREADS = 256, COUNT_W_SMEM = 48 * 1024;
static int g_count_w_blocks_per_sm = 1;  // set by prepare_kernels

void prepare_kernels()
{
    cudaFuncSetAttribute(k_score_cm, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    cudaFuncSetAttribute(k_compare_cm, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    cudaFuncSetAttribute(k_count<EpochTable, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    cudaFuncSetAttribute(k_count<EpochTable32V, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    cudaFuncSetAttribute(k_count<EpochTable, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    cudaFuncSetAttribute(k_count<EpochTable32V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    cudaFuncSetAttribute(k_count_long, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    cudaFuncSetAttribute(k_count_sort<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    cudaFuncSetAttribute(k_count_sort<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    cudaFuncSetAttribute(k_count_w, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    cudaFuncSetAttribute(k_expand_bin, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         bin_smem_bytes_per_warp(BIN_MAX) * (EXPAND_THREADS / 32));
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_count_w, COUNT_W_THREADS, COUNT_W_SMEM);
    g_count_w_blocks_per_sm = nb > 0 ? nb : 1;
    k_fill_log_int<<<(LOGT_MAX + 256) / 256, 256>>>();
    cudaDeviceSynchronize();
}

int count_blocks_per_sm(const Shape &sh)
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_count<EpochTable32V, false>, sh.threads, sh.smem_bytes);
    return nb;
}

int score_blocks_per_sm(const Shape &sh)
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_score_cm, sh.threads, sh.smem_bytes);
    return nb;
}

#define TRACE(name) \
    do {            \
        if (tr) tr(name, s); \
    } while (0)

static int launch_scan(const int *size, int K, int *start, int *cursor, Rcp *recip, int big_thr,
                       int *big_list, int *counters, int *tmp, const int *status, cudaStream_t s, TraceFn tr)
{
    if (K <= SCAN_SINGLE_MAX) {
        TRACE("k_scan_single");
        k_scan_single<<<1, 1024, 0, s>>>(size, K, start, cursor, recip, big_thr, big_list, counters, status);
        return 1;
    }
    const int tiles = scan_tiles(K);
    TRACE("k_scan_tiles");
    k_scan_tiles<<<tiles, 1024, 0, s>>>(size, K, tmp, status);
    // exclusive prefix of the tile sums, in place into tmp[0..tiles] (tmp[tiles] = total)
    TRACE("k_scan_single");
    k_scan_single<<<1, 1024, 0, s>>>(tmp, tiles, tmp, nullptr, nullptr, INT_MAX, nullptr, counters, status);
    TRACE("k_scan_apply");
    k_scan_apply<<<tiles, 1024, 0, s>>>(size, K, tmp, start, cursor, recip, big_thr, big_list, counters, status);
    return 3;
}

// Exclusive prefix of in[0..n) into out[0..n] (out may alias in); tmp holds
// scan_tmp_elems(n) ints.  Returns the number of launches, or -1.
size_t scan_tmp_elems(long long n) { return (size_t)scan_tiles((int)n) + 1; }

int scan_offsets(const int *in, int n, int *out, int *tmp, int *counters, const int *status, cudaStream_t s)
{
    return launch_scan(in, n, out, nullptr, nullptr, INT_MAX, nullptr, counters, tmp, status, s, nullptr);
}

int launch_score(const GraphDev &g, const int *labels, int K, const ScoreWs &ws, const Shape &sh,
                 const PerCommDev *pc, int num_sms, cudaStream_t s, TraceFn tr)
{
    int launches = 0;
    const long long n = g.n;
    const int hist_smem = (K <= 12288) ? K * 4 : 0;
    TRACE("k_hist");
    k_hist<<<grid_for(n, 512, num_sms, 4), 512, hist_smem, s>>>(labels, K, ws.size, nullptr, 0, nullptr, n,
                                                                ws.status, hist_smem ? 1 : 0);
    ++launches;
    launches += launch_scan(ws.size, K, ws.start, ws.cursor, ws.recip, sh.big_community, ws.big_list,
                            ws.counters, ws.scan_tmp, ws.status, s, tr);
    TRACE("k_scatter");
    k_scatter<<<grid_for(n, 512, num_sms, 8), 512, 0, s>>>(labels, nullptr, n, ws.cursor, ws.members, ws.status, 0);
    ++launches;

    ScoreKArgs a;
    a.x.row_ptr = g.row_ptr;
    a.x.col = g.col;
    a.x.labels = labels;
    a.x.members = ws.members;
    a.x.start = ws.start;
    a.x.recip = ws.recip;
    a.x.E = g.n_arcs / 2;
    a.x.n = g.n;
    a.x.n_arcs = g.n_arcs;
    a.x.K = K;
    a.x.err = ws.status;
    a.x.pc_size = pc ? pc->size : nullptr;
    a.x.pc_ein = pc ? pc->ein : nullptr;
    a.x.pc_eout = pc ? pc->eout : nullptr;
    a.x.pc_dens = pc ? pc->dens : nullptr;
    a.x.pc_contr = pc ? pc->contr : nullptr;
    a.x.pc_expn = pc ? pc->expn : nullptr;
    a.x.pc_cond = pc ? pc->cond : nullptr;
    a.x.pc_qds = pc ? pc->qds : nullptr;
    a.big_list = ws.big_list;
    a.ovf_in = ws.ovf_list;
    a.ovf_out = ws.ovf_list;
    a.counters = ws.counters;
    a.gacc = ws.gacc;
    a.status = ws.status;
    a.big_thr = sh.big_community;
    a.plan = plan_smem(sh.threads, sh.smem_bytes);
    const int blocks = community_grid(K, num_sms, sh);
    a.phase = 0;
    TRACE("k_score_cm");
    k_score_cm<<<blocks, sh.threads, sh.smem_bytes, s>>>(a);
    a.phase = 1;
    TRACE("k_score_cm_overflow");
    k_score_cm<<<blocks, sh.threads, sh.smem_bytes, s>>>(a);
    TRACE("k_score_fin");
    k_score_fin<<<1, 32, 0, s>>>(ws.gacc, ws.status, n, g.n_arcs / 2, ws.result, 0);
    TRACE(nullptr);
    launches += 3;
    return cudaGetLastError() == cudaSuccess ? launches : -1;
}

size_t score2_ws_bytes(long long n, long long n_arcs, int K, bool weighted, int bin_mode, bool pack)
{
    return carve_score2_ws(reinterpret_cast<void *>(4096), n, n_arcs, K, weighted, bin_mode, pack).bytes;
}

// Window size, window count and nearness distance of the binned gathers.
static void bin_geometry(long long n, int mode, int *shift, int *nbins, int *near)
{
    int lg = 0;
    while ((1LL << lg) < n) ++lg;  // ceil(log2 n)
    if (mode == 2) {
        *shift = std::max(23, lg - 4);
        *near = 1 << 14;
    } else {
        *shift = std::max(4, lg - 2);
        *near = 0;
    }
    *nbins = (int)(((std::max(n, 1LL) - 1) >> *shift) + 1);
}

ScoreWs carve_score2_ws(void *base, long long n, long long n_arcs, int K, bool weighted, int bin_mode, bool pack)
{
    ScoreWs w{};
    if (weighted) bin_mode = 0;
    if (weighted || bin_mode || K > PACK_MAX_K) pack = false;
    const int tiles = scan_tiles((int)std::max<long long>(n, K));
    char *p = (char *)base;
    w.status = (int *)p;
    w.counters = (int *)(p + 16);
    p += 256;
    w.gacc = (unsigned long long *)p;
    p += align_up(32 * 8, 256);
    w.result = (qm_quality *)p;
    p += align_up(sizeof(qm_quality), 256);
    w.size = (int *)p;
    p += align_up((size_t)K * 4, 256);
    w.inter = (int *)p;
    p += align_up((size_t)K * 4, 256);
    w.inter_hi = (int *)p;
    p += align_up((size_t)K * 4, 256);
    if (weighted) {
        w.wl = (unsigned long long *)p;
        p += align_up((size_t)K * 6 * 8, 256);
    }
    if (bin_mode) {
        w.bin_ctr = (int *)p;
        p += align_up(BC_WORDS * 4, 256);
    }
    w.zero_bytes = (size_t)(p - (char *)base);
    if (bin_mode) {
        bin_geometry(n, bin_mode, &w.bin_shift, &w.bin_nbins, &w.bin_near);
        const long long warps = std::min<long long>((n + 255) / 256, BIN_MAX_BLOCKS) * (EXPAND_THREADS / 32);
        w.bin_chunks = n_arcs / BIN_CHUNK + 1 + warps * w.bin_nbins;
        w.bin_seg = (int *)p;
        p += align_up((size_t)K * 4, 256);
        w.bin_list = (unsigned long long *)p;
        p += align_up((size_t)w.bin_chunks * 8, 256);
        w.bin_sorted = (unsigned long long *)p;
        p += align_up((size_t)w.bin_chunks * 8, 256);
        w.bin_pool = (unsigned long long *)p;
        p += align_up((size_t)w.bin_chunks * BIN_CHUNK * 8, 256);
    }
    if (pack) {
        w.plab = (unsigned long long *)p;
        p += align_up((size_t)((n + 2) / 3) * 8, 256);
    }
    if (weighted) {
        w.nbrw = (float *)p;
        p += align_up((size_t)n_arcs * 4, 256) + 256;
        w.recw = (unsigned long long *)p;
        p += align_up((size_t)K * 4 * 8, 256);
    }
    w.start = (int *)p;
    p += align_up(((size_t)K + 1) * 4, 256);
    w.recip = (Rcp *)p;
    p += align_up((size_t)K * 16, 256);
    w.cursor = (int *)p;
    p += align_up((size_t)K * 4, 256);
    w.big_list = (int *)p;
    p += align_up((size_t)K * 4, 256);
    w.ovf_list = nullptr;
    w.members = (int *)p;
    p += align_up((size_t)n * 4, 256);
    w.aoff = (unsigned *)p;
    p += align_up((size_t)(n + 1) * 4, 256);
    w.nbr = (int *)p;
    p += align_up((size_t)n_arcs * 4, 256) + 256;
    w.rec = (unsigned long long *)p;
    p += align_up((size_t)K * 8 * REC_WORDS, 256);
    w.hdr_big = (RunHdr *)p;
    p += align_up((size_t)K * sizeof(RunHdr), 256);
    w.hdr_small = (RunHdr *)p;
    p += align_up((size_t)K * sizeof(RunHdr), 256);
    w.hdr_long = (RunHdr *)p;
    p += align_up((size_t)K * sizeof(RunHdr), 256);
    w.hdr_mid = (RunHdr *)p;
    p += align_up((size_t)K * sizeof(RunHdr), 256);
    w.scan_tmp = (int *)p;
    p += align_up((size_t)(tiles + 1) * 4, 256);
    w.bytes = (size_t)(p - (char *)base);
    return w;
}

int launch_permute_hist(const int *labels, const int *inv, long long n, int *out, int K, const ScoreWs &ws,
                        int num_sms, cudaStream_t s)
{
    const int hist_smem = (K <= 12288) ? K * 4 : 0;
    k_permute_hist<<<grid_for(n, 512, num_sms, 8), 512, hist_smem, s>>>(labels, inv, n, out, K, ws.size, ws.status,
                                                                       hist_smem ? 1 : 0);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

static int community_grid(long long K, int num_sms, const Shape &sh)
{
    const long long resident = (long long)num_sms * (sh.blocks_per_sm > 0 ? sh.blocks_per_sm : 1);
    return (int)std::max<long long>(1, std::min<long long>(resident, K));
}

// k_expand: 8 blocks per SM, or fewer when the graph has fewer member chunks
// (32 member positions per warp, EXPAND_THREADS / 32 warps per block).
// k_expand: per_sm blocks per SM, or fewer when the graph has fewer member
// chunks.  The gathers from the block encoding (L2-resident, bound by latency)
// take one wave of resident blocks: each block has an equal grid-stride share,
// so blocks of a second wave would start late and end the kernel late.  The
// DRAM-bound gathers from the packed copy keep 8 blocks per SM (measured
// faster there).
static int expand_grid(long long n, int num_sms, int per_sm = 8)
{
    const long long per_block = 32LL * (EXPAND_THREADS / 32);
    return (int)std::max<long long>(1,
                                    std::min<long long>((long long)num_sms * per_sm, (n + per_block - 1) / per_block));
}

template <bool WT, int LAB, bool HI>
static int expand_per_sm()
{
    static std::atomic<int> v{0};
    if (!v.load()) {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_expand<WT, LAB, HI>, EXPAND_THREADS, 0);
        v.store(std::max(1, std::min(nb, 8)));
    }
    return v.load();
}

// Weighted graphs after k_expand<true>: one block per community counts and
// forms the weighted pair sums, then the weighted terms and the result.

static int launch_weighted_tail(const GraphDev &g, int K, const ScoreWs &ws, const PerCommDev *pc, int num_sms,
                                cudaStream_t s, TraceFn tr, Shard own, int launches)
{
    CountCtx x;
    x.nbr = ws.nbr;
    x.aoff = ws.aoff;
    x.start = ws.start;
    x.inter = ws.inter;
    x.recip = ws.recip;
    x.rec = ws.rec;
    x.K = K;
    x.err = ws.status;
    x.full = 0;
    TRACE("k_count_w");
    k_count_w<<<(int)std::min<long long>((long long)num_sms * g_count_w_blocks_per_sm, K), COUNT_W_THREADS,
                COUNT_W_SMEM, s>>>(
        x, ws.nbrw, ws.recw, plan_smem(COUNT_W_THREADS, COUNT_W_SMEM), ws.status, own);
    PerCommDev pcd{};
    if (pc) pcd = *pc;
    TRACE("k_score_terms_w");
    k_score_terms_w<<<grid_for(K, 256, num_sms, 2), 256, 0, s>>>(ws.start, ws.rec, ws.recw, ws.wl, K, g.n_arcs / 2,
                                                                 g.w_lo, g.w_hi, pcd, ws.gacc, ws.status, own);
    launches += 2;
    if (own.p == 1) {
        TRACE("k_score_fin");
        k_score_fin<<<1, 32, 0, s>>>(ws.gacc, ws.status, g.n, g.n_arcs / 2, ws.result, 1);
        ++launches;
    }
    TRACE(nullptr);
    return cudaGetLastError() == cudaSuccess ? launches : -1;
}

// The two-phase plain scoring pipeline (see k_expand / count_community):
//   k_hist -> scan (sizes) -> k_scatter_deg -> scan (member degrees = arc offsets)
//   -> k_expand -> k_classify -> k_count -> k_score_terms -> k_score_fin
int launch_score2(const GraphDev &g, const int *labels, int K, const ScoreWs &ws, const Shape &sh,
                  const PerCommDev *pc, int num_sms, cudaStream_t s, TraceFn tr, int shard_r, int shard_p,
                  bool sizes_ready)
{
    int launches = 0;
    const Shard own{shard_r, shard_p};
    const long long n = g.n;
    if (!sizes_ready) {
        const int hist_smem = (K <= 12288) ? K * 4 : 0;
        TRACE("k_hist");
        k_hist<<<grid_for(n, 512, num_sms, 4), 512, hist_smem, s>>>(labels, K, ws.size, nullptr, 0, nullptr, n,
                                                                    ws.status, hist_smem ? 1 : 0);
        ++launches;
    }
    launches += launch_scan(ws.size, K, ws.start, ws.cursor, ws.recip, INT_MAX, nullptr, ws.counters,
                            ws.scan_tmp, ws.status, s, tr);
    TRACE("k_scatter_deg");
    k_scatter_deg<<<grid_for(n, 512, num_sms, 8), 512, 0, s>>>(labels, g.row_ptr, n, ws.cursor, ws.members,
                                                               (int *)ws.aoff, ws.status);
    ++launches;
    // exclusive prefix of the member degrees, in place: aoff[p] = arcs before member position p
    launches += launch_scan((const int *)ws.aoff, (int)n, (int *)ws.aoff, nullptr, nullptr, INT_MAX, nullptr,
                            ws.counters, ws.scan_tmp, ws.status, s, tr);
    if (g.wt) {
        TRACE("k_expand");
        k_expand<true, LAB_PLAIN, false><<<expand_grid(n, num_sms), EXPAND_THREADS, 0, s>>>(g.row_ptr, g.col, labels, nullptr, ws.members, ws.aoff,
                                                              ws.start, n, ws.inter, nullptr, ws.nbr, ws.status, own, g.wt,
                                                              ws.nbrw, ws.wl);
        ++launches;
        return launch_weighted_tail(g, K, ws, pc, num_sms, s, tr, own, launches);
    }
    const int *packed_len = ws.inter;  // entries of each community's packed run
    const bool half = sh.algo == ALGO_HALF && g.up_ptr && shard_p == 1 && !ws.bin_pool;
    if (half) {
        // each undirected edge gathered once, from its lower end; the scatter
        // cursors are free now and take the segment bases
        unsigned *cbase = (unsigned *)ws.cursor;
        const bool full = pc && pc->qds;
        const dim3 eg(expand_grid(n, num_sms)), eb(EXPAND_THREADS);
        TRACE("k_cbase");
        k_cbase<<<grid_for(K, 256, num_sms, 4), 256, 0, s>>>(ws.start, ws.aoff, K, cbase, ws.status);
        ++launches;
        if (ws.plab) {
            TRACE("k_pack3");
            k_pack3<<<grid_for((n + 2) / 3, 256, num_sms, 8), 256, 0, s>>>(labels, n, ws.plab, ws.status, nullptr);
            ++launches;
        }
        TRACE("k_expand_half");
        if (ws.plab && full)
            k_expand_half<true, true><<<eg, eb, 0, s>>>(g.up_ptr, g.up_col, labels, ws.plab, ws.members, cbase, n,
                                                        ws.inter, ws.inter_hi, ws.nbr, ws.status);
        else if (ws.plab)
            k_expand_half<true, false><<<eg, eb, 0, s>>>(g.up_ptr, g.up_col, labels, ws.plab, ws.members, cbase, n,
                                                         ws.inter, ws.inter_hi, ws.nbr, ws.status);
        else if (full)
            k_expand_half<false, true><<<eg, eb, 0, s>>>(g.up_ptr, g.up_col, labels, nullptr, ws.members, cbase, n,
                                                         ws.inter, ws.inter_hi, ws.nbr, ws.status);
        else
            k_expand_half<false, false><<<eg, eb, 0, s>>>(g.up_ptr, g.up_col, labels, nullptr, ws.members, cbase, n,
                                                          ws.inter, ws.inter_hi, ws.nbr, ws.status);
        ++launches;
        packed_len = ws.inter_hi;
    } else if (ws.bin_pool) {
        BinArgs ba;
        ba.pool = ws.bin_pool;
        ba.list = ws.bin_list;
        ba.sorted = ws.bin_sorted;
        ba.ctr = ws.bin_ctr;
        ba.seg = ws.bin_seg;
        ba.pool_chunks = ws.bin_chunks;
        ba.shift = ws.bin_shift;
        ba.nbins = ws.bin_nbins;
        ba.near = ws.bin_near;
        const int smem = bin_smem_bytes_per_warp(ba.nbins) * (EXPAND_THREADS / 32);
        TRACE("k_expand_bin");
        k_expand_bin<<<std::min(expand_grid(n, num_sms), BIN_MAX_BLOCKS), EXPAND_THREADS, smem, s>>>(
            g.row_ptr, g.col, labels, ws.members, ws.aoff, ws.start, n, ws.inter, ws.nbr, ws.status, own, ba);
        TRACE("k_bin_order");
        k_bin_order<<<num_sms * 2, 256, 0, s>>>(ba, ws.aoff, ws.start, K, ws.status);
        TRACE("k_resolve");
        k_resolve<<<num_sms * 8, RESOLVE_THREADS, 0, s>>>(ba, labels, ws.inter, ws.nbr, ws.status);
        launches += 3;
    } else {
        // without per-community Qds terms each unordered pair of communities is
        // counted by its smaller id only, so only the labels above c are packed
        const bool hi = !(pc && pc->qds);
        const dim3 eg(expand_grid(n, num_sms)), eb(EXPAND_THREADS);
        // on a renumbered graph above BLOCKS_MIN_NODES nodes (any size with
        // algorithm 4) the block encoding is tried first (the packed copy, in
        // the same buffer, only when it does not fit)
        const bool blocks = ws.plab && g.inv && label_blocks(sh.algo, n);
        int *const bx_bad = blocks ? &ws.counters[C_BX_BAD] : nullptr;
        if (blocks) {
            TRACE("k_pack_blocks");
            const long long nb = (n + BLK_NODES - 1) / BLK_NODES;
            k_pack_blocks<<<grid_for((nb + 2 * PACKB_UNROLL - 1) / (2 * PACKB_UNROLL) * 32, 256, num_sms, 8), 256, 0,
                            s>>>(
                labels, n, ws.plab, blocks_xcap(n), &ws.counters[C_BX_COUNT], bx_bad, ws.status);
            ++launches;
        }
        if (ws.plab) {
            TRACE("k_pack3");
            k_pack3<<<grid_for((n + 2) / 3, 256, num_sms, 8), 256, 0, s>>>(labels, n, ws.plab, ws.status, bx_bad);
            ++launches;
        }
        TRACE("k_expand");
        if (blocks) {
            if (hi)
                k_expand<false, LAB_BLOCKS, true><<<expand_grid(n, num_sms, expand_per_sm<false, LAB_BLOCKS, true>()),
                                                    eb, 0, s>>>(g.row_ptr, g.col, labels, ws.plab, ws.members,
                                                                    ws.aoff, ws.start, n, ws.inter, ws.inter_hi,
                                                                    ws.nbr, ws.status, own, nullptr, nullptr,
                                                                    nullptr, bx_bad);
            else
                k_expand<false, LAB_BLOCKS, false><<<expand_grid(n, num_sms,
                                                                 expand_per_sm<false, LAB_BLOCKS, false>()),
                                                     eb, 0, s>>>(g.row_ptr, g.col, labels, ws.plab, ws.members,
                                                                     ws.aoff, ws.start, n, ws.inter, nullptr, ws.nbr,
                                                                     ws.status, own, nullptr, nullptr, nullptr,
                                                                     bx_bad);
            ++launches;
        }
        if (ws.plab && hi)
            k_expand<false, LAB_PACK3, true><<<eg, eb, 0, s>>>(g.row_ptr, g.col, labels, ws.plab, ws.members,
                                                               ws.aoff, ws.start, n, ws.inter, ws.inter_hi, ws.nbr,
                                                               ws.status, own, nullptr, nullptr, nullptr, bx_bad);
        else if (ws.plab)
            k_expand<false, LAB_PACK3, false><<<eg, eb, 0, s>>>(g.row_ptr, g.col, labels, ws.plab, ws.members,
                                                                ws.aoff, ws.start, n, ws.inter, nullptr, ws.nbr,
                                                                ws.status, own, nullptr, nullptr, nullptr, bx_bad);
        else if (hi)
            k_expand<false, LAB_PLAIN, true><<<eg, eb, 0, s>>>(g.row_ptr, g.col, labels, nullptr, ws.members, ws.aoff,
                                                           ws.start, n, ws.inter, ws.inter_hi, ws.nbr, ws.status,
                                                           own, nullptr, nullptr, nullptr);
        else
            k_expand<false, LAB_PLAIN, false><<<eg, eb, 0, s>>>(g.row_ptr, g.col, labels, nullptr, ws.members,
                                                            ws.aoff, ws.start, n, ws.inter, nullptr, ws.nbr,
                                                            ws.status, own, nullptr, nullptr, nullptr);
        ++launches;
        packed_len = hi ? ws.inter_hi : ws.inter;
    }
    const CountPlan cp = plan_count(sh.threads, sh.smem_bytes);
    const bool sorted = sh.algo == ALGO_SORT;
    const SortPlan sp = plan_sort(sh.threads, sh.smem_bytes);
    TRACE("k_classify");
    if (sorted)  // warps sort runs up to SORT_WARP_CAP, blocks up to their buffers
        k_classify<<<grid_for(K, 256, num_sms, 4), 256, 0, s>>>(ws.start, ws.aoff, packed_len, K, SORT_WARP_CAP,
                                                                SORT_WARP_CAP, sp.cap, ws.hdr_big, ws.hdr_small,
                                                                ws.hdr_long, ws.hdr_mid, ws.counters, ws.status, own,
                                                                half ? ws.inter : nullptr);
    else
        k_classify<<<grid_for(K, 256, num_sms, 4), 256, 0, s>>>(ws.start, ws.aoff, packed_len, K, cp.fill_w,
                                                                cp.fill_g, cp.fill, ws.hdr_big, ws.hdr_small,
                                                                ws.hdr_long, ws.hdr_mid, ws.counters, ws.status, own,
                                                                half ? ws.inter : nullptr);
    ++launches;
    CountKArgs a;
    a.x.nbr = ws.nbr;
    a.x.aoff = ws.aoff;
    a.x.start = ws.start;
    a.x.inter = ws.inter;
    a.x.recip = ws.recip;
    a.x.rec = ws.rec;
    a.x.K = K;
    a.x.err = ws.status;
    a.big = ws.hdr_big;
    a.small = ws.hdr_small;
    a.mid = ws.hdr_mid;
    a.counters = ws.counters;
    a.status = ws.status;
    a.plan = cp;
    a.stage_wait = g_stage_wait.load();
    const int count_grid = community_grid(K, num_sms, sh);  // sh.blocks_per_sm: occupancy resolved by the caller
    // S_c of every community only when its per-community Qds term is asked for
    a.x.full = (pc && pc->qds) ? 1 : 0;
    if (sorted) {
        CountSortArgs sa;
        sa.x = a.x;
        sa.big = ws.hdr_big;
        sa.small = ws.hdr_small;
        sa.counters = ws.counters;
        sa.status = ws.status;
        sa.plan = sp;
        int bits = 1;
        while (bits < 31 && (1LL << bits) < (long long)K) ++bits;
        sa.passes = (bits + 7) / 8;
        TRACE("k_count_sort");
        if (sa.x.full) k_count_sort<true><<<count_grid, sh.threads, sh.smem_bytes, s>>>(sa);
        else k_count_sort<false><<<count_grid, sh.threads, sh.smem_bytes, s>>>(sa);
    } else if (K < (1 << 24) - 1) {
        TRACE("k_count");
        if (a.x.full) k_count<EpochTable32V, true><<<count_grid, sh.threads, sh.smem_bytes, s>>>(a);
        else k_count<EpochTable32V, false><<<count_grid, sh.threads, sh.smem_bytes, s>>>(a);
    } else {
        TRACE("k_count");
        if (a.x.full) k_count<EpochTable, true><<<count_grid, sh.threads, sh.smem_bytes, s>>>(a);
        else k_count<EpochTable, false><<<count_grid, sh.threads, sh.smem_bytes, s>>>(a);
    }
    TRACE("k_count_long");
    k_count_long<<<std::min(num_sms, K), 1024, MAX_DYN_SMEM, s>>>(a.x, ws.hdr_long, ws.counters, plan_smem(1024, MAX_DYN_SMEM),
                                                      ws.status);
    launches += 2;
    PerCommDev pcd{};
    if (pc) pcd = *pc;
    TRACE("k_score_terms");
    k_score_terms<<<grid_for(K, 256, num_sms, 2), 256, 0, s>>>(ws.start, ws.rec, K, g.n_arcs / 2, pcd, ws.gacc,
                                                               ws.status, own);
    ++launches;
    if (shard_p == 1) {  // a shard's caller reads the partial sums instead
        TRACE("k_score_fin");
        k_score_fin<<<1, 32, 0, s>>>(ws.gacc, ws.status, n, g.n_arcs / 2, ws.result, 0);
        ++launches;
    }
    TRACE(nullptr);
    return cudaGetLastError() == cudaSuccess ? launches : -1;
}

int launch_score_fin(const unsigned long long *gacc, const int *status, long long n, long long E, qm_quality *out,
                     int weighted, cudaStream_t s)
{
    k_score_fin<<<1, 32, 0, s>>>(gacc, status, n, E, out, weighted);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

int launch_weight_check(const GraphDev &g, const float *wt, int full, int *status, unsigned long long *lim,
                        int num_sms, cudaStream_t s)
{
    k_wcheck<<<grid_for(g.n_arcs, 256, num_sms, 8), 256, 0, s>>>(wt, g.n_arcs, status, lim);
    if (full) k_wsym<<<grid_for(g.n, 256, num_sms, 8), 256, 0, s>>>(g.row_ptr, g.col, wt, g.n, status);
    return cudaGetLastError() == cudaSuccess ? (full ? 2 : 1) : -1;
}

int launch_compare(const int *truth, const int *found, long long n, int ka, int kb,
                   const CompareWs &ws, const Shape &sh, int num_sms, cudaStream_t s, TraceFn tr)
{
    int launches = 0;
    // sizes of the detected communities (the truth sizes are summed from the
    // contingency cells by k_compare_cm, far fewer updates than one per node)
    const int hist_smem = (kb <= 12288) ? kb * 4 : 0;
    TRACE("k_hist");
    k_hist<<<grid_for(n, 512, num_sms, 4), 512, hist_smem, s>>>(found, kb, ws.size_b, nullptr, 0, nullptr, n,
                                                                ws.status, hist_smem ? 1 : 0);
    ++launches;
    const SmemPlan plan = plan_smem(sh.threads, sh.smem_bytes);
    launches += launch_scan(ws.size_b, kb, ws.start, ws.cursor, nullptr, plan.max_used_w, ws.big_list,
                            ws.counters, ws.scan_tmp, ws.status, s, tr);
    TRACE("k_scatter");
    k_scatter<<<grid_for(n, 512, num_sms, 8), 512, 0, s>>>(found, truth, n, ws.cursor, ws.members, ws.status, ka);
    ++launches;
    CompareKArgs a;
    a.x.truth = truth;
    a.x.tl = ws.members;  // truth labels in detected-community order (k_scatter with vals)
    a.x.members = nullptr;
    a.x.start = ws.start;
    a.x.size_a = ws.size_a;
    a.x.size_a_acc = ws.size_a;  // summed from the cells by k_compare_cm
    a.x.rowmax_n = ws.rowmax_n;
    a.x.rowmax_r = ws.rowmax_r;
    a.x.N = n;
    a.x.ka = ka;
    a.x.kb = kb;
    a.x.err = ws.status;
    a.big_list = ws.big_list;
    a.counters = ws.counters;
    a.cells = ws.cells;
    a.gacc = ws.gacc;
    a.status = ws.status;
    a.plan = plan;
    a.x.logt = ws.logt;
    TRACE("k_log_table");
    k_log_table<<<(LOGT_MAX + 256) / 256, 256, 0, s>>>(ws.logt, n);
    ++launches;
    TRACE("k_compare_cm");  // sh.blocks_per_sm: occupancy resolved by the caller
    k_compare_cm<<<community_grid(kb, num_sms, sh), sh.threads, sh.smem_bytes, s>>>(a);
    TRACE("k_compare_cells");
    k_compare_cells<<<grid_for(n, 256, num_sms, 8), 256, 0, s>>>(a.x, ws.cells, ws.counters, ws.size_b, ws.gacc,
                                                                 ws.status);
    TRACE("k_compare_cols");
    k_compare_cols<<<grid_for(kb, 256, num_sms, 2), 256, 0, s>>>(ws.size_b, kb, n, ws.gacc, ws.status);
    TRACE("k_compare_rows");
    k_compare_rows<<<grid_for(ka, 256, num_sms, 2), 256, 0, s>>>(a.x, ws.gacc, ws.status);
    TRACE("k_compare_fin");
    k_compare_fin<<<1, 32, 0, s>>>(ws.gacc, ws.status, n, ws.result);
    TRACE(nullptr);
    launches += 5;
    return cudaGetLastError() == cudaSuccess ? launches : -1;
}

int launch_validate(const GraphDev &g, int full, int *status, unsigned long long *max_deg, int num_sms,
                    cudaStream_t s)
{
    k_validate<<<grid_for(g.n, 256, num_sms, 8), 256, 0, s>>>(g.row_ptr, g.col, g.n, g.n_arcs, full, status,
                                                              max_deg);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace qm
