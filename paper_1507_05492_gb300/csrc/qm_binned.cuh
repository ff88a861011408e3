// qm_binned.cuh -- the far-end label gathers of the expand phase, made
// L2-resident by binning them by destination window (propagation blocking:
// Beamer, Asanovic & Patterson, IPDPS 2017).
//
// The expand phase visits every arc (u, v) of the members of community c and
// needs label[v] (the no-ground-truth decomposition of Sec. III-A: the edges
// inside c, on its boundary, and to which neighbour community).  When the label
// array is several times the L2, gathering label[v] for arbitrary v costs a DRAM
// access each.  Here the arcs whose far end lies close to u (in node-id order)
// are gathered at once, as before; every other arc becomes an 8-byte record
// (c, v) in the bin of v's window (2^shift consecutive node ids).  A second
// kernel then walks the bins window by window, so that the labels it gathers
// come from one window of the label array at a time, which stays in L2, and
// appends each label != c to c's packed run.  The runs end up holding the same
// multisets as with direct gathers (in another order), so every count and sum
// downstream is unchanged.
//
// Records travel through a pool of fixed chunks: each warp stages records per
// bin in shared memory, writes them to its current chunk of that bin in whole
// 128-byte pieces, and lists each chunk when it is closed.  The chunk list is
// then ordered by bin.
#pragma once
// Included by qm_kernels.cu inside namespace qm, after k_expand.

constexpr int BIN_MAX = 16;        // destination windows at most
constexpr int BIN_CHUNK = 256;     // records per pool chunk (2 KB)
constexpr int BIN_FLUSH = 16;      // records written per flush (128 bytes, whole sectors)
constexpr int BIN_SLOTS = 48;      // staged records per (warp, bin): < BIN_FLUSH left over + 32 new
constexpr int BIN_MAX_BLOCKS = 2048;  // blocks of the binning expand at most (sizes the pool)

// Device counters of the binned path (zeroed with the call's workspace).
enum { BC_CHUNKS = 0, BC_LIST = 1, BC_BIN_COUNT = 2, BC_BIN_FILL = 2 + BIN_MAX, BC_ERR = 2 + 2 * BIN_MAX,
       BC_WORDS = 64 };

struct BinArgs {
    unsigned long long *pool;    // [pool_chunks * BIN_CHUNK] records: (c << 32) | v
    unsigned long long *list;    // [pool_chunks] closed chunks: chunk | bin << 32 | count << 40
    unsigned long long *sorted;  // [pool_chunks] the same entries ordered by bin
    int *ctr;                    // [BC_WORDS]
    int *seg;                    // [K] first packed slot of community c: aoff[start[c]]
    long long pool_chunks;
    int shift;                   // window of node v: v >> shift
    int nbins;                   // windows (<= BIN_MAX)
    int near;                    // arcs with |v - u| < near are gathered directly
};

// Per-warp staging in shared memory: records, counts, current chunk and its fill per bin.
struct WarpBins {
    unsigned long long *buf;  // [nbins][BIN_SLOTS]
    int *cnt;                 // [nbins]
    int *chunk;               // [nbins], -1: none open
    int *fill;                // [nbins]
};

__host__ __device__ __forceinline__ int bin_smem_bytes_per_warp(int nbins)
{
    return (nbins * BIN_SLOTS * 8 + 3 * nbins * 4 + 15) & ~15;
}

__device__ __forceinline__ void bin_close(const BinArgs &ba, int ch, int b, int count)
{
    const int i = atomicAdd(&ba.ctr[BC_LIST], 1);
    if (i >= ba.pool_chunks) {  // cannot happen with the pool's sizing
        atomicOr(&ba.ctr[BC_ERR], 1);
        return;
    }
    ba.list[i] = (unsigned long long)(unsigned)ch | ((unsigned long long)b << 32) | ((unsigned long long)count << 40);
    atomicAdd(&ba.ctr[BC_BIN_COUNT + b], 1);
}

// Lane 0: make sure bin b has an open chunk with room for `need` records.
__device__ __forceinline__ void bin_room(const BinArgs &ba, const WarpBins &wb, int b, int need)
{
    if (wb.chunk[b] >= 0 && wb.fill[b] + need <= BIN_CHUNK) return;
    if (wb.chunk[b] >= 0) bin_close(ba, wb.chunk[b], b, wb.fill[b]);
    const int ch = atomicAdd(&ba.ctr[BC_CHUNKS], 1);
    wb.chunk[b] = ch;
    wb.fill[b] = 0;
    if (ch >= ba.pool_chunks) atomicOr(&ba.ctr[BC_ERR], 1);  // cannot happen with the pool's sizing
}

// Writes n <= 32 staged records of bin b (from its front) to the bin's chunk
// and moves the rest of the staging buffer down.  Whole warp.
__device__ __forceinline__ void bin_flush(const BinArgs &ba, const WarpBins &wb, int b, int n, int lane)
{
    if (lane == 0) bin_room(ba, wb, b, n);
    __syncwarp();
    const int ch = wb.chunk[b], f = wb.fill[b], total = wb.cnt[b];
    unsigned long long *src = wb.buf + b * BIN_SLOTS;
    if (lane < n && ch < ba.pool_chunks) __stcs(&ba.pool[(size_t)ch * BIN_CHUNK + f + lane], src[lane]);
    const int rest = total - n;
    unsigned long long keep = 0;
    if (lane < rest) keep = src[n + lane];
    __syncwarp();
    if (lane < rest) src[lane] = keep;
    if (lane == 0) {
        wb.fill[b] = f + n;
        wb.cnt[b] = rest;
    }
    __syncwarp();
}

// Stages one record per lane that has one (far), then flushes every bin that
// holds at least BIN_FLUSH records.  Whole warp.
__device__ __forceinline__ void bin_push(const BinArgs &ba, const WarpBins &wb, bool far, int b,
                                         unsigned long long rec, int lane)
{
    const unsigned fm = __ballot_sync(0xffffffffu, far);
    if (!fm) return;
    unsigned peers = 0;
    int base = 0;
    if (far) {
        peers = __match_any_sync(fm, b);
        base = wb.cnt[b];
        wb.buf[b * BIN_SLOTS + base + __popc(peers & ((1u << lane) - 1u))] = rec;
    }
    __syncwarp();
    if (far && lane == __ffs(peers) - 1) wb.cnt[b] = base + __popc(peers);
    __syncwarp();
    for (;;) {
        const unsigned full = __ballot_sync(0xffffffffu, lane < ba.nbins && wb.cnt[lane] >= BIN_FLUSH);
        if (!full) break;
        bin_flush(ba, wb, __ffs(full) - 1, BIN_FLUSH, lane);
    }
}

// End of a warp's work: writes what is staged and closes every open chunk.
__device__ __forceinline__ void bin_finish(const BinArgs &ba, const WarpBins &wb, int lane)
{
    for (int b = 0; b < ba.nbins; ++b) {
        if (wb.cnt[b] > 0) bin_flush(ba, wb, b, wb.cnt[b], lane);
        if (lane == 0 && wb.chunk[b] >= 0) bin_close(ba, wb.chunk[b], b, wb.fill[b]);
        __syncwarp();
    }
}

// Gathers (or bins) the labels of arcs [e_lo, e_hi) of a run of community c
// (loc(e) is the CSR index of arc e; uref a member of the run, the reference
// point of the nearness test) and packs the gathered labels != c into c's
// segment at cbase.
template <class LOC>
__device__ __forceinline__ void expand_range_bin(unsigned e_lo, unsigned e_hi, int c, unsigned cbase, int uref,
                                                 LOC loc, const int *__restrict__ col,
                                                 const int *__restrict__ labels, int *inter, int *__restrict__ nbr,
                                                 unsigned long long keep, int lane, const BinArgs &ba,
                                                 const WarpBins &wb)
{
    const unsigned lt = (1u << lane) - 1u;
    for (unsigned e0 = e_lo; e0 < e_hi; e0 += 32u * EXPAND_UNROLL) {
        int v[EXPAND_UNROLL], lab[EXPAND_UNROLL];
        bool far[EXPAND_UNROLL];
#pragma unroll
        for (int k = 0; k < EXPAND_UNROLL; ++k) {
            const unsigned e = e0 + lane + 32u * k;
            v[k] = e < e_hi ? __ldcs(&col[loc(e)]) : -1;
        }
#pragma unroll
        for (int k = 0; k < EXPAND_UNROLL; ++k) {
            far[k] = v[k] >= 0 && (long long)abs(v[k] - uref) >= (long long)ba.near;
            lab[k] = (v[k] >= 0 && !far[k]) ? ld_hint(&labels[v[k]], keep) : -1;
        }
        unsigned msk[EXPAND_UNROLL];
        int tot = 0;
#pragma unroll
        for (int k = 0; k < EXPAND_UNROLL; ++k) {
            msk[k] = __ballot_sync(0xffffffffu, lab[k] >= 0 && lab[k] != c);
            tot += __popc(msk[k]);
        }
        if (tot) {
            int pos = 0;
            if (lane == 0) pos = atomicAdd(&inter[c], tot);
            unsigned at = cbase + (unsigned)__shfl_sync(0xffffffffu, pos, 0);
#pragma unroll
            for (int k = 0; k < EXPAND_UNROLL; ++k) {
                if ((msk[k] >> lane) & 1u) __stcs(&nbr[at + __popc(msk[k] & lt)], lab[k]);
                at += __popc(msk[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < EXPAND_UNROLL; ++k)
            bin_push(ba, wb, far[k], far[k] ? (v[k] >> ba.shift) : 0,
                     ((unsigned long long)(unsigned)c << 32) | (unsigned)v[k], lane);
    }
}

// Phase A of the binned path: k_expand's walk over member positions, with the
// far arcs binned instead of gathered.
__global__ void __launch_bounds__(EXPAND_THREADS) k_expand_bin(const long long *__restrict__ row_ptr,
                                                               const int *__restrict__ col,
                                                               const int *__restrict__ labels,
                                                               const int *__restrict__ members,
                                                               const unsigned *__restrict__ aoff,
                                                               const int *__restrict__ start, long long n,
                                                               int *inter, int *__restrict__ nbr, const int *status,
                                                               Shard own, BinArgs ba)
{
    __shared__ unsigned offs_s[EXPAND_THREADS / 32][33];
    __shared__ long long rs_s[EXPAND_THREADS / 32][32];
    __shared__ int cw_s[EXPAND_THREADS / 32][32];
    extern __shared__ __align__(16) unsigned char bin_sm[];
    if (*status) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned *offw = offs_s[w];
    long long *rsw = rs_s[w];
    int *cw = cw_s[w];
    unsigned char *mine = bin_sm + (size_t)w * bin_smem_bytes_per_warp(ba.nbins);
    WarpBins wb;
    wb.buf = (unsigned long long *)mine;
    wb.cnt = (int *)(mine + (size_t)ba.nbins * BIN_SLOTS * 8);
    wb.chunk = wb.cnt + ba.nbins;
    wb.fill = wb.chunk + ba.nbins;
    if (lane < ba.nbins) {
        wb.cnt[lane] = 0;
        wb.chunk[lane] = -1;
        wb.fill[lane] = 0;
    }
    __syncwarp();
    const unsigned long long keep = l2_policy_evict_last();
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long p0 = ((long long)blockIdx.x * (blockDim.x >> 5) + w) * 32; p0 < n; p0 += nwarps * 32) {
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
        int cur_c = -1;
        unsigned cbase = 0;
        if (__popc(segs) <= EXPAND_MAX_SEGS) {
            unsigned rem = segs;
            while (rem) {
                const int lo = __ffs(rem) - 1;
                rem &= rem - 1;
                const int hi = rem ? __ffs(rem) - 1 : nm;
                const unsigned e_lo = offw[lo], e_hi = offw[hi];
                const int uref = __shfl_sync(0xffffffffu, u, lo);
                if (e_lo == e_hi) continue;
                const int c = cw[lo];
                if (!own.owns(c)) continue;
                if (c != cur_c) {
                    cur_c = c;
                    if (lane == 0) cbase = __ldg(&aoff[__ldg(&start[c])]);
                    cbase = __shfl_sync(0xffffffffu, cbase, 0);
                }
                const long long cs = rsw[lo] - (long long)e_lo;  // CSR index of arc e is cs + e
                expand_range_bin(e_lo, e_hi, c, cbase, uref, [cs](unsigned e) { return cs + (long long)e; }, col,
                                 labels, inter, nbr, keep, lane, ba, wb);
            }
        } else {
            while (runs) {
                const int m_lo = __ffs(runs) - 1;
                runs &= runs - 1;
                const int m_hi = runs ? __ffs(runs) - 1 : nm;
                const unsigned e_lo = offw[m_lo], e_hi = offw[m_hi];
                const int uref = __shfl_sync(0xffffffffu, u, m_lo);
                if (e_lo == e_hi) continue;
                const int c = cw[m_lo];
                if (!own.owns(c)) continue;
                if (lane == 0) cbase = __ldg(&aoff[__ldg(&start[c])]);
                cbase = __shfl_sync(0xffffffffu, cbase, 0);
                expand_range_bin(
                    e_lo, e_hi, c, cbase, uref,
                    [=](unsigned e) {
                        const int o = m_lo + upper_bound_smem(offw + m_lo, m_hi - m_lo, e) - 1;
                        return rsw[o] + (long long)(e - offw[o]);
                    },
                    col, labels, inter, nbr, keep, lane, ba, wb);
            }
        }
        __syncwarp();
    }
    bin_finish(ba, wb, lane);
}

// Orders the closed chunks by bin (a counting sort over the few bins) and
// records each community's first packed slot.
__global__ void k_bin_order(BinArgs ba, const unsigned *__restrict__ aoff, const int *__restrict__ start, int K,
                            int *status)
{
    __shared__ int off_s[BIN_MAX];
    if (*(volatile int *)status) return;
    if (ba.ctr[BC_ERR]) {  // the pool overflowed (a sizing error): fail the call
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, 8);
        return;
    }
    const int L = min(ba.ctr[BC_LIST], (int)min(ba.pool_chunks, (long long)INT_MAX));
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < ba.nbins; ++b) {
            off_s[b] = acc;
            acc += ba.ctr[BC_BIN_COUNT + b];
        }
    }
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const long long top = max((long long)L, (long long)K);
    for (long long i0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < top; i0 += stride) {
        const long long i = i0 + lane;
        if (i < K) ba.seg[i] = __ldg(&aoff[__ldg(&start[i])]);
        const bool has = i < L;
        const unsigned act = __ballot_sync(0xffffffffu, has);
        if (!has) continue;
        const unsigned long long ent = ba.list[i];
        const int b = (int)((ent >> 32) & 0xFFu);
        const unsigned peers = __match_any_sync(act, b);
        const int leader = __ffs(peers) - 1;
        int pos = 0;
        if (lane == leader) pos = atomicAdd(&ba.ctr[BC_BIN_FILL + b], __popc(peers));
        pos = __shfl_sync(peers, pos, leader) + __popc(peers & ((1u << lane) - 1u));
        ba.sorted[off_s[b] + pos] = ent;
    }
}

constexpr int RESOLVE_THREADS = 256;

// Phase A, second half: the binned records, window by window.  Warp g takes
// the chunks g, g + W, g + 2W, ... of the bin-ordered list, so all warps move
// through the windows together and the labels they gather come from one or two
// windows of the label array at a time.  Each label != c is appended to c's
// packed run; the lanes of a warp that hold the same community take their
// slots with one atomic.
__global__ void __launch_bounds__(RESOLVE_THREADS) k_resolve(BinArgs ba, const int *__restrict__ labels,
                                                             int *inter, int *__restrict__ nbr, const int *status)
{
    if (*status) return;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int L = min(ba.ctr[BC_LIST], (int)min(ba.pool_chunks, (long long)INT_MAX));
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    const unsigned long long keep = l2_policy_evict_last();
    for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < L; i += nwarps) {
        const unsigned long long ent = __ldg(&ba.sorted[i]);
        const long long ch = (long long)(ent & 0xFFFFFFFFull);
        const int cnt = (int)((ent >> 40) & 0x1FFu);
        if (ch >= ba.pool_chunks) continue;  // flagged by the binning kernel
        const unsigned long long *rec = ba.pool + (size_t)ch * BIN_CHUNK;
        constexpr int U = BIN_CHUNK / 32;
        int c[U], d[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int j = lane + 32 * k;
            c[k] = -1;
            d[k] = -1;
            if (j < cnt) {
                const unsigned long long r = __ldcs(&rec[j]);
                c[k] = (int)(r >> 32);
                d[k] = (int)(r & 0xFFFFFFFFull);  // the far node v for now
            }
        }
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (c[k] >= 0) d[k] = ld_hint(&labels[d[k]], keep);
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const bool cut = c[k] >= 0 && d[k] != c[k];
            const unsigned cm = __ballot_sync(0xffffffffu, cut);
            if (!cm) continue;
            if (cut) {
                const unsigned peers = __match_any_sync(cm, c[k]);
                const int leader = __ffs(peers) - 1;
                int pos = 0;
                if (lane == leader) pos = atomicAdd(&inter[c[k]], __popc(peers));
                pos = __shfl_sync(peers, pos, leader) + __popc(peers & lt);
                __stcs(&nbr[(unsigned)__ldg(&ba.seg[c[k]]) + (unsigned)pos], d[k]);
            }
        }
    }
}
