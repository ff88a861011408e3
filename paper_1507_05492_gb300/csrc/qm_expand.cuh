// qm_expand.cuh -- phase A of the two-phase scoring pipeline (the far-end
// label gathers), shared by the single-partition pipeline (k_expand in
// qm_kernels.cu) and the batched pipeline over many candidate partitions
// (qm_batched.cu).
#pragma once

#include <climits>

#include "qm_community.cuh"

namespace qm {
using namespace qmk;

// Phase A: for each member position p (community order) the labels of the
// neighbours of members[p] are looked up.  A warp takes 32 consecutive member
// positions; they hold one or more runs of members of one community each.  For
// a run of community c the warp spreads the run's arcs over its lanes,
// gathers the neighbour labels, and packs those != c at the front of c's arc
// segment: a ballot gives each lane its place and one atomic on inter[c]
// reserves the room.  inter[c] ends as the number of cut arcs of c,
// |E_c^out| (Sec. II-B.3), and the packed run never outgrows the segment,
// whose length is the volume of c.  No shared-memory table is needed, so the
// kernel runs at full occupancy.
//
// Locating the CSR entry of the e-th arc of a run: when the 32 members form a
// few segments of consecutive node ids (the common case on a graph loaded
// with QM_REORDER), a segment's rows are adjacent in the CSR and its arcs are
// one contiguous range; otherwise a search over the members' arc offsets
// finds the member of each arc.
constexpr int EXPAND_THREADS = 256;

// Community ownership of a sharded call (the decomposition of Sec. III-A:
// community c belongs to process c mod P).  Unsharded calls pass P = 1.
struct Shard {
    int r;  // this shard
    int p;  // number of shards
    __device__ __forceinline__ bool owns(int c) const { return p == 1 || c % p == r; }
};
constexpr int EXPAND_UNROLL = 8;
constexpr int EXPAND_MAX_SEGS = 6;

// Edge weights of a weighted graph (float32, 0 or in [2^-20, 2^20)) as exact
// fixed-point integers: w * 2^43 (an integer below 2^63).
__device__ __forceinline__ unsigned long long w_fixed(float w) { return __float2ull_rn(w * 8796093022208.0f); }

// Packed copy of the labels for the far-end gathers: three 21-bit labels per
// 64-bit word (label ids below 2^21), 8/3 bytes a node instead of 4.  The
// gathers of the expand phase land at random in the label array; a smaller
// array leaves a larger share of it in L2.
constexpr int PACK_BITS = 21;
constexpr long long PACK_MAX_K = 1LL << PACK_BITS;

__device__ __forceinline__ int ld_label3(const unsigned long long *plab, int v, unsigned long long pol)
{
    const unsigned q = (unsigned)v / 3u;
    const unsigned r = (unsigned)v - 3u * q;
    unsigned long long w;
    asm("ld.global.nc.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(w) : "l"(plab + q), "l"(pol));
    return (int)((w >> (PACK_BITS * r)) & 0x1FFFFFull);
}

// Block encoding of the labels of a renumbered graph, for the far-end gathers
// (built per call by k_pack_blocks).  Along the stored node order the labels
// of a partition that follows the graph's clusters change rarely, so 16
// consecutive nodes mostly carry one or two labels: one 64-bit word per 16
// nodes holds labels A ([0, 21)) and B ([21, 42)) and a 16-bit mask ([42, 58))
// whose bit i selects B for the block's node i.  A block of three or more
// labels has bit 63 set and, in bits [0, 32), the offset (in 32-bit words from
// the array's start) of its 16 labels in the exception area after the block
// words.  Half a byte a node instead of the packed copy's 8/3, so that the
// whole encoding of 10^8 nodes stays in L2.
constexpr int BLK_NODES = 16;

__device__ __forceinline__ int ld_label_blk(const unsigned long long *blab, int v, unsigned long long pol)
{
    unsigned long long w;
    asm("ld.global.nc.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(w) : "l"(blab + ((unsigned)v >> 4)), "l"(pol));
    const unsigned i = (unsigned)v & 15u;
    if (!(w >> 63)) return (int)((w >> (((w >> (42u + i)) & 1ull) ? PACK_BITS : 0)) & 0x1FFFFFull);
    return ld_hint((const int *)blab + ((unsigned)w + i), pol);
}

// Label sources of the far-end gathers: the labels as given, the packed copy,
// or the block encoding.
enum { LAB_PLAIN = 0, LAB_PACK3 = 1, LAB_BLOCKS = 2 };

// Gathers the labels of arcs [e_lo, e_hi) of a run of community c (loc(e) is
// the CSR index of arc e; plab is the packed copy or the block encoding, as
// LAB says), counts those != c in inter[c] (the cut arcs of c)
// and packs them into c's segment at cbase; with HI only the labels above c are
// packed (each unordered pair of communities is counted by its smaller id), and
// hi[c] counts them.  On a weighted graph (WT) the arc weights travel with the
// packed labels (nbrw) and each lane sums the fixed-point weights of its intra
// and cut arcs.
template <bool WT, int LAB, bool HI, class LOC>
__device__ __forceinline__ void expand_range(unsigned e_lo, unsigned e_hi, int c, unsigned cbase, LOC loc,
                                             const int *__restrict__ col, const int *__restrict__ labels,
                                             const unsigned long long *__restrict__ plab,
                                             int *inter, int *hi, int *__restrict__ nbr, unsigned long long keep,
                                             int lane, const float *__restrict__ wt, float *__restrict__ nbrw,
                                             u128 &w_in, u128 &w_out)
{
    const unsigned lt = (1u << lane) - 1u;
    for (unsigned e0 = e_lo; e0 < e_hi; e0 += 32u * EXPAND_UNROLL) {
        int lab[EXPAND_UNROLL];
        float wv[EXPAND_UNROLL];
#pragma unroll
        for (int k = 0; k < EXPAND_UNROLL; ++k) {
            const unsigned e = e0 + lane + 32u * k;
            lab[k] = e < e_hi ? __ldcs(&col[loc(e)]) : -1;
            if (WT) wv[k] = e < e_hi ? __ldcs(&wt[loc(e)]) : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < EXPAND_UNROLL; ++k)
            if (lab[k] >= 0)
                lab[k] = LAB == LAB_BLOCKS  ? ld_label_blk(plab, lab[k], keep)
                         : LAB == LAB_PACK3 ? ld_label3(plab, lab[k], keep)
                                            : ld_hint(&labels[lab[k]], keep);
        if (WT) {
#pragma unroll
            for (int k = 0; k < EXPAND_UNROLL; ++k)
                if (lab[k] >= 0) {
                    const unsigned long long f = w_fixed(wv[k]);
                    if (lab[k] == c) w_in += f; else w_out += f;
                }
        }
        unsigned msk[EXPAND_UNROLL];
        int tot = 0, cut = 0;
#pragma unroll
        for (int k = 0; k < EXPAND_UNROLL; ++k) {
            if (HI) cut += __popc(__ballot_sync(0xffffffffu, lab[k] >= 0 && lab[k] != c));
            msk[k] = __ballot_sync(0xffffffffu, HI ? lab[k] > c : (lab[k] >= 0 && lab[k] != c));
            tot += __popc(msk[k]);
        }
        if (HI && cut && lane == 0) atomicAdd(&inter[c], cut);
        if (tot == 0) continue;
        int pos = 0;
        if (lane == 0) pos = atomicAdd(HI ? &hi[c] : &inter[c], tot);
        unsigned at = cbase + (unsigned)__shfl_sync(0xffffffffu, pos, 0);
#pragma unroll
        for (int k = 0; k < EXPAND_UNROLL; ++k) {
            if ((msk[k] >> lane) & 1u) {
                __stcs(&nbr[at + __popc(msk[k] & lt)], lab[k]);
                if (WT) __stcs(&nbrw[at + __popc(msk[k] & lt)], wv[k]);
            }
            at += __popc(msk[k]);
        }
    }
}

// Adds a warp's intra and cut weight sums of community c to its limbs (wl:
// six words per community, intra then cut).
__device__ __forceinline__ void flush_weights(unsigned long long *wl, int c, u128 w_in, u128 w_out, int lane)
{
    for (int d = 16; d > 0; d >>= 1) {
        w_in += shfl_down_u128(w_in, d);
        w_out += shfl_down_u128(w_out, d);
    }
    if (lane == 0) {
        if (w_in) limbs_add(wl + (size_t)c * 6, (i128)w_in);
        if (w_out) limbs_add(wl + (size_t)c * 6 + 3, (i128)w_out);
    }
}

// One warp's share of phase A: the 32 member positions from p0 (fewer at the
// end), their runs of one community each, and the gathers of those runs'
// arcs.  offw (33 entries), rsw and cw (32 each) are the warp's shared-memory
// slices.
template <bool WT, int LAB, bool HI>
__device__ __forceinline__ void expand_chunk(long long p0, long long n, const long long *__restrict__ row_ptr,
                                             const int *__restrict__ col, const int *__restrict__ labels,
                                             const unsigned long long *__restrict__ plab,
                                             const int *__restrict__ members, const unsigned *__restrict__ aoff,
                                             const int *__restrict__ start, int *inter, int *inter_hi,
                                             int *__restrict__ nbr, Shard own, const float *__restrict__ wt,
                                             float *__restrict__ nbrw, unsigned long long *wl, unsigned *offw,
                                             long long *rsw, int *cw, unsigned long long keep, int lane)
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
    int cur_c = -1;
    unsigned cbase = 0;
    if (__popc(segs) <= EXPAND_MAX_SEGS) {
        unsigned rem = segs;
        while (rem) {
            const int lo = __ffs(rem) - 1;
            rem &= rem - 1;
            const int hi = rem ? __ffs(rem) - 1 : nm;
            const unsigned e_lo = offw[lo], e_hi = offw[hi];
            if (e_lo == e_hi) continue;
            const int c = cw[lo];
            if (!own.owns(c)) continue;
            if (c != cur_c) {
                cur_c = c;
                if (lane == 0) cbase = __ldg(&aoff[__ldg(&start[c])]);
                cbase = __shfl_sync(0xffffffffu, cbase, 0);
            }
            const long long cs = rsw[lo] - (long long)e_lo;  // CSR index of arc e is cs + e
            u128 w_in = 0, w_out = 0;
            expand_range<WT, LAB, HI>(e_lo, e_hi, c, cbase, [cs](unsigned e) { return cs + (long long)e; }, col,
                                       labels, plab, inter, inter_hi, nbr, keep, lane, wt, nbrw, w_in, w_out);
            if (WT) flush_weights(wl, c, w_in, w_out, lane);
        }
    } else {
        while (runs) {
            const int m_lo = __ffs(runs) - 1;
            runs &= runs - 1;
            const int m_hi = runs ? __ffs(runs) - 1 : nm;
            const unsigned e_lo = offw[m_lo], e_hi = offw[m_hi];
            if (e_lo == e_hi) continue;
            const int c = cw[m_lo];
            if (!own.owns(c)) continue;
            if (lane == 0) cbase = __ldg(&aoff[__ldg(&start[c])]);
            cbase = __shfl_sync(0xffffffffu, cbase, 0);
            u128 w_in = 0, w_out = 0;
            expand_range<WT, LAB, HI>(
                e_lo, e_hi, c, cbase,
                [=](unsigned e) {
                    const int o = m_lo + upper_bound_smem(offw + m_lo, m_hi - m_lo, e) - 1;
                    return rsw[o] + (long long)(e - offw[o]);
                },
                col, labels, plab, inter, inter_hi, nbr, keep, lane, wt, nbrw, w_in, w_out);
            if (WT) flush_weights(wl, c, w_in, w_out, lane);
        }
    }
    __syncwarp();
}


// ---------------------------------------------------------------- half-edge gathers
//
// On a graph that also holds its upper rows (each node's arcs to itself and to
// higher node ids, a self-loop stored as ~u), every undirected edge is gathered
// once, from its lower end.  An arc of a member of c to community l != c puts
// one entry into the run of the smaller of the two ids: l packed into c's
// segment when l > c, c appended to l's segment (through l's run cursor and
// segment base cbase[l]) when l < c; with FULL both.  Arcs inside c add 2 (a
// self-loop 1) to same2[c], so E_c^out = vol(c) - same2[c] and the runs hold the
// same multisets as gathering every arc from both ends.
template <bool PACK, bool FULL, class LOC>
__device__ __forceinline__ void expand_range_half(unsigned e_lo, unsigned e_hi, int c, unsigned cbase_c, LOC loc,
                                                  const int *__restrict__ up_col, const int *__restrict__ labels,
                                                  const unsigned long long *__restrict__ plab, int *same2,
                                                  int *cursor, const unsigned *__restrict__ cbase,
                                                  int *__restrict__ nbr, unsigned long long keep, int lane)
{
    const unsigned lt = (1u << lane) - 1u;
    for (unsigned e0 = e_lo; e0 < e_hi; e0 += 32u * EXPAND_UNROLL) {
        int lab[EXPAND_UNROLL];
        unsigned intra = 0;
#pragma unroll
        for (int k = 0; k < EXPAND_UNROLL; ++k) {
            const unsigned e = e0 + lane + 32u * k;
            lab[k] = e < e_hi ? __ldcs(&up_col[loc(e)]) : INT_MIN;
        }
#pragma unroll
        for (int k = 0; k < EXPAND_UNROLL; ++k) {
            if (lab[k] == INT_MIN) {
                lab[k] = -1;
            } else if (lab[k] < 0) {  // a self-loop: one arc inside c
                intra += 1u;
                lab[k] = -1;
            } else {
                lab[k] = PACK ? ld_label3(plab, lab[k], keep) : ld_hint(&labels[lab[k]], keep);
                if (lab[k] == c) {
                    intra += 2u;
                    lab[k] = -1;
                }
            }
        }
        intra = __reduce_add_sync(0xffffffffu, intra);
        if (intra && lane == 0) atomicAdd(&same2[c], (int)intra);
        // entries for c's own run
        unsigned msk[EXPAND_UNROLL];
        int tot = 0;
#pragma unroll
        for (int k = 0; k < EXPAND_UNROLL; ++k) {
            msk[k] = __ballot_sync(0xffffffffu, FULL ? lab[k] >= 0 : lab[k] > c);
            tot += __popc(msk[k]);
        }
        if (tot) {
            int pos = 0;
            if (lane == 0) pos = atomicAdd(&cursor[c], tot);
            unsigned at = cbase_c + (unsigned)__shfl_sync(0xffffffffu, pos, 0);
#pragma unroll
            for (int k = 0; k < EXPAND_UNROLL; ++k) {
                if ((msk[k] >> lane) & 1u) __stcs(&nbr[at + __popc(msk[k] & lt)], lab[k]);
                at += __popc(msk[k]);
            }
        }
        // c appended to the runs of the smaller neighbouring ids (FULL: all),
        // lanes of one destination merged into one cursor update; all cursor
        // updates and segment bases of the step are in flight at once
        unsigned peers[EXPAND_UNROLL];
        int base[EXPAND_UNROLL];
        unsigned cb[EXPAND_UNROLL];
#pragma unroll
        for (int k = 0; k < EXPAND_UNROLL; ++k) {
            const bool rem = FULL ? lab[k] >= 0 : (lab[k] >= 0 && lab[k] < c);
            const unsigned rm = __ballot_sync(0xffffffffu, rem);
            peers[k] = rem ? __match_any_sync(rm, lab[k]) : 0u;
        }
#pragma unroll
        for (int k = 0; k < EXPAND_UNROLL; ++k) {
            base[k] = 0;
            if (peers[k] && lane == __ffs(peers[k]) - 1) base[k] = atomicAdd(&cursor[lab[k]], __popc(peers[k]));
            if (peers[k]) cb[k] = __ldg(&cbase[lab[k]]);
        }
#pragma unroll
        for (int k = 0; k < EXPAND_UNROLL; ++k) {
            if (!peers[k]) continue;
            const int b = __shfl_sync(peers[k], base[k], __ffs(peers[k]) - 1);
            nbr[cb[k] + (unsigned)(b + __popc(peers[k] & lt))] = c;
        }
    }
}

// One warp's share of the half-edge phase A: as expand_chunk, over the
// members' upper rows (up_ptr / up_col), with the in-chunk arc offsets summed
// in the warp and each community's segment base read from cbase.
template <bool PACK, bool FULL>
__device__ __forceinline__ void expand_chunk_half(long long p0, long long n, const long long *__restrict__ up_ptr,
                                                  const int *__restrict__ up_col, const int *__restrict__ labels,
                                                  const unsigned long long *__restrict__ plab,
                                                  const int *__restrict__ members, const unsigned *__restrict__ cbase,
                                                  int *same2, int *cursor, int *__restrict__ nbr, unsigned *offw,
                                                  long long *rsw, int *cw, unsigned long long keep, int lane)
{
    const int nm = (int)min(32LL, n - p0);
    int u = -2;
    unsigned d = 0;
    if (lane < nm) {
        u = __ldcs(&members[p0 + lane]);
        rsw[lane] = __ldg(&up_ptr[u]);
        d = (unsigned)(__ldg(&up_ptr[u + 1]) - rsw[lane]);
        cw[lane] = ld_hint(&labels[u], keep);
    }
    unsigned inc = d;
#pragma unroll
    for (int s2 = 1; s2 < 32; s2 <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, inc, s2);
        if (lane >= s2) inc += t;
    }
    if (lane < nm) offw[lane] = inc - d;
    if (lane == nm - 1) offw[nm] = inc;
    __syncwarp();
    const int u_prev = __shfl_up_sync(0xffffffffu, u, 1);
    const bool valid = lane < nm;
    const bool newrun = valid && (lane == 0 || cw[lane] != cw[lane - 1]);
    unsigned runs = __ballot_sync(0xffffffffu, newrun);
    const unsigned segs = __ballot_sync(0xffffffffu, newrun || (valid && u != u_prev + 1));
    if (__popc(segs) <= EXPAND_MAX_SEGS) {
        unsigned rem = segs;
        while (rem) {
            const int lo = __ffs(rem) - 1;
            rem &= rem - 1;
            const int hi = rem ? __ffs(rem) - 1 : nm;
            const unsigned e_lo = offw[lo], e_hi = offw[hi];
            if (e_lo == e_hi) continue;
            const int c = cw[lo];
            const long long cs = rsw[lo] - (long long)e_lo;  // upper-row index of arc e is cs + e
            expand_range_half<PACK, FULL>(e_lo, e_hi, c, __ldg(&cbase[c]),
                                          [cs](unsigned e) { return cs + (long long)e; }, up_col, labels, plab,
                                          same2, cursor, cbase, nbr, keep, lane);
        }
    } else {
        while (runs) {
            const int m_lo = __ffs(runs) - 1;
            runs &= runs - 1;
            const int m_hi = runs ? __ffs(runs) - 1 : nm;
            const unsigned e_lo = offw[m_lo], e_hi = offw[m_hi];
            if (e_lo == e_hi) continue;
            const int c = cw[m_lo];
            expand_range_half<PACK, FULL>(
                e_lo, e_hi, c, __ldg(&cbase[c]),
                [=](unsigned e) {
                    const int o = m_lo + upper_bound_smem(offw + m_lo, m_hi - m_lo, e) - 1;
                    return rsw[o] + (long long)(e - offw[o]);
                },
                up_col, labels, plab, same2, cursor, cbase, nbr, keep, lane);
        }
    }
    __syncwarp();
}

}  // namespace qm
