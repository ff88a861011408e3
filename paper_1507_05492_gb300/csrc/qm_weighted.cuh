// qm_weighted.cuh -- Eqs. (8)-(9) on weighted graphs (included by qm_kernels.cu).
//
// The paper defines Q and Qds for unweighted graphs and notes for the
// weighted case that the densities d_c and d_ci,cj keep the unweighted edge
// counts (so that they stay at most 1) while the other edge amounts become
// weight sums:
//   Q_w   = sum_c [ W_c^in / W - ((2 W_c^in + W_c^out) / (2W))^2 ]
//   Qds_w = sum_ci [ W_ci^in / W d_ci - ((2 W_ci^in + W_ci^out) / (2W) d_ci)^2
//                    - sum_{cj != ci} W_ci,cj / (2W) d_ci,cj ]
// Weights are float32 (0 or in [2^-20, 2^20)); each is an exact fixed-point
// integer w * 2^43, so every weight sum below is exact:
//   - k_expand<true> sums each community's intra-arc weights (2 W_c^in) and
//     cut-arc weights (W_c^out) into three-limb integers, and packs the cut
//     arcs' weights beside their labels;
//   - k_count_w counts each community's run in the shared-memory table
//     (|E_ci,cj| for every neighbour cj) and then, in a second pass over the
//     run, adds for every cut arc (weight w, neighbour cj) the exact product
//     w * |E_ci,cj| * Rcp_cj, so that P_i = sum_j W_ij |E_ij| / |c_j| is a
//     256-bit integer (scale 2^171);
//   - k_score_terms_w forms the FP64 terms of each community once from these
//     integers and adds them in fixed point (Q_w into its own accumulator).
// The six measures of Sec. II-B.3 keep their unweighted counts.
//
// Included inside namespace qm of qm_kernels.cu, after the helpers it uses.

struct U256 {
    unsigned long long w[4];
};

__device__ __forceinline__ void u256_zero(U256 &a) { a.w[0] = a.w[1] = a.w[2] = a.w[3] = 0ull; }

__device__ __forceinline__ void u256_add(U256 &a, const U256 &b)
{
    unsigned long long c = 0ull;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned long long s = a.w[k] + b.w[k];
        const unsigned long long c1 = s < a.w[k] ? 1ull : 0ull;
        const unsigned long long t = s + c;
        const unsigned long long c2 = t < s ? 1ull : 0ull;
        a.w[k] = t;
        c = c1 + c2;
    }
}

// a += x * r for x < 2^96 and a 128-bit reciprocal r (the product is below 2^224).
__device__ __forceinline__ void u256_mac(U256 &a, u128 x, const Rcp &r)
{
    const unsigned long long x0 = (unsigned long long)x, x1 = (unsigned long long)(x >> 64);
    const unsigned long long r0 = r.lo, r1 = r.hi;
    const u128 p00 = (u128)x0 * r0, p01 = (u128)x0 * r1, p10 = (u128)x1 * r0, p11 = (u128)x1 * r1;
    U256 p;
    p.w[0] = (unsigned long long)p00;
    u128 t = (p00 >> 64) + (u128)(unsigned long long)p01 + (u128)(unsigned long long)p10;
    p.w[1] = (unsigned long long)t;
    t = (t >> 64) + (p01 >> 64) + (p10 >> 64) + (u128)(unsigned long long)p11;
    p.w[2] = (unsigned long long)t;
    p.w[3] = (unsigned long long)((t >> 64) + (p11 >> 64));
    u256_add(a, p);
}

__device__ __forceinline__ double u256_to_double(const U256 &a)
{
    double r = (double)a.w[3];
    r = __dadd_rn(__dmul_rn(r, 18446744073709551616.0), (double)a.w[2]);
    r = __dadd_rn(__dmul_rn(r, 18446744073709551616.0), (double)a.w[1]);
    r = __dadd_rn(__dmul_rn(r, 18446744073709551616.0), (double)a.w[0]);
    return r;  // a, rounded (its value times 2^0)
}

// Count of `key` in the table (0 when absent).
__device__ __forceinline__ unsigned long long tab_count(const SmemTable &t, unsigned key)
{
    const unsigned long long tag = (unsigned long long)(key + 1u) << 32;
    unsigned h = tab_hash(key, t.cap);
    for (int probe = 0; probe < t.cap; ++probe) {
        if (!QM_CHK(h, t.cap, 11)) return 0ull;
        const unsigned long long s = ((volatile unsigned long long *)t.slot)[h];
        if ((s & 0xFFFFFFFF00000000ull) == tag) return s & 0xFFFFFFFFull;
        if (s == 0ull) return 0ull;
        h = (h + 1u == (unsigned)t.cap) ? 0u : h + 1u;
    }
    return 0ull;
}

// Block totals of (slots, cnt2, P) delivered to thread 0 (6 words per warp in red).
__device__ __forceinline__ void group_totals_w(unsigned long long &slots, unsigned long long &cnt2, U256 &P,
                                               unsigned long long *red)
{
    slots = warp_sum_u64(slots);
    cnt2 = warp_sum_u64(cnt2);
    for (int d = 16; d > 0; d >>= 1) {
        U256 o;
#pragma unroll
        for (int k = 0; k < 4; ++k) o.w[k] = __shfl_down_sync(0xffffffffu, P.w[k], d);
        u256_add(P, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    block_sync();
    if (lane == 0) {
        red[6 * wid] = slots;
        red[6 * wid + 1] = cnt2;
#pragma unroll
        for (int k = 0; k < 4; ++k) red[6 * wid + 2 + k] = P.w[k];
    }
    block_sync();
    if (threadIdx.x == 0)
        for (int w = 1; w < nw; ++w) {
            slots += red[6 * w];
            cnt2 += red[6 * w + 1];
            U256 o;
#pragma unroll
            for (int k = 0; k < 4; ++k) o.w[k] = red[6 * w + 2 + k];
            u256_add(P, o);
        }
}

// Counts community c's run (entries nbr[a0 .. a0 + m), weights nbrw[...]) with
// the whole block, then adds every entry's weighted pair share.  Runs larger
// than the table split their keys into R hash classes (one pass per class);
// an overflowing pass doubles R.  Writes rec[c] (REC_* words; the unweighted
// pair sum is not formed) and recw[c] = P_c (256-bit).
__device__ __forceinline__ void count_run_weighted(const CountCtx &x, const float *nbrw, unsigned long long *recw,
                                                   int c, unsigned a0, unsigned m, unsigned vol,
                                                   const SmemTable &tab, int tid, int T, unsigned long long *red)
{
    const int *src = x.nbr + a0;
    const float *wsrc = nbrw + a0;
    const unsigned cap_keys = (unsigned)tab.max_used;
    unsigned R = m <= cap_keys ? 1u
                               : (unsigned)min((unsigned long long)R_MAX,
                                               (5ull * m + 4ull * cap_keys - 1) / (4ull * cap_keys));
    for (;;) {
        unsigned long long slots = 0, cnt2 = 0;
        U256 P;
        u256_zero(P);
        bool ok = true;
        for (unsigned r = 0; r < R && ok; ++r) {
            for (unsigned e = tid; e < m; e += T) {
                const int lv = __ldcg(&src[e]);
                if (!QM_CHK(lv, x.K, 6)) continue;
                if (R == 1 || tab_split((unsigned)lv, R) == r) tab_insert(tab, (unsigned)lv);
            }
            block_sync();
            if (*(volatile int *)tab.overflow) {
                ok = false;
                break;
            }
            for (unsigned e = tid; e < m; e += T) {
                const int lv = __ldcg(&src[e]);
                if (!QM_CHK(lv, x.K, 6)) continue;
                if (R > 1 && tab_split((unsigned)lv, R) != r) continue;
                const unsigned long long cnt = tab_count(tab, (unsigned)lv);
                const u128 q = (u128)w_fixed(__ldcg(&wsrc[e])) * (u128)cnt;
                u256_mac(P, q, ld_rcp(&x.recip[lv]));
            }
            block_sync();
            tab_drain(tab, tid, T, [&](int key, long long cnt) {
                if (key < c) return;  // each unordered pair counted once, by its smaller id
                ++slots;
                cnt2 += (unsigned long long)cnt * (unsigned long long)cnt;
            });
            block_sync();
            if (tid == 0) *tab.n_used = 0;
            block_sync();
        }
        if (!ok) {
            tab_wipe(tab, tid, T);
            block_sync();
            if (tid == 0) { *tab.n_used = 0; *tab.overflow = 0; }
            block_sync();
            const unsigned nr = R * 2u;
            if (nr > R_MAX) {
                if (tid == 0) atomicOr(x.err, 2);
                return;
            }
            R = nr;
            continue;
        }
        group_totals_w(slots, cnt2, P, red);
        if (tid == 0) {
            unsigned long long *rc = x.rec + (size_t)c * REC_WORDS;
            rc[REC_SAME] = (unsigned long long)(vol - m);
            rc[REC_VOL] = (unsigned long long)vol;
            rc[REC_SLOTS] = slots;
            rc[REC_CNT2] = cnt2;
            rc[REC_INNER_LO] = 0ull;
            rc[REC_INNER_HI] = 0ull;
            rc[REC_FULL_LO] = 0ull;
            rc[REC_FULL_HI] = 0ull;
#pragma unroll
            for (int k = 0; k < 4; ++k) recw[(size_t)c * 4 + k] = P.w[k];
        }
        block_sync();
        return;
    }
}

// One block per owned non-empty community (grid-stride), whole-block table.
__global__ void __launch_bounds__(1024) k_count_w(CountCtx x, const float *nbrw, unsigned long long *recw,
                                                   SmemPlan p, const int *status, Shard own)
{
    extern __shared__ __align__(16) unsigned char sm[];
    if (*status) return;
    unsigned long long *red = (unsigned long long *)(sm + p.red_off);
    int *ctl = (int *)(sm + p.ctl_off);
    unsigned long long *slot = (unsigned long long *)(sm + p.slot_off);
    int *used = (int *)(sm + p.used_off);
    for (int i = threadIdx.x; i < p.cap; i += blockDim.x) slot[i] = 0ull;
    if (threadIdx.x < 2) ctl[threadIdx.x] = 0;
    block_sync();
    const SmemTable tb{slot, used, &ctl[0], &ctl[1], p.cap, p.max_used};
    for (int c = blockIdx.x; c < x.K; c += gridDim.x) {
        const int s0 = __ldcg(&x.start[c]), s1 = __ldcg(&x.start[c + 1]);
        if (s1 == s0 || !own.owns(c)) continue;
        const unsigned a0 = __ldcg(&x.aoff[s0]), vol = __ldcg(&x.aoff[s1]) - a0;
        const unsigned m = (unsigned)__ldcg(&x.inter[c]);
        count_run_weighted(x, nbrw, recw, c, a0, m, vol, tb, threadIdx.x, blockDim.x, red);
    }
}

// FP64 terms of every owned community from its integers (weighted Eqs. 8-9,
// unweighted Sec. II-B.3), added in fixed point; Q_w goes to GS_QW.
__global__ void k_score_terms_w(const int *start, const unsigned long long *rec, const unsigned long long *recw,
                                const unsigned long long *wl, int K, long long E, unsigned long long w_lo,
                                unsigned long long w_hi, PerCommDev pc, unsigned long long *g, const int *status,
                                Shard own)
{
    __shared__ unsigned long long red[72];
    if (*status) return;
    ScoreAcc acc;
    score_acc_zero(acc);
    i128 qw = 0;
    const double W2 = __dmul_rn(2.0, u128_to_double(((u128)w_hi << 64) | (u128)w_lo));  // 2W * 2^43
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < K; c += gridDim.x * blockDim.x) {
        const long long size = start[c + 1] - start[c];
        if (size == 0 || !own.owns(c)) continue;
        const unsigned long long *rc = rec + (size_t)c * REC_WORDS;
        const unsigned long long same = rc[REC_SAME], vol = rc[REC_VOL];
        const long long ein = (long long)(same / 2), eout = (long long)(vol - same);
        double qs_unweighted, dens, contr, expn, cond;
        community_terms(ein, eout, size, E, qs_unweighted, dens, contr, expn, cond);
        const i128 win2 = limbs_get(wl + (size_t)c * 6), wout = limbs_get(wl + (size_t)c * 6 + 3);
        const double fin = __ddiv_rn(i128_to_double(win2), W2);          // W_c^in / W
        const double fvol = __ddiv_rn(i128_to_double(win2 + wout), W2);  // (2 W_c^in + W_c^out) / (2W)
        const double qwt = __dsub_rn(fin, __dmul_rn(fvol, fvol));
        const double t1 = __dmul_rn(fin, dens), t2 = __dmul_rn(fvol, dens);
        const double self = __dsub_rn(t1, __dmul_rn(t2, t2));
        U256 P;
#pragma unroll
        for (int k = 0; k < 4; ++k) P.w[k] = recw[(size_t)c * 4 + k];
        // P = sum_j W_ij |E_ij| / |c_j| * 2^171 ; penalty = that / (2W |c|)
        const double pen = __ddiv_rn(ldexp(u256_to_double(P), -128), __dmul_rn(W2, (double)size));
        acc.qds_self += fp_from_double(self, SC_QDS);
        acc.qds_pair += fp_from_double(pen, SC_QDS);
        acc.dens += fp_from_double(dens, SC_MEAN);
        acc.contr += fp_from_double(contr, SC_MEAN);
        acc.expn += fp_from_double(expn, SC_MEAN);
        acc.cond += fp_from_double(cond, SC_MEAN);
        acc.vol2 += (u128)vol * (u128)vol;
        acc.ein += (unsigned long long)ein;
        acc.eout += (unsigned long long)eout;
        acc.nonempty += 1;
        acc.slots += rc[REC_SLOTS];
        acc.cnt2 += rc[REC_CNT2];
        qw += fp_from_double(qwt, SC_QDS);
        if (pc.size) pc.size[c] = size;
        if (pc.ein) pc.ein[c] = ein;
        if (pc.eout) pc.eout[c] = eout;
        if (pc.dens) pc.dens[c] = dens;
        if (pc.contr) pc.contr[c] = contr;
        if (pc.expn) pc.expn[c] = expn;
        if (pc.cond) pc.cond[c] = cond;
        if (pc.qds) pc.qds[c] = __dsub_rn(self, pen);
    }
    flush_score_threads(acc, g, red);
    const i128 t = group_sum_i128(qw, blockDim.x, red);
    if (threadIdx.x == 0 && t != 0) limbs_add(g + GS_QW, t);
}

// ---------------------------------------------------------------- load time

// Weight check and total: every weight must be 0 or in [2^-20, 2^20) (NaN
// fails); the fixed-point sum over all arcs (2 W * 2^43) goes to three limbs.
__global__ void k_wcheck(const float *__restrict__ wt, long long n_arcs, int *status, unsigned long long *lim)
{
    u128 s = 0;
    bool bad = false;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n_arcs;
         e += (long long)gridDim.x * blockDim.x) {
        const float w = wt[e];
        if (!(w == 0.0f || (w >= 9.5367431640625e-07f && w < 1048576.0f))) {
            bad = true;
            continue;
        }
        s += w_fixed(w);
    }
    if (bad) atomicOr(status, 2);
    for (int d = 16; d > 0; d >>= 1) s += shfl_down_u128(s, d);
    if ((threadIdx.x & 31) == 0 && s) limbs_add(lim, (i128)s);
}

// Symmetric weights: arc (u, v) and arc (v, u) carry the same weight (rows
// sorted, as the full validation has checked).
__global__ void k_wsym(const long long *__restrict__ row_ptr, const int *__restrict__ col,
                       const float *__restrict__ wt, long long n, int *status)
{
    bool bad = false;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (long long)gridDim.x * blockDim.x) {
        for (long long k = row_ptr[u]; k < row_ptr[u + 1] && !bad; ++k) {
            const int v = col[k];
            long long lo = row_ptr[v], hi = row_ptr[v + 1];
            bool found = false;
            while (lo < hi) {
                const long long mid = (lo + hi) >> 1;
                const int w = col[mid];
                if (w == (int)u) {
                    found = wt[mid] == wt[k];
                    break;
                }
                if (w < (int)u) lo = mid + 1; else hi = mid;
            }
            if (!found) bad = true;
        }
    }
    if (bad) atomicOr(status, 4);
}

