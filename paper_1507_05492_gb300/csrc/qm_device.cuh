// qm_device.cuh -- device building blocks shared by every scoring kernel.
//
// * 128-bit fixed-point accumulation: every floating-point sum of the metrics
//   (Eqs. 1-3, 9 and the means of Sec. II-B.3) is a sum of per-community or
//   per-cell terms.  Each term is evaluated once in FP64 with round-to-nearest
//   operations (the library is built with --fmad=false), converted to a signed
//   128-bit integer at a fixed binary scale, and the integers are added.  Integer
//   addition is associative, so a sum does not depend on how threads, warps,
//   blocks or batches split the work.
// * An open-addressing hash table in shared memory that counts how often each
//   community id occurs (|E_ci,cj| of Eq. 9 and the cells |c n c'| of Eqs. 1-4).
// * The per-community and per-cell term formulas.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qmk {

typedef __int128 i128;
typedef unsigned __int128 u128;

// Binary scales of the fixed-point accumulators (value = integer * 2^-scale).
// Each is chosen so that the largest possible sum stays below 2^126.
constexpr int SC_QDS = 100;   // Qds terms: |sum| <= 3
constexpr int SC_MEAN = 64;   // sums of d_c, 2E_in/|c|, E_out/|c|, conductance: < 2^34
constexpr int SC_VI = 80;     // sum of n log(n^2/(n_a n_b)): |sum| < 43 N < 2^37
constexpr int SC_H = 100;     // NMI numerator / denominator terms: |sum| < 44
constexpr int SC_F = 80;      // F-measure sum of n_a * max ratio: < N < 2^31

// ---------------------------------------------------------------- bounds checks
// Compiled in only with -DQM_BOUNDS_CHECK (a diagnostic build): an index outside
// [0, n) records (site, index, bound) in qm_dbg_rec and the access is skipped.
#ifdef QM_BOUNDS_CHECK
static __device__ unsigned long long qm_dbg_rec[8];
__device__ __forceinline__ bool qm_chk_ex(long long i, long long n, int site, long long e0, long long e1,
                                          long long e2, long long e3)
{
    if (i >= 0 && i < n) return true;
    if (atomicCAS(&qm_dbg_rec[0], 0ull, (unsigned long long)site) == 0ull) {
        qm_dbg_rec[1] = (unsigned long long)i;
        qm_dbg_rec[2] = (unsigned long long)n;
        qm_dbg_rec[4] = (unsigned long long)e0;
        qm_dbg_rec[5] = (unsigned long long)e1;
        qm_dbg_rec[6] = (unsigned long long)e2;
        qm_dbg_rec[7] = (unsigned long long)e3;
    }
    atomicAdd(&qm_dbg_rec[3], 1ull);
    return false;
}
#define QM_CHK(i, n, site) qm_chk_ex((long long)(i), (long long)(n), (site), 0, 0, 0, 0)
#define QM_CHKX(i, n, site, a, b, c, d) \
    qm_chk_ex((long long)(i), (long long)(n), (site), (long long)(a), (long long)(b), (long long)(c), (long long)(d))
#else
#define QM_CHK(i, n, site) true
#define QM_CHKX(i, n, site, a, b, c, d) true
#endif

// ---------------------------------------------------------------- fixed point

__device__ __forceinline__ i128 fp_from_double(double x, int scale)
{
    unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    int ex = (int)((bits >> 52) & 0x7FF);
    unsigned long long man = bits & ((1ull << 52) - 1);
    if (ex == 0 && man == 0) return 0;
    if (ex == 0) ex = 1; else man |= (1ull << 52);
    int sh = ex - 1075 + scale;               // |x| * 2^scale = man * 2^sh
    u128 m = (u128)man, v;
    if (sh >= 0) {
        if (sh > 73) sh = 73;                 // out of range: saturate (never reached in range)
        v = m << sh;
    } else if (sh > -127) {
        v = (m + ((u128)1 << (-sh - 1))) >> (-sh);   // round half up
    } else {
        v = 0;
    }
    return (bits >> 63) ? -(i128)v : (i128)v;
}

__device__ __forceinline__ double fp_to_double(i128 v, int scale)
{
    bool neg = v < 0;
    u128 a = neg ? (u128)(-v) : (u128)v;
    double hi = (double)(unsigned long long)(a >> 64);
    double lo = (double)(unsigned long long)a;
    double r = __dadd_rn(__dmul_rn(hi, 18446744073709551616.0), lo);
    r = ldexp(r, -scale);
    return neg ? -r : r;
}

// A 128-bit sum kept in global memory as three 64-bit limbs so that it can be
// updated with 64-bit atomics: v = L2 * 2^86 + L1 * 2^43 + L0, where L0 and L1
// add up non-negative 43-bit chunks (safe for fewer than 2^21 additions) and
// L2 adds the signed high part.
__device__ __forceinline__ void limbs_add(unsigned long long *L, i128 v)
{
    const u128 mask = (((u128)1) << 43) - 1;
    u128 u = (u128)v;
    unsigned long long l0 = (unsigned long long)(u & mask);
    unsigned long long l1 = (unsigned long long)((u >> 43) & mask);
    long long l2 = (long long)(v >> 86);
    if (l0) atomicAdd(&L[0], l0);
    if (l1) atomicAdd(&L[1], l1);
    if (l2) atomicAdd(&L[2], (unsigned long long)l2);
}

__device__ __forceinline__ void limbs_store(unsigned long long *L, i128 v)
{
    const u128 mask = (((u128)1) << 43) - 1;
    u128 u = (u128)v;
    L[0] = (unsigned long long)(u & mask);
    L[1] = (unsigned long long)((u >> 43) & mask);
    L[2] = (unsigned long long)(long long)(v >> 86);
}

__device__ __forceinline__ i128 limbs_get(const unsigned long long *L)
{
    return (i128)(long long)L[2] * (((i128)1) << 86) + (i128)L[1] * (((i128)1) << 43) + (i128)L[0];
}

__device__ __forceinline__ i128 shfl_down_i128(i128 v, int d)
{
    unsigned long long lo = (unsigned long long)(u128)v;
    unsigned long long hi = (unsigned long long)((u128)v >> 64);
    lo = __shfl_down_sync(0xffffffffu, lo, d);
    hi = __shfl_down_sync(0xffffffffu, hi, d);
    return (i128)(((u128)hi << 64) | (u128)lo);
}

__device__ __forceinline__ i128 warp_sum_i128(i128 v)
{
    for (int d = 16; d > 0; d >>= 1) v += shfl_down_i128(v, d);
    return v;  // valid in lane 0
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    return v;
}

// ---------------------------------------------------------------- exact pair sums
//
// The split penalty of Eq. (9) for community i needs S_i = sum_j |E_ij|^2 / |c_j|
// over the neighbouring communities j.  Each 1/|c_j| is held as the 128-bit
// integer Rcp_j = floor((2^128 - 1) / |c_j|) (relative error below 2^-97 for
// any size below 2^31), and sum_j |E_ij|^2 Rcp_j is accumulated exactly in 192
// bits; S_i is that sum / 2^128.  Integer sums do not depend on the order or
// grouping of their terms, so a pass that adds |E_ij|^2 per key and one that
// adds (2k - 1) Rcp_j for the k-th occurrence of key j (sum over k of 2k - 1
// is |E_ij|^2) give identical bits.

struct __align__(16) Rcp {
    unsigned long long lo, hi;
};

// floor((2^128 - 1) / s) for 1 <= s < 2^31, by long division in 32-bit digits.
__device__ __forceinline__ Rcp rcp_of(long long s)
{
    const unsigned long long d = (unsigned long long)s;
    unsigned long long rem = 0, q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned long long cur = (rem << 32) | 0xFFFFFFFFull;
        q[k] = cur / d;
        rem = cur % d;
    }
    Rcp r;
    r.hi = (q[0] << 32) | q[1];
    r.lo = (q[2] << 32) | q[3];
    return r;
}

// Loads through L2 only (data written earlier in the same launch) / through
// the read-only path.
__device__ __forceinline__ Rcp ld_rcp_cg(const Rcp *p)
{
    const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2 *>(p));
    return Rcp{v.x, v.y};
}

__device__ __forceinline__ Rcp ld_rcp(const Rcp *p)
{
    const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p));
    return Rcp{v.x, v.y};
}

struct U192 {
    unsigned long long w0, w1, w2;
};

__device__ __forceinline__ void u192_zero(U192 &a) { a.w0 = a.w1 = a.w2 = 0ull; }

// a += q * r
__device__ __forceinline__ void u192_mac(U192 &a, unsigned long long q, const Rcp &r)
{
    const u128 p0 = (u128)q * r.lo;
    const u128 p1 = (u128)q * r.hi;
    const u128 t = (((u128)a.w1 << 64) | a.w0) + p0;
    const unsigned long long c = t < p0 ? 1ull : 0ull;
    a.w0 = (unsigned long long)t;
    const u128 t2 = (((u128)(a.w2 + c) << 64) | (unsigned long long)(t >> 64)) + p1;
    a.w1 = (unsigned long long)t2;
    a.w2 = (unsigned long long)(t2 >> 64);
}

// a += r (u192_mac with q = 1)
__device__ __forceinline__ void u192_add_rcp(U192 &a, const Rcp &r)
{
    const u128 r128 = ((u128)r.hi << 64) | r.lo;
    const u128 t = (((u128)a.w1 << 64) | a.w0) + r128;
    a.w2 += t < r128 ? 1ull : 0ull;
    a.w0 = (unsigned long long)t;
    a.w1 = (unsigned long long)(t >> 64);
}

__device__ __forceinline__ void u192_add(U192 &a, const U192 &b)
{
    const u128 lb = ((u128)b.w1 << 64) | b.w0;
    const u128 t = (((u128)a.w1 << 64) | a.w0) + lb;
    a.w2 += b.w2 + (t < lb ? 1ull : 0ull);
    a.w0 = (unsigned long long)t;
    a.w1 = (unsigned long long)(t >> 64);
}

// Warp total (valid in lane 0).
__device__ __forceinline__ U192 u192_warp_sum(U192 a)
{
    for (int d = 16; d > 0; d >>= 1) {
        U192 o;
        o.w0 = __shfl_down_sync(0xffffffffu, a.w0, d);
        o.w1 = __shfl_down_sync(0xffffffffu, a.w1, d);
        o.w2 = __shfl_down_sync(0xffffffffu, a.w2, d);
        u192_add(a, o);
    }
    return a;
}

// S * 2^64 as a 64.64 fixed-point number: the sum shifted right by 64 bits.
__device__ __forceinline__ u128 u192_shr64(const U192 &a) { return ((u128)a.w2 << 64) | a.w1; }

// ---------------------------------------------------------------- accumulators

// Per-thread partial sums of one partition's no-ground-truth metrics.
struct ScoreAcc {
    i128 qds_self;    // sum_c [E_in/|E| d_c - ((2E_in+E_out)/(2|E|) d_c)^2]   (SC_QDS)
    i128 qds_pair;    // sum over ordered (ci,cj) of |E_ij|^2 / (2|E| |ci| |cj|)  (SC_QDS)
    i128 dens;        // sum_c d_c                 (SC_MEAN)
    i128 contr;       // sum_c 2 E_in / |c|        (SC_MEAN)
    i128 expn;        // sum_c E_out / |c|         (SC_MEAN)
    i128 cond;        // sum_c conductance         (SC_MEAN)
    u128 vol2;        // sum_c (2 E_in + E_out)^2  (exact)
    unsigned long long ein;       // sum_c E_in
    unsigned long long eout;      // sum_c E_out
    unsigned long long nonempty;  // communities with |c| > 0
    unsigned long long slots;     // ordered pairs (ci,cj) with |E_ij| > 0
    unsigned long long cnt2;      // sum over ordered pairs of |E_ij|^2
};

__device__ __forceinline__ void score_acc_zero(ScoreAcc &a)
{
    a.qds_self = a.qds_pair = a.dens = a.contr = a.expn = a.cond = 0;
    a.vol2 = 0;
    a.ein = a.eout = a.nonempty = a.slots = a.cnt2 = 0;
}

__device__ __forceinline__ void score_acc_add(ScoreAcc &d, const ScoreAcc &s)
{
    d.qds_self += s.qds_self;
    d.qds_pair += s.qds_pair;
    d.dens += s.dens;
    d.contr += s.contr;
    d.expn += s.expn;
    d.cond += s.cond;
    d.vol2 += s.vol2;
    d.ein += s.ein;
    d.eout += s.eout;
    d.nonempty += s.nonempty;
    d.slots += s.slots;
    d.cnt2 += s.cnt2;
}

// Global (per-partition) accumulator layout, all unsigned long long:
enum {
    GS_QDS_SELF = 0, GS_QDS_PAIR = 3, GS_DENS = 6, GS_CONTR = 9, GS_EXPN = 12, GS_COND = 15,
    GS_VOL2 = 18, GS_EIN = 21, GS_EOUT = 22, GS_NONEMPTY = 23, GS_SLOTS = 24, GS_CNT2 = 25,
    GS_QW = 26,  // weighted graphs: sum_c of the Q_w term (SC_QDS), three limbs
    GS_COUNT = 29
};

// Per-thread partial sums of one comparison (contingency table).
struct CompareAcc {
    i128 vi;     // sum over cells of n log(n^2 / (n_a n_b))        (SC_VI)
    i128 hnum;   // sum over cells of (n/N) log(n N / (n_a n_b))    (SC_H)
    i128 hden;   // sum over communities of both sides of p log p   (SC_H)
    i128 f;      // sum over truth communities of n_a * max ratio   (SC_F)
    unsigned long long a11;     // sum over cells C(n, 2)
    unsigned long long sa;      // sum over truth communities C(n_a, 2)
    unsigned long long sb;      // sum over found communities C(n_b, 2)
    unsigned long long nvd;     // row maxima + column maxima
    unsigned long long cells;   // non-zero cells
    unsigned long long ka;      // non-empty truth communities
    unsigned long long kb;      // non-empty found communities
};

__device__ __forceinline__ void compare_acc_zero(CompareAcc &a)
{
    a.vi = a.hnum = a.hden = a.f = 0;
    a.a11 = a.sa = a.sb = a.nvd = a.cells = a.ka = a.kb = 0;
}

__device__ __forceinline__ void compare_acc_add(CompareAcc &d, const CompareAcc &s)
{
    d.vi += s.vi;
    d.hnum += s.hnum;
    d.hden += s.hden;
    d.f += s.f;
    d.a11 += s.a11;
    d.sa += s.sa;
    d.sb += s.sb;
    d.nvd += s.nvd;
    d.cells += s.cells;
    d.ka += s.ka;
    d.kb += s.kb;
}

enum {
    GC_VI = 0, GC_HNUM = 3, GC_HDEN = 6, GC_F = 9, GC_A11 = 12, GC_SA = 13, GC_SB = 14,
    GC_NVD = 15, GC_CELLS = 16, GC_KA = 17, GC_KB = 18, GC_COUNT = 19
};

// ---------------------------------------------------------------- term formulas

// Eq. (9) self part and the Sec. II-B.3 measures of one non-empty community.
// ein = |E_c^in|, eout = |E_c^out|, s = |c|, E = |E|.
__device__ __forceinline__ void community_terms(long long ein, long long eout, long long s, long long E,
                                                double &qds_self, double &dens, double &contr,
                                                double &expn, double &cond)
{
    const double in = (double)ein, out = (double)eout, sz = (double)s, e = (double)E;
    const double vol = __dadd_rn(__dmul_rn(2.0, in), out);
    dens = (s > 1) ? __ddiv_rn(__dmul_rn(2.0, in), __dmul_rn(sz, __dsub_rn(sz, 1.0))) : 0.0;
    const double t1 = __dmul_rn(__ddiv_rn(in, e), dens);
    const double t2 = __dmul_rn(__ddiv_rn(vol, __dmul_rn(2.0, e)), dens);
    qds_self = __dsub_rn(t1, __dmul_rn(t2, t2));
    contr = __ddiv_rn(__dmul_rn(2.0, in), sz);
    expn = __ddiv_rn(out, sz);
    cond = (vol > 0.0) ? __ddiv_rn(out, vol) : 0.0;
}

// Eq. (9) split-penalty term of the ordered pair (ci, cj):
// |E_ij| / (2|E|) * |E_ij| / (|ci| |cj|).
__device__ __forceinline__ double pair_term(long long cnt, long long si, long long sj, long long E)
{
    const double x = (double)cnt;
    const double a = __ddiv_rn(x, __dmul_rn(2.0, (double)E));
    const double b = __ddiv_rn(x, __dmul_rn((double)si, (double)sj));
    return __dmul_rn(a, b);
}

// Largest integer i whose log(i) (and, per comparison call, log(N / i)) is tabulated.
constexpr int LOGT_MAX = 8192;

// log(i) for 0 < i <= LOGT_MAX (entry 0 unused).  Each translation unit that
// includes this header has its own copy, filled once per device by
// k_fill_log_int from its prepare step; every copy holds the same bits.
static __device__ double qm_log_int[LOGT_MAX + 1];

static __global__ void k_fill_log_int()
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= LOGT_MAX; i += gridDim.x * blockDim.x)
        qm_log_int[i] = i == 0 ? 0.0 : log((double)i);
}

// log(n^2 / (n_a n_b)) of one contingency cell: the logarithm of its Eq. (1)
// term, and (with log(N/n)) of its Eq. (2) term.  When all three counts are
// tabulated and the ratio is below 1/4 or above 4 (|log| > 1.38), the value is
// formed from the table as 2 log n - log n_a - log n_b (absolute error a few
// units of 2^-52 * 18, so the relative error stays below 1e-14); otherwise,
// and in particular near a ratio of 1 where the terms would cancel, one
// logarithm of the ratio is taken.
__device__ __forceinline__ double cell_log(long long n, long long na, long long nb)
{
    const double x = __dmul_rn((double)n, (double)n), y = __dmul_rn((double)na, (double)nb);
    if (n <= LOGT_MAX && na <= LOGT_MAX && nb <= LOGT_MAX && (__dmul_rn(4.0, x) < y || x > __dmul_rn(4.0, y))) {
        const double ln = __ldg(&qm_log_int[n]), la = __ldg(&qm_log_int[na]), lb = __ldg(&qm_log_int[nb]);
        return __dsub_rn(__dsub_rn(__dmul_rn(2.0, ln), la), lb);
    }
    return log(__ddiv_rn(x, y));
}

// log(N / n); every caller evaluates this same expression (directly, or via
// a table of it for small n), so all paths give the same bits.
__device__ __forceinline__ double log_ratio(long long N, long long n)
{
    return log(__ddiv_rn((double)N, (double)n));
}

// Eq. (1) term n log(n^2 / (n_a n_b)) from the cell's logarithm l1.
__device__ __forceinline__ double vi_term_l(long long n, double l1) { return __dmul_rn((double)n, l1); }

// Eq. (2) numerator term (n/N) log(n N / (n_a n_b)) = (n/N) (l1 + log(N/n)),
// from the quotient n/N (nmi_over: the same division, tabulated by callers that
// form many cells of one N).
__device__ __forceinline__ double nmi_over(long long n, long long N) { return __ddiv_rn((double)n, (double)N); }

__device__ __forceinline__ double nmi_num_term_q(double n_over_N, double l1, double log_n_over)
{
    return __dmul_rn(n_over_N, __dadd_rn(l1, log_n_over));
}

__device__ __forceinline__ double nmi_num_term_l(long long n, long long N, double l1, double log_n_over)
{
    return nmi_num_term_q(nmi_over(n, N), l1, log_n_over);
}

// A comparison's tables for cells and communities of at most LOGT_MAX nodes:
// log(N / i) at [i] and i / N at [LOGT_MAX + 1 + i], i = 1 .. LOGT_MAX.
constexpr int LOGT_WORDS = 2 * (LOGT_MAX + 1);

// Eq. (2) denominator term (n_c/N) log(n_c/N) of one community.
__device__ __forceinline__ double entropy_term(long long nc, long long N)
{
    const double p = __ddiv_rn((double)nc, (double)N);
    return __dmul_rn(p, log(p));
}

// Eq. (3) ratio 2 n / (n_a + n_b) of one cell.
__device__ __forceinline__ double f_ratio(long long n, long long na, long long nb)
{
    return __ddiv_rn(__dmul_rn(2.0, (double)n), (double)(na + nb));
}

// ---------------------------------------------------------------- hash table

// Open addressing with linear probing over `cap` 64-bit slots in shared memory.
// A slot holds ((key + 1) << 32) | count; 0 means empty.  `used` lists the
// occupied slot indices so that reading out and clearing cost O(occupied).
struct SmemTable {
    unsigned long long *slot;
    int *used;
    int *n_used;     // shared counter
    int *overflow;   // shared flag
    int cap;
    int max_used;
};

__device__ __forceinline__ unsigned tab_hash(unsigned key, int cap)
{
    return __umulhi(key * 0x9E3779B1u + 0x7F4A7C15u, (unsigned)cap);
}

// Secondary hash that splits keys into R sub-ranges for multi-pass counting.
__device__ __forceinline__ unsigned tab_split(unsigned key, unsigned R)
{
    unsigned h = key * 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h % R;
}

// Adds inc (>= 1) occurrences of key.
__device__ __forceinline__ void tab_insert_n(const SmemTable &t, unsigned key, unsigned inc)
{
    const unsigned long long tag = (unsigned long long)(key + 1u) << 32;
    unsigned h = tab_hash(key, t.cap);
    // Once the table has overflowed its pass is discarded: stop probing.
    if (*(volatile int *)t.overflow) return;
    for (int probe = 0; probe < t.cap; ++probe) {
        if (!QM_CHK(h, t.cap, 8)) return;
        if ((probe & 15) == 15 && *(volatile int *)t.overflow) return;
        unsigned long long cur = ((volatile unsigned long long *)t.slot)[h];
        if (cur == 0ull) {
            unsigned long long prev = atomicCAS(&t.slot[h], 0ull, tag | (unsigned long long)inc);
            if (prev == 0ull) {
                int idx = atomicAdd(t.n_used, 1);
                if (idx < t.max_used) t.used[idx] = (int)h;
                else *t.overflow = 1;
                return;
            }
            cur = prev;
        }
        if ((cur & 0xFFFFFFFF00000000ull) == tag) {
            atomicAdd(&t.slot[h], (unsigned long long)inc);
            return;
        }
        h = (h + 1u == (unsigned)t.cap) ? 0u : h + 1u;
    }
    *t.overflow = 1;
}

__device__ __forceinline__ void tab_insert(const SmemTable &t, unsigned key) { tab_insert_n(t, key, 1u); }

// Warp-aggregated insert: the lanes with `valid` set insert their keys, equal
// keys merged into one update of their count (all 32 lanes call this).
__device__ __forceinline__ void tab_insert_warp(const SmemTable &t, unsigned key, bool valid)
{
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    if (!valid) return;
    const unsigned peers = __match_any_sync(act, key);
    if ((threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) tab_insert_n(t, key, (unsigned)__popc(peers));
}

// ---------------------------------------------------------------- bulk copies
//
// One-dimensional TMA bulk copy global -> shared memory completing on an
// mbarrier (PTX cp.async.bulk / mbarrier.*).  Both addresses must be 16-byte
// aligned and the size a multiple of 16 bytes.

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Orders this thread's earlier shared-memory accesses (and barrier inits)
// before later accesses by the async proxy (bulk copies).
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bulk_load_smem(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Waits for the phase with the given parity to complete; gives up after
// `limit` polls (each poll may itself suspend briefly) and returns false.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, unsigned limit)
{
    for (unsigned i = 0; i < limit; ++i) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(smem_u32(bar)), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// ---------------------------------------------------------------- misc

// How many items a warp claims at a time from a shared list of n items when
// `warps` warps draw from it: about a quarter of an even share, between 1 and
// 32.  Few items (a small graph) then spread over all warps instead of
// queueing behind a few, and many items still take few atomics per warp.
__device__ __forceinline__ int claim_chunk(long long n, long long warps)
{
    const long long c = n / (4 * (warps > 0 ? warps : 1));
    return c < 1 ? 1 : (c > 32 ? 32 : (int)c);
}

// Number of entries of the sorted prefix a[0..n) that are <= x.
__device__ __forceinline__ int upper_bound_smem(const unsigned *a, int n, unsigned x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Block-wide barrier in its non-.aligned PTX form.  __syncthreads() is the
// .aligned barrier, which requires each warp to arrive converged; the block
// routines reach their barriers straight from data-dependent loops (hash-table
// probing, ragged arc loops), so the warp may arrive in several pieces.  The
// non-aligned barrier counts threads, not converged warps, and orders memory
// like __syncthreads().  Every lane of every warp has arrived once it returns,
// so a warp sync then merges the pieces again: without it a warp can stay
// split and issue each later instruction once per piece.  (No caller lets a
// lane exit while others of its warp still reach a block barrier.)
__device__ __forceinline__ void block_sync()
{
    asm volatile("barrier.sync 0;" ::: "memory");
    __syncwarp();
}

__device__ __forceinline__ void group_sync(int group)
{
    if (group == 32) __syncwarp();
    else block_sync();
}

// Barrier of a group of threads that may also be one of the block's equal
// groups of `group` consecutive threads (a multiple of 32): such a group takes
// named barrier 1 + its index (non-aligned, like block_sync).
__device__ __forceinline__ void group_sync_n(int group)
{
    if (group == 32) {
        __syncwarp();
    } else if (group == (int)blockDim.x) {
        block_sync();
    } else {
        asm volatile("barrier.sync %0, %1;" ::"r"(1 + (int)threadIdx.x / group), "r"(group) : "memory");
        __syncwarp();
    }
}

}  // namespace qmk
