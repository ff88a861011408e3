/*
 * qm_oracle.c -- plain, slow CPU statement of the community-quality metrics of
 * Chen, Liu & Szymanski, "Parallel Toolkit for Measuring the Quality of Network
 * Community Structure" (arXiv 1507.05492).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * it is used by tests/, by the smoke check and by the timed CPU baseline of the
 * benchmark.  It shares no code, header, table or helper with the CUDA library.
 *
 * Every metric is the paper's definition written out literally, term by term,
 * in long double with Neumaier-compensated summation.  No blocking, fusion or
 * reordering beyond what the definitions state.
 *
 *   Sec. II-A.1  Eq. (1) VI, Eq. (2) NMI           -> oq_compare
 *   Sec. II-A.2  Eq. (3) F-measure, Eq. (4) NVD    -> oq_compare
 *   Sec. II-A.3  Eq. (5) RI, Eq. (6) ARI, Eq. (7) JI -> oq_compare (pair counts
 *                from the contingency table), oq_pairs_bruteforce (Algorithm 4)
 *   Sec. II-B.1  Eq. (8) modularity Q              -> oq_score
 *   Sec. II-B.2  Eq. (9) modularity density Qds    -> oq_score
 *   Sec. II-B.3  six per-community measures        -> oq_score
 *   weighted graphs (the note beside Eq. 9)        -> oq_score_weighted
 *   label propagation (the detector family of Sec. I, IV-C) -> oq_label_propagation
 *   overlapping communities (covers; the paper's future work, Sec. VI),
 *   the set formulas read literally -> oq_score_cover, oq_compare_cover,
 *                oq_pairs_cover_bruteforce
 *   the same quantities as oq_score with OpenMP threads (all-core CPU
 *   baseline)                                        -> oq_score_omp
 *
 * Readings taken where the paper is silent:
 *   - log is the natural log (Eq. 1);
 *   - d_c = 0 for a one-node community (Eq. 9, 0/0);
 *   - label ids with no member are absent communities, skipped everywhere;
 *   - conductance = 0 when 2|E_in|+|E_out| = 0 (isolated node);
 *   - partition-level value of a per-community measure = unweighted mean over
 *     non-empty communities (Sec. II-B.3 defines them per community only);
 *   - NMI = 1 when both entropies are 0; ARI = 1 and JI = 1 when their
 *     denominators are 0 (both partitions trivial in the same way);
 *   - pairs are unordered (A = |V|(|V|-1)/2, Sec. II-A.3), so the brute force
 *     of Algorithm 4 counts i<j;
 *   - the Qds split penalty sums over ordered pairs (c_i, c_j), j != i, as
 *     written in Eq. (9): each unordered pair contributes to both communities;
 *   - F-measure sums over the ground truth C (first argument) and maximises
 *     over the detected C' (second argument), Eq. (3).
 *
 * Parity pins (tests/test_oracle_*.py): closed forms (two 5-cliques joined by
 * one edge; a two-partition worked example), networkx modularity, scikit-learn
 * pair/information indices, Algorithm 4 brute force, adjacency-matrix and
 * set-intersection brute force, invariants.  The partition-level means of the
 * six measures are pinned only against the reading above ("parity unpinned"
 * against the paper's own toolkit, which prints no values).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OQ_OK 0
#define OQ_EINVAL 1
#define OQ_ENOMEM 2
#define OQ_ECHECK 3 /* an internal identity failed */

/* ---- compensated summation (Neumaier) in long double ---- */
typedef struct { long double s, c; } oq_sum;

static void sum_add(oq_sum *k, long double x)
{
    long double t = k->s + x;
    if (fabsl(k->s) >= fabsl(x))
        k->c += (k->s - t) + x;
    else
        k->c += (x - t) + k->s;
    k->s = t;
}

static long double sum_get(const oq_sum *k) { return k->s + k->c; }

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * Graph validation: the method is defined for an unweighted, undirected graph
 * (Sec. II-B.1).  A symmetric CSR with no self-loops and no repeated arcs is
 * required.  Returns OQ_OK or OQ_EINVAL.
 */
int oq_validate_graph(const int64_t *row_ptr, const int32_t *col, int64_t n)
{
    if (n < 1 || row_ptr[0] != 0)
        return OQ_EINVAL;
    for (int64_t u = 0; u < n; u++)
        if (row_ptr[u + 1] < row_ptr[u])
            return OQ_EINVAL;
    int64_t nnz = row_ptr[n];
    int32_t *sorted = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    if (!sorted)
        return OQ_ENOMEM;
    memcpy(sorted, col, (size_t)nnz * sizeof(int32_t));
    int rc = OQ_OK;
    for (int64_t u = 0; u < n && rc == OQ_OK; u++) {
        int64_t b = row_ptr[u], e = row_ptr[u + 1];
        qsort(sorted + b, (size_t)(e - b), sizeof(int32_t), cmp_i32);
        for (int64_t k = b; k < e; k++) {
            if (sorted[k] < 0 || sorted[k] >= n || sorted[k] == u) { rc = OQ_EINVAL; break; }
            if (k > b && sorted[k] == sorted[k - 1]) { rc = OQ_EINVAL; break; }
        }
    }
    /* symmetry: (u,v) present implies (v,u) present (binary search in v's sorted row) */
    for (int64_t u = 0; u < n && rc == OQ_OK; u++) {
        for (int64_t k = row_ptr[u]; k < row_ptr[u + 1]; k++) {
            int32_t v = col[k];
            int64_t lo = row_ptr[v], hi = row_ptr[v + 1];
            int found = 0;
            while (lo < hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (sorted[mid] == (int32_t)u) { found = 1; break; }
                if (sorted[mid] < (int32_t)u) lo = mid + 1; else hi = mid;
            }
            if (!found) { rc = OQ_EINVAL; break; }
        }
    }
    free(sorted);
    return rc;
}

/*
 * Output layout of oq_score (plain arrays, no shared struct):
 *   dbl[0]  Q                      Eq. (8)
 *   dbl[1]  Qds                    Eq. (9)
 *   dbl[2]  mean intra-edges       Sec. II-B.3, |E_c^in|
 *   dbl[3]  mean intra-density     d_c of Eq. (9)
 *   dbl[4]  mean contraction       2|E_c^in|/|c|
 *   dbl[5]  mean inter-edges       |E_c^out|
 *   dbl[6]  mean expansion         |E_c^out|/|c|
 *   dbl[7]  mean conductance       |E_c^out|/(2|E_c^in|+|E_c^out|)
 *   dbl[8]  sum of |terms| of Q    (conditioning for tolerance checks)
 *   dbl[9]  sum of |terms| of Qds
 *   i64[0]  |V|, i64[1] |E|, i64[2] non-empty communities,
 *   i64[3]  sum_c |E_c^in|, i64[4] cut edges = sum_c |E_c^out| / 2,
 *   i64[5]  distinct unordered community pairs with |E_ij| > 0,
 *   i64[6]  sum over those pairs of |E_ij| squared (integer check value)
 * Per-community arrays (length K, each may be NULL): size, ein, eout (int64);
 * intra_density, contraction, expansion, conductance, qds_term (double).
 * Absent communities (size 0) get zeros.
 */
int oq_score(const int64_t *row_ptr, const int32_t *col, int64_t n,
             const int32_t *label, int32_t K,
             double *dbl, int64_t *i64,
             int64_t *pc_size, int64_t *pc_ein, int64_t *pc_eout,
             double *pc_density, double *pc_contraction, double *pc_expansion,
             double *pc_conductance, double *pc_qds)
{
    if (n < 1 || K < 1)
        return OQ_EINVAL;
    for (int64_t u = 0; u < n; u++)
        if (label[u] < 0 || label[u] >= K)
            return OQ_EINVAL;
    int64_t nnz = row_ptr[n];
    if (nnz <= 0 || (nnz & 1))
        return OQ_EINVAL;
    const int64_t E = nnz / 2; /* |E|, each undirected edge stored as two arcs */

    int64_t *size = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *ein = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *eout = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    uint64_t *keys = (uint64_t *)malloc((size_t)(E > 0 ? E : 1) * sizeof(uint64_t));
    long double *split = (long double *)calloc((size_t)K, sizeof(long double));
    if (!size || !ein || !eout || !keys || !split) {
        free(size); free(ein); free(eout); free(keys); free(split);
        return OQ_ENOMEM;
    }
    int rc = OQ_OK;

    /* community sizes |c| */
    for (int64_t u = 0; u < n; u++)
        size[label[u]]++;

    /* classify each undirected edge once (v > u):
     * inside a community -> |E_c^in|; otherwise it is on the boundary of both
     * communities (|E_c^out|) and joins the pair (min, max) for |E_ci,cj|. */
    int64_t nkeys = 0;
    for (int64_t u = 0; u < n; u++) {
        int32_t lu = label[u];
        for (int64_t k = row_ptr[u]; k < row_ptr[u + 1]; k++) {
            int32_t v = col[k];
            if (v <= u)
                continue;
            int32_t lv = label[v];
            if (lu == lv) {
                ein[lu]++;
            } else {
                eout[lu]++;
                eout[lv]++;
                uint64_t a = (uint64_t)(lu < lv ? lu : lv), b = (uint64_t)(lu < lv ? lv : lu);
                keys[nkeys++] = (a << 32) | b;
            }
        }
    }

    /* identities: sum_c (2 Ein + Eout) = 2|E|; sum Ein + sum Eout / 2 = |E| */
    int64_t s_in = 0, s_out = 0;
    for (int32_t c = 0; c < K; c++) { s_in += ein[c]; s_out += eout[c]; }
    if (2 * s_in + s_out != nnz || s_in + s_out / 2 != E || (s_out & 1) || s_out / 2 != nkeys)
        rc = OQ_ECHECK;

    /* |E_ci,cj| by sorting the pair keys and counting runs */
    qsort(keys, (size_t)nkeys, sizeof(uint64_t), cmp_u64);
    int64_t npairs = 0, sq_check = 0;
    int64_t *pair_sum = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    if (!pair_sum) rc = OQ_ENOMEM;
    for (int64_t s = 0; s < nkeys && rc == OQ_OK;) {
        int64_t t = s;
        while (t < nkeys && keys[t] == keys[s]) t++;
        int64_t cnt = t - s;
        int32_t ci = (int32_t)(keys[s] >> 32), cj = (int32_t)(keys[s] & 0xffffffffu);
        npairs++;
        sq_check += cnt * cnt;
        pair_sum[ci] += cnt;
        pair_sum[cj] += cnt;
        /* Eq. (9): |E_ci,cj| / (2|E|) * d_ci,cj with d_ci,cj = |E_ci,cj| / (|ci||cj|);
         * the ordered sum over c_j != c_i adds this term to both communities. */
        long double eij = (long double)cnt;
        long double term = (eij / (2.0L * (long double)E)) *
                           (eij / ((long double)size[ci] * (long double)size[cj]));
        split[ci] += term;
        split[cj] += term;
        s = t;
    }
    for (int32_t c = 0; c < K && rc == OQ_OK; c++)
        if (pair_sum[c] != eout[c])
            rc = OQ_ECHECK; /* sum_j |E_ij| = |E_i^out| */
    free(pair_sum);

    oq_sum q = {0, 0}, qabs = {0, 0}, qds = {0, 0}, qdsabs = {0, 0};
    oq_sum m_in = {0, 0}, m_dens = {0, 0}, m_contr = {0, 0}, m_out = {0, 0}, m_exp = {0, 0}, m_cond = {0, 0};
    int64_t nonempty = 0;
    const long double LE = (long double)E;
    for (int32_t c = 0; c < K && rc == OQ_OK; c++) {
        if (size[c] == 0) {
            if (pc_size) pc_size[c] = 0;
            if (pc_ein) pc_ein[c] = 0;
            if (pc_eout) pc_eout[c] = 0;
            if (pc_density) pc_density[c] = 0;
            if (pc_contraction) pc_contraction[c] = 0;
            if (pc_expansion) pc_expansion[c] = 0;
            if (pc_conductance) pc_conductance[c] = 0;
            if (pc_qds) pc_qds[c] = 0;
            continue;
        }
        nonempty++;
        long double s = (long double)size[c], in = (long double)ein[c], out = (long double)eout[c];
        /* Eq. (8) */
        long double frac_in = in / LE;
        long double frac_vol = (2.0L * in + out) / (2.0L * LE);
        sum_add(&q, frac_in - frac_vol * frac_vol);
        sum_add(&qabs, fabsl(frac_in) + frac_vol * frac_vol);
        /* Eq. (9): d_c = 2|E_c^in| / (|c|(|c|-1)), 0 for |c| = 1 */
        long double d = size[c] > 1 ? (2.0L * in) / (s * (s - 1.0L)) : 0.0L;
        long double t1 = in / LE * d;
        long double t2 = (2.0L * in + out) / (2.0L * LE) * d;
        long double term = t1 - t2 * t2 - split[c];
        sum_add(&qds, term);
        sum_add(&qdsabs, fabsl(t1) + t2 * t2 + split[c]);
        /* Sec. II-B.3 */
        long double contraction = 2.0L * in / s;
        long double expansion = out / s;
        long double vol = 2.0L * in + out;
        long double conductance = vol > 0 ? out / vol : 0.0L;
        sum_add(&m_in, in);
        sum_add(&m_dens, d);
        sum_add(&m_contr, contraction);
        sum_add(&m_out, out);
        sum_add(&m_exp, expansion);
        sum_add(&m_cond, conductance);
        if (pc_size) pc_size[c] = size[c];
        if (pc_ein) pc_ein[c] = ein[c];
        if (pc_eout) pc_eout[c] = eout[c];
        if (pc_density) pc_density[c] = (double)d;
        if (pc_contraction) pc_contraction[c] = (double)contraction;
        if (pc_expansion) pc_expansion[c] = (double)expansion;
        if (pc_conductance) pc_conductance[c] = (double)conductance;
        if (pc_qds) pc_qds[c] = (double)term;
    }
    if (rc == OQ_OK) {
        long double ne = (long double)nonempty;
        dbl[0] = (double)sum_get(&q);
        dbl[1] = (double)sum_get(&qds);
        dbl[2] = (double)(sum_get(&m_in) / ne);
        dbl[3] = (double)(sum_get(&m_dens) / ne);
        dbl[4] = (double)(sum_get(&m_contr) / ne);
        dbl[5] = (double)(sum_get(&m_out) / ne);
        dbl[6] = (double)(sum_get(&m_exp) / ne);
        dbl[7] = (double)(sum_get(&m_cond) / ne);
        dbl[8] = (double)sum_get(&qabs);
        dbl[9] = (double)sum_get(&qdsabs);
        i64[0] = n;
        i64[1] = E;
        i64[2] = nonempty;
        i64[3] = s_in;
        i64[4] = s_out / 2;
        i64[5] = npairs;
        i64[6] = sq_check;
    }
    free(size); free(ein); free(eout); free(keys); free(split);
    return rc;
}

/*
 * Output layout of oq_compare (C = first argument = ground truth, C' = second):
 *   dbl[0] VI   Eq. (1)          dbl[1] NMI  Eq. (2)
 *   dbl[2] F-measure Eq. (3)     dbl[3] NVD  Eq. (4)
 *   dbl[4] RI   Eq. (5)          dbl[5] ARI  Eq. (6)     dbl[6] JI Eq. (7)
 *   dbl[7] sum |terms| of VI     dbl[8] sum |terms| of the NMI numerator
 *   dbl[9] |NMI denominator|
 *   i64[0] |V|, i64[1] non-empty |C|, i64[2] non-empty |C'|, i64[3] non-zero cells,
 *   i64[4] a11, i64[5] a10, i64[6] a01, i64[7] a00,
 *   i64[8] sum_c max_c' |c n c'| + sum_c' max_c |c' n c|   (NVD numerator)
 */
int oq_compare(const int32_t *a, const int32_t *b, int64_t n, int32_t ka, int32_t kb,
               double *dbl, int64_t *i64)
{
    if (n < 2 || ka < 1 || kb < 1)
        return OQ_EINVAL;
    for (int64_t i = 0; i < n; i++)
        if (a[i] < 0 || a[i] >= ka || b[i] < 0 || b[i] >= kb)
            return OQ_EINVAL;
    int64_t *na = (int64_t *)calloc((size_t)ka, sizeof(int64_t));
    int64_t *nb = (int64_t *)calloc((size_t)kb, sizeof(int64_t));
    uint64_t *keys = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    int64_t *rowmax = (int64_t *)calloc((size_t)ka, sizeof(int64_t));
    int64_t *colmax = (int64_t *)calloc((size_t)kb, sizeof(int64_t));
    long double *rowbest = (long double *)calloc((size_t)ka, sizeof(long double));
    if (!na || !nb || !keys || !rowmax || !colmax || !rowbest) {
        free(na); free(nb); free(keys); free(rowmax); free(colmax); free(rowbest);
        return OQ_ENOMEM;
    }
    for (int64_t i = 0; i < n; i++) {
        na[a[i]]++;
        nb[b[i]]++;
        keys[i] = ((uint64_t)(uint32_t)a[i] << 32) | (uint64_t)(uint32_t)b[i];
    }
    /* contingency cells |c n c'| by sorting (c, c') keys */
    qsort(keys, (size_t)n, sizeof(uint64_t), cmp_u64);
    const long double N = (long double)n;
    oq_sum vi = {0, 0}, viabs = {0, 0}, num = {0, 0}, numabs = {0, 0}, den = {0, 0};
    int64_t ncells = 0, a11 = 0, total = 0;
    for (int64_t s = 0; s < n;) {
        int64_t t = s;
        while (t < n && keys[t] == keys[s]) t++;
        int64_t cnt = t - s;
        int32_t ca = (int32_t)(keys[s] >> 32), cb = (int32_t)(keys[s] & 0xffffffffu);
        ncells++;
        total += cnt;
        long double x = (long double)cnt;
        long double sa = (long double)na[ca], sb = (long double)nb[cb];
        /* Eq. (1) term: |c n c'| log(|c n c'|^2 / (|c||c'|)) */
        long double tv = x * logl(x * x / (sa * sb));
        sum_add(&vi, tv);
        sum_add(&viabs, fabsl(tv));
        /* Eq. (2) numerator term: |c n c'|/|V| log(|c n c'||V| / (|c||c'|)) */
        long double tn = x / N * logl(x * N / (sa * sb));
        sum_add(&num, tn);
        sum_add(&numabs, fabsl(tn));
        /* Eq. (3): max over c' of 2|c n c'| / (|c| + |c'|) */
        long double r = 2.0L * x / (sa + sb);
        if (r > rowbest[ca]) rowbest[ca] = r;
        /* Eq. (4): row and column maxima of |c n c'| */
        if (cnt > rowmax[ca]) rowmax[ca] = cnt;
        if (cnt > colmax[cb]) colmax[cb] = cnt;
        /* Sec. II-A.3: pairs inside one cell are together in both partitions */
        a11 += cnt * (cnt - 1) / 2;
        s = t;
    }
    int rc = (total == n) ? OQ_OK : OQ_ECHECK;
    int64_t sa2 = 0, sb2 = 0, nvdsum = 0, kan = 0, kbn = 0;
    oq_sum f = {0, 0};
    for (int32_t c = 0; c < ka; c++) {
        if (na[c] == 0) continue;
        kan++;
        long double p = (long double)na[c] / N;
        sum_add(&den, p * logl(p));
        sa2 += na[c] * (na[c] - 1) / 2;
        nvdsum += rowmax[c];
        sum_add(&f, (long double)na[c] * rowbest[c]);
    }
    for (int32_t c = 0; c < kb; c++) {
        if (nb[c] == 0) continue;
        kbn++;
        long double p = (long double)nb[c] / N;
        sum_add(&den, p * logl(p));
        sb2 += nb[c] * (nb[c] - 1) / 2;
        nvdsum += colmax[c];
    }
    /* Sec. II-A.3 pair counts from the table: a11 + a10 = sum_c C(|c|,2),
     * a11 + a01 = sum_c' C(|c'|,2), A = C(|V|,2) */
    int64_t A = n * (n - 1) / 2;
    int64_t a10 = sa2 - a11, a01 = sb2 - a11, a00 = A - a11 - a10 - a01;
    if (a10 < 0 || a01 < 0 || a00 < 0)
        rc = OQ_ECHECK;
    if (rc == OQ_OK) {
        long double LA = (long double)A;
        long double l11 = (long double)a11, l10 = (long double)a10, l01 = (long double)a01, l00 = (long double)a00;
        dbl[0] = (double)(-sum_get(&vi) / N);
        long double dd = sum_get(&den);
        dbl[1] = dd != 0.0L ? (double)(-2.0L * sum_get(&num) / dd) : 1.0;
        dbl[2] = (double)(sum_get(&f) / N);
        dbl[3] = (double)(1.0L - (long double)nvdsum / (2.0L * N));
        dbl[4] = (double)((l11 + l00) / LA);
        long double M = (l11 + l10) * (l11 + l01) / LA;  /* Eq. (6) */
        long double ari_den = 0.5L * ((l11 + l10) + (l11 + l01)) - M;
        dbl[5] = ari_den != 0.0L ? (double)((l11 - M) / ari_den) : 1.0;
        long double ji_den = l11 + l10 + l01;
        dbl[6] = ji_den != 0.0L ? (double)(l11 / ji_den) : 1.0;
        dbl[7] = (double)(sum_get(&viabs) / N);
        dbl[8] = (double)(2.0L * sum_get(&numabs));
        dbl[9] = (double)fabsl(dd);
        i64[0] = n; i64[1] = kan; i64[2] = kbn; i64[3] = ncells;
        i64[4] = a11; i64[5] = a10; i64[6] = a01; i64[7] = a00; i64[8] = nvdsum;
    }
    free(na); free(nb); free(keys); free(rowmax); free(colmax); free(rowbest);
    return rc;
}

/*
 * Algorithm 4 (Pthreads pair counting), single thread: every unordered node
 * pair i < j is classified by whether it is together in C and in C'.
 * out[0..3] = a11, a10, a01, a00.  O(|V|^2): tiny inputs only.
 */
int oq_pairs_bruteforce(const int32_t *a, const int32_t *b, int64_t n, int64_t *out)
{
    if (n < 2)
        return OQ_EINVAL;
    int64_t a11 = 0, a10 = 0, a01 = 0, a00 = 0;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = i + 1; j < n; j++) {
            int sa = a[i] == a[j], sb = b[i] == b[j];
            if (sa && sb) a11++;
            else if (sa) a10++;
            else if (sb) a01++;
            else a00++;
        }
    out[0] = a11; out[1] = a10; out[2] = a01; out[3] = a00;
    return OQ_OK;
}

/*
 * Set-intersection form of Eqs. (1)-(4), the cost model of Algorithms 1-2:
 * for every community pair (c, c') count |c n c'| by scanning all nodes.
 * O(|C||C'||V|): tiny inputs only.  dbl[0..3] = VI, NMI, F-measure, NVD.
 */
int oq_compare_bruteforce(const int32_t *a, const int32_t *b, int64_t n, int32_t ka, int32_t kb,
                          double *dbl)
{
    if (n < 2)
        return OQ_EINVAL;
    const long double N = (long double)n;
    oq_sum vi = {0, 0}, num = {0, 0}, den = {0, 0}, f = {0, 0};
    int64_t nvd = 0;
    for (int32_t c = 0; c < ka; c++) {
        int64_t sc = 0;
        for (int64_t i = 0; i < n; i++) sc += a[i] == c;
        if (sc == 0) continue;
        long double best = 0.0L;
        int64_t bestn = 0;
        for (int32_t d = 0; d < kb; d++) {
            int64_t sd = 0, both = 0;
            for (int64_t i = 0; i < n; i++) {
                sd += b[i] == d;
                both += (a[i] == c) && (b[i] == d);
            }
            if (sd == 0 || both == 0) continue;
            long double x = (long double)both;
            sum_add(&vi, x * logl(x * x / ((long double)sc * (long double)sd)));
            sum_add(&num, x / N * logl(x * N / ((long double)sc * (long double)sd)));
            long double r = 2.0L * x / ((long double)sc + (long double)sd);
            if (r > best) best = r;
            if (both > bestn) bestn = both;
        }
        sum_add(&f, (long double)sc * best);
        nvd += bestn;
        long double p = (long double)sc / N;
        sum_add(&den, p * logl(p));
    }
    for (int32_t d = 0; d < kb; d++) {
        int64_t sd = 0;
        for (int64_t i = 0; i < n; i++) sd += b[i] == d;
        if (sd == 0) continue;
        int64_t bestn = 0;
        for (int32_t c = 0; c < ka; c++) {
            int64_t both = 0;
            for (int64_t i = 0; i < n; i++) both += (a[i] == c) && (b[i] == d);
            if (both > bestn) bestn = both;
        }
        nvd += bestn;
        long double p = (long double)sd / N;
        sum_add(&den, p * logl(p));
    }
    dbl[0] = (double)(-sum_get(&vi) / N);
    long double dd = sum_get(&den);
    dbl[1] = dd != 0.0L ? (double)(-2.0L * sum_get(&num) / dd) : 1.0;
    dbl[2] = (double)(sum_get(&f) / N);
    dbl[3] = (double)(1.0L - (long double)nvd / (2.0L * N));
    return OQ_OK;
}

/*
 * Definition-level form of Eqs. (8)-(9) for tiny graphs: for every ordered
 * community pair (ci, cj) count |E_ci,cj| by scanning every arc, and count
 * |E_c^in| and |E_c^out| per community by scanning every arc.  O(K^2 |E|).
 * dbl[0] = Q, dbl[1] = Qds.
 */
int oq_score_bruteforce(const int64_t *row_ptr, const int32_t *col, int64_t n,
                        const int32_t *label, int32_t K, double *dbl)
{
    int64_t nnz = row_ptr[n];
    if (nnz <= 0)
        return OQ_EINVAL;
    const long double E = (long double)(nnz / 2);
    oq_sum q = {0, 0}, qds = {0, 0};
    for (int32_t ci = 0; ci < K; ci++) {
        int64_t size = 0, in_arcs = 0, out_arcs = 0;
        for (int64_t u = 0; u < n; u++) size += label[u] == ci;
        if (size == 0) continue;
        for (int64_t u = 0; u < n; u++) {
            if (label[u] != ci) continue;
            for (int64_t k = row_ptr[u]; k < row_ptr[u + 1]; k++) {
                if (label[col[k]] == ci) in_arcs++;
                else out_arcs++;
            }
        }
        long double in = (long double)(in_arcs / 2), out = (long double)out_arcs;
        long double frac_vol = (2.0L * in + out) / (2.0L * E);
        sum_add(&q, in / E - frac_vol * frac_vol);
        long double s = (long double)size;
        long double d = size > 1 ? 2.0L * in / (s * (s - 1.0L)) : 0.0L;
        long double split = 0.0L;
        for (int32_t cj = 0; cj < K; cj++) {
            if (cj == ci) continue;
            int64_t sj = 0, eij = 0;
            for (int64_t u = 0; u < n; u++) sj += label[u] == cj;
            if (sj == 0) continue;
            for (int64_t u = 0; u < n; u++) {
                if (label[u] != ci) continue;
                for (int64_t k = row_ptr[u]; k < row_ptr[u + 1]; k++)
                    eij += label[col[k]] == cj;
            }
            long double x = (long double)eij;
            split += x / (2.0L * E) * (x / (s * (long double)sj));
        }
        long double t2 = frac_vol * d;
        sum_add(&qds, in / E * d - t2 * t2 - split);
    }
    dbl[0] = (double)sum_get(&q);
    dbl[1] = (double)sum_get(&qds);
    return OQ_OK;
}

/*
 * Per-community evaluation for a sample of community ids (used to check very
 * large inputs one community at a time).  For each sampled community c it
 * collects the members of c, walks their rows, and counts |E_c^in|, |E_c^out|
 * and |E_c,cj| for every neighbouring community cj (sorting the neighbour
 * labels), then forms the bracketed term of Eq. (9) for c.  Community sizes come
 * from one pass over all labels.
 *   ids[m]   sampled community ids (any order, repeats allowed)
 *   out_i64  [m][4]: |c|, |E_c^in|, |E_c^out|, number of distinct cj
 *   out_dbl  [m][2]: Qds term of c (Eq. 9), split penalty sum_j |E_cj|^2/(2|E||c||cj|)
 */
int oq_score_communities(const int64_t *row_ptr, const int32_t *col, int64_t n,
                         const int32_t *label, int32_t K, const int32_t *ids, int64_t m,
                         int64_t *out_i64, double *out_dbl)
{
    if (n < 1 || K < 1 || m < 0)
        return OQ_EINVAL;
    int64_t nnz = row_ptr[n];
    if (nnz <= 0)
        return OQ_EINVAL;
    const long double E = (long double)(nnz / 2);
    int64_t *size = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    if (!size)
        return OQ_ENOMEM;
    for (int64_t u = 0; u < n; u++) {
        if (label[u] < 0 || label[u] >= K) { free(size); return OQ_EINVAL; }
        size[label[u]]++;
    }
    int rc = OQ_OK;
    for (int64_t s = 0; s < m && rc == OQ_OK; s++) {
        const int32_t c = ids[s];
        if (c < 0 || c >= K) { rc = OQ_EINVAL; break; }
        int64_t in_arcs = 0, out_arcs = 0, nb = 0;
        int32_t *nbr = NULL;
        size_t cap = 0;
        for (int64_t u = 0; u < n; u++) {
            if (label[u] != c) continue;
            for (int64_t k = row_ptr[u]; k < row_ptr[u + 1]; k++) {
                int32_t lv = label[col[k]];
                if (lv == c) { in_arcs++; continue; }
                out_arcs++;
                if ((size_t)nb == cap) {
                    cap = cap ? 2 * cap : 1024;
                    int32_t *t = (int32_t *)realloc(nbr, cap * sizeof(int32_t));
                    if (!t) { rc = OQ_ENOMEM; break; }
                    nbr = t;
                }
                nbr[nb++] = lv;
            }
            if (rc != OQ_OK) break;
        }
        if (rc != OQ_OK) { free(nbr); break; }
        qsort(nbr, (size_t)nb, sizeof(int32_t), cmp_i32);
        long double split = 0.0L, sc = (long double)size[c];
        int64_t distinct = 0;
        for (int64_t a = 0; a < nb;) {
            int64_t b = a;
            while (b < nb && nbr[b] == nbr[a]) b++;
            long double x = (long double)(b - a);
            split += (x / (2.0L * E)) * (x / (sc * (long double)size[nbr[a]]));
            distinct++;
            a = b;
        }
        free(nbr);
        long double in = (long double)(in_arcs / 2), out = (long double)out_arcs;
        long double d = size[c] > 1 ? 2.0L * in / (sc * (sc - 1.0L)) : 0.0L;
        long double t1 = in / E * d;
        long double t2 = (2.0L * in + out) / (2.0L * E) * d;
        out_i64[4 * s + 0] = size[c];
        out_i64[4 * s + 1] = in_arcs / 2;
        out_i64[4 * s + 2] = out_arcs;
        out_i64[4 * s + 3] = distinct;
        out_dbl[2 * s + 0] = size[c] ? (double)(t1 - t2 * t2 - split) : 0.0;
        out_dbl[2 * s + 1] = (double)split;
    }
    free(size);
    return rc;
}

/*
 * oq_label_propagation -- plain synchronous label propagation, the O(|E|)
 * detector family whose output C' the paper scores (Sec. I, Sec. IV-C); not
 * SLPA itself, whose exact rules the paper leaves to its cited source (parity
 * against SLPA unpinned).  Rules, applied to every node at once in each round:
 *   - labels start as the node ids;
 *   - a node looks at its neighbours' labels; when deg > 32 it looks only at
 *     the neighbours in row positions floor(i * deg / 32), i = 0..31;
 *   - it takes the label seen most often; it keeps its own label when that is
 *     among the most frequent, else it takes the smallest of them; a node with
 *     no neighbours keeps its label.
 * Afterwards the labels present are renumbered in increasing order of value
 * to 0..K'-1.  The counting is a plain double loop over the (at most 32)
 * labels seen.
 *   out[n]   final labels in [0, K'),  *k_out = K'
 */
int oq_label_propagation(const int64_t *row_ptr, const int32_t *col, int64_t n, int32_t rounds,
                         int32_t *out, int32_t *k_out)
{
    if (n < 1 || rounds < 0)
        return OQ_EINVAL;
    int32_t *cur = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *nxt = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *rank = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    if (!cur || !nxt || !rank) { free(cur); free(nxt); free(rank); return OQ_ENOMEM; }
    for (int64_t u = 0; u < n; u++)
        cur[u] = (int32_t)u;
    for (int32_t r = 0; r < rounds; r++) {
        for (int64_t u = 0; u < n; u++) {
            const int64_t deg = row_ptr[u + 1] - row_ptr[u];
            int32_t seen[32];
            int m = 0;
            for (int64_t i = 0; i < (deg < 32 ? deg : 32); i++) {
                const int64_t pos = deg <= 32 ? i : i * deg / 32;
                seen[m++] = cur[col[row_ptr[u] + pos]];
            }
            int32_t best = cur[u];
            int best_count = 0, own_count = 0;
            for (int a = 0; a < m; a++) {
                int count = 0;
                for (int b = 0; b < m; b++)
                    count += seen[b] == seen[a];
                if (seen[a] == cur[u])
                    own_count = count;
                if (count > best_count || (count == best_count && seen[a] < best)) {
                    best_count = count;
                    best = seen[a];
                }
            }
            if (m > 0 && own_count == best_count)
                best = cur[u];
            nxt[u] = m > 0 ? best : cur[u];
        }
        int32_t *t = cur; cur = nxt; nxt = t;
    }
    for (int64_t u = 0; u < n; u++)
        rank[cur[u]] = 1;
    int32_t k = 0;
    for (int64_t c = 0; c < n; c++) {
        const int32_t present = rank[c];
        rank[c] = k;
        k += present;
    }
    for (int64_t u = 0; u < n; u++)
        out[u] = rank[cur[u]];
    *k_out = k;
    free(cur); free(nxt); free(rank);
    return OQ_OK;
}

/*
 * oq_score_weighted -- Eq. (8) and Eq. (9) on a weighted undirected graph, in
 * the reading the paper's note on the weighted case gives: every edge count
 * that measures amount (|E|, |E_c^in|, |E_c^out|, |E_ci,cj| outside the
 * densities) becomes a sum of edge weights, while the densities d_c and
 * d_ci,cj keep the unweighted counts, so that they stay at most 1:
 *   Q_w   = sum_c [ W_c^in / W - ((2 W_c^in + W_c^out) / (2W))^2 ]
 *   Qds_w = sum_ci [ W_ci^in / W d_ci - ((2 W_ci^in + W_ci^out) / (2W) d_ci)^2
 *                    - sum_{cj != ci} W_ci,cj / (2W) d_ci,cj ]
 * with W the total edge weight, d_c = 2|E_c^in| / (|c|(|c|-1)) and
 * d_ci,cj = |E_ci,cj| / (|ci||cj|).  Edges are visited once (v > u) with the
 * weight stored on arc (u, v); weight[] runs parallel to col[].
 *   dbl[0] Q_w, dbl[1] Qds_w, dbl[2] sum |terms| of Q_w, dbl[3] sum |terms| of Qds_w,
 *   dbl[4] W
 * Returns OQ_EINVAL for a non-positive total weight or a bad label.
 */
typedef struct {
    uint64_t key;
    long double w;
} oq_wkey;

static int cmp_wkey(const void *a, const void *b)
{
    uint64_t x = ((const oq_wkey *)a)->key, y = ((const oq_wkey *)b)->key;
    return x < y ? -1 : (x > y ? 1 : 0);
}

int oq_score_weighted(const int64_t *row_ptr, const int32_t *col, const double *weight, int64_t n,
                      const int32_t *label, int32_t K, double *dbl)
{
    if (n < 1 || K < 1)
        return OQ_EINVAL;
    for (int64_t u = 0; u < n; u++)
        if (label[u] < 0 || label[u] >= K)
            return OQ_EINVAL;
    const int64_t nnz = row_ptr[n];
    if (nnz <= 0 || (nnz & 1))
        return OQ_EINVAL;
    const int64_t E = nnz / 2;
    int64_t *size = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *ein = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    long double *win = (long double *)calloc((size_t)K, sizeof(long double));
    long double *wout = (long double *)calloc((size_t)K, sizeof(long double));
    long double *split = (long double *)calloc((size_t)K, sizeof(long double));
    oq_wkey *keys = (oq_wkey *)malloc((size_t)E * sizeof(oq_wkey));
    if (!size || !ein || !win || !wout || !split || !keys) {
        free(size); free(ein); free(win); free(wout); free(split); free(keys);
        return OQ_ENOMEM;
    }
    for (int64_t u = 0; u < n; u++)
        size[label[u]]++;
    long double W = 0.0L;
    int64_t nkeys = 0;
    for (int64_t u = 0; u < n; u++) {
        const int32_t lu = label[u];
        for (int64_t k = row_ptr[u]; k < row_ptr[u + 1]; k++) {
            const int32_t v = col[k];
            if (v <= u)
                continue;
            const long double w = (long double)weight[k];
            W += w;
            const int32_t lv = label[v];
            if (lu == lv) {
                ein[lu]++;
                win[lu] += w;
            } else {
                wout[lu] += w;
                wout[lv] += w;
                const uint64_t a = (uint64_t)(lu < lv ? lu : lv), b = (uint64_t)(lu < lv ? lv : lu);
                keys[nkeys].key = (a << 32) | b;
                keys[nkeys].w = w;
                nkeys++;
            }
        }
    }
    int rc = W > 0.0L ? OQ_OK : OQ_EINVAL;
    /* per unordered pair: the count |E_ci,cj| and the weight W_ci,cj */
    qsort(keys, (size_t)nkeys, sizeof(oq_wkey), cmp_wkey);
    for (int64_t s = 0; s < nkeys && rc == OQ_OK;) {
        int64_t t = s;
        long double wij = 0.0L;
        while (t < nkeys && keys[t].key == keys[s].key) {
            wij += keys[t].w;
            t++;
        }
        const long double cnt = (long double)(t - s);
        const int32_t ci = (int32_t)(keys[s].key >> 32), cj = (int32_t)(keys[s].key & 0xffffffffu);
        const long double term = (wij / (2.0L * W)) * (cnt / ((long double)size[ci] * (long double)size[cj]));
        split[ci] += term;
        split[cj] += term;
        s = t;
    }
    oq_sum q = {0, 0}, qabs = {0, 0}, qds = {0, 0}, qdsabs = {0, 0};
    for (int32_t c = 0; c < K && rc == OQ_OK; c++) {
        if (size[c] == 0)
            continue;
        const long double s = (long double)size[c];
        const long double fin = win[c] / W, fvol = (2.0L * win[c] + wout[c]) / (2.0L * W);
        sum_add(&q, fin - fvol * fvol);
        sum_add(&qabs, fabsl(fin) + fvol * fvol);
        const long double d = size[c] > 1 ? (2.0L * (long double)ein[c]) / (s * (s - 1.0L)) : 0.0L;
        const long double t1 = fin * d, t2 = fvol * d;
        sum_add(&qds, t1 - t2 * t2 - split[c]);
        sum_add(&qdsabs, fabsl(t1) + t2 * t2 + split[c]);
    }
    if (rc == OQ_OK) {
        dbl[0] = (double)sum_get(&q);
        dbl[1] = (double)sum_get(&qds);
        dbl[2] = (double)sum_get(&qabs);
        dbl[3] = (double)sum_get(&qdsabs);
        dbl[4] = (double)W;
    }
    free(size); free(ein); free(win); free(wout); free(split); free(keys);
    return rc;
}

/* ------------------------------------------------------------------------
 * All-core statement of oq_score for the timed CPU baseline.
 *
 * oq_score_omp computes oq_score's quantities (same dbl[0..9], i64[0..6]
 * layout, no per-community arrays) with OpenMP threads over the host cores,
 * in the same steps: community sizes; each undirected edge classified once
 * (v > u) into |E_c^in|, |E_c^out| and an unordered pair key; the keys sorted
 * and counted by runs into |E_ci,cj| and the Eq. (9) split penalty of both
 * communities; then Eqs. (8)-(9) and the Sec. II-B.3 measures community by
 * community, summed on one thread.  Threads take static node chunks with
 * private counters and key buffers (merged afterwards); the sort buckets the
 * keys by ranges of their smaller community id and sorts each bucket on its
 * own; split penalties go to per-thread arrays added in thread order.  It
 * differs from oq_score only in the order of the long double additions of the
 * split penalties.  Built without -fopenmp it runs on one thread.
 * *threads receives the number of threads used.
 * ------------------------------------------------------------------------ */
#ifdef _OPENMP
#include <omp.h>
#endif

static int oq_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int oq_thread_id(void)
{
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

int oq_score_omp(const int64_t *row_ptr, const int32_t *col, int64_t n, const int32_t *label, int32_t K,
                 double *dbl, int64_t *i64, int32_t *threads)
{
    if (n < 1 || K < 1)
        return OQ_EINVAL;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t u = 0; u < n; u++)
        if (label[u] < 0 || label[u] >= K)
            bad = 1;
    if (bad)
        return OQ_EINVAL;
    const int64_t nnz = row_ptr[n];
    if (nnz <= 0 || (nnz & 1))
        return OQ_EINVAL;
    const int64_t E = nnz / 2;
    const int T = oq_max_threads();
    const size_t TK = (size_t)T * (size_t)K;
    const int B = 4 * T; /* key buckets by ranges of the smaller community id */
    int64_t *tsize = (int64_t *)calloc(TK, sizeof(int64_t));
    int64_t *tein = (int64_t *)calloc(TK, sizeof(int64_t));
    int64_t *teout = (int64_t *)calloc(TK, sizeof(int64_t));
    uint64_t **tkeys = (uint64_t **)calloc((size_t)T, sizeof(uint64_t *));
    int64_t *tn = (int64_t *)calloc((size_t)T, sizeof(int64_t));
    int64_t *tb = (int64_t *)calloc((size_t)T * (size_t)B, sizeof(int64_t)); /* keys per (thread, bucket) */
    int64_t *boff = (int64_t *)calloc((size_t)B + 1, sizeof(int64_t));
    int64_t *size = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *ein = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *eout = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    if (!tsize || !tein || !teout || !tkeys || !tn || !tb || !boff || !size || !ein || !eout) {
        free(tsize); free(tein); free(teout); free(tkeys); free(tn); free(tb); free(boff);
        free(size); free(ein); free(eout);
        return OQ_ENOMEM;
    }
    int nomem = 0;
#pragma omp parallel reduction(| : nomem)
    {
        const int t = oq_thread_id();
        int64_t *ls = tsize + (size_t)t * K, *li = tein + (size_t)t * K, *lo = teout + (size_t)t * K;
        int64_t cap = 1 << 16, cnt = 0;
        uint64_t *buf = (uint64_t *)malloc((size_t)cap * sizeof(uint64_t));
        if (!buf) nomem = 1;
#pragma omp for schedule(static)
        for (int64_t u = 0; u < n; u++) {
            const int32_t lu = label[u];
            ls[lu]++;
            for (int64_t k = row_ptr[u]; k < row_ptr[u + 1]; k++) {
                const int32_t v = col[k];
                if (v <= u) continue;
                const int32_t lv = label[v];
                if (lu == lv) {
                    li[lu]++;
                    continue;
                }
                lo[lu]++;
                lo[lv]++;
                if (!buf) continue;
                if (cnt == cap) {
                    uint64_t *nb = (uint64_t *)realloc(buf, (size_t)cap * 2 * sizeof(uint64_t));
                    if (!nb) { free(buf); buf = NULL; nomem = 1; continue; }
                    buf = nb;
                    cap *= 2;
                }
                const uint64_t a = (uint64_t)(lu < lv ? lu : lv), b = (uint64_t)(lu < lv ? lv : lu);
                buf[cnt++] = (a << 32) | b;
            }
        }
        tkeys[t] = buf;
        tn[t] = cnt;
        if (buf)
            for (int64_t i = 0; i < cnt; i++)
                tb[(size_t)t * B + (int)((buf[i] >> 32) * (uint64_t)B / (uint64_t)K)]++;
    }
    int rc = nomem ? OQ_ENOMEM : OQ_OK;
    /* merged counters */
#pragma omp parallel for schedule(static)
    for (int32_t c = 0; c < K; c++)
        for (int t = 0; t < T; t++) {
            size[c] += tsize[(size_t)t * K + c];
            ein[c] += tein[(size_t)t * K + c];
            eout[c] += teout[(size_t)t * K + c];
        }
    free(tsize); free(tein); free(teout);
    int64_t s_in = 0, s_out = 0, nkeys = 0;
    for (int32_t c = 0; c < K; c++) { s_in += ein[c]; s_out += eout[c]; }
    for (int t = 0; t < T; t++) nkeys += tn[t];
    if (rc == OQ_OK && (2 * s_in + s_out != nnz || s_in + s_out / 2 != E || (s_out & 1) || s_out / 2 != nkeys))
        rc = OQ_ECHECK;
    uint64_t *keys = rc == OQ_OK ? (uint64_t *)malloc((size_t)(nkeys > 0 ? nkeys : 1) * sizeof(uint64_t)) : NULL;
    if (rc == OQ_OK && !keys) rc = OQ_ENOMEM;
    long double *tsplit = NULL;
    int64_t *tpair = NULL;
    int64_t npairs = 0, sq_check = 0;
    if (rc == OQ_OK) {
        /* bucket offsets, then every thread scatters its keys into its slice of each bucket */
        int64_t *at = (int64_t *)malloc((size_t)T * (size_t)B * sizeof(int64_t));
        if (!at) rc = OQ_ENOMEM;
        if (rc == OQ_OK) {
            int64_t acc = 0;
            for (int b = 0; b < B; b++) {
                boff[b] = acc;
                for (int t = 0; t < T; t++) {
                    at[(size_t)t * B + b] = acc;
                    acc += tb[(size_t)t * B + b];
                }
            }
            boff[B] = acc;
#pragma omp parallel for schedule(static)
            for (int t = 0; t < T; t++) {
                int64_t *pos = at + (size_t)t * B;
                for (int64_t i = 0; i < tn[t]; i++) {
                    const uint64_t key = tkeys[t][i];
                    keys[pos[(int)((key >> 32) * (uint64_t)B / (uint64_t)K)]++] = key;
                }
            }
#pragma omp parallel for schedule(dynamic, 1)
            for (int b = 0; b < B; b++)
                qsort(keys + boff[b], (size_t)(boff[b + 1] - boff[b]), sizeof(uint64_t), cmp_u64);
        }
        free(at);
        tsplit = (long double *)calloc(TK, sizeof(long double));
        tpair = (int64_t *)calloc(TK, sizeof(int64_t));
        if (rc == OQ_OK && (!tsplit || !tpair)) rc = OQ_ENOMEM;
    }
    for (int t = 0; t < T; t++) free(tkeys[t]);
    free(tkeys); free(tn); free(tb);
    if (rc == OQ_OK) {
        /* |E_ci,cj| by runs; the Eq. (9) split term goes to both communities */
#pragma omp parallel for schedule(static) reduction(+ : npairs, sq_check)
        for (int b = 0; b < B; b++) {
            const int t = oq_thread_id();
            long double *sp = tsplit + (size_t)t * K;
            int64_t *ps = tpair + (size_t)t * K;
            for (int64_t s = boff[b]; s < boff[b + 1];) {
                int64_t u = s;
                while (u < boff[b + 1] && keys[u] == keys[s]) u++;
                const int64_t cnt = u - s;
                const int32_t ci = (int32_t)(keys[s] >> 32), cj = (int32_t)(keys[s] & 0xffffffffu);
                npairs++;
                sq_check += cnt * cnt;
                ps[ci] += cnt;
                ps[cj] += cnt;
                const long double eij = (long double)cnt;
                const long double term = (eij / (2.0L * (long double)E)) *
                                         (eij / ((long double)size[ci] * (long double)size[cj]));
                sp[ci] += term;
                sp[cj] += term;
                s = u;
            }
        }
    }
    free(keys);
    long double *split = tsplit ? (long double *)calloc((size_t)K, sizeof(long double)) : NULL;
    if (rc == OQ_OK && !split) rc = OQ_ENOMEM;
    if (rc == OQ_OK) {
#pragma omp parallel for schedule(static) reduction(| : bad)
        for (int32_t c = 0; c < K; c++) {
            int64_t p = 0;
            for (int t = 0; t < T; t++) {
                split[c] += tsplit[(size_t)t * K + c];
                p += tpair[(size_t)t * K + c];
            }
            if (p != eout[c]) bad = 1; /* sum_j |E_ij| = |E_i^out| */
        }
        if (bad) rc = OQ_ECHECK;
    }
    free(tsplit); free(tpair);
    if (rc == OQ_OK) {
        oq_sum q = {0, 0}, qabs = {0, 0}, qds = {0, 0}, qdsabs = {0, 0};
        oq_sum m_in = {0, 0}, m_dens = {0, 0}, m_contr = {0, 0}, m_out = {0, 0}, m_exp = {0, 0}, m_cond = {0, 0};
        int64_t nonempty = 0;
        const long double LE = (long double)E;
        for (int32_t c = 0; c < K; c++) {
            if (size[c] == 0) continue;
            nonempty++;
            const long double s = (long double)size[c], in = (long double)ein[c], out = (long double)eout[c];
            const long double frac_in = in / LE, frac_vol = (2.0L * in + out) / (2.0L * LE);
            sum_add(&q, frac_in - frac_vol * frac_vol);
            sum_add(&qabs, fabsl(frac_in) + frac_vol * frac_vol);
            const long double d = size[c] > 1 ? (2.0L * in) / (s * (s - 1.0L)) : 0.0L;
            const long double t1 = in / LE * d, t2 = (2.0L * in + out) / (2.0L * LE) * d;
            sum_add(&qds, t1 - t2 * t2 - split[c]);
            sum_add(&qdsabs, fabsl(t1) + t2 * t2 + split[c]);
            const long double vol = 2.0L * in + out;
            sum_add(&m_in, in);
            sum_add(&m_dens, d);
            sum_add(&m_contr, 2.0L * in / s);
            sum_add(&m_out, out);
            sum_add(&m_exp, out / s);
            sum_add(&m_cond, vol > 0 ? out / vol : 0.0L);
        }
        const long double ne = (long double)nonempty;
        dbl[0] = (double)sum_get(&q);
        dbl[1] = (double)sum_get(&qds);
        dbl[2] = (double)(sum_get(&m_in) / ne);
        dbl[3] = (double)(sum_get(&m_dens) / ne);
        dbl[4] = (double)(sum_get(&m_contr) / ne);
        dbl[5] = (double)(sum_get(&m_out) / ne);
        dbl[6] = (double)(sum_get(&m_exp) / ne);
        dbl[7] = (double)(sum_get(&m_cond) / ne);
        dbl[8] = (double)sum_get(&qabs);
        dbl[9] = (double)sum_get(&qdsabs);
        i64[0] = n;
        i64[1] = E;
        i64[2] = nonempty;
        i64[3] = s_in;
        i64[4] = s_out / 2;
        i64[5] = npairs;
        i64[6] = sq_check;
    }
    free(split); free(size); free(ein); free(eout); free(boff);
    if (threads) *threads = T;
    return rc;
}

/* ------------------------------------------------------------------------
 * Overlapping communities (covers).
 *
 * The paper defines its metrics for disjoint communities and names overlapping
 * ones as future work (Sec. VI).  Every formula is written with node sets
 * (|c|, |c n c'|, edges inside c, edges leaving c, edges between c_i and c_j),
 * so a cover -- a family of node sets in which a node may belong to several
 * communities or to none -- is scored here by reading each set formula
 * literally:
 *   |c|        the members of c;
 *   |E_c^in|   edges with both ends in c;
 *   |E_c^out|  edges with exactly one end in c;
 *   |E_ci,cj|  edges {u, v} with u in c_i \ c_j and v in c_j \ c_i (an edge
 *              that leaves c_i and enters c_j; symmetric in i and j);
 *   |c n c'|   the nodes in both c and c' (one node can add to several cells);
 *   a11 etc.   a pair of nodes is "in the same community" of a cover when the
 *              two share at least one community.
 * Q, Qds, the six measures and Eqs. (1)-(7) then follow their printed formulas
 * unchanged.  For a cover in which every node has exactly one community every
 * quantity equals the partition's.
 *
 * A cover is given node by node: the communities of node u are
 * memb[mptr[u] .. mptr[u+1]), ids in [0, K), strictly increasing.
 * ------------------------------------------------------------------------ */

int oq_validate_cover(const int64_t *mptr, const int32_t *memb, int64_t n, int32_t K)
{
    if (n < 1 || K < 1 || mptr[0] != 0)
        return OQ_EINVAL;
    for (int64_t u = 0; u < n; u++) {
        if (mptr[u + 1] < mptr[u])
            return OQ_EINVAL;
        for (int64_t k = mptr[u]; k < mptr[u + 1]; k++) {
            if (memb[k] < 0 || memb[k] >= K)
                return OQ_EINVAL;
            if (k > mptr[u] && memb[k] <= memb[k - 1])
                return OQ_EINVAL;
        }
    }
    return OQ_OK;
}

/* is c among the sorted communities list[0 .. len) */
static int in_list(const int32_t *list, int64_t len, int32_t c)
{
    for (int64_t k = 0; k < len; k++)
        if (list[k] == c)
            return 1;
    return 0;
}

/*
 * Eqs. (8)-(9) and the six measures of Sec. II-B.3 for a cover, in the layout
 * of oq_score (dbl[0..9], i64[0..6]) except that i64[4] is the sum over
 * communities of |E_c^out| (for a partition, twice the cut edges).  Every
 * undirected edge is visited once (v > u) with its two communities lists A, B:
 * it is inside each c in A n B, on the boundary of each c in A \ B and B \ A,
 * and between every i in A \ B and j in B \ A.
 */
int oq_score_cover(const int64_t *row_ptr, const int32_t *col, int64_t n, const int64_t *mptr,
                   const int32_t *memb, int32_t K, double *dbl, int64_t *i64)
{
    if (oq_validate_cover(mptr, memb, n, K) != OQ_OK)
        return OQ_EINVAL;
    const int64_t nnz = row_ptr[n];
    if (nnz <= 0 || (nnz & 1))
        return OQ_EINVAL;
    const int64_t E = nnz / 2;
    int64_t *size = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *ein = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *eout = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    long double *split = (long double *)calloc((size_t)K, sizeof(long double));
    int64_t nkeys = 0, cap = 1024;
    uint64_t *keys = (uint64_t *)malloc((size_t)cap * sizeof(uint64_t));
    if (!size || !ein || !eout || !split || !keys) {
        free(size); free(ein); free(eout); free(split); free(keys);
        return OQ_ENOMEM;
    }
    int rc = OQ_OK;
    for (int64_t u = 0; u < n; u++)
        for (int64_t k = mptr[u]; k < mptr[u + 1]; k++)
            size[memb[k]]++;
    int64_t vol_check = 0;
    for (int64_t u = 0; u < n && rc == OQ_OK; u++) {
        const int32_t *A = memb + mptr[u];
        const int64_t la = mptr[u + 1] - mptr[u];
        vol_check += (row_ptr[u + 1] - row_ptr[u]) * la;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1] && rc == OQ_OK; e++) {
            const int32_t v = col[e];
            if (v <= u)
                continue;
            const int32_t *B = memb + mptr[v];
            const int64_t lb = mptr[v + 1] - mptr[v];
            for (int64_t x = 0; x < la; x++) {
                if (in_list(B, lb, A[x])) ein[A[x]]++;
                else eout[A[x]]++;
            }
            for (int64_t y = 0; y < lb; y++)
                if (!in_list(A, la, B[y])) eout[B[y]]++;
            for (int64_t x = 0; x < la; x++) {
                if (in_list(B, lb, A[x])) continue;       /* i in A \ B */
                for (int64_t y = 0; y < lb; y++) {
                    if (in_list(A, la, B[y])) continue;   /* j in B \ A */
                    if (nkeys == cap) {
                        uint64_t *nk = (uint64_t *)realloc(keys, (size_t)cap * 2 * sizeof(uint64_t));
                        if (!nk) { rc = OQ_ENOMEM; break; }
                        keys = nk;
                        cap *= 2;
                    }
                    const uint64_t a = (uint64_t)(A[x] < B[y] ? A[x] : B[y]);
                    const uint64_t b = (uint64_t)(A[x] < B[y] ? B[y] : A[x]);
                    keys[nkeys++] = (a << 32) | b;
                }
            }
        }
    }
    /* identity: the volumes sum_c (2|E_c^in| + |E_c^out|) add up the degrees of all memberships */
    int64_t s_in = 0, s_out = 0;
    for (int32_t c = 0; c < K; c++) { s_in += ein[c]; s_out += eout[c]; }
    if (rc == OQ_OK && 2 * s_in + s_out != vol_check)
        rc = OQ_ECHECK;
    qsort(keys, (size_t)nkeys, sizeof(uint64_t), cmp_u64);
    int64_t npairs = 0, sq_check = 0;
    for (int64_t s = 0; s < nkeys && rc == OQ_OK;) {
        int64_t t = s;
        while (t < nkeys && keys[t] == keys[s]) t++;
        const int64_t cnt = t - s;
        const int32_t ci = (int32_t)(keys[s] >> 32), cj = (int32_t)(keys[s] & 0xffffffffu);
        npairs++;
        sq_check += cnt * cnt;
        /* Eq. (9): |E_ci,cj| / (2|E|) * |E_ci,cj| / (|ci||cj|), to both communities */
        const long double eij = (long double)cnt;
        const long double term = (eij / (2.0L * (long double)E)) * (eij / ((long double)size[ci] * (long double)size[cj]));
        split[ci] += term;
        split[cj] += term;
        s = t;
    }
    if (rc == OQ_OK) {
        oq_sum q = {0, 0}, qabs = {0, 0}, qds = {0, 0}, qdsabs = {0, 0};
        oq_sum m_in = {0, 0}, m_dens = {0, 0}, m_contr = {0, 0}, m_out = {0, 0}, m_exp = {0, 0}, m_cond = {0, 0};
        int64_t nonempty = 0;
        const long double LE = (long double)E;
        for (int32_t c = 0; c < K; c++) {
            if (size[c] == 0) continue;
            nonempty++;
            const long double s = (long double)size[c], in = (long double)ein[c], out = (long double)eout[c];
            const long double frac_in = in / LE, frac_vol = (2.0L * in + out) / (2.0L * LE);
            sum_add(&q, frac_in - frac_vol * frac_vol);
            sum_add(&qabs, fabsl(frac_in) + frac_vol * frac_vol);
            const long double d = size[c] > 1 ? (2.0L * in) / (s * (s - 1.0L)) : 0.0L;
            const long double t1 = in / LE * d, t2 = (2.0L * in + out) / (2.0L * LE) * d;
            sum_add(&qds, t1 - t2 * t2 - split[c]);
            sum_add(&qdsabs, fabsl(t1) + t2 * t2 + split[c]);
            const long double vol = 2.0L * in + out;
            sum_add(&m_in, in);
            sum_add(&m_dens, d);
            sum_add(&m_contr, 2.0L * in / s);
            sum_add(&m_out, out);
            sum_add(&m_exp, out / s);
            sum_add(&m_cond, vol > 0 ? out / vol : 0.0L);
        }
        if (nonempty == 0) {
            rc = OQ_EINVAL;  /* no community has a member */
        } else {
            const long double ne = (long double)nonempty;
            dbl[0] = (double)sum_get(&q);
            dbl[1] = (double)sum_get(&qds);
            dbl[2] = (double)(sum_get(&m_in) / ne);
            dbl[3] = (double)(sum_get(&m_dens) / ne);
            dbl[4] = (double)(sum_get(&m_contr) / ne);
            dbl[5] = (double)(sum_get(&m_out) / ne);
            dbl[6] = (double)(sum_get(&m_exp) / ne);
            dbl[7] = (double)(sum_get(&m_cond) / ne);
            dbl[8] = (double)sum_get(&qabs);
            dbl[9] = (double)sum_get(&qdsabs);
            i64[0] = n;
            i64[1] = E;
            i64[2] = nonempty;
            i64[3] = s_in;
            i64[4] = s_out;
            i64[5] = npairs;
            i64[6] = sq_check;
        }
    }
    free(size); free(ein); free(eout); free(split); free(keys);
    return rc;
}

/* do two sorted lists share an element */
static int lists_meet(const int32_t *a, int64_t la, const int32_t *b, int64_t lb)
{
    int64_t x = 0, y = 0;
    while (x < la && y < lb) {
        if (a[x] == b[y]) return 1;
        if (a[x] < b[y]) x++; else y++;
    }
    return 0;
}

/*
 * Eqs. (1)-(7) for two covers, C = (aptr, amemb, ka) the ground truth and
 * C' = (bptr, bmemb, kb) the detected one, in the layout of oq_compare.  The
 * cells |c n c'| come from every node's pairs (c, c') of its two lists, sorted
 * and counted.  The pair counts follow their definition: a pair {i, j} is
 * together in a cover when the two share a community; each pair sharing one
 * in C is found once by walking, for every node i, the members j > i of its
 * communities and marking j.
 */
int oq_compare_cover(const int64_t *aptr, const int32_t *amemb, int32_t ka, const int64_t *bptr,
                     const int32_t *bmemb, int32_t kb, int64_t n, double *dbl, int64_t *i64)
{
    if (n < 2 || oq_validate_cover(aptr, amemb, n, ka) != OQ_OK || oq_validate_cover(bptr, bmemb, n, kb) != OQ_OK)
        return OQ_EINVAL;
    const int64_t ma = aptr[n], mb = bptr[n];
    int64_t *na = (int64_t *)calloc((size_t)ka, sizeof(int64_t));
    int64_t *nb = (int64_t *)calloc((size_t)kb, sizeof(int64_t));
    int64_t *rowmax = (int64_t *)calloc((size_t)ka, sizeof(int64_t));
    int64_t *colmax = (int64_t *)calloc((size_t)kb, sizeof(int64_t));
    long double *rowbest = (long double *)calloc((size_t)ka, sizeof(long double));
    int64_t ncell_cap = 0;
    for (int64_t i = 0; i < n; i++) ncell_cap += (aptr[i + 1] - aptr[i]) * (bptr[i + 1] - bptr[i]);
    uint64_t *keys = (uint64_t *)malloc((size_t)(ncell_cap > 0 ? ncell_cap : 1) * sizeof(uint64_t));
    /* members of every community of both covers (transposes), and the pair marks */
    int64_t *astart = (int64_t *)calloc((size_t)ka + 1, sizeof(int64_t));
    int64_t *bstart = (int64_t *)calloc((size_t)kb + 1, sizeof(int64_t));
    int32_t *amem = (int32_t *)malloc((size_t)(ma > 0 ? ma : 1) * sizeof(int32_t));
    int32_t *bmem = (int32_t *)malloc((size_t)(mb > 0 ? mb : 1) * sizeof(int32_t));
    int64_t *mark = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!na || !nb || !rowmax || !colmax || !rowbest || !keys || !astart || !bstart || !amem || !bmem || !mark) {
        free(na); free(nb); free(rowmax); free(colmax); free(rowbest); free(keys);
        free(astart); free(bstart); free(amem); free(bmem); free(mark);
        return OQ_ENOMEM;
    }
    int64_t nk = 0;
    for (int64_t i = 0; i < n; i++) {
        for (int64_t x = aptr[i]; x < aptr[i + 1]; x++) na[amemb[x]]++;
        for (int64_t y = bptr[i]; y < bptr[i + 1]; y++) nb[bmemb[y]]++;
        for (int64_t x = aptr[i]; x < aptr[i + 1]; x++)
            for (int64_t y = bptr[i]; y < bptr[i + 1]; y++)
                keys[nk++] = ((uint64_t)(uint32_t)amemb[x] << 32) | (uint64_t)(uint32_t)bmemb[y];
    }
    qsort(keys, (size_t)nk, sizeof(uint64_t), cmp_u64);
    const long double N = (long double)n;
    oq_sum vi = {0, 0}, viabs = {0, 0}, num = {0, 0}, numabs = {0, 0}, den = {0, 0};
    int64_t ncells = 0;
    for (int64_t s = 0; s < nk;) {
        int64_t t = s;
        while (t < nk && keys[t] == keys[s]) t++;
        const int64_t cnt = t - s;
        const int32_t ca = (int32_t)(keys[s] >> 32), cb = (int32_t)(keys[s] & 0xffffffffu);
        ncells++;
        const long double x = (long double)cnt, sa = (long double)na[ca], sb = (long double)nb[cb];
        const long double tv = x * logl(x * x / (sa * sb));          /* Eq. (1) term */
        sum_add(&vi, tv);
        sum_add(&viabs, fabsl(tv));
        const long double tn = x / N * logl(x * N / (sa * sb));       /* Eq. (2) numerator term */
        sum_add(&num, tn);
        sum_add(&numabs, fabsl(tn));
        const long double r = 2.0L * x / (sa + sb);                  /* Eq. (3) */
        if (r > rowbest[ca]) rowbest[ca] = r;
        if (cnt > rowmax[ca]) rowmax[ca] = cnt;                       /* Eq. (4) */
        if (cnt > colmax[cb]) colmax[cb] = cnt;
        s = t;
    }
    int64_t nvdsum = 0, kan = 0, kbn = 0;
    oq_sum f = {0, 0};
    for (int32_t c = 0; c < ka; c++) {
        if (na[c] == 0) continue;
        kan++;
        const long double p = (long double)na[c] / N;
        sum_add(&den, p * logl(p));
        nvdsum += rowmax[c];
        sum_add(&f, (long double)na[c] * rowbest[c]);
    }
    for (int32_t c = 0; c < kb; c++) {
        if (nb[c] == 0) continue;
        kbn++;
        const long double p = (long double)nb[c] / N;
        sum_add(&den, p * logl(p));
        nvdsum += colmax[c];
    }
    /* transposes */
    for (int32_t c = 0; c < ka; c++) astart[c + 1] = astart[c] + na[c];
    for (int32_t c = 0; c < kb; c++) bstart[c + 1] = bstart[c] + nb[c];
    {
        int64_t *fa = (int64_t *)malloc((size_t)ka * sizeof(int64_t)), *fb = (int64_t *)malloc((size_t)kb * sizeof(int64_t));
        if (!fa || !fb) {
            free(fa); free(fb);
            free(na); free(nb); free(rowmax); free(colmax); free(rowbest); free(keys);
            free(astart); free(bstart); free(amem); free(bmem); free(mark);
            return OQ_ENOMEM;
        }
        memcpy(fa, astart, (size_t)ka * sizeof(int64_t));
        memcpy(fb, bstart, (size_t)kb * sizeof(int64_t));
        for (int64_t i = 0; i < n; i++) {
            for (int64_t x = aptr[i]; x < aptr[i + 1]; x++) amem[fa[amemb[x]]++] = (int32_t)i;
            for (int64_t y = bptr[i]; y < bptr[i + 1]; y++) bmem[fb[bmemb[y]]++] = (int32_t)i;
        }
        free(fa); free(fb);
    }
    /* pairs together in C (a11 when also together in C'), then pairs together in C' */
    int64_t sameA = 0, sameB = 0, a11 = 0;
    for (int64_t i = 0; i < n; i++) mark[i] = -1;
    for (int64_t i = 0; i < n; i++)
        for (int64_t x = aptr[i]; x < aptr[i + 1]; x++) {
            const int32_t c = amemb[x];
            for (int64_t p = astart[c]; p < astart[c + 1]; p++) {
                const int64_t j = amem[p];
                if (j <= i || mark[j] == i) continue;
                mark[j] = i;
                sameA++;
                if (lists_meet(bmemb + bptr[i], bptr[i + 1] - bptr[i], bmemb + bptr[j], bptr[j + 1] - bptr[j]))
                    a11++;
            }
        }
    for (int64_t i = 0; i < n; i++) mark[i] = -1;
    for (int64_t i = 0; i < n; i++)
        for (int64_t y = bptr[i]; y < bptr[i + 1]; y++) {
            const int32_t c = bmemb[y];
            for (int64_t p = bstart[c]; p < bstart[c + 1]; p++) {
                const int64_t j = bmem[p];
                if (j <= i || mark[j] == i) continue;
                mark[j] = i;
                sameB++;
            }
        }
    const int64_t A = n * (n - 1) / 2;
    const int64_t a10 = sameA - a11, a01 = sameB - a11, a00 = A - a11 - a10 - a01;
    int rc = (a10 < 0 || a01 < 0 || a00 < 0) ? OQ_ECHECK : OQ_OK;
    if (rc == OQ_OK) {
        const long double LA = (long double)A;
        const long double l11 = (long double)a11, l10 = (long double)a10, l01 = (long double)a01, l00 = (long double)a00;
        dbl[0] = (double)(-sum_get(&vi) / N);
        const long double dd = sum_get(&den);
        dbl[1] = dd != 0.0L ? (double)(-2.0L * sum_get(&num) / dd) : 1.0;
        dbl[2] = (double)(sum_get(&f) / N);
        dbl[3] = (double)(1.0L - (long double)nvdsum / (2.0L * N));
        dbl[4] = (double)((l11 + l00) / LA);
        const long double M = (l11 + l10) * (l11 + l01) / LA;  /* Eq. (6) */
        const long double ari_den = 0.5L * ((l11 + l10) + (l11 + l01)) - M;
        dbl[5] = ari_den != 0.0L ? (double)((l11 - M) / ari_den) : 1.0;
        const long double ji_den = l11 + l10 + l01;
        dbl[6] = ji_den != 0.0L ? (double)(l11 / ji_den) : 1.0;
        dbl[7] = (double)(sum_get(&viabs) / N);
        dbl[8] = (double)(2.0L * sum_get(&numabs));
        dbl[9] = (double)fabsl(dd);
        i64[0] = n; i64[1] = kan; i64[2] = kbn; i64[3] = ncells;
        i64[4] = a11; i64[5] = a10; i64[6] = a01; i64[7] = a00; i64[8] = nvdsum;
    }
    free(na); free(nb); free(rowmax); free(colmax); free(rowbest); free(keys);
    free(astart); free(bstart); free(amem); free(bmem); free(mark);
    return rc;
}

/*
 * Pair counts of two covers by visiting every node pair i < j (O(|V|^2),
 * tiny inputs only): together in a cover = the two lists share an id.
 * out[0..3] = a11, a10, a01, a00.
 */
int oq_pairs_cover_bruteforce(const int64_t *aptr, const int32_t *amemb, const int64_t *bptr,
                              const int32_t *bmemb, int64_t n, int64_t *out)
{
    if (n < 2)
        return OQ_EINVAL;
    int64_t a11 = 0, a10 = 0, a01 = 0, a00 = 0;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = i + 1; j < n; j++) {
            const int sa = lists_meet(amemb + aptr[i], aptr[i + 1] - aptr[i], amemb + aptr[j], aptr[j + 1] - aptr[j]);
            const int sb = lists_meet(bmemb + bptr[i], bptr[i + 1] - bptr[i], bmemb + bptr[j], bptr[j + 1] - bptr[j]);
            if (sa && sb) a11++;
            else if (sa) a10++;
            else if (sb) a01++;
            else a00++;
        }
    out[0] = a11; out[1] = a10; out[2] = a01; out[3] = a00;
    return OQ_OK;
}
