// qm_finalize.cuh -- from exact sums to the metric values (shared by the plain
// and the batched kernels so that both produce bit-identical results).
#pragma once

#include "qm_device.cuh"
#include "../../include/qm.h"

namespace qmk {

struct ScoreTotals {
    i128 qds_self, qds_pair, dens, contr, expn, cond, vol2;
    unsigned long long ein, eout, nonempty, slots, cnt2;
};

struct CompareTotals {
    i128 vi, hnum, hden, f;
    unsigned long long a11, sa, sb, nvd, cells, ka, kb;
};

__device__ __forceinline__ double i128_to_double(i128 v) { return fp_to_double(v, 0); }

// Eqs. (8), (9) and the Sec. II-B.3 means.
//   Q = sum_c [E_in/|E| - (vol_c/(2|E|))^2] = (4|E| sum E_in - sum vol_c^2) / (4|E|^2),
// evaluated from exact integers with one rounding of numerator and denominator.
__device__ __forceinline__ void make_quality(const ScoreTotals &t, long long n, long long E,
                                             qm_quality *out)
{
    qm_quality r;
    r.n_nodes = n;
    r.n_edges = E;
    r.n_communities_nonempty = (long long)t.nonempty;
    r.intra_edges_total = (long long)t.ein;
    r.cut_edges_total = (long long)(t.eout / 2);
    r.n_community_pairs = (long long)t.slots;  // each unordered pair counted once
    r.pair_count_sq_sum = (long long)t.cnt2;
    const i128 num = (i128)4 * (i128)E * (i128)t.ein - t.vol2;
    const i128 den = (i128)4 * (i128)E * (i128)E;
    r.modularity = __ddiv_rn(i128_to_double(num), i128_to_double(den));
    r.modularity_density = fp_to_double(t.qds_self - t.qds_pair, SC_QDS);
    const double ne = (double)t.nonempty;
    r.mean_intra_edges = __ddiv_rn((double)t.ein, ne);
    r.mean_inter_edges = __ddiv_rn((double)t.eout, ne);
    r.mean_intra_density = __ddiv_rn(fp_to_double(t.dens, SC_MEAN), ne);
    r.mean_contraction = __ddiv_rn(fp_to_double(t.contr, SC_MEAN), ne);
    r.mean_expansion = __ddiv_rn(fp_to_double(t.expn, SC_MEAN), ne);
    r.mean_conductance = __ddiv_rn(fp_to_double(t.cond, SC_MEAN), ne);
    *out = r;
}

// Eqs. (1)-(7).  Pair counts of Sec. II-A.3 from the contingency table:
//   a11 = sum C(n_cc', 2), a11 + a10 = sum C(|c|, 2) = S_a, a11 + a01 = S_b,
//   A = C(N, 2).  RI, JI and ARI are ratios of exact integers; ARI is Eq. (6)
//   multiplied through by 2A: 2(A a11 - S_a S_b) / (A (S_a + S_b) - 2 S_a S_b).
__device__ __forceinline__ void make_compare(const CompareTotals &t, long long N, qm_compare *out)
{
    qm_compare r;
    const long long A = N * (N - 1) / 2;
    const long long a11 = (long long)t.a11;
    const long long a10 = (long long)t.sa - a11;
    const long long a01 = (long long)t.sb - a11;
    const long long a00 = A - a11 - a10 - a01;
    r.n_nodes = N;
    r.k_truth = (long long)t.ka;
    r.k_found = (long long)t.kb;
    r.n_cells = (long long)t.cells;
    r.a11 = a11;
    r.a10 = a10;
    r.a01 = a01;
    r.a00 = a00;
    r.nvd_sum = (long long)t.nvd;
    const double dn = (double)N;
    r.vi = -__ddiv_rn(fp_to_double(t.vi, SC_VI), dn);
    const double hden = fp_to_double(t.hden, SC_H);
    r.nmi = (t.hden != 0) ? __ddiv_rn(__dmul_rn(-2.0, fp_to_double(t.hnum, SC_H)), hden) : 1.0;
    r.f_measure = __ddiv_rn(fp_to_double(t.f, SC_F), dn);
    r.nvd = __dsub_rn(1.0, __ddiv_rn((double)t.nvd, __dmul_rn(2.0, dn)));
    r.ri = __ddiv_rn((double)(a11 + a00), (double)A);
    const i128 sa = (i128)t.sa, sb = (i128)t.sb, a = (i128)A;
    const i128 ari_num = 2 * (a * (i128)a11 - sa * sb);
    const i128 ari_den = a * (sa + sb) - 2 * sa * sb;
    r.ari = (ari_den != 0) ? __ddiv_rn(i128_to_double(ari_num), i128_to_double(ari_den)) : 1.0;
    const long long ji_den = a11 + a10 + a01;
    r.ji = (ji_den != 0) ? __ddiv_rn((double)a11, (double)ji_den) : 1.0;
    *out = r;
}

}  // namespace qmk
