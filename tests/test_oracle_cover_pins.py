"""Pins of the oracle's cover (overlapping communities) statement.

The paper defines its metrics for disjoint communities and leaves overlapping
ones to future work (Sec. VI); the oracle reads every set formula of Eqs. (1)-(9)
and Sec. II-B.3 literally on a cover (qm_oracle.c states the reading).  Pinned by:
* hand-derived closed forms for two small covers (tests/golden/closed_forms.json);
* covers with one community per node, which must give the partition oracle's
  results (a different code path: sorted labels instead of membership lists);
* an exact-rational brute force written from the set definitions (edges
  classified per community pair by set membership), on random small covers;
* the pair counts against a visit of every node pair;
* invariants: relabelling the communities, permuting the nodes."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from helpers import close, csr_from_edges

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def frac(v):
    return v[0] / v[1] if isinstance(v, list) else v


@pytest.mark.parametrize("case", ["cover_bowtie", "cover_two_triangles"])
def test_closed_forms(oracle_mod, case):
    g = GOLD[case]
    rp, col = csr_from_edges(g["n"], g["edges"])
    mp, mb = oracle_mod.cover_from_lists(g["cover"])
    s = oracle_mod.score_cover(rp, col, mp, mb, g["K"])
    for k in ("modularity", "modularity_density", "mean_intra_edges", "mean_intra_density", "mean_contraction",
              "mean_inter_edges", "mean_expansion", "mean_conductance"):
        assert close(s[k], frac(g[k]), 1.0, 1e-14), (k, s[k], g[k])
    assert s["intra_edges_total"] == g["intra_edges_total"]
    assert s["cut_edges_total"] == g["boundary_total"]
    assert s["n_community_pairs"] == g["n_community_pairs"] and s["pair_count_sq_sum"] == g["pair_count_sq_sum"]
    fp, fb = oracle_mod.cover_from_lists(g["found"])
    c = oracle_mod.compare_cover(mp, mb, g["K"], fp, fb, g["k_found"])
    for k in ("a11", "a10", "a01", "a00"):
        assert c[k] == g[k], k
    for k in ("vi", "nmi", "f_measure", "nvd", "ri", "ari", "ji"):
        assert close(c[k], frac(g[k]), 1.0, 1e-13), (k, c[k], g[k])


def random_cover(rng, n, K, extra):
    """Each node gets one random community, and with probability `extra` a
    second and a third; some nodes get none."""
    lists = []
    for _ in range(n):
        x = {int(rng.integers(K))}
        while rng.random() < extra and len(x) < 3:
            x.add(int(rng.integers(K)))
        if rng.random() < 0.05:
            x = set()
        lists.append(sorted(x))
    return lists


def brute_score(n, edges, lists, K):
    """Q, Qds and the six means by the set definitions, in exact rationals:
    each community is a node set; every edge is tested against each community
    (inside / on the boundary) and each community pair (leaves one, enters the
    other)."""
    sets = [set(i for i in range(n) if c in lists[i]) for c in range(K)]
    E = len(edges)
    live = [c for c in range(K) if sets[c]]
    Q = Qds = Fraction(0)
    means = [Fraction(0)] * 6
    for c in live:
        s = len(sets[c])
        ein = sum(1 for u, v in edges if u in sets[c] and v in sets[c])
        eout = sum(1 for u, v in edges if (u in sets[c]) != (v in sets[c]))
        d = Fraction(2 * ein, s * (s - 1)) if s > 1 else Fraction(0)
        Q += Fraction(ein, E) - Fraction(2 * ein + eout, 2 * E) ** 2
        pen = Fraction(0)
        for j in live:
            if j == c:
                continue
            eij = sum(1 for u, v in edges
                      if (u in sets[c] - sets[j] and v in sets[j] - sets[c]) or
                      (v in sets[c] - sets[j] and u in sets[j] - sets[c]))
            pen += Fraction(eij, 2 * E) * Fraction(eij, s * len(sets[j]))
        Qds += Fraction(ein, E) * d - (Fraction(2 * ein + eout, 2 * E) * d) ** 2 - pen
        vol = 2 * ein + eout
        vals = [Fraction(ein), d, Fraction(2 * ein, s), Fraction(eout), Fraction(eout, s),
                Fraction(eout, vol) if vol else Fraction(0)]
        means = [m + v for m, v in zip(means, vals)]
    return Q, Qds, [m / len(live) for m in means]


def test_random_covers_against_set_brute_force(oracle_mod):
    rng = np.random.default_rng(5)
    names = ("mean_intra_edges", "mean_intra_density", "mean_contraction", "mean_inter_edges", "mean_expansion",
             "mean_conductance")
    for trial in range(25):
        n = int(rng.integers(4, 14))
        m = int(rng.integers(3, n * 3))
        edges = sorted({(min(a, b), max(a, b)) for a, b in rng.integers(0, n, (m, 2)) if a != b})
        if not edges:
            continue
        K = int(rng.integers(1, 6))
        lists = random_cover(rng, n, K, 0.4)
        if not any(lists):
            continue
        rp, col = csr_from_edges(n, edges)
        mp, mb = oracle_mod.cover_from_lists(lists)
        s = oracle_mod.score_cover(rp, col, mp, mb, K)
        Q, Qds, means = brute_score(n, edges, lists, K)
        assert close(s["modularity"], float(Q), s["cond_modularity"]), trial
        assert close(s["modularity_density"], float(Qds), s["cond_modularity_density"]), trial
        for k, v in zip(names, means):
            assert close(s[k], float(v)), (trial, k)


def test_one_community_per_node_equals_partition_oracle(oracle_mod):
    rng = np.random.default_rng(6)
    for trial in range(8):
        n = int(rng.integers(20, 600))
        edges = rng.integers(0, n, (n * 4, 2))
        rp, col = csr_from_edges(n, edges)
        K = int(rng.integers(1, 40))
        lab = rng.integers(0, K, n).astype(np.int32)
        lab2 = rng.integers(0, K + 3, n).astype(np.int32)
        mp, mb = oracle_mod.cover_from_lists([[int(x)] for x in lab])
        mp2, mb2 = oracle_mod.cover_from_lists([[int(x)] for x in lab2])
        a = oracle_mod.score(rp, col, lab, K)
        b = oracle_mod.score_cover(rp, col, mp, mb, K)
        for k in ("n_nodes", "n_edges", "n_communities_nonempty", "intra_edges_total", "n_community_pairs",
                  "pair_count_sq_sum"):
            assert a[k] == b[k], k
        assert b["cut_edges_total"] == 2 * a["cut_edges_total"]  # sum of |E_c^out| counts each cut edge twice
        for k in ("modularity", "modularity_density", "mean_intra_edges", "mean_intra_density", "mean_contraction",
                  "mean_inter_edges", "mean_expansion", "mean_conductance"):
            assert close(b[k], a[k], max(a["cond_modularity"], a["cond_modularity_density"], 1.0), 1e-13), k
        c1 = oracle_mod.compare(lab, lab2, K, K + 3)
        c2 = oracle_mod.compare_cover(mp, mb, K, mp2, mb2, K + 3)
        for k in ("k_truth", "k_found", "n_cells", "a11", "a10", "a01", "a00", "nvd_sum"):
            assert c1[k] == c2[k], k
        for k in ("vi", "nmi", "f_measure", "nvd", "ri", "ari", "ji"):
            assert close(c2[k], c1[k], 1.0, 1e-13), k


def test_cover_pair_counts_against_every_node_pair(oracle_mod):
    rng = np.random.default_rng(7)
    for trial in range(20):
        n = int(rng.integers(2, 150))
        A = random_cover(rng, n, int(rng.integers(1, 12)), 0.5)
        B = random_cover(rng, n, int(rng.integers(1, 12)), 0.5)
        ka = max([c for x in A for c in x], default=0) + 1
        kb = max([c for x in B for c in x], default=0) + 1
        ap, am = oracle_mod.cover_from_lists(A)
        bp, bm = oracle_mod.cover_from_lists(B)
        c = oracle_mod.compare_cover(ap, am, ka, bp, bm, kb)
        assert (c["a11"], c["a10"], c["a01"], c["a00"]) == oracle_mod.pairs_cover_bruteforce(ap, am, bp, bm), trial


def test_invariance_and_validation(oracle_mod):
    rng = np.random.default_rng(8)
    n = 300
    edges = rng.integers(0, n, (1500, 2))
    rp, col = csr_from_edges(n, edges)
    K = 25
    lists = random_cover(rng, n, K, 0.3)
    mp, mb = oracle_mod.cover_from_lists(lists)
    base = oracle_mod.score_cover(rp, col, mp, mb, K)
    # relabel communities
    perm = rng.permutation(K)
    mp2, mb2 = oracle_mod.cover_from_lists([sorted(int(perm[c]) for c in x) for x in lists])
    r = oracle_mod.score_cover(rp, col, mp2, mb2, K)
    # permute node ids
    pn = rng.permutation(n)
    inv = np.argsort(pn)
    e2 = [(int(pn[u]), int(pn[v])) for u, v in zip(np.repeat(np.arange(n), np.diff(rp)), col) if u < v]
    rp3, col3 = csr_from_edges(n, e2)
    mp3, mb3 = oracle_mod.cover_from_lists([lists[int(inv[i])] for i in range(n)])
    p = oracle_mod.score_cover(rp3, col3, mp3, mb3, K)
    for k in ("modularity", "modularity_density", "mean_conductance", "mean_intra_density"):
        assert close(r[k], base[k], 1.0, 1e-13) and close(p[k], base[k], 1.0, 1e-13), k
    for k in ("intra_edges_total", "cut_edges_total", "n_community_pairs", "pair_count_sq_sum"):
        assert r[k] == base[k] == p[k], k
    # malformed covers are refused
    assert not oracle_mod.validate_cover(np.array([0, 2], np.int64), np.array([1, 1], np.int32), 3)  # repeat
    assert not oracle_mod.validate_cover(np.array([0, 2], np.int64), np.array([2, 1], np.int32), 3)  # unsorted
    assert not oracle_mod.validate_cover(np.array([0, 1], np.int64), np.array([3], np.int32), 3)     # out of range
    assert oracle_mod.validate_cover(np.array([0, 0, 2], np.int64), np.array([0, 2], np.int32), 3)
