"""Pins of the CPU oracle to things other than itself (no GPU needed).

* closed forms derived by hand from the paper's equations (tests/golden/closed_forms.json);
* library routines that compute the same textbook quantities: networkx modularity
  (Eq. 8), scikit-learn Rand / adjusted Rand / NMI / mutual information (Eqs. 1, 2, 5, 6);
* brute force: Algorithm 4 (every node pair), the set-intersection form of
  Eqs. (1)-(4), Newman's adjacency-matrix form of Q and an adjacency-matrix
  count of |E_ci,cj| evaluated in exact rationals;
* invariants: Q in [-1/2, 1], relabelling and node permutation invariance,
  symmetry of the symmetric indices, VI = H + H' - 2I, Qds = -1 for singletons,
  Qds = Q for a disjoint union of cliques scored by cliques.
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "closed_forms.json")))


def csr_from_edges(n, edges):
    adj = [set() for _ in range(n)]
    for u, v in edges:
        if u != v:
            adj[u].add(v)
            adj[v].add(u)
    rp = np.zeros(n + 1, np.int64)
    col = []
    for u in range(n):
        rp[u + 1] = rp[u] + len(adj[u])
        col.extend(sorted(adj[u]))
    return rp, np.array(col, np.int32), adj


def two_cliques():
    edges = [(i, j) for i in range(5) for j in range(i + 1, 5)]
    edges += [(i + 5, j + 5) for i in range(5) for j in range(i + 1, 5)]
    edges += [(4, 5)]
    return csr_from_edges(10, edges)


def random_graph(rng, n, p):
    edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
    if not edges:
        edges = [(0, 1)]
    return csr_from_edges(n, edges)


def frac(x):
    return Fraction(x[0], x[1])


def close(a, b, cond=0.0, rel=1e-12):
    return abs(a - b) <= rel * max(abs(b), abs(cond), 1e-300)


def restricted_growth_strings(n):
    """All set partitions of n labelled nodes, as canonical label vectors."""
    def rec(prefix, m):
        if len(prefix) == n:
            yield list(prefix)
            return
        for c in range(m + 1):
            yield from rec(prefix + [c], max(m, c + 1) if c == m else m)
    yield from rec([0], 1)


# ---------------------------------------------------------------- exact brute force

def exact_scores(adj, labels):
    """Q by Newman's adjacency form and Qds by adjacency-matrix pair counts, exact."""
    n = len(adj)
    m = sum(len(a) for a in adj) // 2
    deg = [len(a) for a in adj]
    q = Fraction(0)
    for i in range(n):
        for j in range(n):
            if labels[i] == labels[j]:
                q += Fraction(1 if j in adj[i] else 0) - Fraction(deg[i] * deg[j], 2 * m)
    q /= 2 * m
    comms = sorted(set(labels))
    members = {c: [u for u in range(n) if labels[u] == c] for c in comms}
    between = {}
    for ci in comms:
        for cj in comms:
            between[ci, cj] = sum(1 for u in members[ci] for v in members[cj] if v in adj[u])
    qds = Fraction(0)
    for ci in comms:
        s = len(members[ci])
        ein = Fraction(between[ci, ci], 2)
        eout = sum(between[ci, cj] for cj in comms if cj != ci)
        d = Fraction(2) * ein / (s * (s - 1)) if s > 1 else Fraction(0)
        qds += ein / m * d - ((2 * ein + eout) / Fraction(2 * m) * d) ** 2
        for cj in comms:
            if cj != ci:
                e = between[ci, cj]
                qds -= Fraction(e, 2 * m) * Fraction(e, s * len(members[cj]))
    return q, qds


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("case", ["planted", "one_community", "singletons"])
def test_two_cliques_closed_forms(oracle_mod, case):
    rp, col, _ = two_cliques()
    g = GOLD["two_cliques"][case]
    lab = np.array(g["labels"], np.int32)
    r = oracle_mod.score(rp, col, lab, int(lab.max()) + 1, per_community=True)
    assert r["n_edges"] == 21
    assert close(r["modularity"], float(frac(g["modularity"])), 1.0)
    assert close(r["modularity_density"], float(frac(g["modularity_density"])), 1.0)
    if case == "planted":
        pc = g["per_community"]
        assert r["intra_edges_total"] == 20 and r["cut_edges_total"] == 1
        assert list(r["per_community"]["intra_edges"]) == [10, 10]
        assert list(r["per_community"]["inter_edges"]) == [1, 1]
        for key in ("intra_density", "contraction", "expansion", "conductance"):
            for v in r["per_community"][key]:
                assert close(v, float(frac(pc[key])))
        assert close(r["mean_conductance"], 1 / 21)
        assert close(r["mean_expansion"], 1 / 5)


def test_two_partitions_closed_forms(oracle_mod):
    g = GOLD["two_partitions"]
    r = oracle_mod.compare(g["truth"], g["found"], 2, 2)
    assert (r["a11"], r["a10"], r["a01"], r["a00"]) == (g["a11"], g["a10"], g["a01"], g["a00"])
    for key in ("ri", "ari", "ji", "f_measure", "nvd"):
        assert close(r[key], float(frac(g[key]))), key
    vi = -(4 * math.log(16 / 20) + math.log(1 / 30) + 5 * math.log(25 / 30)) / 10
    assert close(vi, g["vi"], rel=1e-15)
    assert close(r["vi"], g["vi"], rel=1e-13)
    assert close(r["nmi"], g["nmi"], rel=1e-13)


def test_identity_and_extreme_partitions(oracle_mod):
    rng = np.random.default_rng(7)
    for n in (2, 5, 37, 500):
        a = rng.integers(0, max(1, n // 3), n).astype(np.int32)
        k = int(a.max()) + 1
        r = oracle_mod.compare(a, a, k, k)
        assert r["vi"] == 0.0  # every term is log(1) = 0 exactly
        assert close(r["nmi"], 1.0) and close(r["ari"], 1.0) and close(r["ri"], 1.0)
        assert close(r["ji"], 1.0) and close(r["f_measure"], 1.0) and r["nvd"] == 0.0
        # one community against n singletons
        one = np.zeros(n, np.int32)
        sing = np.arange(n, dtype=np.int32)
        r = oracle_mod.compare(one, sing, 1, n)
        assert close(r["ri"], 0.0, 1.0) and close(r["ari"], 0.0, 1.0) and close(r["ji"], 0.0, 1.0)
        assert close(r["nmi"], 0.0, 1.0)
        assert close(r["vi"], math.log(n), rel=1e-13)
        assert close(r["f_measure"], 2 / (n + 1))
        assert close(r["nvd"], (n - 1) / (2 * n))


def test_cliques_special_cases(oracle_mod):
    # K_n as one community: Q = 0, Qds = 0
    for n in (2, 3, 8, 20):
        rp, col, _ = csr_from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
        r = oracle_mod.score(rp, col, np.zeros(n, np.int32), 1)
        assert abs(r["modularity"]) < 1e-15 and abs(r["modularity_density"]) < 1e-15
    # disjoint cliques scored by cliques: d = 1 and no boundary, so Qds = Q (Eq. 9 -> Eq. 8)
    sizes = [3, 4, 6, 2, 9]
    edges, labels, base = [], [], 0
    for c, s in enumerate(sizes):
        edges += [(base + i, base + j) for i in range(s) for j in range(i + 1, s)]
        labels += [c] * s
        base += s
    rp, col, _ = csr_from_edges(base, edges)
    r = oracle_mod.score(rp, col, np.array(labels, np.int32), len(sizes))
    assert close(r["modularity_density"], r["modularity"], 1.0)
    m = sum(s * (s - 1) // 2 for s in sizes)
    q = sum(Fraction(s * (s - 1) // 2, m) - Fraction(s * (s - 1) // 2, m) ** 2 for s in sizes)
    assert close(r["modularity"], float(q))


# ---------------------------------------------------------------- library routines

def test_modularity_matches_networkx(oracle_mod):
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(11)
    for trial in range(25):
        n = int(rng.integers(5, 60))
        rp, col, adj = random_graph(rng, n, float(rng.uniform(0.05, 0.5)))
        k = int(rng.integers(1, n + 1))
        lab = rng.integers(0, k, n).astype(np.int32)
        G = nx.Graph()
        G.add_nodes_from(range(n))
        G.add_edges_from((u, v) for u in range(n) for v in adj[u] if v > u)
        comms = [set(np.flatnonzero(lab == c).tolist()) for c in range(k)]
        comms = [c for c in comms if c]
        ref = nx.community.modularity(G, comms)
        r = oracle_mod.score(rp, col, lab, k)
        assert close(r["modularity"], ref, r["cond_modularity"], rel=1e-12), trial


def test_pair_and_information_indices_match_sklearn(oracle_mod):
    skm = pytest.importorskip("sklearn.metrics")
    from scipy.stats import entropy
    rng = np.random.default_rng(12)
    for trial in range(40):
        n = int(rng.integers(2, 3000))
        ka, kb = int(rng.integers(1, n + 1)), int(rng.integers(1, n + 1))
        a = rng.integers(0, ka, n).astype(np.int32)
        b = rng.integers(0, kb, n).astype(np.int32)
        if trial % 4 == 0:  # correlated partitions
            b = np.where(rng.random(n) < 0.7, a % kb, b).astype(np.int32)
        r = oracle_mod.compare(a, b, ka, kb)
        assert close(r["ri"], skm.rand_score(a, b), rel=1e-12)
        assert close(r["ari"], skm.adjusted_rand_score(a, b), 1.0, rel=1e-10)
        nmi = skm.normalized_mutual_info_score(a, b, average_method="arithmetic")
        assert close(r["nmi"], nmi, 1.0, rel=1e-10)
        mi = skm.mutual_info_score(a, b)
        ha = entropy(np.bincount(a)[np.bincount(a) > 0])
        hb = entropy(np.bincount(b)[np.bincount(b) > 0])
        assert close(r["vi"], ha + hb - 2 * mi, r["cond_vi"] + ha + hb, rel=1e-12)


# ---------------------------------------------------------------- brute force

def test_algorithm4_pair_counts_bit_exact(oracle_mod):
    rng = np.random.default_rng(13)
    for n in (2, 3, 10, 257, 2000):
        for _ in range(3):
            a = rng.integers(0, max(1, int(rng.integers(1, n + 1))), n).astype(np.int32)
            b = rng.integers(0, max(1, int(rng.integers(1, n + 1))), n).astype(np.int32)
            r = oracle_mod.compare(a, b, int(a.max()) + 1, int(b.max()) + 1)
            assert oracle_mod.pairs_bruteforce(a, b) == (r["a11"], r["a10"], r["a01"], r["a00"])
            assert r["a11"] + r["a10"] + r["a01"] + r["a00"] == n * (n - 1) // 2


def test_set_intersection_form(oracle_mod):
    rng = np.random.default_rng(14)
    for _ in range(30):
        n = int(rng.integers(2, 80))
        ka, kb = int(rng.integers(1, 12)), int(rng.integers(1, 12))
        a = rng.integers(0, ka, n).astype(np.int32)
        b = rng.integers(0, kb, n).astype(np.int32)
        r = oracle_mod.compare(a, b, ka, kb)
        bf = oracle_mod.compare_bruteforce(a, b, ka, kb)
        assert close(r["vi"], bf["vi"], r["cond_vi"])
        assert close(r["nmi"], bf["nmi"], 1.0)
        assert close(r["f_measure"], bf["f_measure"])
        assert close(r["nvd"], bf["nvd"], 1.0)
        # F-measure from explicit node sets (Eq. 3), NVD from explicit maxima (Eq. 4)
        A = [set(np.flatnonzero(a == c)) for c in range(ka)]
        B = [set(np.flatnonzero(b == c)) for c in range(kb)]
        f = sum(Fraction(len(c)) * max(Fraction(2 * len(c & d), len(c) + len(d)) for d in B if d)
                for c in A if c) / n
        assert close(r["f_measure"], float(f))
        nvd = 1 - Fraction(sum(max(len(c & d) for d in B) for c in A if c)
                           + sum(max(len(c & d) for c in A) for d in B if d), 2 * n)
        assert close(r["nvd"], float(nvd), 1.0)


def test_scores_against_exact_adjacency_forms(oracle_mod):
    rng = np.random.default_rng(15)
    for trial in range(40):
        n = int(rng.integers(2, 16))
        rp, col, adj = random_graph(rng, n, float(rng.uniform(0.15, 0.8)))
        k = int(rng.integers(1, n + 1))
        lab = rng.integers(0, k, n).astype(np.int32)
        q, qds = exact_scores(adj, lab.tolist())
        r = oracle_mod.score(rp, col, lab, k)
        assert close(r["modularity"], float(q), r["cond_modularity"]), trial
        assert close(r["modularity_density"], float(qds), r["cond_modularity_density"]), trial
        bf = oracle_mod.score_bruteforce(rp, col, lab, k)
        assert close(bf["modularity_density"], float(qds), r["cond_modularity_density"])


def test_exhaustive_partitions_of_seven_nodes(oracle_mod):
    skm = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(16)
    rp, col, adj = random_graph(rng, 7, 0.5)
    truth = np.array([0, 0, 1, 1, 1, 2, 2], np.int32)
    count = 0
    for lab in restricted_growth_strings(7):
        lab = np.array(lab, np.int32)
        k = int(lab.max()) + 1
        q, qds = exact_scores(adj, lab.tolist())
        r = oracle_mod.score(rp, col, lab, k)
        assert close(r["modularity"], float(q), r["cond_modularity"])
        assert close(r["modularity_density"], float(qds), r["cond_modularity_density"])
        assert -0.5 <= r["modularity"] <= 1.0
        c = oracle_mod.compare(truth, lab, 3, k)
        assert close(c["ari"], skm.adjusted_rand_score(truth, lab), 1.0, rel=1e-10)
        assert oracle_mod.pairs_bruteforce(truth, lab) == (c["a11"], c["a10"], c["a01"], c["a00"])
        count += 1
    assert count == 877  # Bell(7)


# ---------------------------------------------------------------- invariants

def test_invariants_relabel_and_permutation(oracle_mod):
    rng = np.random.default_rng(17)
    for _ in range(10):
        n = int(rng.integers(10, 200))
        rp, col, adj = random_graph(rng, n, 0.1)
        k = int(rng.integers(1, 20))
        lab = rng.integers(0, k, n).astype(np.int32)
        r0 = oracle_mod.score(rp, col, lab, k)
        # relabel community ids
        perm_c = rng.permutation(k + 3).astype(np.int32)
        r1 = oracle_mod.score(rp, col, perm_c[lab], k + 3)
        # permute node ids
        p = rng.permutation(n)
        inv = np.empty(n, np.int64)
        inv[p] = np.arange(n)
        edges = [(int(inv[u]), int(inv[v])) for u in range(n) for v in adj[u] if v > u]
        rp2, col2, _ = csr_from_edges(n, edges)
        lab2 = np.empty(n, np.int32)
        lab2[inv] = lab
        r2 = oracle_mod.score(rp2, col2, lab2, k)
        for key in ("modularity", "modularity_density", "mean_conductance", "mean_expansion",
                    "mean_contraction", "mean_intra_density"):
            assert close(r1[key], r0[key], 1.0, 1e-13) and close(r2[key], r0[key], 1.0, 1e-13), key
        for key in ("intra_edges_total", "cut_edges_total", "n_communities_nonempty",
                    "n_community_pairs", "pair_count_sq_sum"):
            assert r1[key] == r0[key] == r2[key]
        assert r0["intra_edges_total"] + r0["cut_edges_total"] == r0["n_edges"]
        # all singletons: Qds = -1 for any graph with at least one edge
        rs = oracle_mod.score(rp, col, np.arange(n, dtype=np.int32), n)
        assert close(rs["modularity_density"], -1.0)


def test_symmetry_of_comparison_indices(oracle_mod):
    rng = np.random.default_rng(18)
    for _ in range(20):
        n = int(rng.integers(2, 500))
        a = rng.integers(0, int(rng.integers(1, 30)), n).astype(np.int32)
        b = rng.integers(0, int(rng.integers(1, 30)), n).astype(np.int32)
        ka, kb = int(a.max()) + 1, int(b.max()) + 1
        r1 = oracle_mod.compare(a, b, ka, kb)
        r2 = oracle_mod.compare(b, a, kb, ka)
        for key in ("vi", "nmi", "ri", "ari", "ji", "nvd"):
            assert close(r1[key], r2[key], 1.0, 1e-13), key
        assert (r1["a10"], r1["a01"]) == (r2["a01"], r2["a10"])


def test_invalid_inputs_rejected(oracle_mod):
    rp, col, _ = two_cliques()
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.score(rp, col, np.array([0] * 9 + [2], np.int32), 2)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.compare([0], [0], 1, 1)
    assert not oracle_mod.validate_graph(np.array([0, 1, 1], np.int64), np.array([1], np.int32))
    assert not oracle_mod.validate_graph(np.array([0, 1], np.int64), np.array([0], np.int32))
    assert oracle_mod.validate_graph(rp, col)
    # a repeated arc: edge {0,1} stored twice in both rows is a multi-edge, which
    # the unweighted simple-graph setting of Sec. II-B.1 excludes, though the
    # CSR is symmetric and has no self-loop
    assert oracle_mod.validate_graph(np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32))
    assert not oracle_mod.validate_graph(np.array([0, 2, 4], np.int64), np.array([1, 1, 0, 0], np.int32))
    # the same repeat inside a larger valid graph (one extra 0-1 arc each way)
    rows = [list(col[rp[u]:rp[u + 1]]) for u in range(len(rp) - 1)]
    rows[0].append(1)
    rows[1].append(0)
    rp2 = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    col2 = np.array([v for r in rows for v in r], np.int32)
    assert not oracle_mod.validate_graph(rp2, col2)


def test_sampled_community_form_matches_whole_graph_oracle(oracle_mod):
    """The per-community routine used on very large inputs agrees with the
    whole-graph oracle's per-community arrays."""
    rng = np.random.default_rng(19)
    for _ in range(5):
        n = int(rng.integers(50, 400))
        rp, col, _ = random_graph(rng, n, 0.08)
        K = int(rng.integers(2, 30))
        lab = rng.integers(0, K, n).astype(np.int32)
        full = oracle_mod.score(rp, col, lab, K, per_community=True)["per_community"]
        ids = rng.integers(0, K, 12).astype(np.int32)
        s = oracle_mod.score_communities(rp, col, lab, K, ids)
        for j, c in enumerate(ids):
            assert s["size"][j] == full["size"][c]
            assert s["intra_edges"][j] == full["intra_edges"][c]
            assert s["inter_edges"][j] == full["inter_edges"][c]
            assert close(s["qds_term"][j], full["qds_term"][c], 1.0, 1e-13)
    rp, col, _ = two_cliques()
    s = oracle_mod.score_communities(rp, col, np.array([0] * 5 + [1] * 5, np.int32), 2, [0, 1])
    assert list(s["distinct_neighbours"]) == [1, 1]
    assert close(s["split"][0], 1 / 42 / 25)


def test_six_measures_and_pair_counts_by_brute_force(oracle_mod):
    """The six measures of Sec. II-B.3 per community and their means over the
    non-empty communities, and the integer pair summaries (distinct unordered
    community pairs joined by an edge, and the sum of |E_ci,cj|^2 over them),
    from adjacency sets in exact rationals.  Label spaces leave ids unused, so
    a mean taken over all K ids instead of the non-empty ones fails."""
    rng = np.random.default_rng(20)
    for trial in range(30):
        n = int(rng.integers(2, 40))
        rp, col, adj = random_graph(rng, n, float(rng.uniform(0.05, 0.6)))
        used = int(rng.integers(1, n + 1))
        K = used + int(rng.integers(1, 6))                 # ids used..K-1 (and gaps) stay empty
        lab = (rng.integers(0, used, n) * (1 + trial % 2)).astype(np.int32)
        K = max(K, int(lab.max()) + 1)
        r = oracle_mod.score(rp, col, lab, K, per_community=True)
        pc = r["per_community"]
        comms = sorted(set(lab.tolist()))
        members = {c: [u for u in range(n) if lab[u] == c] for c in comms}
        means = {k: Fraction(0) for k in ("ie", "id", "co", "oe", "ex", "cd")}
        pairs = {}
        for c in comms:
            s = len(members[c])
            ein = sum(1 for u in members[c] for v in adj[u] if lab[v] == c) // 2
            eout = sum(1 for u in members[c] for v in adj[u] if lab[v] != c)
            for u in members[c]:
                for v in adj[u]:
                    if lab[v] > c:
                        pairs[c, int(lab[v])] = pairs.get((c, int(lab[v])), 0) + 1
            dens = Fraction(2 * ein, s * (s - 1)) if s > 1 else Fraction(0)
            cond = Fraction(eout, 2 * ein + eout) if 2 * ein + eout > 0 else Fraction(0)
            vals = {"ie": Fraction(ein), "id": dens, "co": Fraction(2 * ein, s), "oe": Fraction(eout),
                    "ex": Fraction(eout, s), "cd": cond}
            for k, v in vals.items():
                means[k] += v
            assert pc["size"][c] == s and pc["intra_edges"][c] == ein and pc["inter_edges"][c] == eout
            for key, k in (("intra_density", "id"), ("contraction", "co"), ("expansion", "ex"),
                           ("conductance", "cd")):
                assert close(pc[key][c], float(vals[k])), (trial, key, c)
        for c in set(range(K)) - set(comms):
            assert pc["size"][c] == 0 and pc["intra_edges"][c] == 0 and pc["inter_edges"][c] == 0
        nc = len(comms)
        assert r["n_communities_nonempty"] == nc
        for key, k in (("mean_intra_edges", "ie"), ("mean_intra_density", "id"), ("mean_contraction", "co"),
                       ("mean_inter_edges", "oe"), ("mean_expansion", "ex"), ("mean_conductance", "cd")):
            assert close(r[key], float(means[k] / nc)), (trial, key)
        assert r["n_community_pairs"] == len(pairs)
        assert r["pair_count_sq_sum"] == sum(e * e for e in pairs.values())
        assert r["cut_edges_total"] == sum(pairs.values())


def test_all_core_build_matches_the_serial_oracle(oracle_mod):
    """The OpenMP statement used for the all-core CPU baseline computes the
    serial oracle's quantities: counts exact, sums within the tolerance (only
    the order of the split-penalty additions differs)."""
    rng = np.random.default_rng(77)
    for trial in range(6):
        n = int(rng.integers(30, 3000))
        rp, col, _ = random_graph(rng, n, float(rng.uniform(0.002, 0.05)))
        K = int(rng.integers(1, max(2, n // 3)))
        lab = rng.integers(0, K, n).astype(np.int32)
        a = oracle_mod.score(rp, col, lab, K)
        b = oracle_mod.score_all_cores(rp, col, lab, K)
        assert b["threads"] >= 1
        for k in ("n_nodes", "n_edges", "n_communities_nonempty", "intra_edges_total", "cut_edges_total",
                  "n_community_pairs", "pair_count_sq_sum"):
            assert a[k] == b[k], (trial, k)
        for k in ("modularity", "modularity_density", "mean_intra_edges", "mean_intra_density",
                  "mean_contraction", "mean_inter_edges", "mean_expansion", "mean_conductance"):
            cond = {"modularity": a["cond_modularity"], "modularity_density": a["cond_modularity_density"]}.get(k, 0.0)
            assert close(b[k], a[k], cond), (trial, k, a[k], b[k])
