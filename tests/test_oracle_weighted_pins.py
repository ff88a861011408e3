"""Pins of the oracle's weighted Q and Qds (Eqs. 8-9 in the reading of the
paper's note on weighted graphs: edge amounts weighted, densities unweighted)
to things other than itself: hand-derived closed forms
(tests/golden/closed_forms.json), networkx's weighted modularity, the
unweighted oracle (unit weights, and integer weights against the multigraph
for Q), and invariance under scaling all weights."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "closed_forms.json")))["weighted_triangle_path"]


def weighted_csr(n, edges):
    """edges: (u, v, w); symmetric CSR with sorted rows and parallel weights."""
    rows = [dict() for _ in range(n)]
    for u, v, w in edges:
        rows[u][v] = w
        rows[v][u] = w
    rp = np.zeros(n + 1, np.int64)
    col, wt = [], []
    for u in range(n):
        rp[u + 1] = rp[u] + len(rows[u])
        for v in sorted(rows[u]):
            col.append(v)
            wt.append(rows[u][v])
    return rp, np.array(col, np.int32), np.array(wt, np.float64)


def random_weighted(rng, n, p, wmax=5.0, integer=False):
    edges = []
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < p:
                w = float(rng.integers(1, 4)) if integer else float(rng.uniform(0.05, wmax))
                edges.append((i, j, w))
    if not edges:
        edges = [(0, 1, 1.0)]
    return edges


def close(a, b, cond=0.0, rel=1e-12):
    return abs(a - b) <= rel * max(abs(b), abs(cond), 1e-300)


@pytest.mark.parametrize("case", ["two_groups", "singletons", "one_community"])
def test_closed_forms(oracle_mod, case):
    rp, col, wt = weighted_csr(5, GOLD["edges"])
    c = GOLD[case]
    o = oracle_mod.score_weighted(rp, col, wt, np.array(c["labels"], np.int32), max(c["labels"]) + 1)
    assert close(o["modularity"], float(Fraction(*c["modularity"])))
    assert close(o["modularity_density"], float(Fraction(*c["modularity_density"])))
    assert o["total_weight"] == 6.0


def test_weighted_modularity_matches_networkx(oracle_mod):
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(7)
    for trial in range(6):
        n = int(rng.integers(6, 40))
        edges = random_weighted(rng, n, 0.2)
        rp, col, wt = weighted_csr(n, edges)
        K = int(rng.integers(1, 6))
        labels = rng.integers(0, K, n).astype(np.int32)
        G = nx.Graph()
        G.add_nodes_from(range(n))
        G.add_weighted_edges_from(edges)
        comms = [set(np.flatnonzero(labels == k).tolist()) for k in range(K)]
        comms = [c for c in comms if c]
        ref = nx.community.modularity(G, comms, weight="weight")
        o = oracle_mod.score_weighted(rp, col, wt, labels, K)
        assert close(o["modularity"], ref, o["cond_modularity"], 1e-10), trial


def test_unit_weights_give_the_unweighted_metrics(oracle_mod):
    rng = np.random.default_rng(8)
    for trial in range(5):
        n = int(rng.integers(8, 50))
        edges = [(u, v, 1.0) for u, v, _ in random_weighted(rng, n, 0.15)]
        rp, col, wt = weighted_csr(n, edges)
        K = int(rng.integers(1, 8))
        labels = rng.integers(0, K, n).astype(np.int32)
        w = oracle_mod.score_weighted(rp, col, wt, labels, K)
        u = oracle_mod.score(rp, col, labels, K)
        assert close(w["modularity"], u["modularity"], u["cond_modularity"])
        assert close(w["modularity_density"], u["modularity_density"], u["cond_modularity_density"])


def test_integer_weights_match_the_multigraph_modularity(oracle_mod):
    # Q counts amounts only, so an edge of weight k is k parallel edges
    rng = np.random.default_rng(9)
    for trial in range(4):
        n = int(rng.integers(8, 40))
        edges = random_weighted(rng, n, 0.2, integer=True)
        rp, col, wt = weighted_csr(n, edges)
        multi = [[] for _ in range(n)]
        for u, v, w in edges:
            multi[u] += [v] * int(w)
            multi[v] += [u] * int(w)
        mrp = np.zeros(n + 1, np.int64)
        for u in range(n):
            mrp[u + 1] = mrp[u] + len(multi[u])
        mcol = np.array([v for u in range(n) for v in sorted(multi[u])], np.int32)
        K = int(rng.integers(2, 6))
        labels = rng.integers(0, K, n).astype(np.int32)
        w = oracle_mod.score_weighted(rp, col, wt, labels, K)
        m = oracle_mod.score(mrp, mcol, labels, K)
        assert close(w["modularity"], m["modularity"], m["cond_modularity"])


def test_scaling_all_weights_changes_nothing(oracle_mod):
    rng = np.random.default_rng(10)
    n = 30
    rp, col, wt = weighted_csr(n, random_weighted(rng, n, 0.2))
    labels = rng.integers(0, 4, n).astype(np.int32)
    a = oracle_mod.score_weighted(rp, col, wt, labels, 4)
    b = oracle_mod.score_weighted(rp, col, wt * 7.25, labels, 4)
    assert close(a["modularity"], b["modularity"], a["cond_modularity"])
    assert close(a["modularity_density"], b["modularity_density"], a["cond_modularity_density"])
