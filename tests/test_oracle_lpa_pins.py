"""Pins of the oracle's label propagation (the O(|E|) detector family whose
output C' the paper scores, Sec. I and Sec. IV-C) to hand-derived results on
graphs small enough to follow round by round.  Each case is built so that one
plausible slip fails it: a dropped keep-own-label rule, a largest-instead-of-
smallest tie break, asynchronous instead of synchronous updates, sampling the
first 32 neighbours instead of evenly spaced ones, or a wrong final renumbering.
"""
import numpy as np
import pytest


def csr(n, rows):
    """CSR from explicit neighbour lists, row order kept as given."""
    rp = np.zeros(n + 1, np.int64)
    for u in range(n):
        rp[u + 1] = rp[u] + len(rows[u])
    col = np.array([v for u in range(n) for v in rows[u]], np.int32)
    return rp, col


def undirected(n, edges):
    rows = [[] for _ in range(n)]
    for u, v in edges:
        rows[u].append(v)
        rows[v].append(u)
    return [sorted(r) for r in rows]


@pytest.mark.parametrize("rounds", [0, 1, 2, 3, 6])
def test_matching_swaps_labels_every_round(oracle_mod, rounds):
    # every node has exactly one neighbour: synchronous rounds swap the two
    # labels of an edge, so after an odd count each node holds its partner's id
    n = 20
    rp, col = csr(n, undirected(n, [(2 * i, 2 * i + 1) for i in range(n // 2)]))
    out, k = oracle_mod.label_propagation(rp, col, rounds)
    partner = np.arange(n) ^ 1
    assert k == n
    assert np.array_equal(out, np.arange(n) if rounds % 2 == 0 else partner)


@pytest.mark.parametrize("m", [4, 9, 32])
def test_complete_graph(oracle_mod, m):
    # first propagation round: every label is seen once and the node's own is not among them,
    # so node 0 takes 1 and every other node takes 0; second round: all take 0
    rp, col = csr(m, undirected(m, [(i, j) for i in range(m) for j in range(i + 1, m)]))
    out, k = oracle_mod.label_propagation(rp, col, 1)
    assert k == 2 and out[0] == 1 and np.all(out[1:] == 0)
    out, k = oracle_mod.label_propagation(rp, col, 2)
    assert k == 1 and np.all(out == 0)


def test_disjoint_cliques_and_isolated_nodes(oracle_mod):
    # cliques {0..4} and {5..11}, isolated nodes 12 and 13 (they keep their ids)
    edges = [(i, j) for i in range(5) for j in range(i + 1, 5)]
    edges += [(i, j) for i in range(5, 12) for j in range(i + 1, 12)]
    rp, col = csr(14, undirected(14, edges))
    out, k = oracle_mod.label_propagation(rp, col, 4)
    assert k == 4
    assert list(out) == [0] * 5 + [1] * 7 + [2, 3]


def test_keeps_own_label_on_a_tie(oracle_mod):
    # s=0, b=1, a=2, x=3; edges x-a, x-b, a-b, b-s.
    # first propagation round: x -> 1, a -> 1, b -> 0, s -> 1   (each node sees distinct ids)
    # second round: x sees {1, 0}: own label 1 is tied for most frequent -> keeps 1
    #          a sees {1, 0}: keeps 1;  b sees {1, 1, 1} -> 1;  s sees {0} -> 0
    rp, col = csr(4, undirected(4, [(3, 2), (3, 1), (2, 1), (1, 0)]))
    out, k = oracle_mod.label_propagation(rp, col, 1)
    assert k == 2 and list(out) == [1, 0, 1, 1]
    out, k = oracle_mod.label_propagation(rp, col, 2)
    assert k == 2 and list(out) == [0, 1, 1, 1]


def test_path_oscillates(oracle_mod):
    # 0-1-2: [1, 0, 1] after one round (smallest of tied labels), then [0, 1, 0]
    rp, col = csr(3, undirected(3, [(0, 1), (1, 2)]))
    assert list(oracle_mod.label_propagation(rp, col, 1)[0]) == [1, 0, 1]
    assert list(oracle_mod.label_propagation(rp, col, 2)[0]) == [0, 1, 0]
    assert list(oracle_mod.label_propagation(rp, col, 3)[0]) == [1, 0, 1]


@pytest.mark.parametrize("deg", [33, 40, 64, 100])
def test_high_degree_node_samples_evenly_spaced_neighbours(oracle_mod, deg):
    # Centre 0 joined to leaves 1..deg; leaf l also has a pendant node deg + l.
    # First propagation round: each pendant takes its leaf's id, each leaf takes 0 (the centre
    # is its smallest neighbour id), and the centre takes the smallest leaf id
    # among the row positions it looks at.  The centre's row is ordered so that
    # the positions skipped by the even spacing floor(i * deg / 32) hold the
    # smallest leaf ids: if the oracle looked at all, or at the first 32,
    # neighbours, the centre would share its label with a different pendant.
    sampled = sorted({i * deg // 32 for i in range(32)})
    skipped = [p for p in range(deg) if p not in sampled]
    order = [0] * deg
    leaf_ids = iter(range(1, deg + 1))
    for p in skipped + sampled:       # smallest ids go to the skipped positions
        order[p] = next(leaf_ids)
    n = 1 + 2 * deg
    rows = [order] + [[0, deg + l] for l in range(1, deg + 1)] + [[l] for l in range(1, deg + 1)]
    rp, col = csr(n, rows)
    out, k = oracle_mod.label_propagation(rp, col, 1)
    x = min(order[p] for p in sampled)
    assert x == len(skipped) + 1
    pend = lambda l: deg + l
    assert out[0] == out[pend(x)]
    assert all(out[0] != out[pend(l)] for l in range(1, deg + 1) if l != x)
    assert np.all(out[1:deg + 1] == out[1])
    assert k == deg + 1                 # the centre's new label is shared with one pendant


def test_zero_rounds_is_identity(oracle_mod):
    rp, col = csr(5, undirected(5, [(0, 1), (1, 2), (3, 4)]))
    out, k = oracle_mod.label_propagation(rp, col, 0)
    assert k == 5 and list(out) == [0, 1, 2, 3, 4]
