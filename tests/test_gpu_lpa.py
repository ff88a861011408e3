"""qm_label_propagation (the detector that produces C', Sec. I and Sec. IV-C)
against the oracle: labels and K' bit-exact, on LFR graphs, on the hand-built
graphs of the oracle's pins, for host and device output, and for graphs loaded
with QM_REORDER.  Then the detected partition goes through the comparison
path, as in the paper's detected-vs-truth workload."""
import numpy as np
import pytest
import torch

from helpers import to_dev
from test_oracle_lpa_pins import csr, undirected

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05492_gb300 import qm as q
    return q


@pytest.fixture(scope="module")
def lfr():
    from paper_1507_05492_gb300 import gen
    return gen.lfr_graph(gen.LfrParams(n=60_000, k_max=200, s_max=2000, mu=0.3, seed=31))


@pytest.mark.parametrize("rounds", [0, 1, 2, 5, 12])
def test_lfr_labels_match_oracle(qm, oracle_mod, lfr, rounds):
    g = lfr
    ref, k_ref = oracle_mod.label_propagation(g.row_ptr.numpy(), g.col.numpy(), rounds)
    plain = qm.Graph(*to_dev(g.row_ptr, g.col))
    reord = qm.Graph(*to_dev(g.row_ptr, g.col), reorder=True)
    for gr in (plain, reord):
        lab, k = qm.label_propagation(gr, rounds)
        assert k == k_ref
        assert np.array_equal(lab.cpu().numpy(), ref)
        lab_h, k_h = qm.label_propagation(gr, rounds, device=False)
        assert k_h == k_ref and np.array_equal(lab_h, ref)


def small_cases():
    cases = [("matching", csr(20, undirected(20, [(2 * i, 2 * i + 1) for i in range(10)])), 3),
             ("k9", csr(9, undirected(9, [(i, j) for i in range(9) for j in range(i + 1, 9)])), 1),
             ("tie", csr(4, undirected(4, [(3, 2), (3, 1), (2, 1), (1, 0)])), 2),
             ("path", csr(3, undirected(3, [(0, 1), (1, 2)])), 3)]
    for deg in (33, 40, 64, 100):
        sampled = sorted({i * deg // 32 for i in range(32)})
        skipped = [p for p in range(deg) if p not in sampled]
        order = [0] * deg
        for lid, p in enumerate(skipped + sampled, start=1):
            order[p] = lid
        rows = [order] + [[0, deg + l] for l in range(1, deg + 1)] + [[l] for l in range(1, deg + 1)]
        cases.append((f"star{deg}", csr(1 + 2 * deg, rows), 1))
    return cases


@pytest.mark.parametrize("name,graph,rounds", small_cases(), ids=[c[0] for c in small_cases()])
def test_hand_built_graphs_match_oracle(qm, oracle_mod, name, graph, rounds):
    rp, col = graph
    for r in range(rounds + 1):
        ref, k_ref = oracle_mod.label_propagation(rp, col, r)
        for reorder in (False, True):
            lab, k = qm.label_propagation(qm.Graph(*to_dev(rp, col), reorder=reorder), r)
            assert k == k_ref, (name, r, reorder)
            assert np.array_equal(lab.cpu().numpy(), ref), (name, r, reorder)


def test_isolated_nodes_keep_their_labels(qm, oracle_mod):
    edges = [(i, j) for i in range(5) for j in range(i + 1, 5)]
    rp, col = csr(9, undirected(9, edges))       # nodes 5..8 isolated
    lab, k = qm.label_propagation(qm.Graph(*to_dev(rp, col)), 4)
    assert k == 5 and list(lab.cpu().numpy()) == [0, 0, 0, 0, 0, 1, 2, 3, 4]


def test_bad_arguments_rejected(qm, lfr):
    g = qm.Graph(*to_dev(lfr.row_ptr, lfr.col))
    for rounds in (-1, 1001):
        with pytest.raises(RuntimeError):
            qm.label_propagation(g, rounds)


def test_detected_partition_scored_against_truth(qm, oracle_mod):
    """The paper's detected-vs-truth workload end to end on the device: detect
    C' on an LFR graph with clear communities, then score it (Eqs. 1-9)."""
    from paper_1507_05492_gb300 import gen
    g = gen.lfr_graph(gen.LfrParams(n=100_000, k_max=100, s_max=1000, mu=0.1, seed=5))
    gr = qm.Graph(*to_dev(g.row_ptr, g.col), reorder=True)
    lab, k = qm.label_propagation(gr, 10)
    c = qm.compare(g.labels.cuda(), lab, g.K, k)
    o = oracle_mod.compare(g.labels.numpy(), lab.cpu().numpy(), g.K, k)
    for key in ("nmi", "ari", "vi", "f_measure"):
        assert abs(c[key] - o[key]) <= 1e-12 * max(1.0, abs(o[key])), key
    assert c["nmi"] > 0.8, c
    q = qm.score(gr, lab, k)
    assert q["modularity"] > 0.7, q
