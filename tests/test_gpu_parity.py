"""Parity of the CUDA path (through the C ABI) with the CPU oracle: element by
element on seeded inputs, sizes spanning several blocks and ragged tails, and
the degenerate cases of the method."""
import numpy as np
import pytest
import torch

from helpers import (check_compare, check_quality, close, csr_from_edges, random_graph, star, to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05492_gb300 import qm as q
    return q


@pytest.fixture(scope="module")
def gen():
    from paper_1507_05492_gb300 import gen as g
    return g


def score_both(qm, oracle_mod, rp, col, lab, K, per_community=False, graph=None):
    rp = np.asarray(rp, np.int64)
    col = np.asarray(col, np.int32)
    lab = np.asarray(lab, np.int32)
    g = graph or qm.Graph(*to_dev(rp, col))
    q = qm.score(g, torch.as_tensor(lab).cuda(), K, per_community=per_community)
    o = oracle_mod.score(rp, col, lab, K, per_community=per_community)
    return q, o


# ------------------------------------------------------------------ closed forms through the GPU

def test_two_cliques_closed_forms(qm, oracle_mod):
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))
    edges = [(i, j) for i in range(5) for j in range(i + 1, 5)] + \
            [(i + 5, j + 5) for i in range(5) for j in range(i + 1, 5)] + [(4, 5)]
    rp, col = csr_from_edges(10, edges)
    g = qm.Graph(*to_dev(rp, col), validate=True)
    for case in ("planted", "one_community", "singletons"):
        c = gold["two_cliques"][case]
        lab = np.array(c["labels"], np.int32)
        q = qm.score(g, torch.as_tensor(lab).cuda(), int(lab.max()) + 1)
        num, den = c["modularity"]
        assert close(q["modularity"], num / den, 1.0)
        num, den = c["modularity_density"]
        assert close(q["modularity_density"], num / den, 1.0)
    t = gold["two_partitions"]
    r = qm.compare(torch.tensor(t["truth"], dtype=torch.int32).cuda(),
                   torch.tensor(t["found"], dtype=torch.int32).cuda(), 2, 2)
    assert (r["a11"], r["a10"], r["a01"], r["a00"]) == (16, 4, 5, 20)
    assert close(r["ari"], 40 / 67, 1.0) and close(r["f_measure"], 89 / 99, 1.0)
    assert close(r["vi"], t["vi"], rel=1e-13) and close(r["nmi"], t["nmi"], rel=1e-13)


# ------------------------------------------------------------------ LFR-style inputs

@pytest.mark.parametrize("n,seed", [(1000, 1), (12_345, 2), (100_003, 3)])
def test_score_lfr(qm, gen, oracle_mod, n, seed):
    g = gen.lfr_graph(gen.LfrParams(n=n, seed=seed))
    q, o = score_both(qm, oracle_mod, g.row_ptr, g.col, g.labels, g.K, per_community=True)
    check_quality(q, o, f"lfr n={n}")
    pq, po = q["per_community"], o["per_community"]
    for k in ("size", "intra_edges", "inter_edges"):
        assert np.array_equal(pq[k].cpu().numpy(), po[k]), k
    for k in ("intra_density", "contraction", "expansion", "conductance", "qds_term"):
        a, b = pq[k].cpu().numpy(), po[k]
        assert np.all(np.abs(a - b) <= 1e-12 * np.maximum(np.abs(b), 1e-3)), k


@pytest.mark.parametrize("frac", [0.0, 0.1, 0.5])
def test_compare_lfr(qm, gen, oracle_mod, frac):
    g = gen.lfr_graph(gen.LfrParams(n=20_011, seed=5))
    b = gen.perturb(g.labels, g.K, frac, seed=101)
    c = qm.compare(g.labels.cuda(), b.cuda(), g.K, g.K)
    o = oracle_mod.compare(g.labels.numpy(), b.numpy(), g.K, g.K)
    check_compare(c, o, f"frac={frac}")


def test_candidate_partitions(qm, gen, oracle_mod):
    g = gen.lfr_graph(gen.LfrParams(n=30_000, seed=6))
    graph = qm.Graph(*to_dev(g.row_ptr, g.col))
    for s in range(4):
        lab, K, f = gen.candidate_partition(g.labels, seed=10_000 + s, k_range=(50, 1500))
        q, o = score_both(qm, oracle_mod, g.row_ptr, g.col, lab, K, graph=graph)
        check_quality(q, o, f"candidate {s}")
        c = qm.compare(g.labels.cuda(), lab.cuda(), g.K, K)
        check_compare(c, oracle_mod.compare(g.labels.numpy(), lab.numpy(), g.K, K), f"candidate {s}")


# ------------------------------------------------------------------ degenerate cases

def test_one_community_and_singletons(qm, gen, oracle_mod):
    g = gen.lfr_graph(gen.LfrParams(n=5000, seed=7))
    graph = qm.Graph(*to_dev(g.row_ptr, g.col))
    n = g.n
    for lab, K in ((np.zeros(n, np.int32), 1), (np.arange(n, dtype=np.int32), n)):
        q, o = score_both(qm, oracle_mod, g.row_ptr, g.col, lab, K, graph=graph)
        check_quality(q, o, f"K={K}")
    assert close(q["modularity_density"], -1.0)  # singletons
    one, sing = np.zeros(n, np.int32), np.arange(n, dtype=np.int32)
    c = qm.compare(*to_dev(one, sing), 1, n)
    check_compare(c, oracle_mod.compare(one, sing, 1, n))
    c = qm.compare(*to_dev(sing, one), n, 1)
    check_compare(c, oracle_mod.compare(sing, one, n, 1))
    c = qm.compare(*to_dev(sing, sing), n, n)
    assert c["vi"] == 0.0 and close(c["nmi"], 1.0) and close(c["ari"], 1.0) and c["nvd"] == 0.0


def test_empty_label_ids_and_max_label(qm, oracle_mod):
    rp, col = random_graph(3000, 20_000, seed=8)
    rng = np.random.default_rng(8)
    K = 40_000  # far more ids than nodes: most communities are absent
    lab = rng.integers(0, K, 3000).astype(np.int32)
    lab[0] = K - 1
    q, o = score_both(qm, oracle_mod, rp, col, lab, K)
    check_quality(q, o, "sparse ids")
    truth = rng.integers(0, 7, 3000).astype(np.int32)
    c = qm.compare(*to_dev(truth, lab), 7, K)
    check_compare(c, oracle_mod.compare(truth, lab, 7, K))


def test_label_space_beyond_24_bits(qm, gen, oracle_mod):
    """K >= 2^24 - 1 takes the count tables with 31-bit keys; the result must
    equal, bit for bit, the one for the same partition with compact ids (the
    metrics ignore empty communities and the names of the others)."""
    g = gen.lfr_graph(gen.LfrParams(n=30_000, seed=12))
    graph = qm.Graph(*to_dev(g.row_ptr, g.col))
    K_big = (1 << 24) + 5
    ids = np.random.default_rng(12).choice(K_big, g.K, replace=False).astype(np.int32)
    ids[0] = K_big - 1
    lab = g.labels.numpy()
    q_big = qm.score(graph, torch.from_numpy(ids[lab]).cuda(), K_big)
    q_small = qm.score(graph, g.labels.cuda(), g.K)
    assert q_big == q_small
    check_quality(q_small, oracle_mod.score(g.row_ptr.numpy(), g.col.numpy(), lab, g.K), "compact ids")


def test_star_hub_forces_multipass(qm, oracle_mod):
    """A hub whose community borders 30k other communities overflows every
    shared-memory table; the block path splits its neighbour ids into classes."""
    rp, col = star(30_000)
    n = 30_001
    lab = np.arange(n, dtype=np.int32)
    lab[1:100] = 0  # the hub's community also holds 99 leaves
    q, o = score_both(qm, oracle_mod, rp, col, lab, n)
    check_quality(q, o, "star")
    found = np.zeros(n, np.int32)
    c = qm.compare(*to_dev(lab, found), n, 1)
    check_compare(c, oracle_mod.compare(lab, found, n, 1), "star compare")


def test_isolated_nodes(qm, oracle_mod):
    rp, col = random_graph(2000, 3000, seed=9)
    n = 2500  # nodes 2000..2499 have no edges
    rp = np.concatenate([rp, np.full(n - 2000, rp[-1])])
    rng = np.random.default_rng(9)
    lab = rng.integers(0, 300, n).astype(np.int32)
    lab[2400:] = 299  # a community of isolated nodes only
    lab[lab == 299] = 299
    lab[:2400][lab[:2400] == 299] = 0
    q, o = score_both(qm, oracle_mod, rp, col, lab, 300)
    check_quality(q, o, "isolated")


def test_every_launch_shape_gives_identical_bits(qm, gen, oracle_mod):
    g = gen.lfr_graph(gen.LfrParams(n=40_000, k_max=100, s_max=1000, seed=10))
    graph = qm.Graph(*to_dev(g.row_ptr, g.col))
    lab = g.labels.cuda()
    o = oracle_mod.score(g.row_ptr.numpy(), g.col.numpy(), g.labels.numpy(), g.K)
    ref = None
    for algo in (1, 0, 2, 3, 4, 5):
        for threads, smem, big in ((512, 96 * 1024, 48), (256, 48 * 1024, 16), (1024, 200 * 1024, 400),
                                   (128, 16 * 1024, 1), (512, 20 * 1024, 100_000)):
            qm.set_tuning(graph, g.K, threads, smem, big, algo)
            assert qm.get_tuning(graph, g.K)["algorithm"] == algo
            q = qm.score(graph, lab, g.K)
            check_quality(q, o, f"algorithm {algo} shape {threads}/{smem}/{big}")
            if ref is None:
                ref = q
            assert q == ref, (algo, threads, smem, big)


def test_deterministic_and_host_inputs(qm, gen):
    g = gen.lfr_graph(gen.LfrParams(n=50_000, seed=11))
    graph_dev = qm.Graph(*to_dev(g.row_ptr, g.col))
    graph_host = qm.Graph(g.row_ptr.numpy(), g.col.numpy())
    b = gen.perturb(g.labels, g.K, 0.2, seed=5)
    runs = [qm.score(graph_dev, g.labels.cuda(), g.K) for _ in range(3)]
    runs.append(qm.score(graph_host, g.labels.numpy(), g.K))
    runs.append(qm.score(graph_dev, g.labels.numpy(), g.K))
    assert all(r == runs[0] for r in runs)
    c1 = qm.compare(g.labels.cuda(), b.cuda(), g.K, g.K)
    c2 = qm.compare(g.labels.numpy(), b.numpy(), g.K, g.K)
    assert c1 == c2


def test_per_community_host_outputs(qm, gen, oracle_mod):
    g = gen.lfr_graph(gen.LfrParams(n=8000, seed=12))
    graph = qm.Graph(*to_dev(g.row_ptr, g.col))
    K = g.K + 5  # trailing absent ids get zeros
    q = qm.score(graph, g.labels.numpy(), K, per_community=True)
    o = oracle_mod.score(g.row_ptr.numpy(), g.col.numpy(), g.labels.numpy(), K, per_community=True)
    for k in ("size", "intra_edges", "inter_edges"):
        assert np.array_equal(q["per_community"][k], o["per_community"][k])
    assert np.all(q["per_community"]["qds_term"][g.K:] == 0)


def test_invalid_labels_rejected(qm, gen):
    g = gen.lfr_graph(gen.LfrParams(n=2000, seed=13))
    graph = qm.Graph(*to_dev(g.row_ptr, g.col))
    for bad in (g.K, -1):
        lab = g.labels.clone()
        lab[123] = bad
        with pytest.raises(qm.QmError) as e:
            qm.score(graph, lab.cuda(), g.K)
        assert e.value.status == qm.QM_EINVAL
        with pytest.raises(qm.QmError):
            qm.compare(g.labels.cuda(), lab.cuda(), g.K, g.K)
        for truth in (lab.cuda(), lab.numpy()):          # a ground-truth label out of range
            found = g.labels.cuda() if isinstance(truth, torch.Tensor) else g.labels.numpy()
            with pytest.raises(qm.QmError) as e:
                qm.compare(truth, found, g.K, g.K)
            assert e.value.status == qm.QM_EINVAL
    # the library stays usable after a rejected call
    q = qm.score(graph, g.labels.cuda(), g.K)
    assert q["n_nodes"] == 2000


def test_graph_validation(qm):
    rp, col = random_graph(500, 2000, seed=14)
    g = qm.Graph(*to_dev(rp, col), validate=True)
    assert g.info()["n_edges"] == len(col) // 2
    bad = col.copy()
    bad[0], bad[1] = bad[1], bad[0]  # unsorted row (and possibly asymmetric)
    with pytest.raises(qm.QmError):
        qm.Graph(*to_dev(rp, bad), validate=True)
    oob = col.copy()
    oob[5] = 10_000
    with pytest.raises(qm.QmError):
        qm.Graph(*to_dev(rp, oob))  # ids out of range are always rejected


def test_epoch_wraparound_in_block_tables(qm, oracle_mod):
    """With a small launch shape almost every community goes to a block, and
    each block counts hundreds of communities, so its table epochs wrap (and
    the table is wiped) several times; the results must not change."""
    rp, col = random_graph(400_000, 8_000_000, seed=41)
    rng = np.random.default_rng(41)
    K = 160_000  # ~2.5 nodes and ~100 cut arcs per community
    lab = rng.integers(0, K, 400_000).astype(np.int32)
    graph = qm.Graph(*to_dev(rp, col))
    o = oracle_mod.score(rp, col, lab, K)
    ref = None
    for threads, smem in ((512, 20 * 1024), (128, 16 * 1024), (512, 96 * 1024)):
        qm.set_tuning(graph, K, threads, smem, 48, 1)
        q = qm.score(graph, torch.from_numpy(lab).cuda(), K)
        check_quality(q, o, f"shape {threads}/{smem}")
        if ref is None:
            ref = q
        assert q == ref
