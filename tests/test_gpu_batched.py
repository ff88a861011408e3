"""The batched calls (the two-phase pipeline over all candidates, and the
one-block-per-item kernel for graphs beyond its run limit): every result must
equal, bit for bit, the plain one-partition call on the same inputs (which
itself matches the oracle),
and at the benchmark's batched shape (1,024 candidates per launch on 100,000-node
graphs with mixing 0.1, 0.3 and 0.5) every item matches the oracle."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

from helpers import check_compare, check_quality, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05492_gb300 import qm as q
    return q


@pytest.fixture(scope="module")
def setup(qm):
    from paper_1507_05492_gb300 import gen
    g = gen.lfr_graph(gen.LfrParams(n=20_000, seed=21))
    graph = qm.Graph(*to_dev(g.row_ptr, g.col))
    labs, Ks = [], []
    for p in range(24):
        lab, K, _ = gen.candidate_partition(g.labels, seed=10_000 + p, k_range=(100, 1200))
        labs.append(lab)
        Ks.append(K)
    # pad the label matrix: each row keeps its own K
    L = torch.stack(labs)
    return g, graph, L, Ks


def test_score_batched_equals_plain(qm, setup, oracle_mod):
    g, graph, L, Ks = setup
    out = qm.score_batched(graph, L.cuda(), Ks)
    for p in range(L.shape[0]):
        plain = qm.score(graph, L[p].cuda(), Ks[p])
        assert out[p] == plain, p
    o = oracle_mod.score(g.row_ptr.numpy(), g.col.numpy(), L[3].numpy(), Ks[3])
    check_quality(out[3], o, "batched p=3")


def test_evaluate_batched_equals_plain(qm, setup, oracle_mod):
    g, graph, L, Ks = setup
    truth = g.labels.cuda()
    oq, oc = qm.evaluate_batched(graph, L.cuda(), Ks, truth, g.K)
    for p in range(L.shape[0]):
        assert oq[p] == qm.score(graph, L[p].cuda(), Ks[p]), p
        assert oc[p] == qm.compare(truth, L[p].cuda(), g.K, Ks[p]), p
    check_compare(oc[5], oracle_mod.compare(g.labels.numpy(), L[5].numpy(), g.K, Ks[5]), "p=5")
    # host inputs give the same bits
    oq2, oc2 = qm.evaluate_batched(graph, L.numpy(), Ks, g.labels.numpy(), g.K)
    assert oq2 == oq and oc2 == oc
    # repeated launches replay the captured graph with identical results
    oq3, oc3 = qm.evaluate_batched(graph, L.cuda(), Ks, truth, g.K)
    assert oq3 == oq and oc3 == oc


def test_compare_batched(qm, setup):
    g, graph, L, Ks = setup
    shared = qm.compare_batched(g.labels.cuda(), L.cuda(), g.K, Ks, shared_truth=True)
    per = qm.compare_batched(g.labels.expand(L.shape[0], -1).contiguous().cuda(), L.cuda(),
                             [g.K] * L.shape[0], Ks, shared_truth=False)
    for p in range(L.shape[0]):
        plain = qm.compare(g.labels.cuda(), L[p].cuda(), g.K, Ks[p])
        assert shared[p] == plain and per[p] == plain, p


def test_graphs_of_uneven_sizes(qm, oracle_mod):
    from paper_1507_05492_gb300 import gen
    gs, graphs, labs, Ks = [], [], [], []
    for i, n in enumerate((500, 7_000, 31_337, 2_000, 64_000)):
        g = gen.lfr_graph(gen.LfrParams(n=n, seed=30 + i))
        gs.append(g)
        graphs.append(qm.Graph(*to_dev(g.row_ptr, g.col)))
        lab = gen.perturb(g.labels, g.K, 0.05 * i, seed=40 + i)
        labs.append(lab.cuda())
        Ks.append(g.K)
    out = qm.score_graphs_batched(graphs, labs, Ks)
    for i in range(len(gs)):
        assert out[i] == qm.score(graphs[i], labs[i], Ks[i]), i
        o = oracle_mod.score(gs[i].row_ptr.numpy(), gs[i].col.numpy(), labs[i].cpu().numpy(), Ks[i])
        check_quality(out[i], o, f"graph {i}")


def test_batched_rejects_bad_item(qm, setup):
    g, graph, L, Ks = setup
    bad = L.clone()
    bad[7, 11] = Ks[7]
    with pytest.raises(qm.QmError) as e:
        qm.score_batched(graph, bad.cuda(), Ks)
    assert e.value.status == qm.QM_EINVAL
    out = qm.score_batched(graph, L.cuda(), Ks)  # still usable
    assert out[0] == qm.score(graph, L[0].cuda(), Ks[0])


def test_autotune_batched_keeps_results(qm, setup):
    """qm_autotune_batched tries several launch shapes of the batched kernel and
    caches the fastest; every shape gives the same bits."""
    g, graph, L, Ks = setup
    truth = g.labels.cuda()
    ref_q, ref_c = qm.evaluate_batched(graph, L.cuda(), Ks, truth, g.K)
    t = qm.autotune_batched(graph, L.cuda(), Ks, truth, g.K)
    assert t["threads"] in (256, 512) and t["blocks_per_sm"] >= 1
    got = qm.get_batch_tuning(graph, max(Ks))
    assert (got["threads"], got["smem_bytes"], got["big_community"]) == \
        (t["threads"], t["smem_bytes"], t["big_community"])
    oq, oc = qm.evaluate_batched(graph, L.cuda(), Ks, truth, g.K)
    assert oq == ref_q and oc == ref_c
    for shape in ((256, 64 * 1024, 128), (512, 160 * 1024, 48)):
        qm.set_batch_tuning(graph, max(Ks), *shape)
        oq, oc = qm.evaluate_batched(graph, L.cuda(), Ks, truth, g.K)
        assert oq == ref_q and oc == ref_c, shape
    with pytest.raises(qm.QmError):                      # more threads than the kernel's launch bound
        qm.set_batch_tuning(graph, max(Ks), 1024, 96 * 1024, 128)


def test_batched_count_paths(qm, setup):
    """Candidates whose label ids exceed a group's direct counters take the
    hashed count, runs too long for a warp take whole blocks, and a batch that
    mixes them (under small and large launch shapes) still gives the plain
    bits for scoring and comparison."""
    g, graph, L, Ks = setup
    n = L.shape[1]
    rng = np.random.default_rng(5)
    rows, ks = [L[0], L[1]], [Ks[0], Ks[1]]
    for K in (n, n // 2, 6_000):  # mostly tiny communities over many ids
        rows.append(torch.from_numpy(rng.integers(0, K, n).astype(np.int32)))
        ks.append(K)
    giant = g.labels.clone()
    giant[: n // 2] = 0  # one community of half the nodes: a long run
    rows.append(giant)
    ks.append(g.K)
    M = torch.stack(rows).cuda()
    truth = g.labels.cuda()
    for shape in ((256, 32 * 1024, 128), (512, 96 * 1024, 128)):
        qm.set_batch_tuning(graph, max(ks), *shape)
        sq = qm.score_batched(graph, M, ks)
        oq, oc = qm.evaluate_batched(graph, M, ks, truth, g.K)
        for p in range(len(ks)):
            ref = qm.score(graph, M[p], ks[p])
            assert sq[p] == ref and oq[p] == ref, (shape, p)
            assert oc[p] == qm.compare(truth, M[p], g.K, ks[p]), (shape, p)


def test_batched_waves(qm, setup):
    """Batches larger than a wave run wave after wave (tables, counters and
    prefixes reset per wave) with the same bits as one wave."""
    g, graph, L, Ks = setup
    truth = g.labels.cuda()
    ref_q, ref_c = qm.evaluate_batched(graph, L.cuda(), Ks, truth, g.K)
    try:
        for items in (1, 5, 7):
            qm.debug_set_batch_wave(items)
            oq, oc = qm.evaluate_batched(graph, L.cuda(), Ks, truth, g.K)
            assert oq == ref_q and oc == ref_c, items
            assert qm.score_batched(graph, L.cuda(), Ks) == ref_q, items
    finally:
        qm.debug_set_batch_wave(0)
    with pytest.raises(qm.QmError):
        qm.debug_set_batch_wave(-1)


def test_dense_graph_batches(qm, oracle_mod):
    """A graph whose arcs exceed the two-phase batched pipeline's run limit
    (2^24 - 1) is batched by the one-block-per-item kernel: the same bits as
    the plain calls."""
    from paper_1507_05492_gb300 import gen
    g = gen.lfr_graph(gen.LfrParams(n=120_000, k_mean=150, k_max=300, s_min=400, s_max=1500, seed=71),
                      device="cuda")
    assert g.col.numel() > (1 << 24) - 1
    graph = qm.Graph(g.row_ptr, g.col)
    labs, Ks = gen.candidate_batch(g.labels, 4, seed=30_000, k_range=(50, 400))
    oq, oc = qm.evaluate_batched(graph, labs, Ks, g.labels, g.K)
    for p in range(len(Ks)):
        assert oq[p] == qm.score(graph, labs[p], Ks[p]), p
        assert oc[p] == qm.compare(g.labels, labs[p], g.K, Ks[p]), p
    check_quality(oq[1], oracle_mod.score(g.row_ptr.cpu().numpy(), g.col.cpu().numpy(), labs[1].cpu().numpy(),
                                          Ks[1]), "dense batch item 1")


@pytest.mark.parametrize("workload", ["lfr100k_mu01", "lfr100k_mu03", "lfr100k_mu05"])
def test_full_batch_against_oracle(qm, oracle_mod, workload):
    """One launch of 1,024 candidates (community counts 500-5,000, up to half of
    the nodes moved), scored and compared with the planted partition, exactly as
    bench.py times it; every item of both families against the oracle."""
    from paper_1507_05492_gb300 import gen
    g = gen.lfr_graph(gen.config_params(workload), device="cuda")
    graph = qm.Graph(g.row_ptr, g.col)
    labs, Ks = gen.candidate_batch(g.labels, 1024, seed=10_000)
    oq, oc = qm.evaluate_batched(graph, labs, Ks, g.labels, g.K)
    rp, col, truth = g.row_ptr.cpu().numpy(), g.col.cpu().numpy(), g.labels.cpu().numpy()
    L = labs.cpu().numpy()

    def both(p):
        return (oracle_mod.score(rp, col, L[p], Ks[p]), oracle_mod.compare(truth, L[p], g.K, Ks[p]))

    with ThreadPoolExecutor(max(1, os.cpu_count() or 1)) as ex:
        ref = list(ex.map(both, range(len(Ks))))
    for p, (o_s, o_c) in enumerate(ref):
        check_quality(oq[p], o_s, f"{workload} candidate {p}")
        check_compare(oc[p], o_c, f"{workload} candidate {p}")


def test_large_graph_batches_equal_plain(qm, oracle_mod):
    """Above 2^21 nodes the batched calls run the plain pipelines of every item
    in one captured launch: the same bits as the plain calls, for scoring,
    evaluation against a shared truth, comparisons with shared and per-item
    truths, host inputs and reordered graphs; an out-of-range label in one item
    is reported for the whole call."""
    from paper_1507_05492_gb300 import gen
    g = gen.lfr_graph(gen.LfrParams(n=2_500_000, k_max=100, s_max=1000, seed=61), device="cuda")
    plain = qm.Graph(g.row_ptr, g.col)
    reord = qm.Graph(g.row_ptr, g.col, reorder=True)
    labs, Ks = [], []
    for p in range(5):
        lab, K, _ = gen.candidate_partition(g.labels, seed=20_000 + p, k_range=(5_000, 20_000))
        labs.append(lab)
        Ks.append(K)
    L = torch.stack(labs)
    for graph in (plain, reord):
        oq, oc = qm.evaluate_batched(graph, L, Ks, g.labels, g.K)
        sq = qm.score_batched(graph, L, Ks)
        for p in range(len(Ks)):
            ref = qm.score(graph, L[p], Ks[p])
            assert oq[p] == ref and sq[p] == ref, p
            assert oc[p] == qm.compare(g.labels, L[p], g.K, Ks[p]), p
        oq2, _ = qm.evaluate_batched(graph, L.cpu().numpy(), Ks, g.labels.cpu().numpy(), g.K)
        assert oq2 == oq
    shared = qm.compare_batched(g.labels, L, g.K, Ks, shared_truth=True)
    per = qm.compare_batched(torch.roll(L, 1, 0).contiguous(), L, [Ks[-1]] + Ks[:-1], Ks, shared_truth=False)
    for p in range(len(Ks)):
        assert shared[p] == qm.compare(g.labels, L[p], g.K, Ks[p]), p
        q = (p - 1) % len(Ks)
        assert per[p] == qm.compare(L[q], L[p], Ks[q], Ks[p]), p
    check_quality(oq[2], oracle_mod.score(g.row_ptr.cpu().numpy(), g.col.cpu().numpy(), L[2].cpu().numpy(), Ks[2]),
                  "large batch item 2")
    bad = L.clone()
    bad[3, 17] = Ks[3]
    with pytest.raises(qm.QmError) as e:
        qm.score_batched(plain, bad, Ks)
    assert e.value.status == qm.QM_EINVAL
    assert qm.score_batched(plain, L, Ks)[0] == qm.score(plain, L[0], Ks[0])
