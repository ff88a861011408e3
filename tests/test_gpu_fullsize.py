"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (default launch shape, graph and labels resident on the device).

* 10M nodes (|E| ~ 9.6e7): every output against the whole-graph oracle.
* 100M nodes (|E| ~ 9.6e8): every output against the whole-graph oracle, on
  the graph loaded with QM_REORDER (the order bench.py times) and on the graph
  as given, plus the comparison of the planted partition with a copy with 20%
  of the nodes moved (Eqs. 1-7) against the oracle.  The oracle runs in worker
  threads while the GPU calls are made.
* 100M nodes, sampled: communities checked one by one against the oracle's
  per-community routine, and the totals against identities that hold at any
  size."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

from helpers import check_quality, close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05492_gb300 import qm as q
    return q


def test_ten_million_nodes_against_whole_oracle(qm, oracle_mod):
    from paper_1507_05492_gb300 import gen
    g = gen.lfr_graph(gen.config_params("lfr10m"), device="cuda")
    graph = qm.Graph(g.row_ptr, g.col)
    q = qm.score(graph, g.labels, g.K, per_community=True)
    rp, col, lab = g.row_ptr.cpu().numpy(), g.col.cpu().numpy(), g.labels.cpu().numpy()
    o = oracle_mod.score(rp, col, lab, g.K, per_community=True)
    check_quality(q, o, "lfr10m")
    # the binned far-end gathers give the same bits
    q_plain = qm.score(graph, g.labels, g.K)
    for algo in (2, 3, 5):
        qm.set_tuning(graph, g.K, 512, 96 * 1024, 48, algo)
        assert qm.score(graph, g.labels, g.K) == q_plain, algo
    qm.set_tuning(graph, g.K, 512, 96 * 1024, 48, 1)
    for k in ("size", "intra_edges", "inter_edges"):
        assert np.array_equal(q["per_community"][k].cpu().numpy(), o["per_community"][k]), k
    a, b = q["per_community"]["qds_term"].cpu().numpy(), o["per_community"]["qds_term"]
    assert np.all(np.abs(a - b) <= 1e-12 * np.maximum(np.abs(b), 1e-6))
    # a perturbed partition and the comparison with the planted one, also at full size
    p = gen.perturb(g.labels, g.K, 0.2, seed=9)
    q2 = qm.score(graph, p, g.K)
    check_quality(q2, oracle_mod.score(rp, col, p.cpu().numpy(), g.K), "lfr10m perturbed")
    from helpers import check_compare
    c = qm.compare(g.labels, p, g.K, g.K)
    check_compare(c, oracle_mod.compare(lab, p.cpu().numpy(), g.K, g.K), "lfr10m compare")


def test_hundred_million_nodes_against_whole_oracle(qm, oracle_mod):
    from helpers import check_compare
    from paper_1507_05492_gb300 import gen
    qm.release_cache()  # scratch cached by earlier tests
    torch.cuda.empty_cache()
    g = gen.lfr_graph(gen.config_params("lfr100m"), device="cuda")
    found = gen.perturb(g.labels, g.K, 0.2, seed=9)
    rp, col, lab = g.row_ptr.cpu().numpy(), g.col.cpu().numpy(), g.labels.cpu().numpy()
    found_np = found.cpu().numpy()
    with ThreadPoolExecutor(2) as ex:
        fut_score = ex.submit(oracle_mod.score, rp, col, lab, g.K, True)
        fut_cmp = ex.submit(oracle_mod.compare, lab, found_np, g.K, g.K)
        results = {}
        for reorder in (True, False):
            graph = qm.Graph(g.row_ptr, g.col, reorder=reorder)
            q = qm.score(graph, g.labels, g.K, per_community=True)
            q["per_community"] = {k: v.cpu().numpy() for k, v in q["per_community"].items()}
            q_plain = qm.score(graph, g.labels, g.K)      # the call bench.py times (no per-community output)
            results[reorder] = (q, q_plain)
            graph.close()
            del graph
        c = qm.compare(g.labels, found, g.K, g.K)
        o = fut_score.result()
        oc = fut_cmp.result()
    opc = o["per_community"]
    for reorder, (q, q_plain) in results.items():
        ctx = f"lfr100m reorder={reorder}"
        check_quality(q, o, ctx)
        check_quality(q_plain, o, ctx + " (no per-community output)")
        pc = q["per_community"]
        for k in ("size", "intra_edges", "inter_edges"):
            assert np.array_equal(pc[k], opc[k]), (ctx, k)
        a, b = pc["qds_term"], opc["qds_term"]
        assert np.all(np.abs(a - b) <= 1e-12 * np.maximum(np.abs(b), 1e-6)), ctx
        for k in ("intra_density", "contraction", "expansion", "conductance"):
            assert np.all(np.abs(pc[k] - opc[k]) <= 1e-12 * np.abs(opc[k])), (ctx, k)
    # both node orders give the same bits
    assert {k: v for k, v in results[True][1].items()} == results[False][1]
    check_compare(c, oc, "lfr100m planted vs 20% moved")


def test_hundred_million_nodes_sampled(qm, oracle_mod):
    from paper_1507_05492_gb300 import gen
    g = gen.lfr_graph(gen.config_params("lfr100m"), device="cuda")
    graph = qm.Graph(g.row_ptr, g.col)
    q = qm.score(graph, g.labels, g.K, per_community=True)
    pc = {k: v.cpu().numpy() for k, v in q["per_community"].items()}
    n, E = g.n, g.n_edges
    # identities at any size
    assert q["n_nodes"] == n and q["n_edges"] == E
    assert pc["size"].sum() == n
    assert pc["intra_edges"].sum() == q["intra_edges_total"]
    assert pc["inter_edges"].sum() == 2 * q["cut_edges_total"]
    assert q["intra_edges_total"] + q["cut_edges_total"] == E
    assert q["n_communities_nonempty"] == int((pc["size"] > 0).sum())
    assert q["pair_count_sq_sum"] >= q["n_community_pairs"]
    assert -0.5 <= q["modularity"] <= 1.0
    # Q from the per-community integers (Eq. 8), summed exactly in Python
    vol = 2 * pc["intra_edges"].astype(object) + pc["inter_edges"].astype(object)
    num = 4 * E * int(pc["intra_edges"].sum()) - int(sum(v * v for v in vol))
    assert close(q["modularity"], num / (4 * E * E), 1.0)
    # sampled communities against the oracle, one by one
    rng = np.random.default_rng(5)
    nonempty = np.flatnonzero(pc["size"] > 0)
    big = nonempty[np.argsort(pc["size"][nonempty])[-3:]]
    ids = np.concatenate([rng.choice(nonempty, 13, replace=False), big]).astype(np.int32)
    rp, col, lab = g.row_ptr.cpu().numpy(), g.col.cpu().numpy(), g.labels.cpu().numpy()
    s = oracle_mod.score_communities(rp, col, lab, g.K, ids)
    for j, c in enumerate(ids):
        assert s["size"][j] == pc["size"][c]
        assert s["intra_edges"][j] == pc["intra_edges"][c]
        assert s["inter_edges"][j] == pc["inter_edges"][c]
        assert close(pc["qds_term"][c], s["qds_term"][j], abs(s["qds_term"][j]) + s["split"][j]), c
    # the mean measures are the means of the per-community arrays
    ne = q["n_communities_nonempty"]
    assert close(q["mean_conductance"], float(pc["conductance"].sum()) / ne, rel=1e-11)
    assert close(q["mean_intra_edges"], float(pc["intra_edges"].sum()) / ne)


def test_giant_runs_and_counts_beyond_2_25(qm, oracle_mod):
    """A random 2-way and 3-way split of the 10M-node graph: every community
    has ~5e7 cut arcs (runs far beyond 2^24 entries) and its few keys occur far
    more than 2^25 times, which takes the 64-bit-count general path."""
    from paper_1507_05492_gb300 import gen
    g = gen.lfr_graph(gen.config_params("lfr10m"), device="cuda")
    graph = qm.Graph(g.row_ptr, g.col)
    rp, col = g.row_ptr.cpu().numpy(), g.col.cpu().numpy()
    rng = np.random.default_rng(31)
    for K in (2, 3):
        lab = rng.integers(0, K, g.n).astype(np.int32)
        o = oracle_mod.score(rp, col, lab, K)
        for algo in (1, 0):
            qm.set_tuning(graph, K, 512, 96 * 1024, 48, algo)
            q = qm.score(graph, torch.from_numpy(lab).cuda(), K)
            check_quality(q, o, f"random {K}-way split, algorithm {algo}")
