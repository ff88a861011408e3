"""Overlapping communities (covers) on the GPU through the C ABI, against the
oracle's cover statement: the hand-derived closed forms, covers with one
community per node (which must give the partition calls' bits), LFR-style
covers where a share of the nodes also joins a neighbour's community (graph as
given and renumbered, host and device arrays), empty lists, unused ids, a hub
whose community borders 30,000 others (multi-pass counting), a community of
3,000 overlapping members (pairs beyond the shared-memory list), and malformed
lists."""
import json
import os

import numpy as np
import pytest
import torch

from helpers import check_compare, check_quality, close, csr_from_edges, star

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


@pytest.fixture(scope="module")
def qm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05492_gb300 import qm as q
    return q


def frac(v):
    return v[0] / v[1] if isinstance(v, list) else v


def lists_cover(lists):
    mptr = np.zeros(len(lists) + 1, np.int64)
    mptr[1:] = np.cumsum([len(x) for x in lists])
    memb = np.array([c for x in lists for c in x], dtype=np.int32)
    return mptr, memb


def dev(cover):
    return torch.from_numpy(cover[0]).cuda(), torch.from_numpy(cover[1]).cuda()


def overlap_cover(rp, col, labels, frac_extra, seed):
    """Each node keeps its community; a share of the nodes also joins the
    community of one of their neighbours (when it differs)."""
    rng = np.random.default_rng(seed)
    lists = []
    for u in range(len(labels)):
        x = [int(labels[u])]
        d = rp[u + 1] - rp[u]
        if d and rng.random() < frac_extra:
            v = col[rp[u] + int(rng.integers(d))]
            if labels[v] != labels[u]:
                x = sorted(set(x) | {int(labels[v])})
        lists.append(x)
    return lists_cover(lists)


@pytest.mark.parametrize("case", ["cover_bowtie", "cover_two_triangles"])
def test_closed_forms(qm, case):
    g = GOLD[case]
    rp, col = csr_from_edges(g["n"], g["edges"])
    graph = qm.Graph(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda())
    cov = lists_cover(g["cover"])
    s = qm.score_cover(graph, dev(cov), g["K"])
    for k in ("modularity", "modularity_density", "mean_intra_edges", "mean_intra_density", "mean_contraction",
              "mean_inter_edges", "mean_expansion", "mean_conductance"):
        assert close(s[k], frac(g[k]), 1.0, 1e-14), (k, s[k], g[k])
    assert s["intra_edges_total"] == g["intra_edges_total"] and s["cut_edges_total"] == g["boundary_total"]
    assert s["n_community_pairs"] == g["n_community_pairs"] and s["pair_count_sq_sum"] == g["pair_count_sq_sum"]
    c = qm.compare_covers(dev(cov), g["K"], dev(lists_cover(g["found"])), g["k_found"], g["n"])
    for k in ("a11", "a10", "a01", "a00"):
        assert c[k] == g[k], k
    for k in ("vi", "nmi", "f_measure", "nvd", "ri", "ari", "ji"):
        assert close(c[k], frac(g[k]), 1.0, 1e-13), (k, c[k], g[k])


def test_one_community_per_node_gives_the_partition_bits(qm):
    from paper_1507_05492_gb300 import gen
    g = gen.lfr_graph(gen.LfrParams(n=50_000, k_max=100, s_max=1000, seed=81), device="cuda")
    b = gen.perturb(g.labels, g.K, 0.3, seed=82)
    lab, labb = g.labels.cpu().numpy(), b.cpu().numpy()
    ca = dev(lists_cover([[int(x)] for x in lab]))
    cb = dev(lists_cover([[int(x)] for x in labb]))
    for reorder in (False, True):
        graph = qm.Graph(g.row_ptr, g.col, reorder=reorder)
        for cov, labels in ((ca, g.labels), (cb, b)):
            q = qm.score(graph, labels, g.K)
            s = qm.score_cover(graph, cov, g.K)
            assert s["cut_edges_total"] == 2 * q["cut_edges_total"]
            s["cut_edges_total"] = q["cut_edges_total"]
            assert s == q, reorder
    assert qm.compare_covers(ca, g.K, cb, g.K, g.n) == qm.compare(g.labels, b, g.K, g.K)


@pytest.mark.parametrize("n,extra", [(20_011, 0.1), (150_000, 0.3)])
def test_lfr_covers_against_oracle(qm, oracle_mod, n, extra):
    from paper_1507_05492_gb300 import gen
    g = gen.lfr_graph(gen.LfrParams(n=n, k_max=100, s_max=1000, seed=83 + n % 7), device="cuda")
    rp, col, lab = g.row_ptr.cpu().numpy(), g.col.cpu().numpy(), g.labels.cpu().numpy()
    cov = overlap_cover(rp, col, lab, extra, seed=84)
    found = overlap_cover(rp, col, gen.perturb(g.labels, g.K, 0.2, seed=85).cpu().numpy(), extra / 2, seed=86)
    o = oracle_mod.score_cover(rp, col, cov[0], cov[1], g.K)
    for reorder in (False, True):
        graph = qm.Graph(g.row_ptr, g.col, reorder=reorder)
        s = qm.score_cover(graph, dev(cov), g.K)
        check_quality(s, o, f"cover n={n} reorder={reorder}")
        assert qm.score_cover(graph, cov, g.K) == s  # host arrays: the same bits
    oc = oracle_mod.compare_cover(cov[0], cov[1], g.K, found[0], found[1], g.K)
    c = qm.compare_covers(dev(cov), g.K, dev(found), g.K, g.n)
    check_compare(c, oc, f"cover compare n={n}")
    assert qm.compare_covers(cov, g.K, found, g.K, g.n) == c


def test_empty_lists_unused_ids_and_a_busy_hub(qm, oracle_mod):
    rng = np.random.default_rng(87)
    rp, col = csr_from_edges(4000, rng.integers(0, 4000, (20_000, 2)))
    lists = []
    for u in range(4000):
        r = rng.random()
        lists.append([] if r < 0.1 else sorted({int(rng.integers(0, 900)) * 3 for _ in range(1 + (r > 0.7))}))
    cov = lists_cover(lists)
    K = 3000  # ids are multiples of 3: most are unused
    graph = qm.Graph(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda())
    check_quality(qm.score_cover(graph, dev(cov), K), oracle_mod.score_cover(rp, col, cov[0], cov[1], K), "sparse")
    lists2 = [sorted({int(rng.integers(0, 50))}) if rng.random() > 0.2 else [] for _ in range(4000)]
    c2 = lists_cover(lists2)
    check_compare(qm.compare_covers(dev(cov), K, dev(c2), 50, 4000),
                  oracle_mod.compare_cover(cov[0], cov[1], K, c2[0], c2[1], 50), "sparse compare")
    # a hub in community 0 whose leaves each have their own community (and half also community 0)
    rp, col = star(30_000)
    hub = [[0]] + [[i] if i % 2 else [0, i] for i in range(1, 30_001)]
    cov = lists_cover(hub)
    graph = qm.Graph(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda())
    check_quality(qm.score_cover(graph, dev(cov), 30_001), oracle_mod.score_cover(rp, col, cov[0], cov[1], 30_001),
                  "hub")


def test_large_overlapping_community(qm, oracle_mod):
    """Every node in community 0 and in one of 30 others: community 0 has
    3,000 members with two memberships, more than the shared-memory list
    holds, and every pair of them shares two communities or one."""
    n = 3000
    rng = np.random.default_rng(88)
    A = lists_cover([[0, 1 + int(rng.integers(30))] for _ in range(n)])
    B = lists_cover([[int(rng.integers(40)), 40 + int(rng.integers(5))] for _ in range(n)])
    c = qm.compare_covers(dev(A), 31, dev(B), 45, n)
    o = oracle_mod.compare_cover(A[0], A[1], 31, B[0], B[1], 45)
    check_compare(c, o, "large overlapping community")
    assert (c["a11"], c["a10"], c["a01"], c["a00"]) == oracle_mod.pairs_cover_bruteforce(A[0], A[1], B[0], B[1])


def test_malformed_covers_are_refused(qm):
    rp, col = csr_from_edges(4, [(0, 1), (1, 2), (2, 3)])
    graph = qm.Graph(torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda())
    good = lists_cover([[0], [0, 1], [1], [1]])
    assert qm.score_cover(graph, dev(good), 2)["n_nodes"] == 4
    for bad in ([[0], [1, 0], [1], [1]],      # not increasing
                [[0], [0, 0], [1], [1]],      # repeated
                [[0], [0, 2], [1], [1]]):     # out of range
        with pytest.raises(qm.QmError) as e:
            qm.score_cover(graph, dev(lists_cover(bad)), 2)
        assert e.value.status == qm.QM_EINVAL
        with pytest.raises(qm.QmError) as e:
            qm.compare_covers(dev(lists_cover(bad)), 2, dev(good), 2, 4)
        assert e.value.status == qm.QM_EINVAL
    with pytest.raises(qm.QmError) as e:                       # no community has a member
        qm.score_cover(graph, dev(lists_cover([[], [], [], []])), 2)
    assert e.value.status == qm.QM_EINVAL
    assert qm.score_cover(graph, dev(good), 2)["n_nodes"] == 4  # still usable
