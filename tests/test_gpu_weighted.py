"""Weighted graphs (qm_load_graph_weighted): Q and Qds in the paper's weighted
reading (edge amounts weighted, densities unweighted; the note beside Eq. 9)
against the hand-derived closed forms and the oracle; the counts and the six
measures equal to the unweighted call's; bit-identical results for reordered
graphs, sharded calls and every launch-shape setting; the load-time checks
of the weights; and refusal by the calls that do not take weighted graphs."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

from helpers import to_dev
from test_oracle_weighted_pins import weighted_csr

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "closed_forms.json")))["weighted_triangle_path"]
COUNTS = ["n_nodes", "n_edges", "n_communities_nonempty", "intra_edges_total", "cut_edges_total",
          "n_community_pairs", "pair_count_sq_sum"]
MEANS = ["mean_intra_edges", "mean_intra_density", "mean_contraction", "mean_inter_edges", "mean_expansion",
         "mean_conductance"]


def close(a, b, cond=0.0, rel=1e-12):
    return abs(a - b) <= rel * max(abs(b), abs(cond), 1e-300)


@pytest.fixture(scope="module")
def qm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05492_gb300 import qm as q
    return q


def symmetric_weights(row_ptr, col, lo=0.05, hi=5.0):
    """A float32 weight per arc, equal on (u, v) and (v, u), from a hash of the pair."""
    rp = np.asarray(row_ptr, np.int64)
    v = np.asarray(col, np.int64)
    u = np.repeat(np.arange(len(rp) - 1, dtype=np.int64), np.diff(rp))
    a, b = np.minimum(u, v), np.maximum(u, v)
    h = (a * 2654435761 + b * 40503 + 12345) % (1 << 32)
    return (lo + (h / float(1 << 32)) * (hi - lo)).astype(np.float32)


@pytest.fixture(scope="module")
def setup(qm):
    from paper_1507_05492_gb300 import gen
    g = gen.lfr_graph(gen.LfrParams(n=40_000, k_max=200, s_max=2000, seed=51))
    w = symmetric_weights(g.row_ptr.numpy(), g.col.numpy())
    plain = qm.Graph(*to_dev(g.row_ptr, g.col))
    wg = qm.Graph(*to_dev(g.row_ptr, g.col), weights=w, validate=True)
    wgr = qm.Graph(*to_dev(g.row_ptr, g.col), weights=w, reorder=True)
    rng = np.random.default_rng(51)
    parts = {
        "planted": (g.labels, g.K),
        "perturbed": (gen.perturb(g.labels, g.K, 0.3, seed=8), g.K),
        "random": (torch.from_numpy(rng.integers(0, 600, g.n).astype(np.int32)), 600),
        "singletons": (torch.arange(g.n, dtype=torch.int32), g.n),
        "one": (torch.zeros(g.n, dtype=torch.int32), 1),
    }
    return g, w, plain, wg, wgr, parts


@pytest.mark.parametrize("case", ["two_groups", "singletons", "one_community"])
def test_closed_forms(qm, case):
    rp, col, wt = weighted_csr(5, GOLD["edges"])
    g = qm.Graph(*to_dev(rp, col), weights=wt.astype(np.float32), validate=True)
    c = GOLD[case]
    q = qm.score(g, torch.tensor(c["labels"], dtype=torch.int32).cuda(), max(c["labels"]) + 1)
    assert close(q["modularity"], float(Fraction(*c["modularity"])), 1.0)
    assert close(q["modularity_density"], float(Fraction(*c["modularity_density"])), 1.0)


@pytest.mark.parametrize("name", ["planted", "perturbed", "random", "singletons", "one"])
def test_against_oracle_and_unweighted_counts(qm, oracle_mod, setup, name):
    g, w, plain, wg, wgr, parts = setup
    labels, K = parts[name]
    o = oracle_mod.score_weighted(g.row_ptr.numpy(), g.col.numpy(), w.astype(np.float64), labels.numpy(), K)
    q = qm.score(wg, labels.cuda(), K)
    assert close(q["modularity"], o["modularity"], o["cond_modularity"]), (name, q["modularity"], o)
    assert close(q["modularity_density"], o["modularity_density"], o["cond_modularity_density"]), name
    u = qm.score(plain, labels.cuda(), K)
    for k in COUNTS + MEANS:
        assert q[k] == u[k], (name, k)
    assert qm.score(wgr, labels.cuda(), K) == q, name        # reordered: same bits
    assert qm.score(wg, labels.numpy(), K) == q, name         # host labels


def test_unit_weights_give_the_unweighted_metrics(qm, setup):
    g, _, plain, _, _, parts = setup
    ones = qm.Graph(*to_dev(g.row_ptr, g.col), weights=np.ones(g.col.numel(), np.float32))
    for name in ("planted", "perturbed"):
        labels, K = parts[name]
        a, b = qm.score(ones, labels.cuda(), K), qm.score(plain, labels.cuda(), K)
        assert close(a["modularity"], b["modularity"], 1.0)
        assert close(a["modularity_density"], b["modularity_density"], 1.0)


def test_sharded_and_tuning_give_the_same_bits(qm, setup):
    g, _, _, wg, _, parts = setup
    labels, K = parts["perturbed"]
    ref = qm.score(wg, labels.cuda(), K, per_community=True)
    pc = ref.pop("per_community")
    assert abs(float(pc["qds_term"].sum()) - ref["modularity_density"]) < 1e-9
    for P in (2, 5):
        parts_ = [qm.score_part(wg, labels.cuda(), K, r, P) for r in range(P)]
        assert qm.finalize_part(qm.combine_parts(parts_)) == ref
    qm.set_tuning(wg, K, 512, 96 * 1024, 48, 0)   # the one-kernel pipeline is not used for weighted graphs
    assert qm.score(wg, labels.cuda(), K) == ref


def test_weight_checks(qm, setup):
    g = setup[0]
    rp, col = to_dev(g.row_ptr, g.col)
    base = symmetric_weights(g.row_ptr.numpy(), g.col.numpy())
    for bad in (-1.0, float("nan"), float(2 ** 21), 1e-7):
        w = base.copy()
        w[5] = bad
        with pytest.raises(RuntimeError):
            qm.Graph(rp, col, weights=w)
    w = base.copy()
    w[7] = w[7] * 2                                   # asymmetric: caught by the full check
    with pytest.raises(RuntimeError):
        qm.Graph(rp, col, weights=w, validate=True)
    with pytest.raises(RuntimeError):
        qm.Graph(rp, col, weights=np.zeros(g.col.numel(), np.float32))
    zeros_ok = base.copy()
    zeros_ok[:] = np.where(np.arange(len(base)) % 3 == 0, 0.0, base)
    qm.Graph(rp, col, weights=zeros_ok)               # zero weights are allowed (symmetry not checked here)


def test_batched_calls_refuse_weighted_graphs(qm, setup):
    g, _, _, wg, _, parts = setup
    labels, K = parts["planted"]
    with pytest.raises(RuntimeError):
        qm.score_batched(wg, labels.cuda().unsqueeze(0), [K])
    with pytest.raises(RuntimeError):
        qm.score_graphs_batched([wg], [labels.cuda()], [K])


def test_one_million_nodes_against_oracle(qm, oracle_mod):
    from paper_1507_05492_gb300 import gen
    g = gen.lfr_graph(gen.LfrParams(n=1_000_000, k_max=100, s_max=1000, seed=52))
    w = symmetric_weights(g.row_ptr.numpy(), g.col.numpy(), 0.5, 2.0)
    wg = qm.Graph(*to_dev(g.row_ptr, g.col), weights=w, reorder=True)
    labels = gen.perturb(g.labels, g.K, 0.2, seed=9)
    o = oracle_mod.score_weighted(g.row_ptr.numpy(), g.col.numpy(), w.astype(np.float64), labels.numpy(), g.K)
    q = qm.score(wg, labels.cuda(), g.K)
    assert close(q["modularity"], o["modularity"], o["cond_modularity"])
    assert close(q["modularity_density"], o["modularity_density"], o["cond_modularity_density"])


def test_host_and_device_loads_agree(qm, setup):
    g, w, _, wg, _, parts = setup
    host = qm.Graph(g.row_ptr.numpy(), g.col.numpy(), weights=w, validate=True)
    labels, K = parts["perturbed"]
    assert qm.score(host, labels.cuda(), K) == qm.score(wg, labels.cuda(), K)
