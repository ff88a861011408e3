"""Shared helpers of the GPU parity tests: graph builders and the comparison of
CUDA results with the oracle under the tolerance rule

    counts: bit-exact;   floats: |g - o| <= 1e-12 * max(|o|, sum of |terms|)

where "sum of |terms|" is the conditioning the oracle reports for sums that can
cancel (Q, Qds, VI, NMI) and 1 for indices bounded by 1 in magnitude."""
import numpy as np
import torch

REL = 1e-12

SCORE_COUNTS = ("n_nodes", "n_edges", "n_communities_nonempty", "intra_edges_total", "cut_edges_total",
                "n_community_pairs", "pair_count_sq_sum")
COMPARE_COUNTS = ("n_nodes", "k_truth", "k_found", "n_cells", "a11", "a10", "a01", "a00", "nvd_sum")


def close(g, o, cond=0.0, rel=REL):
    return abs(g - o) <= rel * max(abs(o), abs(cond), 1e-300)


def check_quality(q, o, ctx=""):
    for k in SCORE_COUNTS:
        assert q[k] == o[k], f"{ctx} {k}: gpu {q[k]} oracle {o[k]}"
    assert close(q["modularity"], o["modularity"], o["cond_modularity"]), \
        f"{ctx} Q gpu {q['modularity']!r} oracle {o['modularity']!r}"
    assert close(q["modularity_density"], o["modularity_density"], o["cond_modularity_density"]), \
        f"{ctx} Qds gpu {q['modularity_density']!r} oracle {o['modularity_density']!r}"
    for k in ("mean_intra_edges", "mean_inter_edges", "mean_intra_density", "mean_contraction",
              "mean_expansion", "mean_conductance"):
        assert close(q[k], o[k]), f"{ctx} {k}: gpu {q[k]!r} oracle {o[k]!r}"


def check_compare(c, o, ctx=""):
    for k in COMPARE_COUNTS:
        assert c[k] == o[k], f"{ctx} {k}: gpu {c[k]} oracle {o[k]}"
    for k in ("ri", "ari", "ji", "nvd", "f_measure"):
        assert close(c[k], o[k], 1.0), f"{ctx} {k}: gpu {c[k]!r} oracle {o[k]!r}"
    assert close(c["vi"], o["vi"], o["cond_vi"]), f"{ctx} vi gpu {c['vi']!r} oracle {o['vi']!r}"
    cond_nmi = o["cond_nmi_num"] / max(o["nmi_den_abs"], 1e-300) + abs(o["nmi"])
    assert close(c["nmi"], o["nmi"], cond_nmi), f"{ctx} nmi gpu {c['nmi']!r} oracle {o['nmi']!r}"


def csr_from_edges(n, edges):
    """Symmetric CSR (sorted rows, no loops, no repeats) from an undirected edge list."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    a = np.minimum(e[:, 0], e[:, 1])
    b = np.maximum(e[:, 0], e[:, 1])
    key = np.unique(a * n + b)
    a, b = key // n, key % n
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, src + 1, 1)
    return np.cumsum(rp), dst.astype(np.int32)


def star(n_leaves):
    return csr_from_edges(n_leaves + 1, [(0, i) for i in range(1, n_leaves + 1)])


def random_graph(n, m, seed):
    rng = np.random.default_rng(seed)
    e = rng.integers(0, n, (m, 2))
    return csr_from_edges(n, e)


def to_dev(*arrays):
    return [torch.as_tensor(a).cuda() for a in arrays]
