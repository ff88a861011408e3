"""Sharded scoring (the decomposition by community of Sec. III-A) on one GPU:
the shards of a call, run one after another and combined exactly, must give
the bits of the unsharded qm_score_partition, for every shard count, every
kind of partition, host and device labels, and graphs loaded with QM_REORDER.
The multi-process exchange of the partials is covered on CPU
(tests/test_partials.py)."""
import numpy as np
import pytest
import torch

from helpers import check_quality, to_dev

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
    g = gen.lfr_graph(gen.LfrParams(n=50_000, k_max=200, s_max=2000, seed=41))
    plain = qm.Graph(*to_dev(g.row_ptr, g.col))
    reord = qm.Graph(*to_dev(g.row_ptr, g.col), reorder=True)
    rng = np.random.default_rng(41)
    sparse = rng.integers(0, 100, g.n).astype(np.int32) * 7      # many empty label ids
    parts = {
        "planted": (g.labels, g.K),
        "perturbed": (gen.perturb(g.labels, g.K, 0.3, seed=6), g.K),
        "random": (torch.from_numpy(rng.integers(0, 900, g.n).astype(np.int32)), 900),
        "sparse_ids": (torch.from_numpy(sparse), 700),
        "singletons": (torch.arange(g.n, dtype=torch.int32), g.n),
        "one": (torch.zeros(g.n, dtype=torch.int32), 1),
    }
    return g, plain, reord, parts


def sharded(qm, graph, labels, K, P):
    parts = [qm.score_part(graph, labels, K, r, P) for r in range(P)]
    return qm.finalize_part(qm.combine_parts(parts[::-1]))


@pytest.mark.parametrize("name", ["planted", "perturbed", "random", "sparse_ids", "singletons", "one"])
def test_shards_reproduce_the_unsharded_call(qm, setup, name):
    g, plain, reord, parts = setup
    labels, K = parts[name]
    lab = labels.cuda()
    ref = qm.score(plain, lab, K)
    for P in (1, 2, 3, 8, 64):
        assert sharded(qm, plain, lab, K, P) == ref, (name, P)
    assert sharded(qm, reord, lab, K, 5) == ref, name
    assert sharded(qm, plain, labels.numpy(), K, 4) == ref, name


def test_against_oracle(qm, setup, oracle_mod):
    g, plain, _, parts = setup
    labels, K = parts["perturbed"]
    o = oracle_mod.score(g.row_ptr.numpy(), g.col.numpy(), labels.numpy(), K)
    check_quality(sharded(qm, plain, labels.cuda(), K, 6), o, "6 shards")


def test_shard_partials_are_disjoint_sums(qm, setup):
    """Each shard's counters cover only its own communities: the intra-edge
    totals of the shards add up to the whole, and a shard owning no non-empty
    community contributes nothing."""
    g, plain, _, parts = setup
    labels, K = parts["one"]                          # one community, id 0: shard 0 owns it
    p1 = qm.score_part(plain, labels.cuda(), K, 1, 2)
    assert all(w == 0 for w in p1.words)
    p0 = qm.score_part(plain, labels.cuda(), K, 0, 2)
    assert any(w != 0 for w in p0.words)


def test_errors(qm, setup):
    g, plain, reord, parts = setup
    labels, K = parts["planted"]
    lab = labels.cuda()
    for rank, nranks in ((2, 2), (-1, 2), (0, 0), (0, 65)):
        with pytest.raises(RuntimeError):
            qm.score_part(plain, lab, K, rank, nranks)
    a = qm.score_part(plain, lab, K, 0, 3)
    b = qm.score_part(plain, lab, K, 1, 3)
    with pytest.raises(RuntimeError):
        qm.finalize_part(qm.combine_parts([a, b]))     # shard 2 missing
    other = qm.Graph(*to_dev(torch.tensor([0, 1, 2], dtype=torch.int64), torch.tensor([1, 0], dtype=torch.int32)))
    c = qm.score_part(other, torch.zeros(2, dtype=torch.int32).cuda(), 1, 2, 3)
    with pytest.raises(RuntimeError):
        qm.combine_parts([a, b, c])                    # a partial of another graph


def test_ten_million_nodes_four_shards(qm):
    from paper_1507_05492_gb300 import gen
    g = gen.lfr_graph(gen.config_params("lfr10m"), device=torch.device("cuda", 0))
    graph = qm.Graph(g.row_ptr, g.col, reorder=True)
    ref = qm.score(graph, g.labels, g.K)
    assert sharded(qm, graph, g.labels, g.K, 4) == ref


def test_single_process_sharded_call_on_a_side_stream(qm, setup):
    """dist.score_partition_sharded without a process group (one rank) runs the
    library's shard call and finalisation on the stream it is given."""
    from paper_1507_05492_gb300 import dist as qd
    g, plain, _, parts = setup
    labels, K = parts["perturbed"]
    lab = labels.cuda()
    ref = qm.score(plain, lab, K)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        got = qd.score_partition_sharded(plain, lab, K, stream=st)
    assert got == ref
