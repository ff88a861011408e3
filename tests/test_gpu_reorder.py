"""Graphs loaded with QM_REORDER (renumbered for locality at load time) must give,
bit for bit, the results of the same graph loaded as given, on every entry
point that takes a graph: plain scoring (device and host labels, per-community
outputs, both pipelines), the batched calls, the multi-graph call and the
allocation-free call."""
import ctypes

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
    g = gen.lfr_graph(gen.LfrParams(n=60_000, k_max=200, s_max=2000, seed=21))
    plain = qm.Graph(*to_dev(g.row_ptr, g.col))
    reord = qm.Graph(*to_dev(g.row_ptr, g.col), reorder=True)
    rng = np.random.default_rng(21)
    parts = [(g.labels, g.K),
             (gen.perturb(g.labels, g.K, 0.3, seed=3), g.K),
             (gen.perturb(g.labels, g.K, 0.002, seed=5), g.K),  # a few blocks of three labels
             (torch.from_numpy(rng.integers(0, 500, g.n).astype(np.int32)), 500),
             (torch.arange(g.n, dtype=torch.int32), g.n),
             (torch.zeros(g.n, dtype=torch.int32), 1)]
    return g, plain, reord, parts


def test_reorder_keeps_graph_info(qm, setup):
    g, plain, reord, _ = setup
    a, b = plain.info(), reord.info()
    assert a["n_nodes"] == b["n_nodes"] and a["n_edges"] == b["n_edges"] and a["max_degree"] == b["max_degree"]
    assert b["device_bytes"] == a["device_bytes"] + 4 * g.n


@pytest.mark.parametrize("algo", [1, 0, 2, 3, 4])
def test_plain_scoring_identical(qm, setup, oracle_mod, algo):
    g, plain, reord, parts = setup
    for labels, K in parts:
        for gr in (plain, reord):
            qm.set_tuning(gr, K, 512, 96 * 1024, 48, algo)
        a = qm.score(plain, labels.cuda(), K, per_community=True)
        b = qm.score(reord, labels.cuda(), K, per_community=True)
        c = qm.score(reord, labels.numpy(), K)
        pa, pb = a.pop("per_community"), b.pop("per_community")
        assert a == b == c, K
        for key in pa:
            assert torch.equal(pa[key].cpu(), pb[key].cpu()), key
    labels, K = parts[1]
    o = oracle_mod.score(g.row_ptr.numpy(), g.col.numpy(), labels.numpy(), K)
    check_quality(qm.score(reord, labels.cuda(), K), o, "reordered, perturbed")


def test_batched_calls_identical(qm, setup):
    g, plain, reord, parts = setup
    labels = torch.stack([p[0] for p in parts[:3]]).cuda()
    K = [p[1] for p in parts[:3]]
    assert qm.score_batched(plain, labels, K) == qm.score_batched(reord, labels, K)
    qa, ca = qm.evaluate_batched(plain, labels, K, g.labels.cuda(), g.K)
    qb, cb = qm.evaluate_batched(reord, labels, K, g.labels.cuda(), g.K)
    assert qa == qb and ca == cb
    # a reordered and a plain graph in one multi-graph launch
    outs = qm.score_graphs_batched([reord, plain], [parts[1][0].cuda(), parts[1][0].cuda()], [g.K, g.K])
    assert outs[0] == outs[1] == qm.score(plain, parts[1][0].cuda(), g.K)


def test_allocation_free_call_identical(qm, setup):
    from paper_1507_05492_gb300.qm import QmQuality
    g, plain, reord, parts = setup
    f = qm.lib().qm_score_partition_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    labels, K = parts[1]
    lab = labels.cuda()
    out = QmQuality()
    assert f(reord.handle, lab.data_ptr(), K, ctypes.byref(out), None) == 0, qm.last_error()
    torch.cuda.synchronize()
    got = {name: getattr(out, name) for name, _ in out._fields_}
    assert got == qm.score(plain, lab, K)


@pytest.mark.parametrize("algo", [1, 0, 2, 3, 4])
def test_out_of_range_label_rejected(qm, setup, algo):
    g, plain, reord, parts = setup
    labels, K = parts[0]
    bad = labels.clone()
    bad[12345] = K                                   # one label past the end
    qm.set_tuning(reord, K, 512, 96 * 1024, 48, algo)
    with pytest.raises(RuntimeError):
        qm.score(reord, bad.cuda(), K)
    assert qm.score(reord, labels.cuda(), K) == qm.score(plain, labels.cuda(), K)



def bucketed_graph(qm, g, wb, tb):
    """The graph loaded with QM_REORDER and the two-pass label permutation
    forced on: tiles of 2**tb caller ids, windows of 2**wb new ids."""
    qm.debug_set_perm_buckets(wb, tb, 0)
    try:
        return qm.Graph(*to_dev(g.row_ptr, g.col), reorder=True)
    finally:
        qm.debug_set_perm_buckets(-1, -1, -1)


# 60,000 nodes: (10, 12) gives 59 windows and 15 tiles; (8, 2) 235 windows and
# 15,000 tiles of 4 ids; (15, 16) two windows and one tile; (16, 16) (what
# a graph of up to 293M nodes gets by default) one of each, too large for
# 4-byte labels in shared memory, so that K > 2^24 gathers directly; (1, 15) would need 30,000 windows, more than the
# passes take, so that graph always gathers its labels directly.
@pytest.mark.parametrize("wb,tb,algos", [(10, 12, (1, 0, 4, 7)), (8, 2, (1, 0)), (15, 16, (1,)), (16, 16, (1, 0)),
                                         (1, 15, (1,))])
def test_two_pass_permutation_identical(qm, setup, oracle_mod, wb, tb, algos):
    g, plain, reord, parts = setup
    gb = bucketed_graph(qm, g, wb, tb)
    nw, nt = -(-g.n // 2 ** wb), -(-g.n // 2 ** tb)
    extra = 4 * g.n + 4 * nw * nt + 4 * nt * (nw + 1) if nw <= 8192 else 0
    assert gb.info()["device_bytes"] == reord.info()["device_bytes"] + extra
    # labels of 25 bits (shared memory holds them as 4 bytes, or they are gathered)
    wide = (torch.where(g.labels % 2 == 1, g.labels + 2 ** 24, g.labels), 2 ** 24 + g.K)
    for algo in algos:
        for gr in (plain, gb):
            qm.set_tuning(gr, wide[1], 512, 96 * 1024, 48, algo)
        assert qm.score(plain, wide[0].cuda(), wide[1]) == qm.score(gb, wide[0].cuda(), wide[1]), algo
        for labels, K in parts:
            for gr in (plain, gb):
                qm.set_tuning(gr, K, 512, 96 * 1024, 48, algo)
            a = qm.score(plain, labels.cuda(), K, per_community=True)
            b = qm.score(gb, labels.cuda(), K, per_community=True)
            c = qm.score(gb, labels.numpy(), K)
            pa, pb = a.pop("per_community"), b.pop("per_community")
            assert a == b == c, (algo, K)
            for key in pa:
                assert torch.equal(pa[key].cpu(), pb[key].cpu()), (algo, key)
    labels, K = parts[1]
    o = oracle_mod.score(g.row_ptr.numpy(), g.col.numpy(), labels.numpy(), K)
    check_quality(qm.score(gb, labels.cuda(), K), o, "two-pass permutation, perturbed")
    bad = labels.clone()
    bad[777] = -1                                    # a label below the range
    for algo in algos:
        qm.set_tuning(gb, K, 512, 96 * 1024, 48, algo)
        with pytest.raises(RuntimeError):
            qm.score(gb, bad.cuda(), K)
    assert qm.score(gb, labels.cuda(), K) == qm.score(plain, labels.cuda(), K)


def test_perm_bucket_hook_rejects_bad_bits(qm):
    for wb, tb in ((0, 10), (17, 10), (10, 0), (10, 17)):
        with pytest.raises(RuntimeError):
            qm.debug_set_perm_buckets(wb, tb, 0)
    qm.debug_set_perm_buckets(-1, -1, -1)
