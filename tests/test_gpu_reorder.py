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

