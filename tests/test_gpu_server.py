"""The serving loop: requests of different graph sizes admitted by a memory
budget and batched as they arrive; each result in the mix must equal the
result of the same request scored alone, and, on the serving workload's own
graphs (10k, 1M and 10M nodes), the oracle's result for that request."""
import os
import threading
from concurrent.futures import ThreadPoolExecutor
import time

import numpy as np
import pytest
import torch

from helpers import check_compare, check_quality, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05492_gb300 import gen, qm
    graphs, truths, pools = {}, {}, {}
    for gid, n in (("small", 3_000), ("mid", 60_000), ("large", 400_000)):
        g = gen.lfr_graph(gen.LfrParams(n=n, k_max=100 if n > 100_000 else 50,
                                        s_max=1000 if n > 100_000 else 100, seed=50 + n % 97), device="cuda")
        graphs[gid] = qm.Graph(g.row_ptr, g.col)
        truths[gid] = (g.labels, g.K)
        pools[gid] = [gen.perturb(g.labels, g.K, 0.05 * (i % 10), seed=60 + i) for i in range(12)]
    return qm, graphs, truths, pools


def test_results_in_the_mix_equal_results_alone(env):
    from paper_1507_05492_gb300.server import Server
    qm, graphs, truths, pools = env
    rng = np.random.default_rng(1)
    reqs = []
    for i in range(300):
        gid = ("small", "mid", "large")[rng.integers(3)]
        lab = pools[gid][rng.integers(len(pools[gid]))]
        with_truth = rng.random() < 0.5
        reqs.append((gid, lab, truths[gid][1], truths[gid][0] if with_truth else None,
                     truths[gid][1] if with_truth else None))
    srv = Server(graphs, budget_bytes=2 << 30, max_batch=64, n_streams=3)
    futs = []
    # arrivals in bursts from two client threads, so batches form while others run
    def client(part):
        for r in part:
            futs.append((r, srv.submit(*r)))
            if rng.random() < 0.1:
                time.sleep(0.002)
    ts = [threading.Thread(target=client, args=(reqs[k::2],)) for k in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    results = [(r, f.result(timeout=120)) for r, f in futs]
    srv.close()
    assert max(srv.batch_sizes) > 1, "no request was ever batched"
    for (gid, lab, K, truth, kt), res in results:
        alone = qm.score(graphs[gid], lab, K)
        assert res["quality"] == alone
        if truth is not None:
            assert res["compare"] == qm.compare(truth, lab, kt, K)


def test_admission_respects_budget(env):
    from paper_1507_05492_gb300.server import Server
    qm, graphs, truths, pools = env
    need = qm.workspace_bytes(graphs["large"], truths["large"][1])
    srv = Server(graphs, budget_bytes=int(need * 1.5), max_batch=64, n_streams=4)
    peak = [0]
    orig = srv._take_batch

    def take(head):
        b, total = orig(head)
        peak[0] = max(peak[0], srv.in_flight + total)
        return b, total
    srv._take_batch = take
    futs = [srv.submit("large", pools["large"][i % 12], truths["large"][1]) for i in range(12)]
    for f in futs:
        f.result(timeout=120)
    srv.close()
    assert peak[0] <= int(need * 1.5)
    # a request larger than the whole budget is refused, not queued forever
    tiny = Server(graphs, budget_bytes=1024, n_streams=1)
    f = tiny.submit("large", pools["large"][0], truths["large"][1])
    with pytest.raises(MemoryError):
        f.result(timeout=5)
    tiny.close()


def test_requests_made_just_before_submission(env):
    """Labels produced by device kernels on the submitter's stream and submitted
    at once (before those kernels finish) are read only when complete."""
    from paper_1507_05492_gb300 import gen
    from paper_1507_05492_gb300.server import Server
    qm, graphs, truths, pools = env
    srv = Server(graphs, budget_bytes=2 << 30, max_batch=64, n_streams=3)
    futs = []
    for i in range(24):
        gid = ("small", "mid", "large")[i % 3]
        labels, K = truths[gid]
        lab = gen.perturb(labels, K, 0.3, seed=500 + i)      # queued on the current stream
        futs.append((gid, lab, K, srv.submit(gid, lab, K)))
    results = [(gid, lab, K, f.result(timeout=120)) for gid, lab, K, f in futs]
    srv.close()
    for gid, lab, K, res in results:
        assert res["quality"] == qm.score(graphs[gid], lab, K)


def test_large_graph_batches_run_one_at_a_time(env):
    """Batches on graphs above exclusive_min_nodes never overlap; smaller
    graphs' requests keep running beside them."""
    from paper_1507_05492_gb300.server import Server
    qm, graphs, truths, pools = env
    srv = Server(graphs, budget_bytes=4 << 30, max_batch=4, n_streams=4, exclusive_min_nodes=100_000)
    running, peak = [0], [0]
    lock = threading.Lock()
    orig = srv._run

    def run(batch, stream):
        big = graphs[batch[0].graph_id].n > 100_000
        if big:
            with lock:
                running[0] += 1
                peak[0] = max(peak[0], running[0])
        try:
            orig(batch, stream)
        finally:
            if big:
                with lock:
                    running[0] -= 1
    srv._run = run
    futs = []
    for i in range(24):
        gid = ("large", "small")[i % 2]
        futs.append((gid, pools[gid][i % 12], srv.submit(gid, pools[gid][i % 12], truths[gid][1])))
    results = [(gid, lab, f.result(timeout=120)) for gid, lab, f in futs]
    srv.close()
    assert peak[0] == 1
    for gid, lab, res in results:
        assert res["quality"] == qm.score(graphs[gid], lab, truths[gid][1])



def test_malformed_requests_are_refused_at_submit(env):
    """A request whose tensors do not fit its graph is refused at once; it never
    joins a batch, where it would fail the launch for the others."""
    from paper_1507_05492_gb300.server import Server
    qm, graphs, truths, pools = env
    srv = Server(graphs, budget_bytes=2 << 30, max_batch=64, n_streams=2)
    lab, K = truths["mid"]
    for bad in (lab[:-1], lab.cpu(), lab.to(torch.int64), lab.view(2, -1)):
        with pytest.raises(ValueError):
            srv.submit("mid", bad, K)
    with pytest.raises(ValueError):
        srv.submit("mid", lab, K, truths["small"][0], truths["small"][1])   # truth of another graph
    with pytest.raises(ValueError):
        srv.submit("mid", lab, K, lab)                                        # truth without k_truth
    good = srv.submit("mid", pools["mid"][0], K)
    assert good.result(timeout=60)["quality"] == qm.score(graphs["mid"], pools["mid"][0], K)
    srv.close()


def test_serving_workload_graphs_against_oracle():
    """Poisson-like arrivals over resident 10k-, 1M- and 10M-node graphs (the
    serving configuration), each request a partition with up to half of the
    nodes moved and half of them with a comparison against the planted
    partition; every served result against the oracle."""
    import __graft_entry__
    __graft_entry__.build()
    from oracle import oracle
    from paper_1507_05492_gb300 import gen, qm
    from paper_1507_05492_gb300.server import Server
    graphs, host, pools = {}, {}, {}
    for gid in ("lfr10k", "lfr1m", "lfr10m"):
        g = gen.lfr_graph(gen.config_params(gid), device="cuda")
        graphs[gid] = qm.Graph(g.row_ptr, g.col, reorder=(g.n >= 1_000_000))
        host[gid] = (g.row_ptr.cpu().numpy(), g.col.cpu().numpy(), g.labels.cpu().numpy(), g.K, g.labels)
        pools[gid] = [gen.perturb(g.labels, g.K, 0.5 * i / 5, seed=700 + i) for i in range(6)]
    rng = np.random.default_rng(11)
    srv = Server(graphs, budget_bytes=8 << 30, max_batch=64, n_streams=3)
    futs = []
    for i in range(90):
        gid = ("lfr10k", "lfr1m", "lfr10m")[rng.integers(3)]
        j = int(rng.integers(len(pools[gid])))
        with_truth = bool(rng.random() < 0.5)
        K = host[gid][3]
        truth = host[gid][4] if with_truth else None
        futs.append((gid, j, with_truth, srv.submit(gid, pools[gid][j], K, truth, K if with_truth else None)))
        time.sleep(float(rng.exponential(1 / 400)))
    served = [(gid, j, wt, f.result(timeout=300)) for gid, j, wt, f in futs]
    srv.close()
    need = sorted({(gid, j) for gid, j, _, _ in served})
    need_c = sorted({(gid, j) for gid, j, wt, _ in served if wt})

    def o_score(key):
        gid, j = key
        rp, col, _, K, _ = host[gid]
        return key, oracle.score(rp, col, pools[gid][j].cpu().numpy(), K)

    def o_cmp(key):
        gid, j = key
        _, _, lab, K, _ = host[gid]
        return key, oracle.compare(lab, pools[gid][j].cpu().numpy(), K, K)

    with ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        os_ = dict(ex.map(o_score, need))
        oc_ = dict(ex.map(o_cmp, need_c))
    for gid, j, wt, res in served:
        check_quality(res["quality"], os_[(gid, j)], f"served {gid} partition {j}")
        if wt:
            check_compare(res["compare"], oc_[(gid, j)], f"served {gid} partition {j} vs planted")
    for gr in graphs.values():
        gr.close()
