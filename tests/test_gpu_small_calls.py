"""Calls on small graphs replay a captured CUDA graph of their launches.  The
replayed calls must give the bits of the direct path (taken when tracing is
on), read each call's own labels (host or device), follow changes of K and
launch shape, and drop nothing stale when graphs are freed and loaded again."""
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
def lfr():
    from paper_1507_05492_gb300 import gen
    return gen.lfr_graph(gen.config_params("lfr10k"))


def direct(qm, graph, labels, K):
    qm.trace_enable(True)
    try:
        return qm.score(graph, labels, K)
    finally:
        qm.trace_enable(False)


@pytest.mark.parametrize("reorder", [False, True])
def test_replays_match_the_direct_path(qm, oracle_mod, lfr, reorder):
    from paper_1507_05492_gb300 import gen
    g = lfr
    graph = qm.Graph(*to_dev(g.row_ptr, g.col), reorder=reorder)
    rng = np.random.default_rng(3)
    for trial in range(6):                          # new labels every call, same K
        lab = gen.perturb(g.labels, g.K, 0.05 * trial, seed=trial)
        a = qm.score(graph, lab.cuda(), g.K)
        b = direct(qm, graph, lab.cuda(), g.K)
        assert a == b, trial
        assert qm.score(graph, lab.numpy(), g.K) == a, trial
        if trial % 2 == 0:
            o = oracle_mod.score(g.row_ptr.numpy(), g.col.numpy(), lab.numpy(), g.K)
            check_quality(a, o, f"replayed call {trial}")
    for K in (1, 7, 300):                           # other label counts
        lab = torch.from_numpy(rng.integers(0, K, g.n).astype(np.int32))
        assert qm.score(graph, lab.cuda(), K) == direct(qm, graph, lab.cuda(), K)
    for algo in (0, 1):                             # other launch shapes
        qm.set_tuning(graph, g.K, 256, 48 * 1024, 24, algo)
        assert qm.score(graph, g.labels.cuda(), g.K) == direct(qm, graph, g.labels.cuda(), g.K)


def test_bad_labels_still_reported(qm, lfr):
    graph = qm.Graph(*to_dev(lfr.row_ptr, lfr.col))
    bad = lfr.labels.clone()
    bad[17] = -1
    for _ in range(2):
        with pytest.raises(RuntimeError):
            qm.score(graph, bad.cuda(), lfr.K)
    assert qm.score(graph, lfr.labels.cuda(), lfr.K) == direct(qm, graph, lfr.labels.cuda(), lfr.K)


def test_free_and_reload(qm, lfr):
    """A graph loaded after another was freed (its handle may reuse the freed
    one's address) must not replay the freed graph's captured calls."""
    from paper_1507_05492_gb300 import gen
    other = gen.lfr_graph(gen.LfrParams(n=lfr.n, k_max=50, s_min=20, s_max=100, seed=77))
    K = max(lfr.K, other.K)
    ref_a = ref_b = None
    for _ in range(3):
        a = qm.Graph(*to_dev(lfr.row_ptr, lfr.col))
        qa = qm.score(a, lfr.labels.cuda(), K)
        a.close()
        b = qm.Graph(*to_dev(other.row_ptr, other.col))
        qb = qm.score(b, lfr.labels.cuda(), K)
        assert qb == direct(qm, b, lfr.labels.cuda(), K)
        b.close()
        ref_a, ref_b = ref_a or qa, ref_b or qb
        assert qa == ref_a and qb == ref_b
    assert ref_a != ref_b


def test_sharded_replays(qm, lfr):
    graph = qm.Graph(*to_dev(lfr.row_ptr, lfr.col))
    lab = lfr.labels.cuda()
    ref = qm.score(graph, lab, lfr.K)
    for _ in range(2):
        parts = [qm.score_part(graph, lab, lfr.K, r, 3) for r in range(3)]
        assert qm.finalize_part(qm.combine_parts(parts)) == ref


def test_concurrent_threads(qm, lfr):
    """Calls from several host threads at once (each on its own stream) take
    their own scratch and capture streams and give the serial results."""
    import threading
    from paper_1507_05492_gb300 import gen
    graph = qm.Graph(*to_dev(lfr.row_ptr, lfr.col))
    labs = [gen.perturb(lfr.labels, lfr.K, 0.04 * i, seed=40 + i).cuda() for i in range(8)]
    ref = [direct(qm, graph, lab, lfr.K) for lab in labs]
    errors = []

    def worker(t):
        st = torch.cuda.Stream()
        try:
            for r in range(12):
                i = (t + r) % len(labs)
                with torch.cuda.stream(st):
                    got = qm.score(graph, labs[i], lfr.K, stream=st)
                if got != ref[i]:
                    errors.append((t, r, i))
        except Exception as e:  # reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors[:3]
