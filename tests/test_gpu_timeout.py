"""The bounded device wait of the pair-count kernel (QM_ETIMEOUT).

The kernel stages each long run of packed labels into shared memory with an
asynchronous bulk copy and waits on an mbarrier for a bounded number of polls.
A test hook sets that bound to zero polls, so every such wait expires at its
first check although no copy is withheld: nothing faults or hangs.  The call
must return QM_ETIMEOUT, and with the default bound restored the next call on
the same context must return the oracle's result."""
import pytest

from helpers import check_quality

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1507_05492_gb300 import qm as q
    return q


def test_expired_staging_wait_returns_timeout_and_context_survives(qm, oracle_mod):
    from paper_1507_05492_gb300 import gen
    # communities of up to 1,000 nodes: many runs long enough for the staged block path
    g = gen.lfr_graph(gen.LfrParams(n=300_000, k_max=100, s_min=20, s_max=1000, mu=0.3, seed=91), device="cuda")
    o = oracle_mod.score(g.row_ptr.cpu().numpy(), g.col.cpu().numpy(), g.labels.cpu().numpy(), g.K)
    for reorder in (False, True):
        graph = qm.Graph(g.row_ptr, g.col, reorder=reorder)
        assert qm.get_tuning(graph, g.K)["algorithm"] == 1   # the two-phase pipeline, which stages copies
        check_quality(qm.score(graph, g.labels, g.K), o, "before")
        try:
            qm.debug_set_stage_wait(0)
            for per_community in (False, True):        # replayed and direct launches
                with pytest.raises(qm.QmError) as e:
                    qm.score(graph, g.labels, g.K, per_community=per_community)
                assert e.value.status == qm.QM_ETIMEOUT, e.value
        finally:
            qm.debug_set_stage_wait(-1)
        check_quality(qm.score(graph, g.labels, g.K), o, f"after a timeout, reorder={reorder}")
        q = qm.score(graph, g.labels, g.K, per_community=True)
        check_quality(q, o, "after, per-community output")
        graph.close()
