"""The seeded workload generator gives the same arrays on the CPU and on the
GPU (its random draws are a counter-based function of seed, stream and index,
and every sort of random keys is stable): graphs, perturbations and batched
candidate partitions."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,seed", [(10_000, 1), (200_000, 17)])
def test_graph_identical_on_cpu_and_gpu(n, seed):
    from paper_1507_05492_gb300 import gen
    p = gen.LfrParams(n=n, k_max=100, s_max=1000, seed=seed)
    a = gen.lfr_graph(p)
    b = gen.lfr_graph(p, device="cuda")
    assert a.K == b.K
    assert torch.equal(a.row_ptr, b.row_ptr.cpu())
    assert torch.equal(a.col, b.col.cpu())
    assert torch.equal(a.labels, b.labels.cpu())


def test_partitions_identical_on_cpu_and_gpu():
    from paper_1507_05492_gb300 import gen
    g = gen.lfr_graph(gen.LfrParams(n=50_000, seed=3))
    lab_c, lab_g = g.labels, g.labels.cuda()
    assert torch.equal(gen.perturb(lab_c, g.K, 0.3, seed=5), gen.perturb(lab_g, g.K, 0.3, seed=5).cpu())
    for k_t in (40, 3 * g.K):
        lc, kc = gen.merge_split(lab_c, k_t, seed=6)
        lg, kg = gen.merge_split(lab_g, k_t, seed=6)
        assert kc == kg and torch.equal(lc, lg.cpu())
