"""Host-side helpers for running the scorer on several processes (one GPU each).

The work units of the path are independent (partitions of a resident graph,
or separate graphs), so ranks need no exchange on the data path: each rank
takes its share of the units, and only timings and results are combined at
the end.  The share follows the paper's decomposition of Sec. III-A, unit id
modulo the number of processes.

Works with any torch.distributed backend: NCCL tensors live on the rank's GPU,
gloo tensors on the CPU.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def world() -> tuple[int, int]:
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(), dist.get_rank()
    return 1, 0


def _device():
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def shard(units: int, world_size: int, rank: int) -> list[int]:
    """Unit ids owned by `rank`: id mod world_size == rank (Sec. III-A)."""
    return list(range(rank, units, world_size))


def reduce_scalar(x: float, op: str = "max") -> float:
    ws, _ = world()
    if ws == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op={"max": dist.ReduceOp.MAX, "sum": dist.ReduceOp.SUM,
                           "min": dist.ReduceOp.MIN}[op])
    return float(t.item())


def barrier():
    ws, _ = world()
    if ws == 1:
        return
    if dist.get_backend() == "nccl":
        dist.barrier(device_ids=[torch.cuda.current_device()])
    else:
        dist.barrier()


def gather_sharded(local: dict[int, object], units: int) -> list | None:
    """Collects {unit id: result} from every rank; rank 0 receives the list in
    unit order (None elsewhere).  Every unit must be owned by exactly one rank."""
    ws, rank = world()
    if ws == 1:
        return [local[i] for i in range(units)]
    parts = [None] * ws if rank == 0 else None
    dist.gather_object(local, parts, dst=0)
    if rank != 0:
        return None
    merged = {}
    for p in parts:
        for k, v in p.items():
            if k in merged:
                raise RuntimeError(f"unit {k} scored by two ranks")
            merged[k] = v
    missing = [i for i in range(units) if i not in merged]
    if missing:
        raise RuntimeError(f"units {missing[:5]} were scored by no rank")
    return [merged[i] for i in range(units)]


def score_sharded(score_unit, units: int) -> list | None:
    """Runs score_unit(i) for this rank's share of `units` and gathers all
    results on rank 0 in unit order."""
    ws, rank = world()
    local = {i: score_unit(i) for i in shard(units, ws, rank)}
    return gather_sharded(local, units)


def score_partition_sharded(graph, labels, K: int, stream=None, part_fn=None, finalize_fn=None):
    """One scoring call split over the ranks by community ownership, the
    paper's own decomposition (Sec. III-A): rank r scores the communities
    c with c mod world_size == r, the ranks exchange their exact partial sums
    (one all-gather of 36 int64 words each, the single reduction of the
    paper's processes), and every rank finalises the same total.  Every rank
    holds the whole graph and all labels.  Bit-identical to qm.score.

    part_fn(graph, labels, K, rank, world_size) and finalize_fn(partial) default
    to the library calls; tests pass stand-ins to run the exchange on CPU."""
    from . import qm
    ws, rank = world()
    if part_fn is None:
        part = qm.score_part(graph, labels, K, rank, ws, stream=stream)
    else:
        part = part_fn(graph, labels, K, rank, ws)
    if ws > 1:
        a = torch.from_numpy(qm.part_to_array(part)).to(_device())
        bufs = [torch.empty_like(a) for _ in range(ws)]
        dist.all_gather(bufs, a)
        part = qm.combine_parts([qm.part_from_array(b.cpu().numpy()) for b in bufs])
    return (finalize_fn or (lambda p: qm.finalize_part(p, stream)))(part)

