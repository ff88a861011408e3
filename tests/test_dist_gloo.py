"""Multi-process host logic (world size 2, gloo, CPU): sharding of independent
units by id mod ranks, gathering in unit order, max/sum reductions of timings,
and detection of a unit scored twice or never."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world_size, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    try:
        from paper_1507_05492_gb300 import dist as qd
        out = {}
        ws, r = qd.world()
        out["world"] = (ws, r)
        out["share"] = qd.shard(11, ws, r)
        res = qd.score_sharded(lambda i: {"unit": i, "value": i * i, "rank": r}, 11)
        out["gathered"] = res
        out["max"] = qd.reduce_scalar(1.5 + r, "max")
        out["sum"] = qd.reduce_scalar(10.0 * (r + 1), "sum")
        qd.barrier()
        # a unit claimed by both ranks must be reported
        try:
            qd.gather_sharded({0: "dup"}, 1)
            out["dup_detected"] = False
        except RuntimeError:
            out["dup_detected"] = True
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_gather_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    outs = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert outs[0]["world"] == (2, 0) and outs[1]["world"] == (2, 1)
    assert outs[0]["share"] == [0, 2, 4, 6, 8, 10] and outs[1]["share"] == [1, 3, 5, 7, 9]
    g = outs[0]["gathered"]
    assert [x["unit"] for x in g] == list(range(11)) and all(x["value"] == x["unit"] ** 2 for x in g)
    assert {x["rank"] for x in g} == {0, 1}
    assert outs[1]["gathered"] is None
    assert outs[0]["max"] == outs[1]["max"] == 2.5
    assert outs[0]["sum"] == outs[1]["sum"] == 30.0
    assert outs[0]["dup_detected"]


def test_single_process_fallback():
    from paper_1507_05492_gb300 import dist as qd
    assert qd.world() == (1, 0)
    assert qd.shard(5, 1, 0) == [0, 1, 2, 3, 4]
    assert qd.score_sharded(lambda i: i + 1, 3) == [1, 2, 3]
    assert qd.reduce_scalar(3.0) == 3.0
