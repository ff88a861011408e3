"""Host-side checks of sharded scoring (no GPU): the exact combination of
shard partials (qm_partials_combine) against Python integers, its error
cases, the coverage check of qm_partial_finalize, and the exchange of
partials between two gloo ranks (score_partition_sharded with stand-in shard
and finalise steps)."""
import os
import random
import socket

import pytest
import torch.multiprocessing as mp

TRIPLE_AT, U64_FIRST, U64_COUNT = [0, 3, 6, 9, 12, 15, 18, 26], 21, 5
TRIPLES = len(TRIPLE_AT)
MASK43 = (1 << 43) - 1


@pytest.fixture(scope="module")
def qm():
    from paper_1507_05492_gb300 import build
    build.build()
    from paper_1507_05492_gb300 import qm as q
    return q


def put_value(words, k, v, rng):
    """Stores v as limbs L2 * 2^86 + L1 * 2^43 + L0 (L2 signed), with L0 and L1
    left unnormalised the way repeated 43-bit atomic additions leave them."""
    l2 = v >> 86
    rem = v - (l2 << 86)
    l1, l0 = rem >> 43, rem & MASK43
    carry = rng.randrange(0, min(l1, 1 << 20) + 1)
    l1, l0 = l1 - carry, l0 + (carry << 43)
    t = TRIPLE_AT[k]
    words[t], words[t + 1], words[t + 2] = l0, l1, l2 & ((1 << 64) - 1)


def get_value(words, k):
    t = TRIPLE_AT[k]
    l0, l1, l2 = words[t], words[t + 1], words[t + 2]
    if l2 >= 1 << 63:
        l2 -= 1 << 64
    return (l2 << 86) + (l1 << 43) + l0


def make_partial(qm, rng, rank, nranks, n=1000, e=5000):
    p = qm.QmPartial()
    p.n_nodes, p.n_edges, p.nranks, p.ranks_mask = n, e, nranks, 1 << rank
    vals = [rng.randrange(-(1 << 118), 1 << 118) for _ in range(TRIPLES)]
    cnts = [rng.randrange(0, 1 << 58) for _ in range(U64_COUNT)]
    w = [0] * qm.PARTIAL_WORDS
    for k, v in enumerate(vals):
        put_value(w, k, v, rng)
    for k, c in enumerate(cnts):
        w[U64_FIRST + k] = c
    for i, x in enumerate(w):
        p.words[i] = x
    return p, vals, cnts


@pytest.mark.parametrize("nranks", [1, 2, 5, 64])
def test_combine_is_exact(qm, nranks):
    rng = random.Random(nranks)
    parts = [make_partial(qm, rng, r, nranks) for r in range(nranks)]
    tot = qm.combine_parts([p for p, _, _ in parts])
    assert tot.ranks_mask == (1 << nranks) - 1 if nranks < 64 else (1 << 64) - 1
    assert tot.n_nodes == 1000 and tot.n_edges == 5000 and tot.nranks == nranks
    w = list(tot.words)
    for k in range(TRIPLES):
        assert get_value(w, k) == sum(v[k] for _, v, _ in parts)
        t = TRIPLE_AT[k]
        assert w[t] <= MASK43 and w[t + 1] <= MASK43    # normalised again
    for k in range(U64_COUNT):
        assert w[U64_FIRST + k] == sum(c[k] for _, _, c in parts)
    # any grouping gives the same words
    if nranks >= 2:
        a = qm.combine_parts([p for p, _, _ in parts[: nranks // 2]])
        b = qm.combine_parts([p for p, _, _ in parts[nranks // 2:]])
        assert list(qm.combine_parts([b, a]).words) == w


def test_combine_rejects_mismatches(qm):
    rng = random.Random(3)
    a, _, _ = make_partial(qm, rng, 0, 2)
    b, _, _ = make_partial(qm, rng, 1, 2)
    c, _, _ = make_partial(qm, rng, 0, 2)
    with pytest.raises(RuntimeError):
        qm.combine_parts([a, c])                       # shard 0 twice
    d, _, _ = make_partial(qm, rng, 1, 2, n=999)
    with pytest.raises(RuntimeError):
        qm.combine_parts([a, d])                       # another graph
    e, _, _ = make_partial(qm, rng, 1, 3)
    with pytest.raises(RuntimeError):
        qm.combine_parts([a, e])                       # another shard count
    with pytest.raises(RuntimeError):
        qm.combine_parts([])
    assert qm.combine_parts([a, b]).ranks_mask == 3


def test_finalize_needs_every_shard(qm):
    # rejected before any device work, so this runs without a GPU
    rng = random.Random(4)
    a, _, _ = make_partial(qm, rng, 0, 3)
    b, _, _ = make_partial(qm, rng, 2, 3)
    with pytest.raises(RuntimeError):
        qm.finalize_part(qm.combine_parts([a, b]))


def test_transport_round_trip(qm):
    rng = random.Random(5)
    a, _, _ = make_partial(qm, rng, 63, 64)
    b = qm.part_from_array(qm.part_to_array(a))
    assert (b.n_nodes, b.n_edges, b.nranks, b.ranks_mask) == (a.n_nodes, a.n_edges, a.nranks, a.ranks_mask)
    assert list(b.words) == list(a.words)


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
        from paper_1507_05492_gb300 import qm

        def part_fn(graph, labels, K, r, ws):
            p, _, _ = make_partial(qm, random.Random(100 + r), r, ws)
            return p

        got = qd.score_partition_sharded(None, None, 0, part_fn=part_fn, finalize_fn=lambda p: p)
        q.put((rank, (got.ranks_mask, got.nranks, list(got.words))))
    finally:
        dist.destroy_process_group()


def test_two_ranks_exchange_partials(qm):
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
    assert outs[0] == outs[1]
    mask, nranks, words = outs[0]
    assert mask == 3 and nranks == 2
    parts = [make_partial(qm, random.Random(100 + r), r, 2) for r in range(2)]
    for k in range(TRIPLES):
        assert get_value(words, k) == sum(v[k] for _, v, _ in parts)
    for k in range(U64_COUNT):
        assert words[U64_FIRST + k] == sum(c[k] for _, _, c in parts)
