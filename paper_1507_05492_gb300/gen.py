"""Seeded LFR-style synthetic workloads (graphs with planted communities).

This module holds no metric arithmetic: it only makes inputs.  Both the CUDA
path and the CPU oracle are fed the arrays it returns.

The paper measures on LFR benchmark graphs (Sec. IV-C: power-law degrees with
exponent gamma = 2, power-law community sizes with exponent beta = 1, mixing
mu = 0.3) and on detected partitions from SLPA.  Neither the LFR program nor
SLPA is available, so this generator restates the LFR recipe from those
parameters, and perturbed copies of the planted partition stand in for detected
ones:

1. degrees: continuous power law on [x_min, k_max], x_min solved so the mean is
   ``k_mean``, rounded to integers;
2. community sizes: power law with exponent ``beta`` on [s_min, s_max], drawn
   until they cover ``n`` nodes, the remainder spread over the first ones;
3. each degree splits into k_in = round((1 - mu) k) and k_out = k - k_in;
4. nodes, in descending k_in, take uniformly random free slots of communities
   larger than k_in (k_in is capped at size - 1 when none is left);
5. intra stubs are paired at random inside each community, inter stubs at random
   across the graph (configuration model); self-loops, repeated edges and inter
   pairs landing inside one community are dropped;
6. node ids are shuffled by a seeded permutation and a symmetric CSR is built
   (int64 row offsets, int32 column ids, sorted rows).

All random numbers come from a counter-based SplitMix64 hash of
(seed, stream, index), evaluated with int64 tensor ops, so the draws do not
depend on the device or on the order of evaluation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

_M64 = 1 << 64


def _s64(x: int) -> int:
    x %= _M64
    return x - _M64 if x >= (1 << 63) else x


_GOLDEN = _s64(0x9E3779B97F4A7C15)
_MIX1 = _s64(0xBF58476D1CE4E5B9)
_MIX2 = _s64(0x94D049BB133111EB)


def _srl(x: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of an int64 tensor."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def _splitmix64(x: torch.Tensor) -> torch.Tensor:
    z = x + _GOLDEN
    z = (z ^ _srl(z, 30)) * _MIX1
    z = (z ^ _srl(z, 27)) * _MIX2
    return z ^ _srl(z, 31)


def _splitmix64_int(x: int) -> int:
    z = (x + 0x9E3779B97F4A7C15) % _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) % _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) % _M64
    return z ^ (z >> 31)


class Rng:
    """Counter-based generator: value = SplitMix64(base(seed, stream) + index)."""

    def __init__(self, seed: int, device):
        self.seed = int(seed)
        self.device = torch.device(device)

    def bits(self, stream: int, count: int, offset: int = 0) -> torch.Tensor:
        base = _splitmix64_int(_splitmix64_int(self.seed) ^ (int(stream) * 0x632BE59BD9B4E019 % _M64))
        idx = torch.arange(offset, offset + count, dtype=torch.int64, device=self.device)
        return _splitmix64(idx + _s64(base))

    def bits_at(self, stream: int, idx: torch.Tensor) -> torch.Tensor:
        base = _splitmix64_int(_splitmix64_int(self.seed) ^ (int(stream) * 0x632BE59BD9B4E019 % _M64))
        return _splitmix64(idx.to(torch.int64) + _s64(base))

    def uniform(self, stream: int, count: int) -> torch.Tensor:
        return _srl(self.bits(stream, count), 11).to(torch.float64) * (2.0 ** -53)

    def key40(self, stream: int, count: int) -> torch.Tensor:
        return _srl(self.bits(stream, count), 24)


# ------------------------------------------------------------------ power laws

def _powerlaw_mean(a: float, b: float, g: float) -> float:
    if abs(g - 1.0) < 1e-12:
        return (b - a) / math.log(b / a)
    if abs(g - 2.0) < 1e-12:
        return math.log(b / a) / (1.0 / a - 1.0 / b)
    return ((b ** (2 - g) - a ** (2 - g)) / (2 - g)) / ((b ** (1 - g) - a ** (1 - g)) / (1 - g))


def _powerlaw_sample(u: torch.Tensor, a: float, b: float, g: float) -> torch.Tensor:
    """Inverse CDF of p(x) ~ x^-g on [a, b]."""
    if abs(g - 1.0) < 1e-12:
        return a * torch.pow(torch.tensor(b / a, dtype=torch.float64, device=u.device), u)
    e = 1.0 - g
    return torch.pow(a ** e + u * (b ** e - a ** e), 1.0 / e)


def solve_xmin(k_mean: float, k_max: float, gamma: float) -> float:
    lo, hi = 1.0, float(k_max)
    if _powerlaw_mean(lo, k_max, gamma) > k_mean:
        return lo
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if _powerlaw_mean(mid, k_max, gamma) < k_mean:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@dataclass
class LfrParams:
    n: int
    k_mean: float = 20.0
    k_max: int = 50
    gamma: float = 2.0
    s_min: int = 20
    s_max: int = 100
    beta: float = 1.0
    mu: float = 0.3
    seed: int = 1
    permute: bool = True


@dataclass
class Graph:
    row_ptr: torch.Tensor  # int64 [n + 1]
    col: torch.Tensor      # int32 [2 |E|]
    labels: torch.Tensor   # int32 [n], planted partition
    K: int                 # number of planted communities
    stats: dict

    @property
    def n(self) -> int:
        return self.row_ptr.numel() - 1

    @property
    def n_edges(self) -> int:
        return self.col.numel() // 2


def _community_sizes(p: LfrParams, rng: Rng, dev) -> torch.Tensor:
    n = p.n
    if n <= p.s_min:
        return torch.tensor([n], dtype=torch.int64, device=dev)
    mean_s = _powerlaw_mean(p.s_min, p.s_max, p.beta)
    m = int(math.ceil(n / mean_s * 1.3)) + 16
    off = 0
    chunks = []
    total = 0
    while total < n:
        u = rng.uniform(2, m) if off == 0 else _srl(rng.bits(2, m, off), 11).to(torch.float64) * 2.0 ** -53
        s = torch.round(_powerlaw_sample(u, p.s_min, p.s_max, p.beta)).to(torch.int64)
        s = s.clamp_(p.s_min, p.s_max)
        chunks.append(s)
        total += int(s.sum())
        off += m
    sizes = torch.cat(chunks)
    cs = torch.cumsum(sizes, 0)
    last = int(torch.searchsorted(cs, torch.tensor([n], device=dev)).item())  # first cs >= n
    sizes = sizes[: last + 1].clone()
    prev = int(cs[last - 1]) if last > 0 else 0
    rem = n - prev
    if rem >= p.s_min or last == 0:
        sizes[last] = rem
    else:
        sizes = sizes[:last].clone()
        k = sizes.numel()
        add = torch.full((k,), rem // k, dtype=torch.int64, device=dev)
        add[: rem % k] += 1
        sizes += add
    return sizes


def lfr_graph(p: LfrParams, device="cpu") -> Graph:
    """Build one seeded LFR-style graph with its planted partition."""
    dev = torch.device(device)
    rng = Rng(p.seed, dev)
    n = p.n

    # 1. degrees
    xmin = solve_xmin(p.k_mean, p.k_max, p.gamma)
    deg = torch.round(_powerlaw_sample(rng.uniform(1, n), xmin, float(p.k_max), p.gamma)).to(torch.int64)
    deg.clamp_(1, p.k_max)

    # 2. community sizes
    sizes = _community_sizes(p, rng, dev)
    K = sizes.numel()

    # 3. internal / external split
    k_in = torch.round((1.0 - p.mu) * deg.to(torch.float64)).to(torch.int64)
    k_in = torch.minimum(k_in, deg)

    # 4. assignment of nodes to community slots, largest k_in first
    slot_comm = torch.repeat_interleave(torch.arange(K, device=dev), sizes)
    slot_size = sizes[slot_comm]
    free = torch.ones(n, dtype=torch.bool, device=dev)
    node_comm = torch.full((n,), -1, dtype=torch.int64, device=dev)
    order = torch.argsort(((p.k_max - k_in) << 40) | rng.key40(3, n), stable=True)
    kin_sorted = k_in[order]
    s_small = int(sizes.min())
    values, counts = torch.unique_consecutive(kin_sorted, return_counts=True)
    start = 0
    pending = []
    for t, c in zip(values.tolist(), counts.tolist()):
        seg = order[start:start + c]
        start += c
        if t < s_small:
            pending.append(seg)
            continue
        cand = torch.nonzero(free & (slot_size > t)).flatten()
        take = min(c, cand.numel())
        if take > 0:
            pick = cand[torch.argsort(rng.bits_at(4 + t, cand), stable=True)[:take]]
            node_comm[seg[:take]] = slot_comm[pick]
            free[pick] = False
        if take < c:
            pending.append(seg[take:])
    if pending:
        rest = torch.cat(pending)
        cand = torch.nonzero(free).flatten()
        pick = cand[torch.argsort(rng.bits_at(200, cand), stable=True)]
        node_comm[rest] = slot_comm[pick[: rest.numel()]]
    cap = sizes[node_comm] - 1
    excess = (k_in - cap).clamp_(min=0)
    k_in -= excess
    k_out = deg - k_in

    # 5a. intra stubs, paired at random inside each community
    nodes = torch.arange(n, device=dev)
    s_node = torch.repeat_interleave(nodes, k_in)
    s_comm = node_comm[s_node]
    perm = torch.argsort((s_comm << 40) | rng.key40(5, s_node.numel()), stable=True)
    s_node = s_node[perm]
    s_comm = s_comm[perm]
    del perm
    seg_len = torch.bincount(s_comm, minlength=K)
    seg_start = torch.cumsum(seg_len, 0) - seg_len
    pos = torch.arange(s_node.numel(), device=dev) - seg_start[s_comm]
    first = torch.nonzero(((pos & 1) == 0) & (pos + 1 < seg_len[s_comm])).flatten()
    eu = s_node[first]
    ev = s_node[first + 1]
    del s_node, s_comm, pos, first

    # 5b. inter stubs, paired at random across the graph
    o_node = torch.repeat_interleave(nodes, k_out)
    o_node = o_node[torch.argsort(rng.key40(6, o_node.numel()), stable=True)]
    half = o_node.numel() // 2
    ou = o_node[0:2 * half:2]
    ov = o_node[1:2 * half:2]
    keep = node_comm[ou] != node_comm[ov]
    ou, ov = ou[keep], ov[keep]
    del o_node, keep

    u = torch.cat([eu, ou])
    v = torch.cat([ev, ov])
    del eu, ev, ou, ov
    keep = u != v
    u, v = u[keep], v[keep]
    lo = torch.minimum(u, v)
    hi = torch.maximum(u, v)
    del u, v, keep
    ekey = torch.unique(lo * n + hi)
    del lo, hi

    # 6. seeded node permutation and symmetric CSR
    if p.permute:
        new_id = torch.empty(n, dtype=torch.int64, device=dev)
        new_id[torch.argsort(rng.key40(7, n), stable=True)] = nodes
    else:
        new_id = nodes
    a = new_id[ekey // n]
    b = new_id[ekey % n]
    m = ekey.numel()
    del ekey
    src = torch.cat([a, b])
    dst = torch.cat([b, a])
    del a, b
    akey = torch.sort(src * n + dst).values
    del src, dst
    src = akey // n
    col = (akey % n).to(torch.int32)
    del akey
    counts_row = torch.bincount(src, minlength=n)
    del src
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    row_ptr[1:] = torch.cumsum(counts_row, 0)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    labels[new_id] = node_comm.to(torch.int32)

    stats = dict(n=n, n_edges=m, K=K, x_min=xmin, mean_degree=2.0 * m / n,
                 max_degree=int(counts_row.max()) if n else 0)
    return Graph(row_ptr=row_ptr, col=col, labels=labels, K=K, stats=stats)


def mixing_fraction(g: Graph) -> float:
    """Achieved mu: the fraction of arcs whose endpoints have different planted labels."""
    src = torch.repeat_interleave(torch.arange(g.n, device=g.col.device), g.row_ptr[1:] - g.row_ptr[:-1])
    lab = g.labels.to(torch.int64)
    return float((lab[src] != lab[g.col.to(torch.int64)]).double().mean())


# ------------------------------------------------------------------ partitions

def compact(labels: torch.Tensor) -> tuple[torch.Tensor, int]:
    """Relabel to ids 0..K-1 in order of first appearance of each sorted id."""
    uniq, inv = torch.unique(labels, return_inverse=True)
    return inv.to(torch.int32), int(uniq.numel())


def perturb(labels: torch.Tensor, K: int, frac: float, seed: int, stream: int = 101) -> torch.Tensor:
    """Move floor(frac * n) nodes, chosen without replacement, each to a uniformly
    random other community among 0..K-1 (K >= 2)."""
    n = labels.numel()
    rng = Rng(seed, labels.device)
    m = int(math.floor(frac * n))
    out = labels.clone()
    if m == 0 or K < 2:
        return out
    chosen = torch.argsort(rng.key40(stream, n), stable=True)[:m]
    shift = 1 + (rng.uniform(stream + 1, m) * (K - 1)).to(torch.int64).clamp_(max=K - 2)
    out[chosen] = ((labels[chosen].to(torch.int64) + shift) % K).to(torch.int32)
    return out


def merge_split(labels: torch.Tensor, k_target: int, seed: int, stream: int = 300) -> tuple[torch.Tensor, int]:
    """Merge random pairs of communities (K > k_target) or split random communities
    into two random halves (K < k_target) until there are k_target communities."""
    lab, K = compact(labels.to(torch.int64))
    lab = lab.to(torch.int64)
    rng = Rng(seed, labels.device)
    dev = labels.device
    rnd = 0
    while K != k_target:
        rnd += 1
        if K > k_target:
            d = min(K - k_target, K // 2)
            order = torch.argsort(rng.key40(stream + 2 * rnd, K), stable=True)
            target = torch.arange(K, device=dev)
            target[order[1:2 * d:2]] = order[0:2 * d:2]
            lab, K = compact(target[lab])
            lab = lab.to(torch.int64)
        else:
            sizes = torch.bincount(lab, minlength=K)
            splittable = torch.nonzero(sizes >= 2).flatten()
            if splittable.numel() == 0:
                break
            d = min(k_target - K, splittable.numel())
            pick = splittable[torch.argsort(rng.bits_at(stream + 2 * rnd, splittable), stable=True)[:d]]
            new_id = torch.full((K,), -1, dtype=torch.int64, device=dev)
            new_id[pick] = K + torch.arange(d, device=dev)
            n = lab.numel()
            key = (lab << 40) | rng.key40(stream + 2 * rnd + 1, n)
            order = torch.argsort(key, stable=True)
            sl = lab[order]
            seg_start = torch.cumsum(sizes, 0) - sizes
            pos = torch.arange(n, device=dev) - seg_start[sl]
            move = (new_id[sl] >= 0) & (pos >= sizes[sl] // 2)
            moved_nodes = order[move]
            lab[moved_nodes] = new_id[lab[moved_nodes]]
            K += d
    return lab.to(torch.int32), K


def candidate_partition(planted: torch.Tensor, seed: int, k_range=(500, 5000), frac_max=0.5):
    """A candidate partition: planted labels, merged/split to a random community
    count in ``k_range``, then a random fraction in [0, frac_max] of nodes moved."""
    rng = Rng(seed, "cpu")
    u = rng.uniform(1, 2).tolist()
    k_t = k_range[0] + int(u[0] * (k_range[1] - k_range[0] + 1))
    k_t = min(k_t, k_range[1], planted.numel())
    f = u[1] * frac_max
    lab, K = merge_split(planted, k_t, seed)
    lab = perturb(lab, K, f, seed, stream=401)
    lab, K = compact(lab)
    return lab, K, f


# named workloads ----------------------------------------------------------

def config_params(name: str, seed: int | None = None) -> LfrParams:
    """Parameters of the named synthetic workloads (LFR recipe of Sec. IV-C with
    mean degree 20)."""
    table = {
        "lfr10k": LfrParams(n=10_000, k_mean=20, k_max=50, s_min=20, s_max=100, mu=0.3, seed=1),
        "lfr10m": LfrParams(n=10_000_000, k_mean=20, k_max=100, s_min=20, s_max=1000, mu=0.3, seed=2),
        "lfr100m": LfrParams(n=100_000_000, k_mean=20, k_max=100, s_min=20, s_max=1000, mu=0.3, seed=3),
        "lfr100k_mu01": LfrParams(n=100_000, k_mean=20, k_max=50, s_min=20, s_max=100, mu=0.1, seed=4),
        "lfr100k_mu03": LfrParams(n=100_000, k_mean=20, k_max=50, s_min=20, s_max=100, mu=0.3, seed=5),
        "lfr100k_mu05": LfrParams(n=100_000, k_mean=20, k_max=50, s_min=20, s_max=100, mu=0.5, seed=6),
        "lfr1m": LfrParams(n=1_000_000, k_mean=20, k_max=100, s_min=20, s_max=1000, mu=0.3, seed=8),
        # the 100M-node recipe at 32M nodes: its label array (128 MB) is about
        # the L2's size, so profiler captures of a few GB still see DRAM behaviour
        "lfr32m": LfrParams(n=32_000_000, k_mean=20, k_max=100, s_min=20, s_max=1000, mu=0.3, seed=10),
    }
    p = table[name]
    if seed is not None:
        p.seed = seed
    return p


def candidate_batch(planted: torch.Tensor, P: int, seed: int, k_range=(500, 5000), frac_max=0.5):
    """P candidate partitions (see candidate_partition) as a [P, n] int32 matrix on
    the planted labels' device, with their label-id counts."""
    rows, Ks = [], []
    for p in range(P):
        lab, K, _ = candidate_partition(planted, seed + p, k_range=k_range, frac_max=frac_max)
        rows.append(lab)
        Ks.append(K)
    return torch.stack(rows), Ks
