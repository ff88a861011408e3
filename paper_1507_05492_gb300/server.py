"""Serving loop: resident graphs, scoring requests admitted by a device-memory
budget and batched as they arrive (continuous batching).

Requests carry a partition of one of the resident graphs and optionally a
ground truth to compare with.  Worker threads, one CUDA stream each, repeatedly
take the oldest pending request's graph and as many pending requests of that
graph as the batch limit and the free memory budget allow, and run them as one
batched launch (small graphs: one persistent kernel for the whole batch) or as
consecutive plain calls (large graphs, where one call already fills the GPU).
Requests that arrive while launches are in flight join the next batch a free
worker forms, so their work overlaps on the device.  Results are bit-identical
to scoring each request alone (the library's sums are order-independent).
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import threading
import time

import numpy as np
import torch

from . import qm


class Request:
    __slots__ = ("graph_id", "labels", "K", "truth", "k_truth", "future", "t_arrival", "t_done", "bytes", "ready")

    def __init__(self, graph_id, labels, K, truth, k_truth, nbytes):
        self.graph_id = graph_id
        self.labels = labels
        self.K = int(K)
        self.truth = truth
        self.k_truth = None if k_truth is None else int(k_truth)
        self.future = cf.Future()
        self.t_arrival = time.perf_counter()
        self.t_done = None
        self.bytes = nbytes
        self.ready = None  # event on the submitter's stream after which the tensors are complete


class Server:
    """graphs: {graph_id: qm.Graph}.  budget_bytes bounds the scratch memory of
    the launches in flight.  Graphs with at most `batch_max_nodes` nodes are
    scored by the batched persistent kernel, larger ones call by call.  Work on
    graphs of more than `exclusive_min_nodes` nodes (one call fills the GPU)
    runs one batch at a time, so that such requests do not slow each other
    down; requests on smaller graphs keep running beside it."""

    def __init__(self, graphs: dict, budget_bytes: int, max_batch: int = 512, n_streams: int = 4,
                 batch_max_nodes: int = 300_000, exclusive_min_nodes: int = 2_000_000, device=None):
        self.graphs = graphs
        self.budget = int(budget_bytes)
        self.max_batch = max_batch
        self.batch_max_nodes = batch_max_nodes
        self.exclusive_min_nodes = exclusive_min_nodes
        self.exclusive_busy = False
        dev = torch.device(device if device is not None else "cuda")
        self.device = dev if dev.index is not None else torch.device("cuda", torch.cuda.current_device())
        self.pending = collections.deque()
        self.cv = threading.Condition()
        self.in_flight = 0
        self.closed = False
        self.launches = 0
        self.batch_sizes = []
        self.workers = []
        # each worker has a stream of normal priority and one of high priority;
        # batches on the largest graphs take the high one, so that the small
        # graphs' work running beside them does not stretch the latency tail
        for i in range(n_streams):
            streams = (torch.cuda.Stream(device=self.device, priority=0),
                       torch.cuda.Stream(device=self.device, priority=-1))
            t = threading.Thread(target=self._worker, args=streams, daemon=True, name=f"qm-server-{i}")
            t.start()
            self.workers.append(t)

    # ---------------------------------------------------------------- client side

    def request_bytes(self, graph_id, K, k_truth=None) -> int:
        g = self.graphs[graph_id]
        return qm.workspace_bytes(g, K, k_truth)

    def submit(self, graph_id, labels: torch.Tensor, K: int, truth: torch.Tensor | None = None,
               k_truth: int | None = None) -> cf.Future:
        # a malformed request is refused here: inside a batch it would fail the
        # launch for every request batched with it
        n = self.graphs[graph_id].n
        for name, t in (("labels", labels), ("truth", truth)):
            if t is not None and (not isinstance(t, torch.Tensor) or t.dtype != torch.int32 or
                                  tuple(t.shape) != (n,) or not t.is_contiguous() or t.device != self.device):
                raise ValueError(f"{name} must be a contiguous int32 tensor of shape ({n},) on {self.device}")
        if truth is not None and k_truth is None:
            raise ValueError("a ground truth needs its label count k_truth")
        nbytes = self.request_bytes(graph_id, K, k_truth if truth is not None else None)
        if nbytes > self.budget:
            f = cf.Future()
            f.set_exception(MemoryError(f"request needs {nbytes} bytes, budget is {self.budget}"))
            return f
        r = Request(graph_id, labels, K, truth, k_truth, nbytes)
        r.future.request = r  # latency bookkeeping: arrival and completion times
        # the request's tensors may still be in the making on the submitter's
        # stream: the worker's stream waits for this point before reading them
        r.ready = torch.cuda.Event()
        r.ready.record(torch.cuda.current_stream(self.device))
        with self.cv:
            if self.closed:
                raise RuntimeError("server closed")
            self.pending.append(r)
            self.cv.notify()
        return r.future

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        for t in self.workers:
            t.join()

    # ---------------------------------------------------------------- worker side

    def _exclusive(self, gid) -> bool:
        return self.graphs[gid].n > self.exclusive_min_nodes

    def _head(self):
        """The oldest pending request that may start now (None if none): its graph
        is not one whose work runs one batch at a time while such a batch runs."""
        for r in self.pending:
            if not (self.exclusive_busy and self._exclusive(r.graph_id)):
                return r
        return None

    def _take_batch(self, head):
        """The head request's graph; then every pending request of that graph
        (FIFO) while the batch limit and the memory budget allow."""
        gid = head.graph_id
        batch, total = [], 0
        rest = collections.deque()
        while self.pending and len(batch) < self.max_batch:
            r = self.pending.popleft()
            if r.graph_id == gid and self.in_flight + total + r.bytes <= self.budget:
                batch.append(r)
                total += r.bytes
            else:
                rest.append(r)
                if r.graph_id == gid:
                    break  # budget exhausted: later requests of this graph wait too
        rest.extend(self.pending)
        self.pending = rest
        return batch, total

    def _ready(self):
        head = self._head() if self.pending else None
        return head if head is not None and self.in_flight + head.bytes <= self.budget else None

    def _worker(self, stream, stream_hi):
        torch.cuda.set_device(self.device)
        while True:
            with self.cv:
                while not self.closed and self._ready() is None:
                    self.cv.wait(timeout=0.05)
                head = self._ready()
                if head is None:
                    if self.closed and not self.pending:
                        return
                    self.cv.wait(timeout=0.05)  # closing: wait for the batches in flight
                    continue
                batch, total = self._take_batch(head)
                if not batch:
                    continue
                exclusive = self._exclusive(head.graph_id)
                if exclusive:
                    self.exclusive_busy = True
                self.in_flight += total
                self.launches += 1
                self.batch_sizes.append(len(batch))
            st = stream_hi if exclusive else stream
            try:
                with torch.cuda.stream(st):
                    self._run(batch, st)
            except Exception as e:  # every request of a failed launch sees the error
                for r in batch:
                    if not r.future.done():
                        r.future.set_exception(e)
            finally:
                with self.cv:
                    self.in_flight -= total
                    if exclusive:
                        self.exclusive_busy = False
                    self.cv.notify_all()

    def _run(self, batch, stream):
        g = self.graphs[batch[0].graph_id]
        done = time.perf_counter
        for r in batch:
            stream.wait_event(r.ready)
        if g.n <= self.batch_max_nodes and len(batch) > 1:
            with_truth = [r for r in batch if r.truth is not None]
            without = [r for r in batch if r.truth is None]
            if without:
                L = torch.stack([r.labels for r in without])
                out = qm.score_batched(g, L, [r.K for r in without], stream=stream)
                t = done()
                for r, q in zip(without, out):
                    r.t_done = t
                    r.future.set_result({"quality": q})
            # requests with a ground truth: group those sharing one truth tensor
            groups = collections.defaultdict(list)
            for r in with_truth:
                groups[(r.truth.data_ptr(), r.k_truth)].append(r)
            for (_, kt), rs in groups.items():
                L = torch.stack([r.labels for r in rs])
                oq, oc = qm.evaluate_batched(g, L, [r.K for r in rs], rs[0].truth, kt, stream=stream)
                t = done()
                for r, q, c in zip(rs, oq, oc):
                    r.t_done = t
                    r.future.set_result({"quality": q, "compare": c})
        else:
            for r in batch:
                q = qm.score(g, r.labels, r.K, stream=stream)
                res = {"quality": q}
                if r.truth is not None:
                    res["compare"] = qm.compare(r.truth, r.labels, r.k_truth, r.K, stream=stream)
                r.t_done = done()
                r.future.set_result(res)


def serve_plain(graphs, requests, stream=None):
    """Baseline: the same requests served FIFO, one call per request, one stream.
    requests: list of (t_arrival_offset, graph_id, labels, K, truth, k_truth)."""
    lat, t0 = [], time.perf_counter()
    for (ta, gid, lab, K, truth, kt) in requests:
        now = time.perf_counter() - t0
        if now < ta:
            time.sleep(ta - now)
        g = graphs[gid]
        qm.score(g, lab, K, stream=stream)
        if truth is not None:
            qm.compare(truth, lab, kt, K, stream=stream)
        lat.append(time.perf_counter() - t0 - ta)
    return lat, time.perf_counter() - t0


def _make_workload(duration_s, rate, seed, device, pool_per_graph=24):
    from . import gen
    sizes = {"lfr10k": "lfr10k", "lfr1m": "lfr1m", "lfr10m": "lfr10m"}
    graphs, pools, truths = {}, {}, {}
    for gid, cfg in sizes.items():
        g = gen.lfr_graph(gen.config_params(cfg), device=device)
        # resident graphs of a million nodes and more are renumbered for locality at load
        graphs[gid] = qm.Graph(g.row_ptr, g.col, reorder=g.n >= 1_000_000)
        truths[gid] = (g.labels, g.K)
        rng = np.random.default_rng(seed)
        pools[gid] = [gen.perturb(g.labels, g.K, float(rng.uniform(0, 0.5)), seed=seed + i)
                      for i in range(pool_per_graph)]
        del g
    return graphs, pools, truths


def _arrivals(pools, truths, rate, seed, duration_s=None, count=None):
    """Poisson arrivals at `rate` per second for duration_s seconds (or the
    first `count` of them): each request a uniformly chosen graph, a partition
    from its pool, and with probability 1/2 a comparison with the planted one."""
    rng = np.random.default_rng(seed)
    t, reqs = 0.0, []
    gids = list(pools)
    while True:
        t += rng.exponential(1.0 / rate)
        if (duration_s is not None and t > duration_s) or (count is not None and len(reqs) >= count):
            break
        gid = gids[rng.integers(len(gids))]
        lab = pools[gid][rng.integers(len(pools[gid]))]
        K = truths[gid][1]
        if rng.random() < 0.5:
            reqs.append((t, gid, lab, K, truths[gid][0], truths[gid][1]))
        else:
            reqs.append((t, gid, lab, K, None, None))
    return reqs


def _pct(xs, q):
    return float(np.percentile(np.asarray(xs) * 1e3, q)) if xs else None


def _serve(graphs, reqs, budget_bytes, n_streams):
    """The requests through a Server at their arrival times: latencies
    (arrival to result) and elapsed seconds, and the server's batch record."""
    srv = Server(graphs, budget_bytes, n_streams=n_streams)
    objs, t0 = [], time.perf_counter()
    for (ta, gid, lab, K, truth, kt) in reqs:
        now = time.perf_counter() - t0
        if now < ta:
            time.sleep(ta - now)
        objs.append(srv.submit(gid, lab, K, truth, kt))
    _ = [f.result() for f in objs]
    el = time.perf_counter() - t0
    srv.close()
    lat = [f.request.t_done - f.request.t_arrival for f in objs]
    return lat, el, srv


def _both(graphs, reqs, budget_bytes, n_streams):
    lat, el, srv = _serve(graphs, reqs, budget_bytes, n_streams)
    lat_p, el_p = serve_plain(graphs, reqs)
    return {"requests": len(reqs),
            "served": {"p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99), "partitions_per_s": len(reqs) / el,
                       "launches": srv.launches, "mean_batch": float(np.mean(srv.batch_sizes)),
                       "max_batch": int(max(srv.batch_sizes))},
            "plain": {"p50_ms": _pct(lat_p, 50), "p99_ms": _pct(lat_p, 99), "partitions_per_s": len(reqs) / el_p}}


def run_benchmark(duration_s=60.0, rate=200.0, seed=11, budget_bytes=8 << 30, n_streams=4,
                  sweep_rates=(1000.0, 5000.0, 20000.0), sweep_requests=1500):
    """Poisson arrivals over three resident graphs (10k, 1M, 10M nodes), half of
    the requests with a ground-truth comparison.  Returns p50/p99 latency and
    partitions/s of the served loop and of the plain FIFO baseline (one call per
    request, one stream) on the same arrivals: for duration_s seconds at `rate`,
    for `sweep_requests` requests at each of the sweep rates (where batching
    starts to pay), and for a burst where every request arrives at once."""
    device = torch.device("cuda", torch.cuda.current_device())
    graphs, pools, truths = _make_workload(duration_s, rate, seed, device)
    reqs = _arrivals(pools, truths, rate, seed, duration_s=duration_s)
    torch.cuda.synchronize()

    # warm both paths alike before timing either (scratch pools of the
    # concurrent workers, captured graphs of the small calls): a burst of the
    # first requests through a server and through the plain loop
    warm = [(0.0,) + r[1:] for r in reqs[:min(len(reqs), 96)]]
    srv = Server(graphs, budget_bytes, n_streams=n_streams)
    _ = [f.result() for f in [srv.submit(gid, lab, K, truth, kt) for (_, gid, lab, K, truth, kt) in warm]]
    srv.close()
    serve_plain(graphs, warm)
    torch.cuda.synchronize()

    out = {"rate_per_s": rate, "duration_s": duration_s} | _both(graphs, reqs, budget_bytes, n_streams)
    out["sweep"] = {}
    for i, r in enumerate(sweep_rates):
        rq = _arrivals(pools, truths, r, seed + 1 + i, count=sweep_requests)
        out["sweep"][str(int(r))] = _both(graphs, rq, budget_bytes, n_streams)
    # burst: everything arrives at t = 0 (throughput)
    burst = [(0.0,) + r[1:] for r in reqs[:sweep_requests]]
    srv = Server(graphs, budget_bytes, n_streams=n_streams)
    t0 = time.perf_counter()
    objs = [srv.submit(gid, lab, K, truth, kt) for (_, gid, lab, K, truth, kt) in burst]
    _ = [f.result() for f in objs]
    el = time.perf_counter() - t0
    srv.close()
    out["burst_requests"] = len(burst)
    out["burst_served_partitions_per_s"] = len(burst) / el
    _, el_p = serve_plain(graphs, burst)
    out["burst_plain_partitions_per_s"] = len(burst) / el_p
    for g in graphs.values():
        g.close()
    return out
